"""Pins of the learned-start oracle (oracle/learned.py)."""

import numpy as np
import pytest

import awg_inputs as gi
import oracle as O
import oracle.learned as L


@pytest.fixture(scope="module")
def small():
    p = gi.channels2d(48, q=3, nchan=4, contrast=1e4, seed=9, overlap=2, tau=0.1)
    st = O.setup_problem(p, dense=True)
    return p, st


def test_gradient_matches_finite_differences():
    """Backpropagation against central finite differences of the loss."""
    rng = np.random.default_rng(0)
    F = rng.standard_normal((40, L.NF))
    t = rng.uniform(0, 1, 40)
    th = L.init_params(3) + 0.1 * rng.standard_normal(L.NPARAM)
    _, g = L.loss_and_grad(th, F, t)
    h = 1e-6
    fd = np.zeros_like(th)
    for k in range(L.NPARAM):
        e = np.zeros_like(th)
        e[k] = h
        fd[k] = (L.loss_and_grad(th + e, F, t)[0] - L.loss_and_grad(th - e, F, t)[0]) / (2 * h)
    assert np.max(np.abs(g - fd)) <= 1e-6 * max(1.0, np.max(np.abs(fd)))


def test_adam_first_step_is_signed_lr():
    """First Adam step: m_hat / sqrt(v_hat) = g / |g|, so theta moves by lr."""
    th = np.zeros(5)
    g = np.array([1.0, -2.0, 3.0, -4.0, 0.5])
    th1, m, v = L.adam_step(th, g, np.zeros(5), np.zeros(5), 1, lr=0.1, eps=0.0)
    assert np.allclose(th1, -0.1 * np.sign(g))


def test_leverage_is_projector_diagonal():
    """sum of the unnormalised leverage = rank; invariant to a change of basis."""
    rng = np.random.default_rng(1)
    Y = rng.standard_normal((30, 3))
    g = L.leverage(Y)
    Q, _ = np.linalg.qr(Y)
    raw = np.sum(Q * Q, axis=1)
    assert abs(raw.sum() - 3) < 1e-12
    assert np.allclose(g * raw.max(), raw)
    M = rng.standard_normal((3, 3))
    assert np.allclose(L.leverage(Y @ M), g)


def test_features_definition():
    """Multiplicity and row-sum features against their definitions."""
    p = gi.poisson2d(12, qx=2, overlap=1)
    st = O.setup_problem(p, dense=True)
    mult = 1.0 / st.d
    F = L.node_features(st.A, st.subs[0], mult)
    assert np.allclose(F[:, 1], (mult[st.subs[0]] - 1) / 3)
    A = st.A.toarray()
    rs = A[st.subs[0]].sum(axis=1) / np.diag(A)[st.subs[0]]
    assert np.allclose(F[:, 4], rs)
    assert np.allclose(F[:, 0], 0.0)  # constant coefficient: every log-diag equals the mean


def test_block_eigensolve_finds_the_extra_modes(small):
    """The block iteration returns the pencil's eigenvalues below tau outside
    the kernel (dense eigh of the pencil as the reference), and the
    certificate accepts [kernel, extra modes] but rejects a set missing one."""
    p, st = small
    found = 0
    for s in range(st.N):
        MA, MB, K = L.pencil(st, s)
        lam = st.geneo_lam[s]
        scale = max(1.0, np.abs(lam).max())
        extra = lam[(lam > 1e-9 * scale) & (lam < st.tau)]
        T = st.Ds[s][:, None] * st.splits[s].A_plus_pinv() * st.Ds[s][None, :]
        X0 = np.random.default_rng(s).standard_normal((MA.shape[0], 6))
        th, X, it, cert = L.block_eigensolve(MA, MB, K, T, X0, st.tau)
        assert cert
        got = th[th < st.tau]
        assert got.size == extra.size
        assert np.allclose(got, extra, rtol=1e-8, atol=1e-12)
        Kq = K @ np.linalg.inv(np.linalg.cholesky(K.T @ MB @ K)).T if K.shape[1] else K
        Xs = X[:, th < st.tau]
        U = np.hstack([Kq, Xs])
        assert L.certificate(MA, MB, U, st.tau * (1 - 1e-6))
        if U.shape[1] > 0:
            assert not L.certificate(MA, MB, U[:, :-1], st.tau * (1 - 1e-6))
        found += got.size
    assert found > 0
