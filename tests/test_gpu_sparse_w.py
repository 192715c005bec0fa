"""A sparser second coarse space (the paper's conclusion, Section 6, leaves
sparser approximations of W open): the float64 form with a truncated W
(awg_options.w_drop_tol = theta: the entries |W_ij| >= theta max_i |W_ij|
kept, stored by rows and by columns, F = W^T A W rebuilt from them) against
the oracle's truncate_W at the same theta, through the C ABI:

* H_3,ad and H_3,hyb applies within the float64 apply tolerance
  (max(1e-11, kappa_loc eps)), entry by entry and in norm (H_3,inex is not
  built on a truncated W: Thm. 7's inner matrix assumes W = A_+^-1 Vhat;
  its stage reports AWG_ERR_STATE);
* PCG (host-driven and graph-driven) iterations within 5 % of the oracle's
  PCG with its truncated H_3,ad, true relative residual <= 1e-8;
* the kept entries reported by awg_get_info equal the oracle's count;
* the mixed forms keep the full W (their apply matches the untruncated
  oracle to 1e-4), and the float64 block form reports AWG_ERR_STATE.

Which entries fall below the threshold depends on the basis of W, that
is, on the eigenvectors V^s_- chosen within any multiple eigenvalue of
B^s; the two sides pick those independently.  Exact parity is therefore
checked on problems without symmetry (random coefficients and partitions:
the 3D log-normal generator with k-means parts, a random SPD graph
Laplacian, channels at random rows), and only where no entry of the
oracle's W lies within 1e-7 of the threshold (relative); on symmetric
problems (Poisson, whose subdomains' spectra have multiple eigenvalues) the
truncated solve is checked through what holds in any basis: the PCG
iterations of the oracle's truncated run and a true residual <= 1e-8.
"""

import numpy as np
import pytest

import awg_inputs as gi
import oracle as O

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

THETA = 1e-4
CASES = {
    "channels64": lambda: gi.channels2d(64, q=2, nchan=3, contrast=1e6, seed=11, overlap=2, tau=0.1),
    "grf3d14": lambda: gi.grf3d(L=14, k=12, corr_len=3.0),
    "random_spd400": lambda: gi.random_spd(400, nparts=6, density=0.02, seed=9, overlap=1, tau=0.1),
}
SYMMETRIC = {"config1": lambda: gi.config1()}
_PAIRS = {}


def _pair(name):
    if name not in _PAIRS:
        from paper_2106_10913_gb300 import AWGSolver
        p = CASES[name]()
        st = O.setup_problem(p, dense=p.n <= 6000)
        cmax = np.abs(st.W).max(axis=0)
        rel = np.abs(np.abs(st.W) - THETA * cmax[None, :]) / (THETA * cmax[None, :])
        if rel.min() <= 1e-7:
            pytest.skip("an entry of W lies at the truncation threshold")
        stt = O.truncate_W(st, THETA)
        sol = AWGSolver(p.rowptr, p.colidx, p.val, p.part, p.nparts, p.overlap, p.tau, precisions=0b0011,
                        w_drop_tol=THETA, variant=0)
        _PAIRS[name] = (p, sol, st, stt)
    return _PAIRS[name]


@pytest.fixture(scope="module", params=list(CASES))
def pair(request):
    return _pair(request.param)


def _rel(a, b):
    a, b = np.asarray(a), np.asarray(b)
    return max(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300),
               float(np.max(np.abs(a - b), initial=0.0)) / max(float(np.max(np.abs(b), initial=0.0)), 1e-300))


def test_kept_entries(pair):
    p, sol, st, stt = pair
    from paper_2106_10913_gb300 import awg_get_info
    kept = awg_get_info(sol.h)["w_kept"]
    assert kept == np.count_nonzero(stt.W)
    print(f"[{p.name}: truncated W keeps {kept} of {st.W.size} entries ({100 * kept / st.W.size:.1f} %)]")


@pytest.mark.parametrize("stage", ["h3ad", "h3hyb"])
def test_truncated_apply(pair, stage):
    p, sol, st, stt = pair
    ref = {"h3ad": O.H3_ad_apply, "h3hyb": O.H3_hyb_apply}[stage]
    tol = max(1e-11, O.local_condition(st) * np.finfo(float).eps)
    for seed in (1, 2):
        x = np.random.default_rng(seed).standard_normal(p.n)
        y = sol.apply(torch.from_numpy(x).cuda(), stage=stage).cpu().numpy()
        assert _rel(y, ref(stt, x)) <= tol, seed


def test_truncated_pcg(pair):
    p, sol, st, stt = pair
    from paper_2106_10913_gb300 import FP64, awg_pcg_block_async
    b = p.b if p.b.ndim == 1 else p.b[0]
    ref = O.pcg(lambda v: st.A @ v, b, lambda r: O.H3_ad_apply(stt, r), rtol=1e-8)
    x, its, rel, status = sol.pcg(torch.from_numpy(b).cuda(), rtol=1e-8)
    assert status == 0 and rel[0] <= 1e-8
    assert abs(its[0] - ref.iters) <= max(1.0, 0.05 * ref.iters), (its[0], ref.iters)
    assert np.linalg.norm(st.A @ x.cpu().numpy() - b) <= 1e-8 * np.linalg.norm(b) * (1 + 1e-12)
    # the graph-driven single-right-hand-side solve on the same form
    bb = torch.from_numpy(b[None, :].copy()).cuda()
    xx = torch.zeros_like(bb)
    it_d = torch.zeros(1, dtype=torch.int32, device="cuda")
    rl_d = torch.zeros(1, dtype=torch.float64, device="cuda")
    st_d = torch.full((1,), -1, dtype=torch.int32, device="cuda")
    awg_pcg_block_async(sol.h, bb, xx, it_d, rl_d, st_d, 1e-8, precision=FP64)
    torch.cuda.synchronize()
    assert int(st_d.item()) == 0 and float(rl_d.item()) <= 1e-8
    assert abs(int(it_d.item()) - ref.iters) <= max(1.0, 0.05 * ref.iters)
    print(f"[{p.name}: truncated-W PCG {its[0]} iterations (oracle {ref.iters})]")


def test_mixed_forms_keep_full_W(pair):
    p, sol, st, stt = pair
    from paper_2106_10913_gb300 import FP64, MIXED_FP32, AWGError, awg_apply_block
    x = np.random.default_rng(3).standard_normal(p.n)
    y = sol.apply(torch.from_numpy(x).cuda(), precision=MIXED_FP32).cpu().numpy()
    assert _rel(y, O.H3_ad_apply(st, x)) <= 1e-4
    X = torch.from_numpy(np.random.default_rng(4).standard_normal((3, p.n))).cuda()
    with pytest.raises(AWGError):
        awg_apply_block(sol.h, "h3ad", X, torch.empty_like(X), precision=FP64)
    with pytest.raises(AWGError):
        sol.apply(torch.from_numpy(x).cuda(), stage="h3inex")


@pytest.mark.parametrize("name", list(SYMMETRIC))
def test_truncated_pcg_symmetric_problem(name):
    """Poisson (multiple eigenvalues in the subdomains' spectra): the
    truncated-W solve reaches 1e-8 in the oracle's iterations (within 5 %)."""
    from paper_2106_10913_gb300 import AWGSolver
    p = SYMMETRIC[name]()
    st = O.setup_problem(p, dense=p.n <= 6000)
    stt = O.truncate_W(st, THETA)
    sol = AWGSolver(p.rowptr, p.colidx, p.val, p.part, p.nparts, p.overlap, p.tau, w_drop_tol=THETA)
    try:
        b = p.b if p.b.ndim == 1 else p.b[0]
        ref = O.pcg(lambda v: st.A @ v, b, lambda r: O.H3_ad_apply(stt, r), rtol=1e-8)
        x, its, rel, status = sol.pcg(torch.from_numpy(b).cuda(), rtol=1e-8)
        assert status == 0 and rel[0] <= 1e-8
        assert abs(its[0] - ref.iters) <= max(1.0, 0.05 * ref.iters), (its[0], ref.iters)
        assert np.linalg.norm(st.A @ x.cpu().numpy() - b) <= 1e-8 * np.linalg.norm(b) * (1 + 1e-12)
    finally:
        sol.close()
