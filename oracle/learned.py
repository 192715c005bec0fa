"""Oracle of the learned start block for the GenEO eigensolve.

TEST INFRASTRUCTURE ONLY (see the package header).

The GenEO coarse space of Thm. 4 needs, per subdomain, the eigenvectors of
the pencil (M_A, M_B) = (D^s^-1 A^s_+ D^s^-1, R^s A_+ R^sT) with eigenvalue
below tau (Def. 9).  Their kernel part D^s V^s_- is known exactly (Remark
after Thm. 5); the remaining "extra" modes are found by a block
preconditioned Rayleigh-Ritz iteration, as the paper's own remark (after
Def. 9) suggests with iterative eigensolvers.  A small network proposes where
the extra modes live (their leverage: the diagonal of the orthogonal
projector onto their span, per node) and the start block is that profile
applied to a random block.  This module holds the plain FP64 reference of:

  * the per-node features (computed from A alone),
  * the network's forward and backward passes (gradient-checked against
    central finite differences in the tests),
  * the training target (normalised leverage of the exact extra modes),
  * the block eigensolver and the inertia certificate that judges it.

Network: 5 features -> 16 tanh -> 16 tanh -> 1 sigmoid (385 parameters,
packed as W1[16x5] row-major, b1[16], W2[16x16], b2[16], w3[16], b3[1]).
"""

from __future__ import annotations

import numpy as np
import scipy.linalg as sla

NF, H1, H2 = 5, 16, 16
NPARAM = H1 * NF + H1 + H2 * H1 + H2 + H2 + 1


# ---------------------------------------------------------------- features
def node_features(A, idx: np.ndarray, mult: np.ndarray) -> np.ndarray:
    """Per-node features of one subdomain (rows of a (m, 5) array):
      f0 = (log10 A_pp - mean over the subdomain of log10 A_qq) / 6
      f1 = (multiplicity_p - 1) / 3
      f2 = mean of f0 over the neighbours of p inside the subdomain (0 if none)
      f3 = max of f0 over those neighbours (f0_p if none)
      f4 = (sum_j A_pj over the whole row) / A_pp
    """
    A = A.tocsr()
    m = len(idx)
    pos = {int(g): k for k, g in enumerate(idx)}
    diag = np.array([A[g, g] for g in idx], dtype=float)
    lg = np.log10(diag)
    f0 = (lg - lg.mean()) / 6.0
    F = np.zeros((m, NF))
    F[:, 0] = f0
    F[:, 1] = (mult[idx] - 1.0) / 3.0
    for k, g in enumerate(idx):
        cols = A.indices[A.indptr[g]:A.indptr[g + 1]]
        vals = A.data[A.indptr[g]:A.indptr[g + 1]]
        nb = [pos[int(c)] for c in cols if int(c) != int(g) and int(c) in pos]
        if nb:
            F[k, 2] = f0[nb].mean()
            F[k, 3] = f0[nb].max()
        else:
            F[k, 2] = 0.0
            F[k, 3] = f0[k]
        F[k, 4] = vals.sum() / diag[k]
    return F


# ------------------------------------------------------------------ network
def unpack(theta: np.ndarray):
    o = 0
    W1 = theta[o:o + H1 * NF].reshape(H1, NF); o += H1 * NF
    b1 = theta[o:o + H1]; o += H1
    W2 = theta[o:o + H2 * H1].reshape(H2, H1); o += H2 * H1
    b2 = theta[o:o + H2]; o += H2
    w3 = theta[o:o + H2]; o += H2
    b3 = theta[o]
    return W1, b1, W2, b2, w3, b3


def init_params(seed: int = 0) -> np.ndarray:
    """Glorot-uniform weights, zero biases."""
    rng = np.random.default_rng(seed)
    th = np.zeros(NPARAM)
    o = 0
    for fan_out, fan_in in ((H1, NF), (H2, H1), (1, H2)):
        lim = np.sqrt(6.0 / (fan_in + fan_out))
        th[o:o + fan_out * fan_in] = rng.uniform(-lim, lim, fan_out * fan_in)
        o += fan_out * fan_in + fan_out
    return th


def forward(theta: np.ndarray, F: np.ndarray):
    """Network output per row of F and the activations for backward."""
    W1, b1, W2, b2, w3, b3 = unpack(theta)
    z1 = F @ W1.T + b1
    a1 = np.tanh(z1)
    z2 = a1 @ W2.T + b2
    a2 = np.tanh(z2)
    z3 = a2 @ w3 + b3
    out = 1.0 / (1.0 + np.exp(-z3))
    return out, (F, a1, a2, out)


def loss_and_grad(theta: np.ndarray, F: np.ndarray, t: np.ndarray):
    """Mean squared error L = mean_p (out_p - t_p)^2 and dL/dtheta by
    backpropagation (chain rule written out layer by layer)."""
    out, (F, a1, a2, out) = forward(theta, F)
    P = F.shape[0]
    W1, b1, W2, b2, w3, b3 = unpack(theta)
    err = out - t
    L = float(np.mean(err ** 2))
    d_out = 2.0 * err / P                      # dL/dout
    d_z3 = d_out * out * (1.0 - out)           # sigmoid'
    g_w3 = a2.T @ d_z3
    g_b3 = d_z3.sum()
    d_a2 = np.outer(d_z3, w3)
    d_z2 = d_a2 * (1.0 - a2 ** 2)              # tanh'
    g_W2 = d_z2.T @ a1
    g_b2 = d_z2.sum(axis=0)
    d_a1 = d_z2 @ W2
    d_z1 = d_a1 * (1.0 - a1 ** 2)
    g_W1 = d_z1.T @ F
    g_b1 = d_z1.sum(axis=0)
    g = np.concatenate([g_W1.ravel(), g_b1, g_W2.ravel(), g_b2, g_w3, [g_b3]])
    return L, g


def adam_step(theta, g, m, v, t, lr=1e-2, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam update (Kingma & Ba), returns the new (theta, m, v)."""
    m = b1 * m + (1 - b1) * g
    v = b2 * v + (1 - b2) * g * g
    mh = m / (1 - b1 ** t)
    vh = v / (1 - b2 ** t)
    return theta - lr * mh / (np.sqrt(vh) + eps), m, v


# ---------------------------------------------------------------- targets
def leverage(Y: np.ndarray) -> np.ndarray:
    """Diagonal of the orthogonal projector onto range(Y), normalised to a
    maximum of 1 (all zeros when Y has no columns)."""
    m = Y.shape[0]
    if Y.shape[1] == 0:
        return np.zeros(m)
    Q, _ = np.linalg.qr(Y)
    g = np.sum(Q * Q, axis=1)
    return g / g.max()


def extra_modes(st, s: int):
    """Columns of the exact Y_L (Def. 9) of subdomain s beyond the kernel of
    M_A: eigenvalue above the zero tolerance and below tau."""
    lam = st.geneo_lam[s]
    Y = st.Y[s]
    scale = max(1.0, float(np.abs(lam).max()))
    keep = lam[:Y.shape[1]] > 1e-9 * scale
    return Y[:, keep]


# ------------------------------------------------------- block eigensolver
def pencil(st, s: int):
    """(M_A, M_B, K) of subdomain s: M_A = D^-1 A^s_+ D^-1, M_B = R^s A_+ R^sT
    (Section 4.4 item 4), K = D^s V^s_- (the kernel of M_A)."""
    import oracle.awg_oracle as O
    Ds = st.Ds[s]
    spl = st.splits[s]
    MA = spl.A_plus() / np.outer(Ds, Ds)
    MB = O.local_A_plus_block(st, s)
    K = Ds[:, None] * spl.V_minus
    return 0.5 * (MA + MA.T), 0.5 * (MB + MB.T), K


def block_eigensolve(MA, MB, K, T, X0, tau, tol=1e-13, maxit=200, mu=None):
    """Block inverse iteration with Rayleigh-Ritz for the smallest
    eigenpairs of (M_A, M_B) in the M_B-orthogonal complement of range(K):
      X <- P T M_B X  (T a generalised inverse of M_A, P the M_B-orthogonal
      projector off range(K)), then Rayleigh-Ritz on span(X).
    After each step, once every Ritz pair with value < tau has a norm-wise
    backward error ||M_A x - theta M_B x|| / ((||M_A||_F + |theta| ||M_B||_F)
    ||x||) <= tol, the certificate below is tried with U = [M_B-orthonormal
    K, those Ritz vectors] and mu = tau (1 - 1e-6); the iteration stops when
    it holds.  Returns (theta, X, iterations, certified)."""
    mu = tau * (1 - 1e-6) if mu is None else mu
    nA, nB = np.linalg.norm(MA), np.linalg.norm(MB)
    MBK = MB @ K
    KMK = K.T @ MBK
    Kq = K @ np.linalg.inv(np.linalg.cholesky(KMK)).T if K.shape[1] else K
    def proj(Y):
        if K.shape[1] == 0:
            return Y
        return Y - K @ np.linalg.solve(KMK, MBK.T @ Y)
    X = proj(X0)
    for it in range(1, maxit + 1):
        Y = proj(T @ (MB @ X))
        At = Y.T @ MA @ Y
        Bt = Y.T @ MB @ Y
        th, C = sla.eigh(0.5 * (At + At.T), 0.5 * (Bt + Bt.T))
        X = Y @ C
        R = MA @ X - (MB @ X) * th
        den = (nA + np.abs(th) * nB) * np.linalg.norm(X, axis=0)
        rel = np.linalg.norm(R, axis=0) / den
        below = th < tau
        if np.all(rel[below] <= tol):
            if certificate(MA, MB, np.hstack([Kq, X[:, below]]), mu):
                return th, X, it, True
    return th, X, maxit, False


def certificate(MA, MB, U, mu, sigma=2.0) -> bool:
    """True when M_A - mu M_B + sigma (M_B U)(M_B U)^T is positive definite,
    U M_B-orthonormal.  By Sylvester's law of inertia this holds exactly
    when U spans every eigenvector of (M_A, M_B) with eigenvalue below mu
    (and sigma >= mu)."""
    BU = MB @ U
    S = MA - mu * MB + sigma * (BU @ BU.T)
    try:
        np.linalg.cholesky(0.5 * (S + S.T))
        return True
    except np.linalg.LinAlgError:
        return False
