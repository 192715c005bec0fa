"""FP64 CPU oracle of the AWG preconditioners and of PCG (arXiv 2106.10913).

TEST INFRASTRUCTURE ONLY: imported by tests, by the smoke check and by the
benchmark's CPU-baseline leg, never by the solver library.

Notation follows the paper:
  Omega^s   overlapping index sets (Def. 1), R^s restriction (Def. 2),
  D, D^s    partition of unity (Def. 3), M_mu pair multiplicity and B^s
  (Def. 5), V^s_-, L^s_-, V^s_+, L^s_+ eigen-split of B^s (Def. 6),
  A_+, A_- (Def. 7), H^NN, H^AS_+ and H^AS (Def. 8), Y_L (Def. 9), GenEO
  coarse spaces with H^NN_hyb (Thm. 4), H^AS_+,hyb / H^AS_+,ad (Thm. 3) and
  H^AS_hyb (Thm. 5), W, Pi_3, H_3,ad, H_3,hyb (Def. 10), H_3,inex (Thm. 7).

Readings of points the paper leaves open (each also listed in the design
notes of the repository):
  * overlap growth (Def. 1 gives no construction): Omega^s starts from the
    dofs owned by s and grows by ``overlap`` layers of graph neighbours in the
    stored pattern of A;
  * "A_ij != 0" in Def. 5 is the stored (structural) pattern;
  * zero eigenvalues of B^s (Def. 6 and the Remark after Thm. 2 put them in
    L_-): |lambda| <= 1e-12 max|lambda(B^s)| counts as zero; those vectors
    belong to V^s_- (kernel of A^s_+) but are left out of the second coarse
    space, as Section 4.4 item 1 requires;
  * Y_L selects lambda < tau strictly (Def. 9);
  * E = Z^T A_+ Z (Thm. 4) and F = W^T A W (Def. 10);
  * PCG stops on the unpreconditioned recurrence residual
    ||r_k|| / ||b|| <= rtol with x_0 = 0, then checks the true residual
    (PETSc's preconditioned-norm test is available for the paper's tables);
  * W is exact by default; ``build_W_pcg`` builds it the paper's way (PCG
    with H_2 to a tolerance), ``truncate_W`` drops its small entries;
  * the two-pencil coarse space of H^AS_hyb (Thm. 5) takes both pencils'
    columns side by side (a dependent union leaves E singular, recorded).

``sampled_local_geneo`` evaluates the eigen-splits and GenEO pencils of
chosen subdomains of a problem too large for ``setup`` (used for parity
checks at full size).

Parity of each function is pinned by tests in ``tests/test_oracle_*.py``
against closed forms, exact invariants from the paper's theorems, dense
inverses and brute force.
"""

from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np
import scipy.linalg as sla
import scipy.sparse as sp
import scipy.sparse.linalg as spla

ZERO_EIG_RTOL = 1e-12


# ---------------------------------------------------------------------------
# Section 2.1: subdomains, restriction, minimal overlap
# ---------------------------------------------------------------------------

def csr_from(rowptr, colidx, val, n) -> sp.csr_matrix:
    return sp.csr_matrix((np.asarray(val, float), np.asarray(colidx), np.asarray(rowptr)),
                         shape=(n, n))


def grow_subdomains(A: sp.csr_matrix, part: np.ndarray, nparts: int, overlap: int):
    """Omega^s (Def. 1): the dofs owned by s plus ``overlap`` layers of
    neighbours, where j is a neighbour of i when A_ij is stored."""
    S = A.copy()
    S.data = np.ones_like(S.data)
    S = S.astype(bool)
    subs = []
    for s in range(nparts):
        mask = np.asarray(part) == s
        for _ in range(overlap):
            mask = mask | (S.T.dot(mask.astype(np.int64)) > 0)
        subs.append(np.nonzero(mask)[0].astype(np.int64))
    return subs


def restriction(idx: np.ndarray, n: int) -> sp.csr_matrix:
    """R^s (Def. 2): rows of the identity selected by Omega^s."""
    m = len(idx)
    return sp.csr_matrix((np.ones(m), (np.arange(m), idx)), shape=(m, n))


def minimal_overlap_holds(A: sp.csr_matrix, subs) -> bool:
    """Assumption 1 checked by brute force over every stored (i, j)."""
    n = A.shape[0]
    covered = sp.csr_matrix((n, n), dtype=bool)
    for idx in subs:
        ind = np.zeros(n, dtype=bool)
        ind[idx] = True
        Is = sp.diags(ind.astype(float))
        covered = covered + (Is @ (A != 0).astype(float) @ Is).astype(bool)
    pattern = A.copy()
    pattern.data = np.ones_like(pattern.data)
    pat = pattern.astype(bool).tocoo()
    cov = covered.tocsr()
    return bool(np.all(np.asarray(cov[pat.row, pat.col]).ravel()))


# ---------------------------------------------------------------------------
# Section 2.2: partition of unity, colouring constant
# ---------------------------------------------------------------------------

def partition_of_unity(subs, n: int):
    """D = (sum_t R^tT R^t)^-1 and D^s = R^s D R^sT (Def. 3).  Returns the
    diagonal of D and the list of diagonals of D^s."""
    mult = np.zeros(n)
    for idx in subs:
        R = restriction(idx, n)
        mult += np.asarray((R.T @ R).diagonal()).ravel()
    if np.any(mult == 0):
        raise ValueError("the subdomains do not cover Omega (Def. 1)")
    d = 1.0 / mult
    return d, [d[idx] for idx in subs]


def colouring_constant(subs, A_plus_blocks_nonzero) -> int:
    """A valid N(M) (Def. 4) by greedy colouring of the graph s ~ t iff the
    block R^s M R^tT is non-zero.  ``A_plus_blocks_nonzero(s, t)`` decides it.
    Greedy colouring gives an upper bound of the optimal constant, which keeps
    every bound that uses N valid."""
    N = len(subs)
    colour = [-1] * N
    for s in range(N):
        used = {colour[t] for t in range(N) if t != s and colour[t] >= 0
                and A_plus_blocks_nonzero(s, t)}
        c = 0
        while c in used:
            c += 1
        colour[s] = c
    return max(colour) + 1


# ---------------------------------------------------------------------------
# Section 3.1: pair multiplicity and the splitting B^s (Def. 5, Thm. 1)
# ---------------------------------------------------------------------------

def pair_multiplicity(A: sp.csr_matrix, subs) -> sp.csr_matrix:
    """M_mu = sum_s R^sT R^s S(A) R^sT R^s with S(A) the stored pattern."""
    n = A.shape[0]
    S = A.copy()
    S.data = np.ones_like(S.data)
    M = sp.csr_matrix((n, n))
    for idx in subs:
        R = restriction(idx, n)
        P = R.T @ R
        M = M + P @ S @ P
    return M.tocsr()


def splitting_matrix(A: sp.csr_matrix, Mmu: sp.csr_matrix) -> sp.csr_matrix:
    """B = A (Hadamard /) M_mu on the stored entries of A (Def. 5)."""
    A = A.tocsr().copy()
    A.sort_indices()
    Mmu = Mmu.tocsr()
    coo = A.tocoo()
    mm = np.asarray(Mmu[coo.row, coo.col]).ravel()
    if np.any(mm == 0):
        raise ValueError("minimal overlap (Assumption 1) does not hold")
    return sp.csr_matrix((coo.data / mm, (coo.row, coo.col)), shape=A.shape)


def local_B(B: sp.csr_matrix, idx: np.ndarray) -> np.ndarray:
    """B^s = R^s B R^sT as a dense n^s x n^s array (Def. 5)."""
    return B[idx][:, idx].toarray()


# ---------------------------------------------------------------------------
# Section 3.2: eigen-split of B^s and A_+, A_- (Def. 6, Def. 7, Thm. 2)
# ---------------------------------------------------------------------------

@dataclass
class LocalSplit:
    """Eigen-split B^s = A^s_+ - A^s_- of one subdomain (Def. 6)."""
    lam: np.ndarray          # all eigenvalues, non-decreasing
    V: np.ndarray            # orthonormal eigenvectors
    n_minus: int             # columns of V^s_- (non-positive eigenvalues)
    n_strict: int            # of which strictly negative (enter W)
    tol0: float

    @property
    def V_minus(self):
        return self.V[:, :self.n_minus]

    @property
    def L_minus(self):
        return self.lam[:self.n_minus]

    @property
    def V_plus(self):
        return self.V[:, self.n_minus:]

    @property
    def L_plus(self):
        return self.lam[self.n_minus:]

    @property
    def V_strict(self):
        return self.V[:, :self.n_strict]

    @property
    def L_strict(self):
        return self.lam[:self.n_strict]

    def A_plus(self):
        """A^s_+ = V^s_+ L^s_+ V^s_+^T."""
        return (self.V_plus * self.L_plus) @ self.V_plus.T

    def A_minus(self):
        """A^s_- = -V^s_- L^s_- V^s_-^T."""
        return -(self.V_minus * self.L_minus) @ self.V_minus.T

    def A_plus_pinv(self):
        """(A^s_+)^dagger = V^s_+ (L^s_+)^-1 V^s_+^T (eq. defining H^NN)."""
        return (self.V_plus / self.L_plus) @ self.V_plus.T


def eigen_split(Bs: np.ndarray, zero_rtol: float = ZERO_EIG_RTOL) -> LocalSplit:
    """Diagonalise B^s and split its spectrum at zero (Def. 6).

    Eigenvalues with lambda <= tol0 = zero_rtol * max|lambda| go to L^s_-
    (zeros included, as the Remark after Thm. 2 states); those with
    lambda < -tol0 are the strictly negative ones used for W (Section 4.4).
    """
    lam, V = sla.eigh(Bs)
    tol0 = zero_rtol * (np.max(np.abs(lam)) if lam.size else 0.0)
    n_minus = int(np.sum(lam <= tol0))
    n_strict = int(np.sum(lam < -tol0))
    return LocalSplit(lam, V, n_minus, n_strict, tol0)


# ---------------------------------------------------------------------------
# Everything that follows works on a Setup record.
# ---------------------------------------------------------------------------

@dataclass
class Setup:
    A: sp.csr_matrix
    n: int
    subs: list
    d: np.ndarray
    Ds: list
    B: sp.csr_matrix
    splits: list
    tau: float
    # GenEO
    Y: list = field(default_factory=list)          # Y_L per subdomain
    geneo_lam: list = field(default_factory=list)  # full pencil spectra
    Z: sp.csc_matrix = None
    E: np.ndarray = None
    E_cho: tuple = None
    # second coarse space
    Vhat: sp.csc_matrix = None
    W: np.ndarray = None
    F: np.ndarray = None
    F_cho: tuple = None
    dense: bool = False
    A_plus_dense: np.ndarray = None
    info: dict = field(default_factory=dict)
    # choice of H_2 (Thms. 3-5): "nn_hyb" = H^NN_hyb(tau_sharp),
    # "asp_hyb" = H^AS_+,hyb(tau_flat), "asp_ad" = H^AS_+,ad(tau_flat),
    # "as_hyb" = H^AS_hyb(tau_sharp, tau_flat)
    h2: str = "nn_hyb"
    as_cho: list = field(default_factory=list)     # Cholesky of the local matrices of H^AS_+ / H^AS
    geneo_split: list = field(default_factory=list)  # H^AS: (k1, k2) columns per subdomain from each pencil

    @property
    def N(self):
        return len(self.subs)

    @property
    def n0(self):
        return 0 if self.Z is None else self.Z.shape[1]

    @property
    def n_minus(self):
        return 0 if self.Vhat is None else self.Vhat.shape[1]


def A_minus_apply(st: Setup, x: np.ndarray) -> np.ndarray:
    """A_- x = sum_s R^sT A^s_- R^s x (Def. 7), with A^s_- in its factored
    form -V^s_- L^s_- V^s_-^T.  Works on a vector or on the columns of a
    matrix."""
    y = np.zeros_like(x, dtype=float)
    for idx, spl in zip(st.subs, st.splits):
        if spl.n_minus == 0:
            continue
        Vm = spl.V_minus
        c = Vm.T @ x[idx]
        y[idx] += Vm @ ((-spl.L_minus)[:, None] * c if c.ndim == 2 else (-spl.L_minus) * c)
    return y


def A_plus_apply(st: Setup, x: np.ndarray) -> np.ndarray:
    """A_+ x = A x + A_- x (Thm. 2 (i))."""
    return st.A @ x + A_minus_apply(st, x)


def assemble_dense(st: Setup, which: str) -> np.ndarray:
    """Dense A_+ or A_- = sum_s R^sT A^s_pm R^s (Def. 7); small n only."""
    M = np.zeros((st.n, st.n))
    for idx, spl in zip(st.subs, st.splits):
        loc = spl.A_plus() if which == "plus" else spl.A_minus()
        M[np.ix_(idx, idx)] += loc
    return M


def local_A_plus_from(A: sp.csr_matrix, subs, split_of, s: int) -> np.ndarray:
    """R^s A_+ R^sT through Section 4.4 item 4:
    R^s A R^sT - sum_t R^s R^tT V^t_- L^t_- V^t_-^T R^t R^sT, with the
    eigen-split of subdomain t given by split_of(t) (asked only for the
    subdomains that meet Omega^s)."""
    idx = subs[s]
    M = A[idx][:, idx].toarray()
    for t, jdx in enumerate(subs):
        common, ps, pt = np.intersect1d(idx, jdx, return_indices=True)
        if common.size == 0:
            continue
        spl = split_of(t)
        if spl.n_minus == 0:
            continue
        Vt = spl.V_minus[pt]
        M[np.ix_(ps, ps)] += (Vt * (-spl.L_minus)) @ Vt.T
    return M


def local_A_plus_block(st: Setup, s: int) -> np.ndarray:
    """R^s A_+ R^sT of a set-up problem (Section 4.4 item 4)."""
    return local_A_plus_from(st.A, st.subs, lambda t: st.splits[t], s)


# ---------------------------------------------------------------------------
# Section 3.3: one-level H^NN (Def. 8)
# ---------------------------------------------------------------------------

def H_NN_apply(st: Setup, r: np.ndarray) -> np.ndarray:
    """H^NN r = sum_s R^sT D^s V^s_+ (L^s_+)^-1 V^s_+^T D^s R^s r."""
    z = np.zeros_like(r, dtype=float)
    for idx, Ds, spl in zip(st.subs, st.Ds, st.splits):
        d = Ds if r.ndim == 1 else Ds[:, None]
        lp = spl.L_plus if r.ndim == 1 else spl.L_plus[:, None]
        t = d * r[idx]
        c = spl.V_plus.T @ t
        z[idx] += d * (spl.V_plus @ (c / lp))
    return z


def local_A_plus(st: Setup, s: int) -> np.ndarray:
    """R^s A_+ R^sT: a principal block of the dense A_+ (small n), else
    through Section 4.4 item 4."""
    if st.dense:
        idx = st.subs[s]
        return st.A_plus_dense[np.ix_(idx, idx)]
    return local_A_plus_block(st, s)


def H_plus_AS_apply(st: Setup, r: np.ndarray) -> np.ndarray:
    """H^AS_+ r = sum_s R^sT (R^s A_+ R^sT)^-1 R^s r (Def. 8); the local
    matrices are principal blocks of the spd A_+, so spd, and are solved by
    Cholesky."""
    if not st.as_cho:
        st.as_cho = [sla.cho_factor(0.5 * (M + M.T), lower=True)
                     for M in (local_A_plus(st, s) for s in range(st.N))]
    z = np.zeros_like(r, dtype=float)
    for idx, cho in zip(st.subs, st.as_cho):
        z[idx] += sla.cho_solve(cho, r[idx])
    return z


def H_AS_apply(st: Setup, r: np.ndarray) -> np.ndarray:
    """H^AS r = sum_s R^sT (R^s A R^sT)^-1 R^s r (Def. 8); the local
    matrices are principal blocks of the spd A, solved by Cholesky."""
    if not st.as_cho:
        st.as_cho = [sla.cho_factor(st.A[idx][:, idx].toarray(), lower=True) for idx in st.subs]
    z = np.zeros_like(r, dtype=float)
    for idx, cho in zip(st.subs, st.as_cho):
        z[idx] += sla.cho_solve(cho, r[idx])
    return z


def H1_apply(st: Setup, r: np.ndarray) -> np.ndarray:
    """The one-level preconditioner inside the chosen H_2: H^NN (Thm. 4),
    H^AS_+ (Thm. 3) or H^AS (Thm. 5)."""
    if st.h2 == "nn_hyb":
        return H_NN_apply(st, r)
    return H_AS_apply(st, r) if st.h2 == "as_hyb" else H_plus_AS_apply(st, r)


# ---------------------------------------------------------------------------
# Section 3.4: GenEO coarse space for H^NN (Def. 9, Thm. 4)
# ---------------------------------------------------------------------------

def Y_L(M_A: np.ndarray, M_B: np.ndarray, tau: float):
    """Y_L(tau, M_A, M_B) (Def. 9): the M_B-normalised eigenvectors of the
    pencil whose eigenvalue is below tau, and the whole spectrum."""
    lam, Yfull = sla.eigh(M_A, M_B)
    m = lam.size
    if m == 0 or lam[-1] < tau:
        mL = m
    else:
        mL = int(np.argmax(lam >= tau))
    return Yfull[:, :mL], lam


def geneo_local(spl, Ds: np.ndarray, M_B: np.ndarray, tau: float):
    """Y_L(tau, D^s^-1 A^s_+ D^s^-1, M_B) of one subdomain (Def. 9, Thm. 4)."""
    M_A = (spl.A_plus() / Ds[:, None]) / Ds[None, :]
    return Y_L(0.5 * (M_A + M_A.T), 0.5 * (M_B + M_B.T), tau)


def sampled_local_geneo(A: sp.csr_matrix, subs, Ds, B: sp.csr_matrix, samples, tau: float,
                        zero_rtol: float = ZERO_EIG_RTOL):
    """Def. 6 and Thm. 4's pencil on chosen subdomains of a problem too large
    for ``setup``: the eigen-splits of the sampled subdomains and of every
    subdomain that meets them (the A_- terms of R^s A_+ R^sT), then Y_L of
    each sampled pencil.  Returns, per sample, (eigen-split, Y_L, pencil
    spectrum, R^s A_+ R^sT)."""
    cache = {}

    def split_of(t):
        if t not in cache:
            cache[t] = eigen_split(local_B(B, subs[t]), zero_rtol)
        return cache[t]

    out = []
    for s in samples:
        M_B = local_A_plus_from(A, subs, split_of, s)
        Y, lam = geneo_local(split_of(s), Ds[s], M_B, tau)
        out.append((split_of(s), Y, lam, M_B))
    return out


def geneo_nn(st: Setup, tau: float) -> None:
    """V^0_NN(tau) = sum_s range(R^sT Y_L(tau, D^s^-1 A^s_+ D^s^-1,
    R^s A_+ R^sT)) and E = R^0 A_+ R^0T (Thm. 4)."""
    cols, rows, vals = [], [], []
    col = 0
    st.Y, st.geneo_lam = [], []
    for s, (idx, Ds, spl) in enumerate(zip(st.subs, st.Ds, st.splits)):
        Ys, lam = geneo_local(spl, Ds, local_A_plus(st, s), tau)
        st.Y.append(Ys)
        st.geneo_lam.append(lam)
        k = Ys.shape[1]
        if k:
            rr, cc = np.meshgrid(idx, np.arange(col, col + k), indexing="ij")
            rows.append(rr.ravel())
            cols.append(cc.ravel())
            vals.append(Ys.ravel())
            col += k
    _coarse_from_columns(st, col, rows, cols, vals)


def geneo_as(st: Setup, tau_sharp: float, tau_flat: float) -> None:
    """V^0_AS(tau_sharp, tau_flat) (Thm. 5): per subdomain the columns of
    Y_L(1/tau_flat, D^s^-1 A^s_+ D^s^-1, R^s A R^sT) followed by those of
    Y_L(tau_sharp, R^s A R^sT, R^s A_+ R^sT), prolonged by R^sT, and
    E = Z^T A_+ Z.  The two sets are taken together as the basis the
    theorem assumes; a union that is not linearly independent leaves E
    singular, which is recorded in st.info["E_singular"]."""
    cols, rows, vals = [], [], []
    col = 0
    st.Y, st.geneo_lam, st.geneo_split = [], [], []
    for s, (idx, Ds, spl) in enumerate(zip(st.subs, st.Ds, st.splits)):
        M_A = (spl.A_plus() / Ds[:, None]) / Ds[None, :]
        M_A = 0.5 * (M_A + M_A.T)
        RAR = st.A[idx][:, idx].toarray()
        RApR = local_A_plus(st, s)
        RApR = 0.5 * (RApR + RApR.T)
        Y1, lam1 = Y_L(M_A, RAR, 1.0 / tau_flat)
        Y2, lam2 = Y_L(RAR, RApR, tau_sharp)
        Ys = np.hstack([Y1, Y2])
        st.Y.append(Ys)
        st.geneo_lam.append((lam1, lam2))
        st.geneo_split.append((Y1.shape[1], Y2.shape[1]))
        k = Ys.shape[1]
        if k:
            rr, cc = np.meshgrid(idx, np.arange(col, col + k), indexing="ij")
            rows.append(rr.ravel())
            cols.append(cc.ravel())
            vals.append(Ys.ravel())
            col += k
    _coarse_from_columns(st, col, rows, cols, vals)


def _coarse_from_columns(st: Setup, n0: int, rows, cols, vals) -> None:
    """Z from the prolonged local columns, E = Z^T A_+ Z and its Cholesky
    factor (Assumption 3 asks for a basis: a singular E is recorded)."""
    if n0:
        st.Z = sp.csc_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                             shape=(st.n, n0))
        AZ = A_plus_apply(st, st.Z.toarray()) if st.n * n0 <= 4e7 else _A_plus_sparse_cols(st, st.Z)
        st.E = np.asarray(st.Z.T @ AZ)
        st.E = 0.5 * (st.E + st.E.T)
        try:
            st.E_cho = sla.cho_factor(st.E, lower=True)
        except np.linalg.LinAlgError:
            st.E_cho = None
            st.info["E_singular"] = True
    else:
        st.Z = sp.csc_matrix((st.n, 0))
        st.E = np.zeros((0, 0))
        st.E_cho = None


def _A_plus_sparse_cols(st: Setup, Z: sp.csc_matrix) -> np.ndarray:
    """A_+ Z column block by column block (keeps memory bounded)."""
    out = np.zeros((st.n, Z.shape[1]))
    step = max(1, int(2e7 // st.n))
    for c0 in range(0, Z.shape[1], step):
        blk = Z[:, c0:c0 + step].toarray()
        out[:, c0:c0 + step] = A_plus_apply(st, blk)
    return out


def coarse_E_solve(st: Setup, y: np.ndarray) -> np.ndarray:
    if st.n0 == 0:
        return np.zeros((0,) + y.shape[1:])
    return sla.cho_solve(st.E_cho, y)


def Pi_apply(st: Setup, x: np.ndarray) -> np.ndarray:
    """Pi^NN x = x - Z E^-1 Z^T A_+ x (Thm. 4)."""
    if st.n0 == 0:
        return x.copy()
    return x - st.Z @ coarse_E_solve(st, st.Z.T @ A_plus_apply(st, x))


def Pi_T_apply(st: Setup, x: np.ndarray) -> np.ndarray:
    """Pi^NN^T x = x - A_+ Z E^-1 Z^T x."""
    if st.n0 == 0:
        return x.copy()
    return x - A_plus_apply(st, st.Z @ coarse_E_solve(st, st.Z.T @ x))


def H2_apply(st: Setup, r: np.ndarray) -> np.ndarray:
    """The two-level preconditioner H_2 for A_+ chosen by st.h2:
      H^NN_hyb(tau_sharp) r  = Pi H^NN Pi^T r + Z E^-1 Z^T r    (Thm. 4)
      H^AS_+,hyb(tau_flat) r = Pi H^AS_+ Pi^T r + Z E^-1 Z^T r  (Thm. 3)
      H^AS_+,ad(tau_flat) r  = H^AS_+ r + Z E^-1 Z^T r          (Thm. 3)
      H^AS_hyb(tau_sharp, tau_flat) r = Pi H^AS Pi^T r + Z E^-1 Z^T r (Thm. 5)
    with Pi = I - Z E^-1 Z^T A_+ and E = Z^T A_+ Z in every case."""
    if st.h2 == "asp_ad":
        u = H_plus_AS_apply(st, r)
    else:
        u = Pi_apply(st, H1_apply(st, Pi_T_apply(st, r)))
    if st.n0:
        u = u + st.Z @ coarse_E_solve(st, st.Z.T @ r)
    return u


# ---------------------------------------------------------------------------
# Section 4: the second coarse space and the AWG preconditioners
# ---------------------------------------------------------------------------

def build_Vhat(st: Setup) -> None:
    """[R^1T V^1_- | ... | R^NT V^N_-] restricted to strictly negative
    eigenvalues (Section 4.4 item 1)."""
    rows, cols, vals = [], [], []
    col = 0
    for idx, spl in zip(st.subs, st.splits):
        k = spl.n_strict
        if k:
            rr, cc = np.meshgrid(idx, np.arange(col, col + k), indexing="ij")
            rows.append(rr.ravel())
            cols.append(cc.ravel())
            vals.append(spl.V_strict.ravel())
            col += k
    if col:
        st.Vhat = sp.csc_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                                shape=(st.n, col))
    else:
        st.Vhat = sp.csc_matrix((st.n, 0))


def Lambda_strict(st: Setup) -> np.ndarray:
    """|L^s_-| of the strictly negative eigenvalues, in the column order of
    Vhat."""
    return np.concatenate([-spl.L_strict for spl in st.splits]) if st.n_minus else np.zeros(0)


def solve_A_plus(st: Setup, rhs: np.ndarray) -> np.ndarray:
    """A_+^-1 rhs, exactly.

    Small problems: Cholesky of the densely assembled A_+.  Large problems:
    A_+ = A + U C U^T with U = Vhat and C = diag|L_-| (A^s_- in factored form,
    zero eigenvalues dropped), so the Woodbury identity (eq. (Woodbury), here
    for a positive update) gives A_+^-1 = A^-1 - A^-1 U (C^-1 + U^T A^-1 U)^-1
    U^T A^-1 with A^-1 from a sparse LU of A.
    """
    if st.dense:
        cho = st.info.get("A_plus_cho")
        if cho is None:
            cho = sla.cho_factor(st.A_plus_dense, lower=True)
            st.info["A_plus_cho"] = cho
        return sla.cho_solve(cho, rhs)
    lu = st.info.get("A_lu")
    if lu is None:
        lu = spla.splu(st.A.tocsc())
        st.info["A_lu"] = lu
    X = lu.solve(np.ascontiguousarray(rhs))
    if st.n_minus == 0:
        return X
    U = st.Vhat
    AU = st.info.get("A_inv_U")
    if AU is None:
        AU = lu.solve(U.toarray())
        st.info["A_inv_U"] = AU
    cap = np.diag(1.0 / Lambda_strict(st)) + np.asarray(U.T @ AU)
    return X - AU @ np.linalg.solve(cap, np.asarray(U.T @ X))


def build_W(st: Setup) -> None:
    """W = A_+^-1 [R^sT V^s_-] (Section 4.4 item 1, solved exactly) and
    F = W^T A W (Def. 10)."""
    build_Vhat(st)
    if st.n_minus == 0:
        st.W = np.zeros((st.n, 0))
        st.F = np.zeros((0, 0))
        st.F_cho = None
        return
    if st.dense or st.n * st.n_minus <= _W_BLOCKED_ABOVE:
        st.W = solve_A_plus(st, st.Vhat.toarray())
        F = st.W.T @ (st.A @ st.W)
    else:
        # F = W^T (A W), a block of columns of A W at a time (only one
        # n x n_- array is held)
        st.W = _solve_A_plus_Vhat(st)
        F = np.empty((st.n_minus, st.n_minus))
        for j0 in range(0, st.n_minus, _W_BLOCK[2]):
            j1 = min(st.n_minus, j0 + _W_BLOCK[2])
            F[:, j0:j1] = st.W.T @ (st.A @ st.W[:, j0:j1])
    st.F = 0.5 * (F + F.T)
    st.F_cho = sla.cho_factor(st.F, lower=True)


# Problems whose n x n_- arrays hold more values than this take the blocked
# route below (same steps; the rounding of the blocked products differs in
# the last bits): the elasticity workload's oracle run (n = 295 680,
# n_- = 6659) needs it to fit in 62 GB of host memory.
_W_BLOCKED_ABOVE = 1 << 28
# block sizes of that route: columns of A^-1 U, rows of the update, columns of A W
_W_BLOCK = (256, 16384, 512)


def _solve_A_plus_Vhat(st: Setup) -> np.ndarray:
    """W = A_+^-1 U for U = Vhat on a large problem, by the same Woodbury
    form as solve_A_plus with rhs = U: X = A^-1 U, then
    W = X - X (C^-1 + U^T X)^-1 U^T X, computed in place in X (the steps
    and their order are those of solve_A_plus, in blocks of columns for the
    solves and of rows for the update, so that only one n x n_- array is
    held)."""
    lu = st.info.get("A_lu")
    if lu is None:
        lu = spla.splu(st.A.tocsc())
        st.info["A_lu"] = lu
    U = st.Vhat.tocsc()
    X = np.empty((st.n, st.n_minus), order="F")
    for j0 in range(0, st.n_minus, _W_BLOCK[0]):  # A^-1 U, a block of columns at a time
        j1 = min(st.n_minus, j0 + _W_BLOCK[0])
        X[:, j0:j1] = lu.solve(U[:, j0:j1].toarray())
    cap = np.diag(1.0 / Lambda_strict(st)) + np.asarray(U.T @ X)
    G = np.linalg.solve(cap, np.asarray(U.T @ X))
    for i0 in range(0, st.n, _W_BLOCK[1]):  # X - X G, a block of rows at a time
        i1 = min(st.n, i0 + _W_BLOCK[1])
        X[i0:i1] -= X[i0:i1] @ G
    return X


def build_W_pcg(st: Setup, rtol: float) -> Setup:
    """W by the paper's own route (Section 4.4 item 2): each column
    A_+^-1 R^sT v^s_- by PCG preconditioned with H_2 from x_0 = 0, stopped
    at the relative tolerance rtol on the preconditioned residual (PETSc's
    default test, with which the paper's experiments ran; Table 4 varies
    rtol), then F = W^T A W from that W.  Returns a copy of the setup."""
    import dataclasses
    if st.n_minus == 0:
        return dataclasses.replace(st, info=dict(st.info))
    V = st.Vhat.toarray()
    W = np.zeros_like(V)
    for j in range(V.shape[1]):
        W[:, j] = pcg(lambda v: A_plus_apply(st, v), V[:, j], lambda r: H2_apply(st, r), rtol=rtol,
                      norm="preconditioned").x
    F = W.T @ (st.A @ W)
    F = 0.5 * (F + F.T)
    return dataclasses.replace(st, W=W, F=F, F_cho=sla.cho_factor(F, lower=True), info=dict(st.info))


def truncate_W(st: Setup, theta: float) -> Setup:
    """A sparser second coarse space (the conclusion, Section 6, leaves
    sparser approximations of it open): a copy of the setup whose W drops
    the entries below theta * max_i |W_ij| of their column, with F = W^T A W
    rebuilt from the truncated W so that H_3 stays spd.  theta = 0 keeps
    W.  Thm. 8's bounds need range(W) = range(A_+^-1 V_-) and no longer
    hold; W F^-1 W^T A is still an A-orthogonal projector.  Columns that
    truncation makes linearly dependent leave F singular: recorded in
    info["F_singular"] (F_cho = None)."""
    import dataclasses
    if st.n_minus == 0:
        return dataclasses.replace(st, info=dict(st.info))
    cmax = np.abs(st.W).max(axis=0)
    Wt = np.where(np.abs(st.W) >= theta * cmax[None, :], st.W, 0.0)
    F = Wt.T @ (st.A @ Wt)
    F = 0.5 * (F + F.T)
    info = dict(st.info)
    try:
        cho = sla.cho_factor(F, lower=True)
    except np.linalg.LinAlgError:
        cho = None
        info["F_singular"] = True
    return dataclasses.replace(st, W=Wt, F=F, F_cho=cho, info=info)


def coarse_F_solve(st: Setup, y: np.ndarray) -> np.ndarray:
    if st.n_minus == 0:
        return np.zeros((0,) + y.shape[1:])
    return sla.cho_solve(st.F_cho, y)


def H3_ad_apply(st: Setup, r: np.ndarray) -> np.ndarray:
    """H_3,ad r = H_2 r + W (W^T A W)^-1 W^T r (Def. 10)."""
    z = H2_apply(st, r)
    if st.n_minus:
        z = z + st.W @ coarse_F_solve(st, st.W.T @ r)
    return z


def Pi3_apply(st: Setup, x: np.ndarray) -> np.ndarray:
    """Pi_3 x = x - W (W^T A W)^-1 W^T A x (Def. 10)."""
    if st.n_minus == 0:
        return x.copy()
    return x - st.W @ coarse_F_solve(st, st.W.T @ (st.A @ x))


def Pi3_T_apply(st: Setup, x: np.ndarray) -> np.ndarray:
    if st.n_minus == 0:
        return x.copy()
    return x - st.A @ (st.W @ coarse_F_solve(st, st.W.T @ x))


def H3_hyb_apply(st: Setup, r: np.ndarray) -> np.ndarray:
    """H_3,hyb r = Pi_3 H_2 Pi_3^T r + W (W^T A W)^-1 W^T r (Def. 10)."""
    z = Pi3_apply(st, H2_apply(st, Pi3_T_apply(st, r)))
    if st.n_minus:
        z = z + st.W @ coarse_F_solve(st, st.W.T @ r)
    return z


def H3_inex_apply(st: Setup, r: np.ndarray) -> np.ndarray:
    """H_3,inex r = H_2 r + A_+^-1 V (C^-1 - V^T A_+^-1 V)^-1 V^T A_+^-1 r
    (Thm. 7), with A_- = V C V^T, V = Vhat and C = diag|L_-| (the Woodbury
    identity holds for any such factorisation)."""
    z = H2_apply(st, r)
    if st.n_minus:
        C = Lambda_strict(st)
        V = st.Vhat
        inner = np.diag(1.0 / C) - np.asarray(V.T @ st.W)   # W = A_+^-1 V
        z = z + st.W @ np.linalg.solve(inner, st.W.T @ r)
    return z


# ---------------------------------------------------------------------------
# Setup driver
# ---------------------------------------------------------------------------

def setup(rowptr, colidx, val, n, part=None, nparts=None, overlap=1, tau=0.1, subsets=None,
          dense=None, zero_rtol=ZERO_EIG_RTOL, with_W=True, h2="nn_hyb", tau_flat=10.0) -> Setup:
    """Build every ingredient of H_3 from A alone (Sections 2-4).  ``tau``
    is tau_sharp of H^NN_hyb (Thm. 4); with h2 = "asp_hyb" / "asp_ad" the
    coarse space is V^0_AS,+(tau_flat) of Thm. 3, the eigenvectors of the
    same pencil below 1 / tau_flat; with h2 = "as_hyb" it is
    V^0_AS(tau, tau_flat) of Thm. 5 (two pencils)."""
    if h2 not in ("nn_hyb", "asp_hyb", "asp_ad", "as_hyb"):
        raise ValueError(f"unknown H_2 {h2!r}")
    if h2 in ("asp_hyb", "asp_ad"):
        tau = 1.0 / tau_flat
    A = csr_from(rowptr, colidx, val, n)
    if subsets is not None:
        subs = [np.asarray(s, dtype=np.int64) for s in subsets]
    else:
        subs = grow_subdomains(A, part, nparts, overlap)
    d, Ds = partition_of_unity(subs, n)
    Mmu = pair_multiplicity(A, subs)
    B = splitting_matrix(A, Mmu)
    splits = [eigen_split(local_B(B, idx), zero_rtol) for idx in subs]
    dense = (n <= 6000) if dense is None else dense
    st = Setup(A=A, n=n, subs=subs, d=d, Ds=Ds, B=B, splits=splits, tau=tau, dense=dense, h2=h2)
    if dense:
        st.A_plus_dense = assemble_dense(st, "plus")
    if h2 == "as_hyb":
        geneo_as(st, tau, tau_flat)
    else:
        geneo_nn(st, tau)
    if with_W:
        build_W(st)
    return st


def setup_problem(prob, **kw) -> Setup:
    """Setup from an ``awg_inputs.Problem``."""
    return setup(prob.rowptr, prob.colidx, prob.val, prob.n, part=prob.part,
                 nparts=prob.nparts, overlap=prob.overlap, tau=kw.pop("tau", prob.tau),
                 subsets=prob.subsets, **kw)


def local_condition(st: Setup) -> float:
    """max_s lambda_max(A^s_+) / lambda_min+(A^s_+): the condition number of
    the local pseudo-inverses (with H^AS_+, max_s cond(R^s A_+ R^sT)).  Any backward-stable evaluation of
    (A^s_+)^+ t (this oracle's eigenvector form, or a Cholesky route) has a
    forward error of order local_condition * eps, which bounds how closely
    two correct implementations of H^NN can agree."""
    if st.h2 == "as_hyb":  # H^AS: the local solvers are (R^s A R^sT)^-1
        return float(max(np.linalg.cond(st.A[idx][:, idx].toarray()) for idx in st.subs))
    if st.h2 != "nn_hyb":  # H^AS_+: the local solvers are (R^s A_+ R^sT)^-1
        return float(max(np.linalg.cond(0.5 * (M + M.T)) for M in (local_A_plus(st, s) for s in range(st.N))))
    return float(max(s.L_plus.max() / s.L_plus.min() for s in st.splits if s.L_plus.size))


def mode_counts(st: Setup) -> np.ndarray:
    """Per-subdomain GenEO mode count m^s (columns of Y_L)."""
    return np.array([Y.shape[1] for Y in st.Y], dtype=np.int64)


def minus_counts(st: Setup) -> np.ndarray:
    """Per-subdomain counts (n^s_-, strictly negative)."""
    return np.array([[s.n_minus, s.n_strict] for s in st.splits], dtype=np.int64)


# ---------------------------------------------------------------------------
# PCG (Saad, Algorithm 9.1, as cited in Section 1) and its Lanczos estimates
# ---------------------------------------------------------------------------

@dataclass
class PCGResult:
    x: np.ndarray
    iters: int
    relres: float
    true_relres: float
    converged: bool
    alphas: list
    betas: list
    history: list


def pcg(A_apply, b: np.ndarray, M_apply=None, rtol: float = 1e-8, maxit: int = 1000,
        x0=None, norm: str = "unpreconditioned") -> PCGResult:
    """Preconditioned CG (Saad, Algorithm 9.1, with x_0 = 0 by default).

    ``norm="unpreconditioned"``: stop when ||r_k|| / ||b|| <= rtol on the
    recurrence residual, then confirm on the true residual b - A x_k and keep
    iterating while the true residual is still above rtol (stopping if the
    recurrence residual has fallen 1e6 below rtol, where rounding makes the
    true residual unattainable).
    ``norm="preconditioned"``: stop when ||z_k|| / ||z_0|| <= rtol with
    z_k = H r_k, the default test of PETSc's CG, with which the paper's
    experiments were run (Section 5).
    """
    M_apply = (lambda v: v.copy()) if M_apply is None else M_apply
    x = np.zeros_like(b) if x0 is None else x0.copy()
    r = b - A_apply(x)
    bnorm = np.linalg.norm(b)
    if bnorm == 0.0:
        return PCGResult(x, 0, 0.0, 0.0, True, [], [], [0.0])
    z = M_apply(r)
    z0norm = np.linalg.norm(z)
    p = z.copy()
    rz = float(r @ z)
    alphas, betas = [], []
    hist = [np.linalg.norm(r) / bnorm if norm == "unpreconditioned" else 1.0]
    it = 0
    converged = False
    while it < maxit:
        q = A_apply(p)
        pq = float(p @ q)
        if not pq > 0.0:
            break
        alpha = rz / pq
        x = x + alpha * p
        r = r - alpha * q
        it += 1
        alphas.append(alpha)
        z = M_apply(r)
        if norm == "unpreconditioned":
            rel = np.linalg.norm(r) / bnorm
            hist.append(rel)
            if rel <= rtol:
                true_rel = np.linalg.norm(b - A_apply(x)) / bnorm
                if true_rel <= rtol or rel <= 1e-6 * rtol:
                    converged = true_rel <= rtol
                    break
        else:
            rel = np.linalg.norm(z) / z0norm
            hist.append(rel)
            if rel <= rtol:
                converged = True
                break
        rz_new = float(r @ z)
        if rz_new == 0.0:
            converged = True
            break
        beta = rz_new / rz
        betas.append(beta)
        rz = rz_new
        p = z + beta * p
    true_rel = np.linalg.norm(b - A_apply(x)) / bnorm
    return PCGResult(x, it, hist[-1], true_rel, converged, alphas, betas, hist)


def lanczos_extremes(alphas, betas):
    """Extreme eigenvalues of H A estimated from the CG coefficients through
    the Lanczos tridiagonal matrix T_k."""
    k = len(alphas)
    if k == 0:
        return float("nan"), float("nan")
    d = np.zeros(k)
    e = np.zeros(max(k - 1, 0))
    for j in range(k):
        d[j] = 1.0 / alphas[j] + (betas[j - 1] / alphas[j - 1] if j > 0 else 0.0)
        if j < k - 1:
            e[j] = math.sqrt(betas[j]) / alphas[j]
    ev = sla.eigh_tridiagonal(d, e, eigvals_only=True)
    return float(ev[0]), float(ev[-1])


# ---------------------------------------------------------------------------
# Dense helpers for small problems (tests)
# ---------------------------------------------------------------------------

def dense_operator(apply, n: int) -> np.ndarray:
    """The n x n matrix of a linear map, column by column."""
    I = np.eye(n)
    return apply(I)


def spectrum_HA(H: np.ndarray, A: np.ndarray) -> np.ndarray:
    """Eigenvalues of H A for SPD H, A through the similar matrix
    A^1/2 H A^1/2 (real and sorted)."""
    L = np.linalg.cholesky(A)
    S = L.T @ H @ L
    return np.sort(np.linalg.eigvalsh(0.5 * (S + S.T)))


def A_plus_blocks_nonzero_fn(st: Setup):
    """Predicate for ``colouring_constant`` with M = A_+: R^s A_+ R^tT is
    non-zero when some subdomain u meets both Omega^s and Omega^t (A^u_+ is
    dense on Omega^u) or when A couples them."""
    N = st.N
    n = st.n
    memb = sp.csr_matrix((np.ones(sum(len(s) for s in st.subs)),
                          (np.concatenate([np.full(len(s), k) for k, s in enumerate(st.subs)]),
                           np.concatenate(st.subs))), shape=(N, n))
    meet = (memb @ memb.T).toarray() > 0          # Omega^s meets Omega^u
    reach = (meet.astype(float) @ meet.astype(float)) > 0
    return lambda s, t: bool(reach[s, t])
