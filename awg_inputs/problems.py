"""Problem generators: sparse SPD matrices, partitions and right-hand sides.

Every generator is deterministic given its seed (NumPy ``default_rng``) and
uses only elementwise IEEE arithmetic whose result does not depend on the
machine (no BLAS reductions), so the x86 host and the Arm GPU host build
identical problems.

Matrices are returned in CSR form with ``int32`` row pointers and column
indices (sorted within each row, no duplicates) and ``float64`` values.  The
sparsity pattern is the structural pattern of the discretisation: an entry
that is assembled is stored even if its value cancels to zero.

Workloads (sizes and distributions of the paper's experiments and of their
scaled-up GPU versions):

* ``poisson2d``      vertex-centred 5-point Laplacian (4/-1), Dirichlet
                     neighbours eliminated.
* ``channels2d``     cell-centred finite volumes, harmonic-mean face
                     transmissibilities, Dirichlet faces at half-cell distance,
                     coefficient 1 with seeded horizontal high-contrast
                     channels of width 2 cells.
* ``grf3d``          7-point finite volumes with a log-normal coefficient
                     (Gaussian random field) and a k-means partition.
* ``elasticity2d``   Q1 plane-strain linear elasticity with layered Young's
                     modulus, clamped left edge (Section 5, eq. (elasticity)).
* ``random_spd``     random sparse SPD matrices (graph Laplacian plus a
                     positive diagonal) with random partitions, for property
                     tests.
"""

from __future__ import annotations

from dataclasses import dataclass, field
from typing import Optional

import numpy as np
import scipy.sparse as sp


@dataclass
class Problem:
    """A linear system A x = b with a non-overlapping partition of its dofs.

    ``part[i]`` is the subdomain that owns dof ``i`` before overlap growth
    (values ``0..nparts-1``).  ``subsets``, when given, lists explicit
    overlapping index sets instead (used by the paper's own example, whose
    subdomains are closed unit squares that share their interfaces).
    ``b`` has shape ``(n,)`` for one right-hand side or ``(nrhs, n)`` for
    several (each right-hand side contiguous).
    """

    name: str
    n: int
    rowptr: np.ndarray
    colidx: np.ndarray
    val: np.ndarray
    part: np.ndarray
    nparts: int
    overlap: int
    tau: float
    b: np.ndarray
    subsets: Optional[list] = None
    meta: dict = field(default_factory=dict)

    @property
    def nnz(self) -> int:
        return int(self.rowptr[-1])

    def csr(self) -> sp.csr_matrix:
        return sp.csr_matrix((self.val, self.colidx, self.rowptr),
                             shape=(self.n, self.n))


def _to_csr(rows, cols, vals, n):
    """Sum duplicates into a CSR matrix with sorted int32 indices."""
    rows = np.asarray(rows, dtype=np.int64)
    cols = np.asarray(cols, dtype=np.int64)
    vals = np.asarray(vals, dtype=np.float64)
    # Sort by (row, col) and sum duplicates in a fixed order so that the
    # result is machine independent.
    key = rows * n + cols
    order = np.argsort(key, kind="stable")
    key = key[order]
    vals = vals[order]
    uniq, start = np.unique(key, return_index=True)
    summed = np.add.reduceat(vals, start) if len(vals) else vals
    r = (uniq // n).astype(np.int64)
    c = (uniq % n).astype(np.int32)
    rowptr = np.zeros(n + 1, dtype=np.int64)
    np.add.at(rowptr, r + 1, 1)
    rowptr = np.cumsum(rowptr).astype(np.int32)
    return rowptr, c, summed.astype(np.float64)


def box_partition(nx: int, ny: int, qx: int, qy: int, nz: int = 1, qz: int = 1):
    """Owner of every grid point for a qx x qy (x qz) box partition.

    Box edges are at floor(i*L/q); point (x, y, z) has index
    (z*ny + y)*nx + x.
    """
    bx = (np.arange(nx) * qx) // nx
    by = (np.arange(ny) * qy) // ny
    bz = (np.arange(nz) * qz) // nz
    owner = (bz[:, None, None] * qy + by[None, :, None]) * qx + bx[None, None, :]
    return owner.reshape(-1).astype(np.int32)


# ---------------------------------------------------------------------------
# 2D Poisson, vertex centred
# ---------------------------------------------------------------------------

def poisson2d(nx: int = 64, ny: Optional[int] = None, qx: int = 4, qy: Optional[int] = None,
              overlap: int = 1, tau: float = 0.1, seed: int = 0, nrhs: int = 1,
              scale: float = 1.0) -> Problem:
    """5-point 4/-1 stencil on the nx x ny interior nodes of a Dirichlet grid."""
    ny = nx if ny is None else ny
    qy = qx if qy is None else qy
    n = nx * ny
    idx = np.arange(n).reshape(ny, nx)
    rows = [idx.ravel()]
    cols = [idx.ravel()]
    vals = [np.full(n, 4.0 * scale)]
    for dy, dx in ((0, 1), (0, -1), (1, 0), (-1, 0)):
        ys, xs = np.meshgrid(np.arange(ny), np.arange(nx), indexing="ij")
        yt, xt = ys + dy, xs + dx
        ok = (yt >= 0) & (yt < ny) & (xt >= 0) & (xt < nx)
        rows.append(idx[ys[ok], xs[ok]])
        cols.append(idx[yt[ok], xt[ok]])
        vals.append(np.full(int(ok.sum()), -1.0 * scale))
    rowptr, colidx, val = _to_csr(np.concatenate(rows), np.concatenate(cols),
                                  np.concatenate(vals), n)
    part = box_partition(nx, ny, qx, qy)
    b = _rhs(n, seed, nrhs)
    return Problem(f"poisson2d_{nx}x{ny}_q{qx}x{qy}_ov{overlap}", n, rowptr, colidx, val,
                   part, qx * qy, overlap, tau, b,
                   meta=dict(kind="poisson2d", nx=nx, ny=ny, qx=qx, qy=qy))


def _rhs(n, seed, nrhs):
    rng = np.random.default_rng(seed)
    if nrhs == 1:
        return rng.standard_normal(n)
    return rng.standard_normal((nrhs, n))


# ---------------------------------------------------------------------------
# 2D / 3D finite-volume diffusion
# ---------------------------------------------------------------------------

def _fv_matrix(kappa: np.ndarray):
    """Cell-centred FV matrix on a unit-spacing grid (2D or 3D).

    Face transmissibility between neighbouring cells is the harmonic mean
    2 k_i k_j / (k_i + k_j); a Dirichlet boundary face contributes 2 k_i to the
    diagonal (the boundary is half a cell away).  ``kappa`` is indexed
    [z, y, x] (or [y, x]).
    """
    shape = kappa.shape
    n = kappa.size
    idx = np.arange(n).reshape(shape)
    diag = np.zeros(shape)
    rows, cols, vals = [], [], []
    for ax in range(kappa.ndim):
        a = np.moveaxis(kappa, ax, 0)
        ia = np.moveaxis(idx, ax, 0)
        ka, kb = a[:-1], a[1:]
        t = 2.0 * ka * kb / (ka + kb)
        i0, i1 = ia[:-1].ravel(), ia[1:].ravel()
        tf = t.ravel()
        rows += [i0, i1]
        cols += [i1, i0]
        vals += [-tf, -tf]
        d = np.moveaxis(diag, ax, 0)
        d[:-1] += t
        d[1:] += t
        d[0] += 2.0 * a[0]
        d[-1] += 2.0 * a[-1]
    rows.append(idx.ravel())
    cols.append(idx.ravel())
    vals.append(diag.ravel())
    return _to_csr(np.concatenate(rows), np.concatenate(cols), np.concatenate(vals), n)


def _channel_field(L: int, nchan: int, contrast: float, rng) -> np.ndarray:
    kappa = np.ones((L, L))
    y0 = rng.integers(0, L - 1, size=nchan)  # start rows in [0, L-2]
    for y in y0:
        kappa[y, :] = contrast
        kappa[y + 1, :] = contrast
    return kappa


def channels2d(L: int = 512, q: int = 16, nchan: int = 20, contrast: float = 1e6,
               seed: int = 2, overlap: int = 2, tau: float = 0.1, rhs_seed: int = 0,
               nrhs: int = 1) -> Problem:
    """L x L cells, coefficient 1 with ``nchan`` horizontal channels of width 2
    at ``contrast`` (start rows drawn with replacement from default_rng(seed)),
    q x q box partition."""
    rng = np.random.default_rng(seed)
    kappa = _channel_field(L, nchan, contrast, rng)
    rowptr, colidx, val = _fv_matrix(kappa)
    n = L * L
    part = box_partition(L, L, q, q)
    b = _rhs(n, rhs_seed, nrhs)
    return Problem(f"channels2d_{L}_q{q}_c{nchan}_ov{overlap}", n, rowptr, colidx, val,
                   part, q * q, overlap, tau, b,
                   meta=dict(kind="channels2d", nx=L, ny=L, qx=q, qy=q, contrast=contrast,
                             nchan=nchan))


def _grf(shape_full, corr_len, rng):
    """Periodic Gaussian random field with covariance exp(-r^2/(2 l^2))."""
    noise = rng.standard_normal(shape_full)
    grids = np.meshgrid(*[np.minimum(np.arange(s), s - np.arange(s)) for s in shape_full],
                        indexing="ij")
    r2 = sum(g.astype(np.float64) ** 2 for g in grids)
    cov = np.exp(-r2 / (2.0 * corr_len ** 2))
    spec = np.maximum(np.fft.fftn(cov).real, 0.0)
    field = np.fft.ifftn(np.fft.fftn(noise) * np.sqrt(spec)).real
    return field


def _nearest_centroid(X: np.ndarray, cent: np.ndarray, cand: int = 8) -> np.ndarray:
    """Index of the nearest centroid of every point, the lowest index among
    exactly equal squared distances (what a brute-force argmin returns).
    A k-d tree over the centroids proposes `cand` candidates per point; their
    squared distances are recomputed exactly (integer coordinates, centroids
    on a 2^-10 grid) and compared; a point whose candidates do not settle it
    (the last candidate as close as the first) is done by brute force."""
    from scipy.spatial import cKDTree
    k = cent.shape[0]
    cand = min(cand, k)
    _, nb = cKDTree(cent).query(X, k=cand, workers=-1)  # per-point queries, on every host core
    nb = nb.reshape(X.shape[0], cand)
    d2 = np.zeros(nb.shape)
    for ax in range(X.shape[1]):
        diff = X[:, ax:ax + 1] - cent[nb, ax]
        d2 += diff * diff
    best = d2.min(axis=1)
    # lowest centroid index among the candidates at the minimum
    out = np.where(d2 == best[:, None], nb, k).min(axis=1)
    if cand < k:
        hard = np.nonzero(d2[:, -1] <= best)[0]
        for h0 in range(0, hard.size, 4096):  # brute force, a block of points at a time
            hs = hard[h0:h0 + 4096]
            dd = ((X[hs][:, None, :] - cent[None, :, :]) ** 2).sum(axis=2)
            out[hs] = np.argmin(dd, axis=1)
    return out.astype(np.int64)


def _kmeans_partition(coords: np.ndarray, k: int, rng, sweeps: int = 100) -> np.ndarray:
    """Lloyd's k-means with Forgy initialisation; ties go to the lower index.

    Centroids are rounded to multiples of 2^-10 so that every squared
    distance to an integer coordinate is exact in float64: the assignment is
    identical on every machine.
    """
    npts = coords.shape[0]
    init = rng.choice(npts, size=k, replace=False)
    cent = coords[init].astype(np.float64)
    assign = np.full(npts, -1, dtype=np.int64)
    X = coords.astype(np.float64)
    for _ in range(sweeps):
        new = _nearest_centroid(X, cent)
        if np.array_equal(new, assign):
            break
        assign = new
        for ax in range(coords.shape[1]):
            sums = np.bincount(assign, weights=coords[:, ax].astype(np.float64), minlength=k)
            cnt = np.bincount(assign, minlength=k)
            keep = cnt > 0
            cent[keep, ax] = np.round(sums[keep] / cnt[keep] * 1024.0) / 1024.0
    # relabel to consecutive ids (an empty cluster would leave a gap)
    used, lab = np.unique(assign, return_inverse=True)
    return lab.astype(np.int32), len(used)


def grf3d(L: int = 96, k: int = 512, sigma: float = 3.0, corr_len: float = 8.0,
          seed: int = 3, overlap: int = 2, tau: float = 0.1, rhs_seed: int = 0,
          pad: Optional[int] = None, kmeans_sweeps: int = 100) -> Problem:
    """L^3 cells, kappa = exp(sigma * g) with g a Gaussian random field drawn
    on a periodic (L+pad)^3 grid, cropped and normalised to zero mean and unit
    sample variance; k-means partition of the cell centres."""
    pad = (L // 3) if pad is None else pad
    rng = np.random.default_rng(seed)
    full = L + pad
    g = _grf((full, full, full), corr_len, rng)[:L, :L, :L]
    g = (g - g.mean()) / g.std()
    kappa = np.exp(sigma * g)
    rowptr, colidx, val = _fv_matrix(kappa)
    n = L ** 3
    zz, yy, xx = np.meshgrid(np.arange(L), np.arange(L), np.arange(L), indexing="ij")
    coords = np.stack([xx.ravel(), yy.ravel(), zz.ravel()], axis=1)
    part, nparts = _kmeans_partition(coords, k, rng, sweeps=kmeans_sweeps)
    b = _rhs(n, rhs_seed, 1)
    return Problem(f"grf3d_{L}_k{k}_ov{overlap}", n, rowptr, colidx, val, part, nparts,
                   overlap, tau, b, meta=dict(kind="grf3d", L=L, sigma=sigma))


# ---------------------------------------------------------------------------
# Q1 plane-strain elasticity (Section 5)
# ---------------------------------------------------------------------------

def _q1_element_stiffness(hx: float, hy: float, E: float, nu: float) -> np.ndarray:
    """8x8 stiffness of a rectangular Q1 element, 2x2 Gauss quadrature.

    Dof order: node (0,0),(1,0),(1,1),(0,1) counter-clockwise, (u_x, u_y) per
    node.  Bilinear form 2 mu eps(u):eps(v) + L div(u) div(v) with
    mu = E/(2(1+nu)), L = E nu/((1+nu)(1-2nu)).
    """
    mu = E / (2.0 * (1.0 + nu))
    lam = E * nu / ((1.0 + nu) * (1.0 - 2.0 * nu))
    C = np.array([[lam + 2 * mu, lam, 0.0], [lam, lam + 2 * mu, 0.0], [0.0, 0.0, mu]])
    xi_n = np.array([-1.0, 1.0, 1.0, -1.0])
    eta_n = np.array([-1.0, -1.0, 1.0, 1.0])
    g = 1.0 / np.sqrt(3.0)
    K = np.zeros((8, 8))
    for xi in (-g, g):
        for eta in (-g, g):
            dN_dxi = 0.25 * xi_n * (1 + eta * eta_n)
            dN_deta = 0.25 * eta_n * (1 + xi * xi_n)
            dN_dx = dN_dxi * (2.0 / hx)
            dN_dy = dN_deta * (2.0 / hy)
            Bm = np.zeros((3, 8))
            Bm[0, 0::2] = dN_dx
            Bm[1, 1::2] = dN_dy
            Bm[2, 0::2] = dN_dy
            Bm[2, 1::2] = dN_dx
            K += Bm.T @ C @ Bm * (hx * hy / 4.0)
    return K


def elasticity2d(nex: int, ney: int, Lx: float, Ly: float, E_of_row, nu: float = 0.3,
                 owner_of_node=None, nparts: int = 1, overlap: int = 2, tau: float = 0.1,
                 rhs: str = "random", rhs_seed: int = 0, nrhs: int = 1, subsets_of_node=None,
                 name: str = "elasticity2d") -> Problem:
    """Q1 plane-strain elasticity on an nex x ney element mesh of [0,Lx]x[0,Ly],
    left edge clamped.  ``E_of_row(j)`` gives Young's modulus of element row j.

    Node (i, j) (i along x, j along y) with i >= 1 is free; its dofs are
    2*((j*(nex)) + (i-1)) + {0: u_x, 1: u_y}.
    """
    hx, hy = Lx / nex, Ly / ney
    nnx = nex + 1
    free_nx = nnx - 1
    n_nodes = free_nx * (ney + 1)
    n = 2 * n_nodes

    def node_id(i, j):
        return j * free_nx + (i - 1)

    rows, cols, vals = [], [], []
    f = np.zeros(n)
    Ecache = {}
    for j in range(ney):
        E = float(E_of_row(j))
        if E not in Ecache:
            Ecache[E] = _q1_element_stiffness(hx, hy, E, nu)
        Ke = Ecache[E]
        ii = np.arange(nex)
        corners = [(ii, j), (ii + 1, j), (ii + 1, j + 1), (ii, j + 1)]
        dofs = np.zeros((nex, 8), dtype=np.int64)
        freemask = np.ones((nex, 8), dtype=bool)
        for c, (ci, cj) in enumerate(corners):
            nid = node_id(ci, cj)
            free = ci >= 1
            dofs[:, 2 * c] = np.where(free, 2 * nid, -1)
            dofs[:, 2 * c + 1] = np.where(free, 2 * nid + 1, -1)
            freemask[:, 2 * c] = free
            freemask[:, 2 * c + 1] = free
        for a in range(8):
            for bb in range(8):
                ok = freemask[:, a] & freemask[:, bb]
                rows.append(dofs[ok, a])
                cols.append(dofs[ok, bb])
                vals.append(np.full(int(ok.sum()), Ke[a, bb]))
        if rhs == "gravity":
            # int g . phi over the element: each corner gets area/4 of g_y
            for c in range(4):
                d = dofs[:, 2 * c + 1]
                okd = d >= 0
                np.add.at(f, d[okd], -9.81 * hx * hy / 4.0)
    rowptr, colidx, val = _to_csr(np.concatenate(rows), np.concatenate(cols),
                                  np.concatenate(vals), n)
    if rhs == "gravity":
        b = f
    else:
        b = _rhs(n, rhs_seed, nrhs)
    part = np.zeros(n, dtype=np.int32)
    if owner_of_node is not None:
        jj, iin = np.meshgrid(np.arange(ney + 1), np.arange(1, nnx), indexing="ij")
        own = owner_of_node(iin.ravel(), jj.ravel())
        part[0::2] = own
        part[1::2] = own
    subsets = None
    if subsets_of_node is not None:
        jj, iin = np.meshgrid(np.arange(ney + 1), np.arange(1, nnx), indexing="ij")
        node_sets = subsets_of_node(iin.ravel(), jj.ravel())
        subsets = []
        for s in node_sets:
            s = np.asarray(s, dtype=np.int64)
            subsets.append(np.sort(np.concatenate([2 * s, 2 * s + 1])).astype(np.int32))
    return Problem(name, n, rowptr, colidx, val, part, nparts, overlap, tau, b,
                   subsets=subsets, meta=dict(kind="elasticity2d", nex=nex, ney=ney))


def paper_elasticity(layers: int = 6, E1: float = 1e11, E2: float = 1e7, nu: float = 0.3,
                     tau: float = 0.1) -> Problem:
    """The test case of Section 5: [0,3]^2, h = 1/21 (n = 8064), nine closed
    unit-square subdomains that share only their interfaces, gravity load.

    Hard layers (E1) where the fractional part of y lies in [1/7,2/7] and
    [3/7,4/7] (six layers), also [5/7,6/7] for nine layers, only [1/7,2/7]
    for three layers; ``layers=0`` gives homogeneous E1.
    """
    nex = ney = 63
    bands = {0: [], 3: [(3, 6)], 6: [(3, 6), (9, 12)], 9: [(3, 6), (9, 12), (15, 18)]}[layers]

    def E_of_row(j):
        if layers == 0:
            return E1
        r = j % 21  # element row inside a unit of 21 rows; centre (r+0.5)/21
        for lo, hi in bands:
            if lo <= r < hi:
                return E1
        return E2

    def subsets_of_node(i, j):
        sets = []
        for sy in range(3):
            for sx in range(3):
                m = (i >= 21 * sx) & (i <= 21 * (sx + 1)) & (j >= 21 * sy) & (j <= 21 * (sy + 1))
                sets.append(np.nonzero(m)[0])
        return sets

    def owner_of_node(i, j):
        return (np.minimum(j // 21, 2) * 3 + np.minimum(i // 21, 2)).astype(np.int32)

    return elasticity2d(nex, ney, 3.0, 3.0, E_of_row, nu=nu, owner_of_node=owner_of_node,
                        nparts=9, overlap=0, tau=tau, rhs="gravity",
                        subsets_of_node=subsets_of_node,
                        name=f"paper_elasticity_{layers}layers")


def paper_long_domain(N: int, E1: float = 1e11, E2: float = 1e7, nu: float = 0.3,
                      tau: float = 0.1) -> Problem:
    """The weak-scaling case of Section 5 (Table 6): [0,N] x [0,1], h = 1/14,
    hard layers (E1) for y in [1/7,2/7] and [3/7,4/7], E2 elsewhere, left
    edge clamped, gravity load, N closed unit-square subdomains in a row
    that share only their interfaces."""
    nex, ney = 14 * N, 14
    bands = [(2, 4), (6, 8)]  # element rows whose centres lie in the two layers

    def E_of_row(j):
        return E1 if any(lo <= j < hi for lo, hi in bands) else E2

    def subsets_of_node(i, j):
        return [np.nonzero((i >= 14 * sx) & (i <= 14 * (sx + 1)))[0] for sx in range(N)]

    def owner_of_node(i, j):
        return np.minimum(i // 14, N - 1).astype(np.int32)

    return elasticity2d(nex, ney, float(N), 1.0, E_of_row, nu=nu, owner_of_node=owner_of_node,
                        nparts=N, overlap=0, tau=tau, rhs="gravity", subsets_of_node=subsets_of_node,
                        name=f"paper_long_domain_{N}")


# ---------------------------------------------------------------------------
# Random SPD matrices for property tests
# ---------------------------------------------------------------------------

def random_spd(n: int = 60, nparts: int = 4, density: float = 0.08, seed: int = 0,
               overlap: int = 1, tau: float = 0.1, shift: float = 1e-2) -> Problem:
    """Weighted random-graph Laplacian plus a small positive diagonal (SPD),
    random owner of each dof."""
    rng = np.random.default_rng(seed)
    m = max(n, int(density * n * n / 2))
    i = rng.integers(0, n, size=m)
    j = rng.integers(0, n, size=m)
    keep = i != j
    i, j = i[keep], j[keep]
    w = rng.uniform(0.1, 2.0, size=i.size)
    # make it connected along a path so that the matrix is irreducible
    pi = np.arange(n - 1)
    i = np.concatenate([i, pi])
    j = np.concatenate([j, pi + 1])
    w = np.concatenate([w, rng.uniform(0.1, 2.0, size=n - 1)])
    rows = np.concatenate([i, j, i, j])
    cols = np.concatenate([j, i, i, j])
    vals = np.concatenate([-w, -w, w, w])
    rows = np.concatenate([rows, np.arange(n)])
    cols = np.concatenate([cols, np.arange(n)])
    vals = np.concatenate([vals, shift * rng.uniform(0.5, 1.5, size=n)])
    rowptr, colidx, val = _to_csr(rows, cols, vals, n)
    part = rng.integers(0, nparts, size=n).astype(np.int32)
    # every part non-empty
    part[:nparts] = np.arange(nparts)
    b = _rhs(n, seed + 1, 1)
    return Problem(f"random_spd_{n}_{nparts}_{seed}", n, rowptr, colidx, val, part, nparts,
                   overlap, tau, b, meta=dict(kind="random_spd"))


# ---------------------------------------------------------------------------
# Batches
# ---------------------------------------------------------------------------

def batch_channels(nprob: int = 128, seed0: int = 5000, Lmin: int = 128, Lmax: int = 768,
                   overlap: int = 2, tau: float = 0.1):
    """Independent channel problems: side L ~ U{Lmin..Lmax}, q x q boxes with
    q = 8 + round(16 (L - 128)/640), round(20 L/512) channels of width 2 at
    contrast 10^U(4,6)."""
    probs = []
    for j in range(nprob):
        rng = np.random.default_rng(seed0 + j)
        L = int(rng.integers(Lmin, Lmax + 1))
        q = 8 + int(round(16 * (L - 128) / 640))
        nchan = int(round(20 * L / 512))
        contrast = float(10.0 ** rng.uniform(4, 6))
        kappa = _channel_field(L, nchan, contrast, rng)
        rowptr, colidx, val = _fv_matrix(kappa)
        n = L * L
        b = rng.standard_normal(n)
        probs.append(Problem(f"batch{j}_L{L}_q{q}", n, rowptr, colidx, val,
                             box_partition(L, L, q, q), q * q, overlap, tau, b,
                             meta=dict(kind="channels2d", nx=L, ny=L, qx=q, qy=q,
                                       contrast=contrast, nchan=nchan)))
    return probs


# ---------------------------------------------------------------------------
# Named workloads
# ---------------------------------------------------------------------------

def block_rhs(p: Problem, nrhs: int, seed: int = 1) -> np.ndarray:
    """Right-hand sides of the batched (multi-right-hand-side) solves:
    row 0 is the problem's own b, rows 1 .. nrhs-1 are N(0, 1) draws from
    default_rng(seed) (nrhs x n, row-major)."""
    b0 = p.b if p.b.ndim == 1 else p.b[0]
    rest = np.random.default_rng(seed).standard_normal((nrhs - 1, p.n))
    return np.concatenate([b0[None, :], rest])


def config1() -> Problem:
    """2D Poisson 64x64 (n = 4096), 4x4 boxes, overlap 1, tau = 0.1."""
    return poisson2d(64, qx=4, overlap=1, tau=0.1, seed=0)


def config2() -> Problem:
    """512x512 channels at 1e6 (n = 262144), 16x16 boxes, overlap 2, tau = 0.1."""
    return channels2d(512, q=16, nchan=20, contrast=1e6, seed=2, overlap=2, tau=0.1)


def small_channels(L: int = 128, q: int = 4, nchan: int = 5, seed: int = 2, overlap: int = 2,
                   tau: float = 0.1, contrast: float = 1e6) -> Problem:
    """A smaller instance of the config-2 generator (same subdomain size 32x32
    when L/q = 32); channel count scaled with L."""
    return channels2d(L, q=q, nchan=nchan, contrast=contrast, seed=seed, overlap=overlap,
                      tau=tau)


def config3(L: int = 96, k: int = 512) -> Problem:
    """3D GRF diffusion 96^3 (n = 884736), k-means into 512 parts, overlap 2."""
    return grf3d(L, k=k)


def config4(nex: int = 384, nrhs: int = 32, seed: int = 7, q: int = 16) -> Problem:
    """Q1 elasticity 384x384 on the unit square, left edge clamped, layered E
    (thicknesses U{4..24} elements, alternating 1 and 1e5 starting with 1),
    16x16 node boxes, overlap 2, 32 random right-hand sides.  Smaller meshes
    with q = nex / 24 keep the subdomains' size (the coefficient draws of the
    learned start's training and evaluation)."""
    rng = np.random.default_rng(seed)
    rowE = np.empty(nex)
    j, k = 0, 0
    while j < nex:
        t = int(rng.integers(4, 25))
        rowE[j:j + t] = 1.0 if k % 2 == 0 else 1e5
        j += t
        k += 1
    def owner_of_node(i, jn):
        bx = np.minimum((i * q) // (nex + 1), q - 1)
        by = np.minimum((jn * q) // (nex + 1), q - 1)
        return (by * q + bx).astype(np.int32)

    return elasticity2d(nex, nex, 1.0, 1.0, lambda r: rowE[r], nu=0.3,
                        owner_of_node=owner_of_node, nparts=q * q, overlap=2, tau=0.1,
                        rhs="random", rhs_seed=0, nrhs=nrhs, name=f"elasticity2d_{nex}")


def config5(nprob: int = 128):
    """128 independent channel problems (see ``batch_channels``)."""
    return batch_channels(nprob)
