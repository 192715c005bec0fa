"""Float64-accurate products with the dense coarse inverses on the tensor
cores (the two coarse solves of H_3: E^-1 of Thm. 4 and F^-1 of Def. 10, and
the H_3,inex inner inverse of Thm. 7), through the C ABI
(awg_coarse_apply_block).

Both operands are cut into eight 7-bit integer slices whose bfloat16
products are exact in float32; the recombined result must agree with the
float64 GEMM of the same matrix ENTRY BY ENTRY to 1e-14 of the largest
entry of its column (a float64 GEMM itself is accurate to about
dim * 2^-53 of |M| |X|), for 16-, 32- and 64-wide kernels with zero padding
columns, a zero column, columns of very different scales, and with the
reduction split every 256 terms (the path that coarse spaces above 4032
take).  The products also match an independent float64 solve with the
coarse matrix itself (E or F from the handle, NumPy) to cond(M) eps.
Finally the block apply of H_3,ad with the tensor-core products (default)
and with the float64 CUDA-core products (second handle) both match the
oracle to the FP64 apply tolerance.
"""

import numpy as np
import pytest

import awg_inputs as gi
import oracle as O

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

CASES = {
    "channels64": lambda: gi.channels2d(64, q=2, nchan=3, contrast=1e6, seed=11, overlap=2, tau=0.1),
    "channels192": lambda: gi.channels2d(192, q=6, nchan=8, contrast=1e6, seed=7, overlap=2, tau=0.1),
    "config1": lambda: gi.config1(),
}
_SOL = {}


def _solver(name):
    if name not in _SOL:
        from paper_2106_10913_gb300 import AWGSolver
        p = CASES[name]()
        _SOL[name] = (p, AWGSolver(p.rowptr, p.colidx, p.val, p.part, p.nparts, p.overlap, p.tau,
                                   precisions=0b1011))
    return _SOL[name]


def _rhs(dim, nrhs, seed):
    rng = np.random.default_rng(seed)
    X = rng.standard_normal((nrhs, dim))
    X *= np.logspace(0, -9, nrhs)[:, None]          # columns of very different scales
    X[:, ::5] *= 1e-6                               # small entries inside a column
    if nrhs > 2:
        X[1] = 0.0                                  # a zero column
    return X


def _coarse(sol, which, X, prec, engine):
    from paper_2106_10913_gb300 import awg_coarse_apply_block
    x = torch.from_numpy(np.ascontiguousarray(X)).cuda()
    y = torch.full_like(x, float("nan"))
    awg_coarse_apply_block(sol.h, which, x, y, precision=prec, engine=engine)
    return y.cpu().numpy()


@pytest.mark.parametrize("engine", [1, 2])
@pytest.mark.parametrize("nrhs", [3, 20, 40, 64])
@pytest.mark.parametrize("which,form", [("Einv", "fp64"), ("Finv", "fp64"), ("Finv", "fp16"), ("Finv", "fp32")])
@pytest.mark.parametrize("name", list(CASES))
def test_slice_products_match_float64_gemm(name, which, form, nrhs, engine):
    from paper_2106_10913_gb300 import FP64, MIXED_FP16, MIXED_FP32
    p, sol = _solver(name)
    prec = {"fp64": FP64, "fp16": MIXED_FP16, "fp32": MIXED_FP32}[form]
    dim = sol.info["n0"] if which == "Einv" else sol.info["n_minus"]
    if dim == 0:
        pytest.skip("empty coarse space")
    X = _rhs(dim, nrhs, 300 + nrhs)
    Y64 = _coarse(sol, which, X, prec, 0)
    Yt = _coarse(sol, which, X, prec, engine)
    assert np.all(np.isfinite(Yt))
    for c in range(nrhs):
        ref = Y64[c]
        scale = np.max(np.abs(ref))
        if scale == 0.0:
            assert np.all(Yt[c] == 0.0), c
            continue
        assert np.max(np.abs(Yt[c] - ref)) <= 1e-14 * scale, (c, float(np.max(np.abs(Yt[c] - ref)) / scale))
        assert np.linalg.norm(Yt[c] - ref) <= 1e-14 * np.linalg.norm(ref), c


@pytest.mark.parametrize("which", ["Einv", "Finv"])
@pytest.mark.parametrize("name", list(CASES))
def test_slice_products_solve_the_coarse_problem(name, which):
    """M X against a float64 solve with the coarse matrix itself (E = Z^T A_+ Z
    or F = W^T A W, read from the handle): agreement to cond(M) eps."""
    from paper_2106_10913_gb300 import FP64
    p, sol = _solver(name)
    dim = sol.info["n0"] if which == "Einv" else sol.info["n_minus"]
    if dim == 0:
        pytest.skip("empty coarse space")
    C = sol.array("E" if which == "Einv" else "F").reshape(dim, dim)
    X = _rhs(dim, 20, 77)
    Yt = _coarse(sol, which, X, FP64, 1)
    ref = np.linalg.solve(C, X.T).T
    cond = np.linalg.cond(C)
    for c in range(X.shape[0]):
        if not np.any(X[c]):
            continue
        assert np.linalg.norm(Yt[c] - ref[c]) <= 100 * cond * 2.3e-16 * np.linalg.norm(ref[c]), c


@pytest.mark.parametrize("coarse_tc", [1, 0])
def test_block_apply_with_either_coarse_engine(coarse_tc):
    """H_3,ad on 40 columns with the tensor-core coarse products (default) and
    with the float64 CUDA-core ones: both within the FP64 apply tolerance of
    the oracle, entry by entry."""
    from paper_2106_10913_gb300 import AWGSolver, FP64, awg_apply_block
    p = CASES["channels192"]()
    sol = AWGSolver(p.rowptr, p.colidx, p.val, p.part, p.nparts, p.overlap, p.tau,
                    coarse_tensor_cores=coarse_tc)
    try:
        st = O.setup_problem(p, dense=False)
        X = np.random.default_rng(5).standard_normal((40, p.n))
        x = torch.from_numpy(X).cuda()
        y = torch.full_like(x, float("nan"))
        awg_apply_block(sol.h, "h3ad", x, y, precision=FP64)
        Y = y.cpu().numpy()
        tol = max(1e-11, O.local_condition(st) * np.finfo(float).eps)
        for c in range(X.shape[0]):
            ref = O.H3_ad_apply(st, X[c])
            assert np.max(np.abs(Y[c] - ref)) <= tol * np.max(np.abs(ref)), c
            assert np.linalg.norm(Y[c] - ref) <= tol * np.linalg.norm(ref), c
    finally:
        sol.close()
