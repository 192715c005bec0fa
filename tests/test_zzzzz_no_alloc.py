"""awg_apply_hnn_noalloc: H^NN x for callers that may not allocate device
memory while they apply the preconditioner (frameworks that own all device
memory through their own pool, loops that cannot afford cudaMalloc).  On two
calls in a row, whose shared static scratch keeps the previous call's
values, it must agree with the regular entry point (awg_apply_stage with
the H^NN stage) and, entry by entry, with the oracle's H^NN (Def. 8).

This file is collected last on purpose, and passes alone in a fresh process
as well as after the other GPU tests.
"""

import ctypes

import numpy as np
import pytest

import awg_inputs as gi
import oracle as O

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

FP64_RTOL = 1e-11   # tolerance of the FP64 apply in the other GPU tests
FP32_RTOL = 1e-4    # tolerance of the float32 storage path


@pytest.fixture(scope="module")
def solver():
    import __graft_entry__ as g
    g.build()
    from paper_2106_10913_gb300 import AWGSolver
    p = gi.config1()
    sol = AWGSolver(p.rowptr, p.colidx, p.val, p.part, p.nparts, p.overlap, p.tau,
                    precisions=0b011)
    st = O.setup_problem(p, dense=True)
    yield p, sol, st
    sol.close()


def _rel(a, b):
    return float(torch.linalg.norm(a - b) / torch.linalg.norm(b))


@pytest.mark.parametrize("precision,tol", [(0, FP64_RTOL), (1, FP32_RTOL)])
def test_noalloc_matches_regular_entry_point(solver, precision, tol):
    from paper_2106_10913_gb300 import awg_apply_stage, load_library
    p, sol, st = solver
    lib = load_library()
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    rng = np.random.default_rng(2024 + precision)
    for call in range(2):  # two calls in a row share the static scratch
        xh = rng.standard_normal(p.n)
        x = torch.from_numpy(xh).cuda()
        y_ref = awg_apply_stage(sol.h, "hnn", x, torch.empty_like(x), precision)
        y = torch.full_like(x, float("nan"))
        status = lib.awg_apply_hnn_noalloc(sol.h, precision, x.data_ptr(), y.data_ptr(), stream)
        assert status == 0, f"call {call}: status {status}"
        torch.cuda.synchronize()
        assert torch.isfinite(y).all()
        assert _rel(y, y_ref) <= tol, f"call {call}"
        # against the oracle's H^NN, entry by entry and in norm
        yo = O.H_NN_apply(st, xh)
        yh = y.cpu().numpy()
        assert np.max(np.abs(yh - yo)) <= tol * np.max(np.abs(yo)), f"call {call}"
        assert np.linalg.norm(yh - yo) <= tol * np.linalg.norm(yo), f"call {call}"


def test_noalloc_rejects_bad_arguments(solver):
    from paper_2106_10913_gb300 import load_library
    p, sol, _ = solver
    lib = load_library()
    x = torch.zeros(p.n, dtype=torch.float64, device="cuda")
    assert lib.awg_apply_hnn_noalloc(sol.h, 2, x.data_ptr(), x.data_ptr(), None) == 1
    assert lib.awg_apply_hnn_noalloc(None, 0, x.data_ptr(), x.data_ptr(), None) == 1
