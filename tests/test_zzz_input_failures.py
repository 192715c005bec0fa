"""Failures made by the input, on the GPU path: each returns its status code
(no trap, no hang) and leaves the library usable.

* setup: a row without its diagonal (AWG_ERR_NOT_SPD), a structurally
  asymmetric pattern (AWG_ERR_NOT_SYMMETRIC), column indices out of order
  and a partition value out of range or an empty part (AWG_ERR_INVALID_ARG),
  subdomains that break minimal overlap, overlap 0 (AWG_ERR_MIN_OVERLAP);
* PCG: a right-hand side with a NaN (AWG_ERR_BREAKDOWN: p.Ap is not a
  positive number), an iteration cap of one (AWG_ERR_MAXIT), a zero
  right-hand side (AWG_OK after no iteration, x = 0); the same handle then
  solves a proper right-hand side to 1e-8.
"""

import numpy as np
import pytest

import awg_inputs as gi

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

OK, INVALID_ARG, MIN_OVERLAP, NOT_SPD, BREAKDOWN, MAXIT, NOT_SYMMETRIC = 0, 1, 2, 3, 5, 6, 9


def _problem():
    return gi.poisson2d(12, qx=2, overlap=1, tau=0.1, seed=0)


def _status(rowptr, colidx, val, part, nparts, overlap, **opts):
    from paper_2106_10913_gb300 import AWGSolver
    from paper_2106_10913_gb300.awg import AWGError
    try:
        AWGSolver(rowptr, colidx, val, part, nparts, overlap, 0.1, **opts).close()
        return OK
    except AWGError as e:
        return e.status


def _drop(p, i, j):
    """CSR of p without the stored entry (i, j)."""
    rp, ci, va = p.rowptr.astype(np.int64), p.colidx.copy(), p.val.copy()
    k = rp[i] + int(np.nonzero(ci[rp[i]:rp[i + 1]] == j)[0][0])
    ci, va = np.delete(ci, k), np.delete(va, k)
    rp = rp.copy()
    rp[i + 1:] -= 1
    return rp.astype(np.int32), ci.astype(np.int32), va


def test_setup_rejects_bad_inputs():
    p = _problem()
    assert _status(p.rowptr, p.colidx, p.val, p.part, p.nparts, p.overlap) == OK
    rp, ci, va = _drop(p, 5, 5)
    assert _status(rp, ci, va, p.part, p.nparts, p.overlap) == NOT_SPD
    j = int(p.colidx[p.rowptr[5]:p.rowptr[6]][0])  # an off-diagonal neighbour of row 5
    assert j != 5
    rp, ci, va = _drop(p, 5, j)
    assert _status(rp, ci, va, p.part, p.nparts, p.overlap) == NOT_SYMMETRIC
    ci = p.colidx.copy()
    a = p.rowptr[7]
    ci[a], ci[a + 1] = ci[a + 1], ci[a]
    assert _status(p.rowptr, ci, p.val, p.part, p.nparts, p.overlap) == INVALID_ARG
    part = p.part.copy()
    part[0] = p.nparts
    assert _status(p.rowptr, p.colidx, p.val, part, p.nparts, p.overlap) == INVALID_ARG
    assert _status(p.rowptr, p.colidx, p.val, p.part, p.nparts + 1, p.overlap) == INVALID_ARG
    assert _status(p.rowptr, p.colidx, p.val, p.part, p.nparts, 0) == MIN_OVERLAP


def test_pcg_failures_leave_the_handle_usable():
    from paper_2106_10913_gb300 import AWGSolver
    p = _problem()
    sol = AWGSolver(p.rowptr, p.colidx, p.val, p.part, p.nparts, p.overlap, p.tau, maxit=1)
    try:
        b = torch.from_numpy(p.b).cuda()
        bad = b.clone()
        bad[3] = float("nan")
        _, its, _, st = sol.pcg(bad, rtol=1e-8, check=False)
        assert st == BREAKDOWN and its[0] == 1
        _, its, _, st = sol.pcg(b, rtol=1e-8, check=False)
        assert st == MAXIT and its[0] == 1
        x, its, rel, st = sol.pcg(torch.zeros_like(b), rtol=1e-8, check=False)
        assert st == OK and its[0] == 0 and rel[0] == 0.0 and not torch.any(x)
    finally:
        sol.close()
    sol = AWGSolver(p.rowptr, p.colidx, p.val, p.part, p.nparts, p.overlap, p.tau)
    try:
        bad = torch.from_numpy(p.b).cuda()
        bad[3] = float("nan")
        _, _, _, st = sol.pcg(bad, rtol=1e-8, check=False)
        assert st == BREAKDOWN
        x, its, rel, st = sol.pcg(torch.from_numpy(p.b).cuda(), rtol=1e-8, check=False)
        assert st == OK and rel[0] <= 1e-8 and its[0] > 1
    finally:
        sol.close()
