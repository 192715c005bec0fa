"""GPU path on small instances of the other workload generators, against the
CPU oracle on the same seeded inputs (through the C ABI):

* Q1 plane-strain elasticity with layered Young's modulus (1 / 1e5), left
  edge clamped, 16 x 16 node boxes, 8 random right-hand sides (the
  generator of the 384 x 384, 32-right-hand-side workload, at 48 x 48);
* 3D diffusion with a log-normal random coefficient and a k-means partition
  of uneven subdomain sizes (the generator of the 96^3 workload, at 14^3
  with 12 parts);
* a batch of independent channel problems of different sizes (the batch
  generator, 3 problems of sides 40-64) solved at the same time on three
  streams through the graph-driven PCG.

Bit-exact: eigenvalue and GenEO mode counts.  Floating point: the H_3,ad
apply within 1e-11 relative (or kappa_loc * eps), PCG iterations within 5 %
of the oracle's and true relative residuals <= 1e-8 on every column.
"""

import numpy as np
import pytest

import awg_inputs as gi
import oracle as O

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

CASES = {
    "elasticity48": lambda: gi.config4(nex=48, nrhs=8),
    "grf3d14": lambda: gi.grf3d(L=14, k=12, corr_len=3.0),
}
_PAIRS = {}


def _pair(name):
    if name not in _PAIRS:
        from paper_2106_10913_gb300 import AWGSolver
        p = CASES[name]()
        sol = AWGSolver(p.rowptr, p.colidx, p.val, p.part, p.nparts, p.overlap, p.tau, precisions=0b1001)
        st = O.setup_problem(p, dense=p.n <= 6000)
        _PAIRS[name] = (p, sol, st)
    return _PAIRS[name]


@pytest.fixture(scope="module", params=list(CASES))
def pair(request):
    return _pair(request.param)


def _rel(a, b):
    """Relative error of a against b, in the 2-norm and entry by entry
    (largest |a_i - b_i| over the largest |b_i|): the larger of the two, so
    that one wrong entry cannot hide inside the norm of a long vector."""
    a, b = np.asarray(a), np.asarray(b)
    return max(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300),
               float(np.max(np.abs(a - b), initial=0.0)) / max(float(np.max(np.abs(b), initial=0.0)), 1e-300))


def _rhs(p):
    return p.b if p.b.ndim == 2 else p.b[None, :]


def test_counts_exact(pair):
    p, sol, st = pair
    mm = O.minus_counts(st)
    assert sol.array("n_minus").tolist() == mm[:, 0].tolist()
    assert sol.array("n_strict").tolist() == mm[:, 1].tolist()
    assert sol.array("modes").tolist() == O.mode_counts(st).tolist()
    assert sol.info["n0"] == st.n0 and sol.info["n_minus"] == st.n_minus


def test_apply_parity(pair):
    p, sol, st = pair
    x = np.random.default_rng(8).standard_normal(p.n)
    y = sol.apply(torch.from_numpy(x).cuda(), stage="h3ad").cpu().numpy()
    tol = max(1e-11, O.local_condition(st) * np.finfo(float).eps)
    assert _rel(y, O.H3_ad_apply(st, x)) <= tol


@pytest.mark.parametrize("form", ["fp64", "fp16"])
def test_block_pcg(pair, form):
    p, sol, st = pair
    from paper_2106_10913_gb300 import FP64, MIXED_FP16, awg_pcg_block
    prec = {"fp64": FP64, "fp16": MIXED_FP16}[form]
    B = np.ascontiguousarray(_rhs(p))
    b = torch.from_numpy(B).cuda()
    x = torch.zeros_like(b)
    status, its, rels = awg_pcg_block(sol.h, b, x, 1e-8, precision=prec, check=False)
    assert status == 0
    X = x.cpu().numpy()
    for c in range(B.shape[0]):
        assert rels[c] <= 1e-8
        assert np.linalg.norm(st.A @ X[c] - B[c]) <= 1e-8 * np.linalg.norm(B[c]) * (1 + 1e-12)
        if form == "fp64":
            ref = O.pcg(lambda v: st.A @ v, B[c], lambda r: O.H3_ad_apply(st, r), rtol=1e-8)
            assert abs(its[c] - ref.iters) <= max(1, round(0.05 * ref.iters)), (c, its[c], ref.iters)


def test_batch_problems_concurrent():
    """Three independent problems of the batch generator enqueued on three
    streams from one host thread (graph-driven single-RHS solves): each
    takes the oracle's iterations (float64) and reaches 1e-8."""
    from paper_2106_10913_gb300 import AWGSolver, FP64, awg_pcg_block_async
    probs = gi.batch_channels(3, Lmin=40, Lmax=64)
    sols = [AWGSolver(q.rowptr, q.colidx, q.val, q.part, q.nparts, q.overlap, q.tau) for q in probs]
    try:
        streams = [torch.cuda.Stream() for _ in probs]
        outs = []
        torch.cuda.synchronize()
        for q, s_, strm in zip(probs, sols, streams):
            b = torch.from_numpy(q.b[None, :].copy()).cuda()
            x = torch.zeros_like(b)
            its = torch.zeros(1, dtype=torch.int32, device="cuda")
            rel = torch.zeros(1, dtype=torch.float64, device="cuda")
            st_ = torch.full((1,), -1, dtype=torch.int32, device="cuda")
            awg_pcg_block_async(s_.h, b, x, its, rel, st_, 1e-8, precision=FP64, stream=strm)
            outs.append((x, its, rel, st_))
        torch.cuda.synchronize()
        for q, (x, its, rel, st_) in zip(probs, outs):
            ost = O.setup_problem(q, dense=q.n <= 6000)
            ref = O.pcg(lambda v: ost.A @ v, q.b, lambda r: O.H3_ad_apply(ost, r), rtol=1e-8)
            assert int(st_.item()) == 0 and float(rel.item()) <= 1e-8
            assert abs(int(its.item()) - ref.iters) <= max(1, round(0.05 * ref.iters))
            X = x.cpu().numpy()[0]
            assert np.linalg.norm(ost.A @ X - q.b) <= 1e-8 * np.linalg.norm(q.b) * (1 + 1e-12)
    finally:
        for s_ in sols:
            s_.close()
