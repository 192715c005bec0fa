"""Multi-right-hand-side (block) path against the CPU oracle, column by column
(through the C ABI: awg_apply_block, awg_pcg_block).

* every stage of the block apply (A, A_+, H^NN, H_2 and the three H_3
  variants: H_3,ad, H_3,hyb of Def. 10, H_3,inex of Thm. 7) for 3, 20 and
  40 columns (the 16-, 32- and 64-wide kernels; padding columns included)
  matches the oracle's single-vector operator on each column to the FP64
  apply tolerance (1e-11, or kappa_loc * eps on ill-conditioned local
  problems);
* the mixed block forms (float32 internal vectors; W in float32 on the CUDA
  cores, float16 / bfloat16 on the tensor cores) meet the reduced-precision
  tolerances of the single-RHS forms, and the tensor-core W passes agree
  with the CUDA-core ones;
* block PCG: per column, true relative residual <= 1e-8 and iteration count
  within 5 % of the oracle's PCG on the same column, for every variant.
"""

import numpy as np
import pytest

import awg_inputs as gi
import oracle as O

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

APPLY_RTOL = 1e-11
MIXED_RTOL = 1e-4
BF16_RTOL = 64 * 2.0 ** -8

CASES = {
    "channels24": lambda: gi.channels2d(24, q=3, nchan=3, contrast=1e3, seed=5, overlap=2, tau=0.1),
    "random_spd60": lambda: gi.random_spd(60, nparts=4, density=0.06, seed=3, overlap=1, tau=0.1),
    "config1": lambda: gi.config1(),
    "channels64": lambda: gi.channels2d(64, q=2, nchan=3, contrast=1e6, seed=11, overlap=2, tau=0.1),
}
_PAIRS = {}


def _pair(name):
    if name not in _PAIRS:
        from paper_2106_10913_gb300 import AWGSolver
        p = CASES[name]()
        sol = AWGSolver(p.rowptr, p.colidx, p.val, p.part, p.nparts, p.overlap, p.tau, precisions=0b1111)
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


def _ref_op(st, stage):
    return {
        "spmv": lambda v: st.A @ v,
        "aplus": lambda v: O.A_plus_apply(st, v),
        "hnn": lambda v: O.H_NN_apply(st, v),
        "h2": lambda v: O.H2_apply(st, v),
        "h3ad": lambda v: O.H3_ad_apply(st, v),
        "h3hyb": lambda v: O.H3_hyb_apply(st, v),
        "h3inex": lambda v: O.H3_inex_apply(st, v),
    }[stage]


def _block_apply(sol, stage, X, prec):
    from paper_2106_10913_gb300 import awg_apply_block
    x = torch.from_numpy(np.ascontiguousarray(X)).cuda()
    y = torch.full_like(x, float("nan"))
    awg_apply_block(sol.h, stage, x, y, precision=prec)
    torch.cuda.synchronize()
    return y.cpu().numpy()


@pytest.mark.parametrize("nrhs", [3, 20, 40])
@pytest.mark.parametrize("stage", ["spmv", "aplus", "hnn", "h2", "h3ad", "h3hyb", "h3inex"])
def test_block_stage_parity_fp64(pair, stage, nrhs):
    p, sol, st = pair
    from paper_2106_10913_gb300 import FP64
    X = np.random.default_rng(100 + nrhs).standard_normal((nrhs, p.n))
    Y = _block_apply(sol, stage, X, FP64)
    op = _ref_op(st, stage)
    tol = max(APPLY_RTOL, O.local_condition(st) * np.finfo(float).eps)
    errs = [_rel(Y[c], op(X[c])) for c in range(nrhs)]
    assert max(errs) <= tol, f"worst column error {max(errs):.3e}"


# float16 W in H_3,hyb / H_3,inex: every W pass and the coarse matrices built
# from the stored W carry its rounding (u16 = 2^-11); with every entry of W
# rounded uniformly at random in the oracle, the applies of these workloads
# move by at most 6.3 u16 (H_3,inex on random_spd60; H_3,ad at most 2.8 u16)
VARIANT_FP16_RTOL = 8 * 2.0 ** -11


@pytest.mark.parametrize("form", ["fp32", "fp16"])
@pytest.mark.parametrize("stage", ["h3hyb", "h3inex"])
def test_block_mixed_apply_variants(pair, stage, form):
    """H_3,hyb and H_3,inex in the mixed block forms (float32 vectors, W in
    float32 / float16 on the tensor cores)."""
    p, sol, st = pair
    from paper_2106_10913_gb300 import MIXED_FP16, MIXED_FP32
    prec = {"fp32": MIXED_FP32, "fp16": MIXED_FP16}[form]
    X = np.random.default_rng(17).standard_normal((40, p.n))
    Y = _block_apply(sol, stage, X, prec)
    op = _ref_op(st, stage)
    errs = [_rel(Y[c], op(X[c])) for c in range(X.shape[0])]
    assert max(errs) <= (MIXED_RTOL if form == "fp32" else VARIANT_FP16_RTOL), f"worst column error {max(errs):.3e}"


_VARIANT_SOLVERS = {}


def _variant_solver(name, variant):
    key = (name, variant)
    if key not in _VARIANT_SOLVERS:
        from paper_2106_10913_gb300 import AWGSolver
        p, _, st = _pair(name)
        _VARIANT_SOLVERS[key] = AWGSolver(p.rowptr, p.colidx, p.val, p.part, p.nparts, p.overlap, p.tau,
                                          precisions=0b1011, variant=variant)
    return _VARIANT_SOLVERS[key]


@pytest.mark.parametrize("variant", ["hyb", "inex"])
@pytest.mark.parametrize("name", ["channels64", "config1"])
def test_block_pcg_variants(name, variant):
    """awg_pcg_block (and the graph-driven awg_pcg_block_async) with the
    handle's variant H_3,hyb / H_3,inex: per column the oracle's PCG
    iterations with the same preconditioner (within 5 %, float64) and true
    relative residuals <= 1e-8 (float64, and float16 W for H_3,hyb /
    float32 W for H_3,inex, whose Woodbury inner matrix C^-1 - Vhat^T W is
    ill-conditioned where A is, and so amplifies the storage error of W)."""
    from paper_2106_10913_gb300 import FP64, MIXED_FP16, MIXED_FP32, awg_pcg_block
    p, _, st = _pair(name)
    sol = _variant_solver(name, {"hyb": 1, "inex": 2}[variant])
    M = {"hyb": lambda r: O.H3_hyb_apply(st, r), "inex": lambda r: O.H3_inex_apply(st, r)}[variant]
    B = np.random.default_rng(23).standard_normal((6, p.n))
    b = torch.from_numpy(B).cuda()
    for prec in (FP64, MIXED_FP16 if variant == "hyb" else MIXED_FP32):
        x = torch.zeros_like(b)
        status, its, rels = awg_pcg_block(sol.h, b, x, 1e-8, precision=prec, check=False)
        assert status == 0
        X = x.cpu().numpy()
        for c in range(B.shape[0]):
            assert rels[c] <= 1e-8
            assert np.linalg.norm(st.A @ X[c] - B[c]) <= 1e-8 * np.linalg.norm(B[c]) * (1 + 1e-12)
            if prec == FP64 and c < 3:
                ref = O.pcg(lambda v: st.A @ v, B[c], M, rtol=1e-8)
                assert abs(its[c] - ref.iters) <= max(1, round(0.05 * ref.iters)), (c, its[c], ref.iters)
        xa, itsa, rela, sta = _async_solve(sol, B, prec)
        torch.cuda.synchronize()
        assert int(sta.item()) == 0
        XA = xa.cpu().numpy()
        for c in range(B.shape[0]):
            assert abs(int(itsa[c].item()) - its[c]) <= 1
            assert float(rela[c].item()) <= 1e-8
            assert np.linalg.norm(st.A @ XA[c] - B[c]) <= 1e-8 * np.linalg.norm(B[c]) * (1 + 1e-12)


@pytest.mark.parametrize("form", ["fp32", "fp16", "bf16"])
def test_block_mixed_apply(pair, form):
    p, sol, st = pair
    from paper_2106_10913_gb300 import MIXED_BF16, MIXED_FP16, MIXED_FP32
    prec = {"fp32": MIXED_FP32, "fp16": MIXED_FP16, "bf16": MIXED_BF16}[form]
    X = np.random.default_rng(7).standard_normal((20, p.n))
    Y = _block_apply(sol, "h3ad", X, prec)
    errs = [_rel(Y[c], O.H3_ad_apply(st, X[c])) for c in range(X.shape[0])]
    assert max(errs) <= (BF16_RTOL if form == "bf16" else MIXED_RTOL)


@pytest.mark.parametrize("nrhs", [1, 32, 64])
@pytest.mark.parametrize("form", ["fp16", "bf16"])
def test_block_tensor_cores_match_cuda_cores(form, nrhs):
    """The tcgen05 W passes against the CUDA-core W passes on the same
    16-bit W (second handle with block_tensor_cores = 0): they differ only by
    the 16-bit split of the right-hand sides (about 2^-22 of each column's
    largest entry for float16, 2^-16 for bfloat16) and the order of the
    float32 sums."""
    from paper_2106_10913_gb300 import AWGSolver, MIXED_BF16, MIXED_FP16
    p, sol, st = _pair("channels64")
    ref = AWGSolver(p.rowptr, p.colidx, p.val, p.part, p.nparts, p.overlap, p.tau, precisions=0b1111,
                    block_tensor_cores=0)
    try:
        prec = {"fp16": MIXED_FP16, "bf16": MIXED_BF16}[form]
        X = np.random.default_rng(11 + nrhs).standard_normal((nrhs, p.n))
        Ya = _block_apply(sol, "h3ad", X, prec)
        Yb = _block_apply(ref, "h3ad", X, prec)
        tol = 1e-5 if form == "fp16" else 1e-3
        errs = [_rel(Ya[c], Yb[c]) for c in range(nrhs)]
        assert np.all(np.isfinite(Ya)) and max(errs) <= tol, f"worst column {max(errs):.3e}"
        # two different code paths (split right-hand sides, other sum order)
        assert not np.array_equal(Ya, Yb)
    finally:
        ref.close()


def _check_pcg(p, st, B, X, its, rels, status):
    assert status == 0
    for c in range(B.shape[0]):
        ref = O.pcg(lambda v: st.A @ v, B[c], lambda r: O.H3_ad_apply(st, r), rtol=1e-8)
        assert rels[c] <= 1e-8
        assert abs(its[c] - ref.iters) <= max(1, round(0.05 * ref.iters)), (c, its[c], ref.iters)
        assert np.linalg.norm(st.A @ X[c] - B[c]) <= 1e-8 * np.linalg.norm(B[c]) * (1 + 1e-12)


@pytest.mark.parametrize("form", ["fp64", "fp32", "fp16", "bf16"])
def test_block_pcg_parity(pair, form):
    p, sol, st = pair
    from paper_2106_10913_gb300 import FP64, MIXED_BF16, MIXED_FP16, MIXED_FP32, awg_pcg_block
    prec = {"fp64": FP64, "fp32": MIXED_FP32, "fp16": MIXED_FP16, "bf16": MIXED_BF16}[form]
    B = np.random.default_rng(21).standard_normal((6, p.n))
    b = torch.from_numpy(B).cuda()
    x = torch.zeros_like(b)
    status, its, rels = awg_pcg_block(sol.h, b, x, 1e-8, precision=prec, check=False)
    X = x.cpu().numpy()
    if form in ("fp64", "fp32"):
        _check_pcg(p, st, B, X, its, rels, status)
    else:
        # the 16-bit W forms change the preconditioner (more iterations for
        # bfloat16): the residual must still reach 1e-8 on every column
        assert status == 0 and max(rels) <= 1e-8
        for c in range(B.shape[0]):
            assert np.linalg.norm(st.A @ X[c] - B[c]) <= 1e-8 * np.linalg.norm(B[c]) * (1 + 1e-12)


def test_block_pcg_many_columns():
    """70 columns: one group of 64 and one of 6, zero columns included."""
    from paper_2106_10913_gb300 import FP64, awg_pcg_block
    p, sol, st = _pair("random_spd60")
    B = np.random.default_rng(3).standard_normal((70, p.n))
    B[5] = 0.0
    b = torch.from_numpy(B).cuda()
    x = torch.full_like(b, 7.0)
    status, its, rels = awg_pcg_block(sol.h, b, x, 1e-8, precision=FP64, check=False)
    X = x.cpu().numpy()
    assert status == 0
    assert its[5] == 0 and rels[5] == 0.0 and np.all(X[5] == 0.0)
    keep = [c for c in range(70) if c != 5]
    _check_pcg(p, st, B[keep], X[keep], [its[c] for c in keep], [rels[c] for c in keep], 0)


def test_block_pcg_matches_single_rhs(pair):
    """Column c of a block solve follows the single-RHS solve of column c."""
    p, sol, st = pair
    from paper_2106_10913_gb300 import FP64, awg_pcg, awg_pcg_block
    B = np.random.default_rng(5).standard_normal((4, p.n))
    b = torch.from_numpy(B).cuda()
    xb = torch.zeros_like(b)
    _, its_b, _ = awg_pcg_block(sol.h, b, xb, 1e-8, precision=FP64)
    for c in range(4):
        x1 = torch.zeros_like(b[c])
        _, its1, _ = awg_pcg(sol.h, b[c].contiguous(), x1, 1e-8, precision=FP64)
        assert abs(its1[0] - its_b[c]) <= 1
        assert _rel(xb[c].cpu().numpy(), x1.cpu().numpy()) <= 1e-6


def test_block_apply_rejects_bad_sizes():
    from paper_2106_10913_gb300 import FP64, awg_apply_block
    from paper_2106_10913_gb300.awg import AWGError
    p, sol, st = _pair("random_spd60")
    x = torch.zeros((65, p.n), dtype=torch.float64, device="cuda")
    with pytest.raises(AWGError):
        awg_apply_block(sol.h, "h3ad", x, x.clone(), precision=FP64)
    with pytest.raises(AWGError):
        awg_apply_block(sol.h, 7, x[:2], x[:2].clone(), precision=FP64)


def _async_solve(sol, B, prec, stream=None):
    from paper_2106_10913_gb300 import awg_pcg_block_async
    b = torch.from_numpy(np.ascontiguousarray(B)).cuda()
    x = torch.full_like(b, 3.0)
    its = torch.zeros(B.shape[0], dtype=torch.int32, device="cuda")
    rel = torch.zeros(B.shape[0], dtype=torch.float64, device="cuda")
    st = torch.full((1,), -1, dtype=torch.int32, device="cuda")
    torch.cuda.synchronize()
    awg_pcg_block_async(sol.h, b, x, its, rel, st, 1e-8, precision=prec, stream=stream)
    return x, its, rel, st


@pytest.mark.parametrize("form", ["fp64", "fp16"])
def test_block_pcg_async_matches_sync(pair, form):
    """The graph-driven solve (device-side loop and stopping test) takes the
    iterations of the host-driven block solve and reaches 1e-8 on every
    column; a second call reuses the captured loop graph."""
    p, sol, st = pair
    from paper_2106_10913_gb300 import FP64, MIXED_FP16, awg_pcg_block
    prec = {"fp64": FP64, "fp16": MIXED_FP16}[form]
    for seed in (31, 32):
        B = np.random.default_rng(seed).standard_normal((5, p.n))
        x, its, rel, status = _async_solve(sol, B, prec)
        torch.cuda.synchronize()
        xs = torch.zeros((5, p.n), dtype=torch.float64, device="cuda")
        _, its_s, _ = awg_pcg_block(sol.h, torch.from_numpy(B).cuda(), xs, 1e-8, precision=prec)
        X = x.cpu().numpy()
        assert int(status.item()) == 0
        for c in range(5):
            assert abs(int(its[c].item()) - its_s[c]) <= 1
            assert float(rel[c].item()) <= 1e-8
            assert np.linalg.norm(st.A @ X[c] - B[c]) <= 1e-8 * np.linalg.norm(B[c]) * (1 + 1e-12)


def test_block_pcg_async_concurrent_problems():
    """Two handles (independent problems) enqueued on two streams from one
    host thread (their solves overlap on the device) reach 1e-8 each."""
    from paper_2106_10913_gb300 import MIXED_FP16
    pa, sa, sta = _pair("channels64")
    pb, sb, stb = _pair("config1")
    Ba = np.random.default_rng(41).standard_normal((3, pa.n))
    Bb = np.random.default_rng(42).standard_normal((20, pb.n))
    s1, s2 = torch.cuda.Stream(), torch.cuda.Stream()
    xa, ia, ra, sa_ = _async_solve(sa, Ba, MIXED_FP16, stream=s1)
    xb, ib, rb, sb_ = _async_solve(sb, Bb, MIXED_FP16, stream=s2)
    torch.cuda.synchronize()
    assert int(sa_.item()) == 0 and int(sb_.item()) == 0
    for (p, st, B, x) in ((pa, sta, Ba, xa), (pb, stb, Bb, xb)):
        X = x.cpu().numpy()
        for c in range(B.shape[0]):
            assert np.linalg.norm(st.A @ X[c] - B[c]) <= 1e-8 * np.linalg.norm(B[c]) * (1 + 1e-12)


@pytest.mark.parametrize("form", ["fp64", "fp16"])
def test_pcg_async_single_rhs(pair, form):
    """One right-hand side through the graph-driven loop (single-RHS apply in
    the body): the iterations of awg_pcg and a 1e-8 residual."""
    p, sol, st = pair
    from paper_2106_10913_gb300 import FP64, MIXED_FP16, awg_pcg
    prec = {"fp64": FP64, "fp16": MIXED_FP16}[form]
    B = np.random.default_rng(51).standard_normal((1, p.n))
    x, its, rel, status = _async_solve(sol, B, prec)
    torch.cuda.synchronize()
    x1 = torch.zeros(p.n, dtype=torch.float64, device="cuda")
    _, its1, _ = awg_pcg(sol.h, torch.from_numpy(B[0]).cuda(), x1, 1e-8, precision=prec)
    assert int(status.item()) == 0
    assert abs(int(its[0].item()) - its1[0]) <= 1
    assert float(rel[0].item()) <= 1e-8
    X = x.cpu().numpy()
    assert np.linalg.norm(st.A @ X[0] - B[0]) <= 1e-8 * np.linalg.norm(B[0]) * (1 + 1e-12)


def test_block_pcg_async_two_groups(pair):
    """More than 64 columns: two column groups solve side by side on the
    handle's two slots (own workspace, streams and loop graphs); every
    column takes the host-driven solve's iterations and reaches 1e-8."""
    p, sol, st = pair
    from paper_2106_10913_gb300 import MIXED_FP16, awg_pcg_block
    B = np.random.default_rng(61).standard_normal((77, p.n))
    B[70] = 0.0
    x, its, rel, status = _async_solve(sol, B, MIXED_FP16)
    torch.cuda.synchronize()
    xs = torch.zeros((77, p.n), dtype=torch.float64, device="cuda")
    _, its_s, _ = awg_pcg_block(sol.h, torch.from_numpy(B).cuda(), xs, 1e-8, precision=MIXED_FP16)
    assert int(status.item()) == 0
    X = x.cpu().numpy()
    assert int(its[70].item()) == 0 and np.all(X[70] == 0.0)
    for c in range(77):
        if c == 70:
            continue
        assert abs(int(its[c].item()) - its_s[c]) <= 1
        assert float(rel[c].item()) <= 1e-8
        assert np.linalg.norm(st.A @ X[c] - B[c]) <= 1e-8 * np.linalg.norm(B[c]) * (1 + 1e-12)


@pytest.mark.parametrize("nrhs", [1, 40])
def test_profile_modes(nrhs):
    """awg_profile: with PROF_COUNT alone the solve's launches are counted and
    no kernel class is timed; with every class and PROF_SERIAL each class of
    the H_3,ad solve is timed, and the solve (its side branch run in order on
    the main stream) gives the same x, bit for bit, as the unprofiled one."""
    from paper_2106_10913_gb300 import (MIXED_FP16, PROF_COUNT, PROF_SERIAL, awg_pcg, awg_pcg_block,
                                        awg_profile, awg_profile_read)
    p, sol, st = _pair("channels64")
    B = gi.block_rhs(p, nrhs)
    b = torch.from_numpy(np.ascontiguousarray(B if nrhs > 1 else B[0])).cuda()

    def solve():
        x = torch.zeros_like(b)
        if nrhs > 1:
            awg_pcg_block(sol.h, b, x, 1e-8, MIXED_FP16)
        else:
            awg_pcg(sol.h, b, x, 1e-8, MIXED_FP16)
        torch.cuda.synchronize()
        return x

    x0 = solve()
    awg_profile(sol.h, PROF_COUNT)
    x1 = solve()
    pc = awg_profile_read(sol.h)
    awg_profile(sol.h, 0xFF | PROF_SERIAL)
    x2 = solve()
    ps = awg_profile_read(sol.h)
    awg_profile(sol.h, 0)
    assert pc["launches"] > 0 and all(v == 0 for v in pc["count"].values())
    assert ps["launches"] == pc["launches"]
    for k in ("spmv", "local", "wt", "wd", "coarse", "subdomain", "prolong", "vector"):
        assert ps["count"][k] > 0 and ps["ms"][k] > 0.0, k
    assert torch.equal(x0, x1) and torch.equal(x0, x2)
