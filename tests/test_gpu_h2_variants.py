"""The other H_2 choices on the GPU against the CPU oracle on the same
seeded inputs, through the C ABI: H^AS_+,hyb(tau_flat) and
H^AS_+,ad(tau_flat) of Thm. 3 (local solvers (R^s A_+ R^sT)^-1, coarse space
of the GenEO pencil below 1 / tau_flat) and H^AS_hyb(tau_sharp, tau_flat) of
Thm. 5 (local solvers (R^s A R^sT)^-1, coarse space of two pencils; tau_sharp
= 0.5 so that the second pencil contributes on the channel and random
problems):

* bit-exact: eigenvalue counts and GenEO mode counts;
* every stage of the single-RHS apply (H^AS_+, H_2, the three H_3) and of
  the block apply within 1e-11 relative, or kappa * eps with kappa the
  largest condition number of the local matrices (R^s A_+ R^sT or R^s A R^sT)
  where the local solves are ill-conditioned; the float32 forms within 1e-4;
* PCG: true relative residual <= 1e-8 and iterations within 5 % of the
  oracle's PCG with the same preconditioner.
"""

import dataclasses

import numpy as np
import pytest

import awg_inputs as gi
import oracle as O

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

APPLY_RTOL = 1e-11
MIXED_RTOL = 1e-4
TAU_FLAT = 10.0
TAU_SHARP_AS = 0.5
H2S = ("asp_hyb", "asp_ad", "as_hyb")

CASES = {
    "channels24": lambda: gi.channels2d(24, q=3, nchan=3, contrast=1e3, seed=5, overlap=2, tau=0.1),
    "random_spd60": lambda: gi.random_spd(60, nparts=4, density=0.06, seed=3, overlap=1, tau=0.1),
    "config1": lambda: gi.config1(),
    "channels64": lambda: gi.channels2d(64, q=2, nchan=3, contrast=1e6, seed=11, overlap=2, tau=0.1),
}
_ORACLE = {}
_SOLVERS = {}


def _oracle(name, h2):
    """One oracle setup per problem and coarse space: the two AS_+ choices
    share V^0_AS,+(tau_flat) (Thm. 3) and W, so the additive one reuses the
    hybrid one's pieces."""
    fam = "as" if h2 == "as_hyb" else "asp"
    if (name, fam) not in _ORACLE:
        p = CASES[name]()
        kw = {"h2": "as_hyb", "tau": TAU_SHARP_AS} if fam == "as" else {"h2": "asp_hyb"}
        _ORACLE[(name, fam)] = (p, O.setup_problem(p, dense=p.n <= 6000, tau_flat=TAU_FLAT, **kw))
    p, st = _ORACLE[(name, fam)]
    return p, (st if st.h2 == h2 else dataclasses.replace(st, h2=h2, as_cho=st.as_cho))


def _pair(name, h2):
    key = (name, h2)
    if key not in _SOLVERS:
        from paper_2106_10913_gb300 import AWGSolver, H2_AS_HYB, H2_ASP_AD, H2_ASP_HYB
        p, st = _oracle(name, h2)
        tau = TAU_SHARP_AS if h2 == "as_hyb" else p.tau
        sol = AWGSolver(p.rowptr, p.colidx, p.val, p.part, p.nparts, p.overlap, tau, precisions=0b1011,
                        h2={"asp_hyb": H2_ASP_HYB, "asp_ad": H2_ASP_AD, "as_hyb": H2_AS_HYB}[h2],
                        tau_flat=TAU_FLAT)
        _SOLVERS[key] = (p, sol, st)
    return _SOLVERS[key]


@pytest.fixture(scope="module", params=[(c, h) for c in CASES for h in H2S],
                ids=[f"{c}-{h}" for c in CASES for h in H2S])
def pair(request):
    return _pair(*request.param)


def _rel(a, b):
    """Relative error of a against b, in the 2-norm and entry by entry
    (largest |a_i - b_i| over the largest |b_i|): the larger of the two, so
    that one wrong entry cannot hide inside the norm of a long vector."""
    a, b = np.asarray(a), np.asarray(b)
    return max(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300),
               float(np.max(np.abs(a - b), initial=0.0)) / max(float(np.max(np.abs(b), initial=0.0)), 1e-300))


def _ref_op(st, stage):
    return {
        "hnn": lambda v: O.H1_apply(st, v),
        "h2": lambda v: O.H2_apply(st, v),
        "h3ad": lambda v: O.H3_ad_apply(st, v),
        "h3hyb": lambda v: O.H3_hyb_apply(st, v),
        "h3inex": lambda v: O.H3_inex_apply(st, v),
    }[stage]


def _tol(st):
    return max(APPLY_RTOL, O.local_condition(st) * np.finfo(float).eps)


def test_second_pencil_contributes():
    """The H^AS_hyb cases exercise both pencils of Thm. 5."""
    for name in ("channels24", "random_spd60", "channels64"):
        _, st = _oracle(name, "as_hyb")
        assert sum(k2 for _, k2 in st.geneo_split) > 0, name


def test_counts_exact(pair):
    p, sol, st = pair
    mm = O.minus_counts(st)
    assert sol.array("n_minus").tolist() == mm[:, 0].tolist()
    assert sol.array("modes").tolist() == O.mode_counts(st).tolist()
    assert sol.info["n0"] == st.n0 and sol.info["n_minus"] == st.n_minus


@pytest.mark.parametrize("stage", ["hnn", "h2", "h3ad", "h3hyb", "h3inex"])
def test_stage_parity(pair, stage):
    p, sol, st = pair
    x = np.random.default_rng(321).standard_normal(p.n)
    y = sol.apply(torch.from_numpy(x).cuda(), stage=stage).cpu().numpy()
    assert _rel(y, _ref_op(st, stage)(x)) <= _tol(st)


@pytest.mark.parametrize("stage", ["h2", "h3ad", "h3hyb"])
def test_block_parity(pair, stage):
    """20 columns through the block apply, float64 and float32 forms."""
    p, sol, st = pair
    from paper_2106_10913_gb300 import FP64, MIXED_FP32, awg_apply_block
    X = np.random.default_rng(9).standard_normal((20, p.n))
    op = _ref_op(st, stage)
    ref = [op(X[c]) for c in range(20)]
    for prec, tol in ((FP64, _tol(st)), (MIXED_FP32, MIXED_RTOL)):
        x = torch.from_numpy(X).cuda()
        y = torch.full_like(x, float("nan"))
        awg_apply_block(sol.h, stage, x, y, precision=prec)
        Y = y.cpu().numpy()
        errs = [_rel(Y[c], ref[c]) for c in range(20)]
        assert max(errs) <= tol, (prec, max(errs))


def test_pcg(pair):
    """awg_pcg (float64) takes the oracle's iterations with H_3,ad over this
    H_2; the block solve in the float16 form reaches 1e-8 on every column."""
    p, sol, st = pair
    from paper_2106_10913_gb300 import MIXED_FP16, awg_pcg_block
    b = p.b if p.b.ndim == 1 else p.b[0]
    x, its, rel, status = sol.pcg(torch.from_numpy(b).cuda(), rtol=1e-8)
    assert status == 0 and rel[0] <= 1e-8
    X = x.cpu().numpy()
    assert np.linalg.norm(st.A @ X - b) <= 1e-8 * np.linalg.norm(b) * (1 + 1e-12)
    ref = O.pcg(lambda v: st.A @ v, b, lambda r: O.H3_ad_apply(st, r), rtol=1e-8)
    assert abs(its[0] - ref.iters) <= max(1, round(0.05 * ref.iters)), (its[0], ref.iters)
    B = np.random.default_rng(4).standard_normal((5, p.n))
    xb = torch.zeros((5, p.n), dtype=torch.float64, device="cuda")
    status, itsb, rels = awg_pcg_block(sol.h, torch.from_numpy(B).cuda(), xb, 1e-8, precision=MIXED_FP16,
                                       check=False)
    assert status == 0
    XB = xb.cpu().numpy()
    for c in range(5):
        assert np.linalg.norm(st.A @ XB[c] - B[c]) <= 1e-8 * np.linalg.norm(B[c]) * (1 + 1e-12)
