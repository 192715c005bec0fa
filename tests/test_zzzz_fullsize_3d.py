"""The 3D workload at full size: log-normal diffusion on 96^3 cells
(n = 884 736; sigma 3, correlation length 8), 512 uneven k-means subdomains
grown by 2 layers, tau = 0.1 (awg_inputs.config3), set up on the GPU with
the dense GenEO eigensolver.  The CPU oracle cannot set up the whole
problem, so it is compared where it can be:

* bit-exact over the whole problem: every Omega^s, the pair multiplicities
  M_mu and the partition of unity D;
* on two sampled subdomains (the first and one in the middle of the
  partition), from the oracle's eigen-splits of each sample and of every
  subdomain that meets it: n^s_-, the strictly negative count and the
  GenEO mode count exactly, the eigenvalues of V^s_- to 1e-12 of
  max |lambda(B^s)|, and the GenEO subspace within the largest principal
  angle the eigensolvers' accuracy allows (as for the 512 x 512 problem:
  ten times 1e-13 sqrt(kappa(M_B)) over the relative gap at tau, never
  below 1e-8);
* 16 right-hand sides in one graph-driven block solve with float16 W:
  every column at a true relative residual <= 1e-8 (status 0), the
  iterations reported.
"""

import numpy as np
import pytest
import scipy.linalg as sla

import awg_inputs as gi
import oracle as O

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

SAMPLES = [0, 255]
NRHS = 16
_STATE = {}


def _full():
    if not _STATE:
        from paper_2106_10913_gb300 import GENEO_DENSE, AWGSolver
        p = gi.config3()
        sol = AWGSolver(p.rowptr, p.colidx, p.val, p.part, p.nparts, p.overlap, p.tau, precisions=0b1001,
                        geneo_solver=GENEO_DENSE)
        A = O.csr_from(p.rowptr, p.colidx, p.val, p.n)
        subs = O.grow_subdomains(A, p.part, p.nparts, p.overlap)
        _STATE.update(p=p, sol=sol, A=A, subs=subs)
    return _STATE


def test_structure_exact_3d():
    S = _full()
    p, sol, A, subs = S["p"], S["sol"], S["A"], S["subs"]
    assert sol.array("ns").tolist() == [len(s) for s in subs]
    assert np.array_equal(sol.array("sub_idx"), np.concatenate(subs))
    Mmu = O.pair_multiplicity(A, subs)
    coo = A.tocoo()
    assert np.array_equal(sol.array("mmu"), np.asarray(Mmu.tocsr()[coo.row, coo.col]).ravel())
    d, _ = O.partition_of_unity(subs, p.n)
    assert np.array_equal(sol.array("dvec"), d)
    S["Mmu"] = Mmu


def test_sampled_subdomains_3d():
    S = _full()
    p, sol, A, subs = S["p"], S["sol"], S["A"], S["subs"]
    Mmu = S.get("Mmu")
    if Mmu is None:
        Mmu = O.pair_multiplicity(A, subs)
    _, Ds = O.partition_of_unity(subs, p.n)
    B = O.splitting_matrix(A, Mmu)
    out = O.sampled_local_geneo(A, subs, Ds, B, SAMPLES, p.tau)
    nm, nst, modes = sol.array("n_minus"), sol.array("n_strict"), sol.array("modes")
    ns = sol.array("ns").astype(np.int64)
    lam_m = sol.array("lam_minus")
    nm_ptr = np.concatenate([[0], np.cumsum(nm)])
    Z = sol.array("Z_blocks")
    z_off = np.concatenate([[0], np.cumsum(ns * modes)])
    for s, (spl, Y, lam, M_B) in zip(SAMPLES, out):
        assert (int(nm[s]), int(nst[s])) == (spl.n_minus, spl.n_strict), s
        assert int(modes[s]) == Y.shape[1], s
        scale = np.max(np.abs(spl.lam))
        assert np.max(np.abs(np.sort(lam_m[nm_ptr[s]:nm_ptr[s + 1]]) - np.sort(spl.L_minus)),
                      initial=0.0) <= 1e-12 * scale
        m = Y.shape[1]
        print(f"[3D subdomain {s}: n^s = {len(subs[s])}, n^s_- = {spl.n_minus}, modes = {m}]")
        if m == 0:
            continue
        Zs = Z[z_off[s]:z_off[s + 1]].reshape(m, int(ns[s])).T  # column-major n^s x m^s
        ev = np.linalg.eigvalsh(0.5 * (M_B + M_B.T))
        gap = (lam[m] - lam[m - 1]) / lam[m] if m < lam.size else 1.0
        tol = max(1e-8, 10 * 1e-13 * np.sqrt(ev[-1] / ev[0]) / gap)
        assert np.max(sla.subspace_angles(Zs, Y)) < tol, (s, tol)


def test_block_solve_3d():
    S = _full()
    p, sol, A = S["p"], S["sol"], S["A"]
    from paper_2106_10913_gb300 import MIXED_FP16, awg_pcg_block_async
    Bh = np.ascontiguousarray(gi.block_rhs(p, NRHS))
    b = torch.from_numpy(Bh).cuda()
    x = torch.zeros_like(b)
    its = torch.zeros(NRHS, dtype=torch.int32, device="cuda")
    rel = torch.zeros(NRHS, dtype=torch.float64, device="cuda")
    st = torch.full((1,), -1, dtype=torch.int32, device="cuda")
    awg_pcg_block_async(sol.h, b, x, its, rel, st, 1e-8, precision=MIXED_FP16)
    torch.cuda.synchronize()
    assert int(st.item()) == 0
    X = x.cpu().numpy()
    R = A @ X.T - Bh.T
    true_rel = np.linalg.norm(R, axis=0) / np.linalg.norm(Bh, axis=1)
    assert np.all(true_rel <= 1e-8 * (1 + 1e-12)), float(true_rel.max())
    print(f"[3D block solve, float16 W: n0 = {sol.info['n0']}, n_- = {sol.info['n_minus']}, "
          f"iterations {its.cpu().numpy().tolist()}]")
