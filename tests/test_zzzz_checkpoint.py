"""awg_save / awg_load: a handle read back from its file reports the same
setup results (counts, D, M_mu, eigenvalues, E, F, bit for bit) and applies
and solves exactly as the handle that wrote it.  The single-RHS applies
match bit for bit (their grid sizes are stored with the handle); the block
path builds its float32 copies and re-runs its timing-based autotuner on
first use, so its split sums may be ordered differently: there the
iterations agree within one and both reach 1e-8."""

import numpy as np
import pytest

import awg_inputs as gi

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

INFO_KEYS = ["n", "nnz", "nparts", "sum_ns", "max_ns", "n0", "n_minus", "n_minus_all", "w_iters", "w_relres",
             "setup_ms", "geneo_its_max", "geneo_its_sum", "geneo_dense", "wt_blocks", "wd_blocks"]
ARRAYS = ["ns", "sub_idx", "n_minus", "n_strict", "modes", "lam_minus", "mmu", "dvec", "E", "F"]


def test_round_trip(tmp_path):
    from paper_2106_10913_gb300 import AWGSolver, FP64, MIXED_FP16, awg_pcg_block
    p = gi.channels2d(64, q=2, nchan=3, contrast=1e6, seed=11, overlap=2, tau=0.1)
    sol = AWGSolver(p.rowptr, p.colidx, p.val, p.part, p.nparts, p.overlap, p.tau, precisions=0b1001)
    path = tmp_path / "channels64.awg"
    sol.save(path)
    loaded = AWGSolver.load(path)
    try:
        for k in INFO_KEYS:
            assert loaded.info[k] == sol.info[k], k
        for what in ARRAYS:
            assert np.array_equal(loaded.array(what), sol.array(what)), what
        x = torch.from_numpy(np.random.default_rng(5).standard_normal(p.n)).cuda()
        for prec in (FP64, MIXED_FP16):
            assert torch.equal(loaded.apply(x, precision=prec), sol.apply(x, precision=prec))
            for stage in ("hnn", "h2", "h3hyb", "h3inex"):
                assert torch.equal(loaded.apply(x, precision=prec, stage=stage),
                                   sol.apply(x, precision=prec, stage=stage)), (prec, stage)
        b = torch.from_numpy(p.b).cuda()
        x1, its1, rel1, _ = sol.pcg(b, rtol=1e-8)
        x2, its2, rel2, _ = loaded.pcg(b, rtol=1e-8)
        assert its1 == its2 and rel1 == rel2 and torch.equal(x1, x2)
        B = torch.from_numpy(np.random.default_rng(6).standard_normal((20, p.n))).cuda()
        runs = []
        for s_ in (sol, loaded):
            xb = torch.zeros_like(B)
            st, its, rels = awg_pcg_block(s_.h, B, xb, 1e-8, precision=MIXED_FP16, check=False)
            assert st == 0 and max(rels) <= 1e-8
            runs.append(its)
        assert all(abs(a - c) <= 1 for a, c in zip(*runs))
    finally:
        loaded.close()
        sol.close()


def test_damaged_files_are_refused(tmp_path):
    """A file whose tables disagree with each other (a subdomain size above
    max_ns, a prefix table that decreases) or whose device buffer carries
    fewer bytes than the tables imply is refused with AWG_ERR_IO (11), before
    any buffer is read past its end."""
    import ctypes
    import struct
    from paper_2106_10913_gb300 import AWGSolver, load_library
    p = gi.channels2d(64, q=2, nchan=3, contrast=1e6, seed=11, overlap=2, tau=0.1)
    sol = AWGSolver(p.rowptr, p.colidx, p.val, p.part, p.nparts, p.overlap, p.tau)
    path = tmp_path / "good.awg"
    sol.save(path)
    data = path.read_bytes()
    ns = sol.array("ns").astype(np.int32)
    dvec = sol.array("dvec")
    sol.close()
    N = ns.size
    # host table of the subdomain sizes: element count, then the sizes
    tab = struct.pack("<Q", N) + ns.tobytes()
    i_ns = data.index(tab)
    # host table of the subdomain pointers, right after it
    ptr = np.concatenate([[0], np.cumsum(ns)]).astype(np.int32)
    tab_ptr = struct.pack("<Q", N + 1) + ptr.tobytes()
    i_ptr = data.index(tab_ptr)
    # device buffer D: byte count, then the values
    buf_d = struct.pack("<Q", dvec.size * 8) + dvec.tobytes()
    i_d = data.index(buf_d)
    big = ns.copy()
    big[0] = ns.max() + 1
    bad_ptr = ptr.copy()
    bad_ptr[1], bad_ptr[2] = bad_ptr[2], bad_ptr[1]
    cases = {
        "n^s above max_ns": data[:i_ns + 8] + big.tobytes() + data[i_ns + 8 + 4 * N:],
        "decreasing pointers": data[:i_ptr + 8] + bad_ptr.tobytes() + data[i_ptr + 8 + 4 * (N + 1):],
        "short buffer": data[:i_d] + struct.pack("<Q", dvec.size * 8 - 8) + data[i_d + 8:],
    }
    lib = load_library()
    for name, blob in cases.items():
        f = tmp_path / "bad.awg"
        f.write_bytes(blob)
        h = ctypes.c_void_p(123)
        assert lib.awg_load(str(f).encode(), None, ctypes.byref(h)) == 11, name
        assert not h.value, name
    # the untouched file still loads
    h = ctypes.c_void_p()
    assert lib.awg_load(str(path).encode(), None, ctypes.byref(h)) == 0 and h.value
    lib.awg_destroy(h)
