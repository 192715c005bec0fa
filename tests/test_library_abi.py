"""The C-ABI library builds, loads and exports every entry point that
include/awg.h declares (no GPU needed: no compute call is made)."""

import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "awg.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(awg_[a-z_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    import __graft_entry__ as g
    g.build()
    import paper_2106_10913_gb300 as pkg
    return pkg.load_library()


def test_header_declares_api():
    names = _declared()
    for required in ("awg_setup", "awg_apply", "awg_pcg", "awg_destroy"):
        assert required in names


def test_library_exports_every_declared_symbol(lib):
    for name in _declared():
        assert hasattr(lib, name), f"{name} declared in include/awg.h but not exported"


def test_binding_covers_exports(lib):
    import paper_2106_10913_gb300 as pkg
    assert sorted(pkg.EXPORTED) == _declared()


def test_host_only_calls(lib):
    """Calls that need no device: defaults and status names."""
    import paper_2106_10913_gb300 as pkg
    o = pkg.default_options()
    assert o.variant == 0 and o.precisions == 1 and o.zero_rtol == 1e-12 and o.maxit == 1000
    assert o.geneo_solver == 0 and o.geneo_block == 8 and o.geneo_maxit == 60 and o.autotune == 1
    assert not o.learned_params
    assert lib.awg_status_string(0) == b"AWG_OK"
    assert lib.awg_status_string(2) == b"AWG_ERR_MIN_OVERLAP"
    # argument errors are rejected before any CUDA call
    h = ctypes.c_void_p()
    st = lib.awg_setup(0, 0, None, None, None, None, 1, 1, 0.1, None, None, ctypes.byref(h))
    assert st == 1 and not h.value
    assert lib.awg_get_info(None, None) == 1
    # the learned start needs its parameters; the network calls check sizes
    o = pkg.default_options(geneo_solver=2)
    st = lib.awg_setup(4, 4, 1, 1, 1, 1, 1, 1, 0.1, ctypes.byref(o), None, ctypes.byref(h))
    assert st == 1 and not h.value
    assert lib.awg_learned_forward(-1, None, None, None, 0, None) == 1
    assert lib.awg_learned_grad(0, None, None, None, None, 0, None) == 1
    assert lib.awg_learned_train(1, None, None, None, 1, 1e-2, 0, None, None) == 1
    assert lib.awg_learned_data(None, None, None, None) == 1
    assert ctypes.sizeof(pkg.awg.awg_options) == 112
    assert o.w16_keep == 0.1
    d = pkg.default_options()
    assert d.block_tensor_cores == 1 and d.h2 == pkg.H2_NN_HYB and d.tau_flat == 10.0
    assert d.coarse_tensor_cores == 1 and d.w_drop_tol == 0.0
    for bad in ({"coarse_tensor_cores": 2}, {"w_drop_tol": -1.0}, {"w_drop_tol": 1.0},
                {"w_drop_tol": 1e-4, "variant": 2}):
        o = pkg.default_options(**bad)
        assert lib.awg_setup(4, 4, 1, 1, 1, 1, 1, 1, 0.1, ctypes.byref(o), None, ctypes.byref(h)) == 1, bad
    # H_2 choice and tau_flat are checked before any device work
    for bad in ({"h2": 4}, {"h2": -1}, {"h2": pkg.H2_ASP_AD, "tau_flat": 0.0}):
        o = pkg.default_options(**bad)
        assert lib.awg_setup(4, 4, 1, 1, 1, 1, 1, 1, 0.1, ctypes.byref(o), None, ctypes.byref(h)) == 1
    # the block and graph-driven entry points reject bad arguments before
    # touching the device
    assert lib.awg_apply_block(None, 4, 0, None, None, 1, 1, None) == 1
    assert lib.awg_status_string(11) == b"AWG_ERR_IO"
    assert lib.awg_pcg_block(None, 0, None, None, 1, 1, 1e-8, None, None, None) == 1
    assert lib.awg_pcg_block_async(None, 0, None, None, 1, 1, 1e-8, None, None, None, None) == 1
    assert lib.awg_coarse_apply_block(None, 0, 0, 1, None, None, 1, None) == 1


def test_product_does_not_import_oracle():
    """The solver package never imports the oracle or falls back to the CPU."""
    pkgdir = os.path.join(ROOT, "paper_2106_10913_gb300")
    for dp, _, files in os.walk(pkgdir):
        for f in files:
            if f.endswith(".py"):
                txt = open(os.path.join(dp, f)).read()
                assert "import oracle" not in txt and "from oracle" not in txt, f


def test_checkpoint_file_errors(lib, tmp_path):
    """awg_save / awg_load reject bad arguments and files that are not
    handle files (missing, another tag, another version, truncated, tables
    that disagree with the scalars) before any device work."""
    import struct
    import paper_2106_10913_gb300 as pkg
    h = ctypes.c_void_p(123)
    assert lib.awg_save(None, b"x") == 1
    assert lib.awg_load(None, None, ctypes.byref(h)) == 1 and not h.value
    assert lib.awg_load(b"x", None, None) == 1
    assert lib.awg_load(str(tmp_path / "missing").encode(), None, ctypes.byref(h)) == 11 and not h.value
    osz = ctypes.sizeof(pkg.awg.awg_options)
    ver = 2  # the current format version
    cases = {
        "tag": b"NOTAHNDL" + struct.pack("<II", ver, osz),
        "version": b"AWGHNDL\n" + struct.pack("<II", ver - 1, osz),
        "options": b"AWGHNDL\n" + struct.pack("<II", ver, osz + 8),
        "truncated": b"AWGHNDL\n" + struct.pack("<II", ver, osz) + b"\0" * 16,
        "inconsistent": b"AWGHNDL\n" + struct.pack("<II", ver, osz) + b"\0" * 4096,
    }
    for name, data in cases.items():
        f = tmp_path / name
        f.write_bytes(data)
        h = ctypes.c_void_p(123)
        assert lib.awg_load(str(f).encode(), None, ctypes.byref(h)) == 11, name
        assert not h.value, name


def test_binding_constants_match_header():
    """The binding's profile classes and mask bits are the header's values."""
    import re
    from paper_2106_10913_gb300 import awg as A
    src = open(os.path.join(ROOT, "include", "awg.h")).read()
    vals = {m.group(1): m.group(2) for m in re.finditer(r"(AWG_PROF_[A-Z]+)\s*=\s*([^,}]+?)\s*[,}]", src)}
    assert int(eval(vals["AWG_PROF_SERIAL"])) == A.PROF_SERIAL
    assert int(eval(vals["AWG_PROF_COUNT"])) == A.PROF_COUNT
    for i, name in enumerate(A.PROF_NAMES):
        assert int(vals["AWG_PROF_" + name.upper()]) == i, name
