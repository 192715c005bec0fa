"""bench.py's roofline arithmetic on a made-up profile (no GPU): the
dominant class is the one with the largest summed event time; achieved =
algorithmic bytes per launch over the average launch time; frac =
achieved / the measured copy bandwidth; traffic = the measured DRAM ratio
times the algorithmic bytes for the classes captured (64-column float16-W
form), null otherwise; the iteration line divides block_bytes' total by the
time per iteration."""

import pytest

import bench

torch = pytest.importorskip("torch")


def _info():
    ns = [300, 310, 280, 295]
    return {"n": 1024, "n_minus": 40, "nnz": 5000, "n0": 36, "sum_ns": sum(ns),
            "dense_total": sum(m * m for m in ns), "ns": ns, "z_entries": sum(ns) * 9, "vm_entries": sum(ns) * 10}


def _form(prec, dom_ms):
    ms = {"spmv": 1.0, "local": 1.0, "wt": 1.0, "wd": 1.0, "coarse": 1.0, "subdomain": 1.0, "prolong": 1.0,
          "vector": 1.0}
    ms.update(dom_ms)
    prof = {"ms": ms, "count": {k: 4 for k in ms}, "profiled_solve_ms": sum(ms.values())}
    return {"prec": prec, "block": True, "nrhs": 64, "prof": prof, "ms": 120.0, "steps": 2, "iters": 10}


def test_roofline_local_class_with_traffic():
    from paper_2106_10913_gb300 import MIXED_FP16
    info = _info()
    r = bench.roofline_of(_form(MIXED_FP16, {"local": 8.0}), info)
    per, it_bytes = bench.block_bytes(info, 64, MIXED_FP16)
    assert r["kernel"].startswith("k_local_bimg")
    assert r["avg_launch_ms"] == pytest.approx(2.0)
    assert r["algorithmic_bytes_per_launch"] == pytest.approx(per["local"])
    assert r["achieved"] == pytest.approx(per["local"] / 2e-3 / 1e9)
    assert r["frac"] == pytest.approx(r["achieved"] / r["peak"])
    assert r["traffic"] == pytest.approx(bench.DRAM_RATIO_K64_FP16["local"] * per["local"])
    assert r["kernel_share_of_solve"] == pytest.approx(8.0 / 15.0)
    assert r["iteration"]["ms"] == pytest.approx(120.0 / 2 / 10)
    assert r["iteration"]["algorithmic_bytes"] == pytest.approx(it_bytes)


def test_roofline_without_capture_has_no_traffic():
    from paper_2106_10913_gb300 import MIXED_FP16, MIXED_FP32
    info = _info()
    assert bench.roofline_of(_form(MIXED_FP16, {"vector": 9.0}), info)["traffic"] is None
    assert bench.roofline_of(_form(MIXED_FP32, {"local": 9.0}), info)["traffic"] is None


def test_block_bytes_local_images():
    from paper_2106_10913_gb300 import MIXED_FP16
    info = _info()
    per, _ = bench.block_bytes(info, 64, MIXED_FP16)
    tiles = sum(((m + 127) // 128) * ((m + 31) // 32) for m in info["ns"])
    assert per["local"] == tiles * 16384 + 3 * info["sum_ns"] * 64 * 4
