"""Thin ctypes binding of libawg (include/awg.h).

Argument marshalling only: every step of setup, apply and PCG runs in the
library's CUDA kernels.  Tensors are PyTorch CUDA tensors (device memory and
streams are PyTorch's); the library is loaded from ``lib/libawg.so`` next to
this file and importing fails loudly if it has not been built.
"""

from __future__ import annotations

import ctypes
import os
from typing import Optional

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "lib", "libawg.so")

AWG_OK = 0
STATUS = {0: "AWG_OK", 1: "AWG_ERR_INVALID_ARG", 2: "AWG_ERR_MIN_OVERLAP", 3: "AWG_ERR_NOT_SPD",
          4: "AWG_ERR_EIG", 5: "AWG_ERR_BREAKDOWN", 6: "AWG_ERR_MAXIT", 7: "AWG_ERR_OOM",
          8: "AWG_ERR_CUDA", 9: "AWG_ERR_NOT_SYMMETRIC", 10: "AWG_ERR_STATE", 11: "AWG_ERR_IO"}
H3_AD, H3_HYB, H3_INEX = 0, 1, 2
FP64, MIXED_FP32, MIXED_BF16, MIXED_FP16 = 0, 1, 2, 3
# H^NN_hyb(tau) (Thm. 4), H^AS_+,hyb / ,ad(tau_flat) (Thm. 3), H^AS_hyb(tau, tau_flat) (Thm. 5)
H2_NN_HYB, H2_ASP_HYB, H2_ASP_AD, H2_AS_HYB = 0, 1, 2, 3
STAGE = {"spmv": 0, "aplus": 1, "hnn": 2, "h2": 3, "h3ad": 4, "h3hyb": 5, "h3inex": 6}
ARRAY = {"ns": (0, np.int32), "sub_idx": (1, np.int32), "n_minus": (2, np.int32),
         "n_strict": (3, np.int32), "modes": (4, np.int32), "lam_minus": (5, np.float64),
         "mmu": (6, np.float64), "dvec": (7, np.float64), "E": (8, np.float64),
         "F": (9, np.float64), "W": (10, np.float64), "Z": (11, np.float64), "Z_blocks": (12, np.float64)}


class AWGError(RuntimeError):
    def __init__(self, status: int, where: str):
        self.status = status
        super().__init__(f"{where}: {STATUS.get(status, status)}")


class awg_options(ctypes.Structure):
    _fields_ = [("variant", ctypes.c_int), ("precisions", ctypes.c_int),
                ("zero_rtol", ctypes.c_double), ("w_rtol", ctypes.c_double),
                ("w_maxit", ctypes.c_int), ("maxit", ctypes.c_int), ("verbose", ctypes.c_int),
                ("w_precision", ctypes.c_int), ("geneo_solver", ctypes.c_int),
                ("geneo_block", ctypes.c_int), ("geneo_maxit", ctypes.c_int),
                ("learned_params", ctypes.c_void_p), ("autotune", ctypes.c_int),
                ("w16_keep", ctypes.c_double), ("block_tensor_cores", ctypes.c_int),
                ("h2", ctypes.c_int), ("tau_flat", ctypes.c_double),
                ("coarse_tensor_cores", ctypes.c_int), ("w_drop_tol", ctypes.c_double)]


class awg_info(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int), ("nnz", ctypes.c_int), ("nparts", ctypes.c_int),
                ("sum_ns", ctypes.c_int64), ("max_ns", ctypes.c_int), ("n0", ctypes.c_int),
                ("n_minus", ctypes.c_int), ("n_minus_all", ctypes.c_int),
                ("w_iters", ctypes.c_int), ("w_relres", ctypes.c_double),
                ("setup_ms", ctypes.c_double * 8), ("device_bytes", ctypes.c_size_t),
                ("geneo_its_max", ctypes.c_int), ("geneo_its_sum", ctypes.c_int64),
                ("geneo_dense", ctypes.c_int), ("wt_blocks", ctypes.c_int * 4),
                ("wd_blocks", ctypes.c_int * 4), ("block_wt_ctas", ctypes.c_int * 3),
                ("block_dense_bps", ctypes.c_int * 3), ("w_kept", ctypes.c_int64)]


EXPORTED = ["awg_default_options", "awg_status_string", "awg_setup", "awg_destroy",
            "awg_get_info", "awg_apply", "awg_apply_stage", "awg_pcg", "awg_get_array",
            "awg_profile", "awg_profile_read", "awg_apply_hnn_noalloc", "awg_learned_data",
            "awg_learned_forward", "awg_learned_grad", "awg_learned_train", "awg_profile_trace",
            "awg_apply_block", "awg_pcg_block", "awg_pcg_block_async", "awg_save", "awg_load",
            "awg_coarse_apply_block"]
LEARNED_NPARAM, LEARNED_NFEAT = 385, 5
GENEO_DENSE, GENEO_BLOCK, GENEO_LEARNED = 0, 1, 2
PROF_NAMES = ["spmv", "local", "wt", "wd", "coarse", "subdomain", "prolong", "vector"]
# further awg_profile mask bits: serialise the apply's two streams while
# profiling; count launches only
PROF_SERIAL, PROF_COUNT = 1 << 8, 1 << 9

_lib = None


def load_library(path: str = LIB_PATH):
    """Load libawg.so and declare its signatures (raises if absent)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise ImportError(f"libawg.so not found at {path}; build it with "
                          "`python -c 'import __graft_entry__ as g; g.build()'`")
    lib = ctypes.CDLL(path)
    P, I, D, S = ctypes.c_void_p, ctypes.c_int, ctypes.c_double, ctypes.c_size_t
    lib.awg_default_options.argtypes = [ctypes.POINTER(awg_options)]
    lib.awg_default_options.restype = None
    lib.awg_status_string.argtypes = [I]
    lib.awg_status_string.restype = ctypes.c_char_p
    lib.awg_setup.argtypes = [I, I, P, P, P, P, I, I, D, ctypes.POINTER(awg_options), P,
                              ctypes.POINTER(P)]
    lib.awg_setup.restype = I
    lib.awg_destroy.argtypes = [P]
    lib.awg_destroy.restype = None
    lib.awg_get_info.argtypes = [P, ctypes.POINTER(awg_info)]
    lib.awg_get_info.restype = I
    lib.awg_apply.argtypes = [P, I, P, P, I, I, P]
    lib.awg_apply.restype = I
    lib.awg_apply_stage.argtypes = [P, I, I, P, P, P]
    lib.awg_apply_stage.restype = I
    lib.awg_pcg.argtypes = [P, I, P, P, I, I, D, ctypes.POINTER(I), ctypes.POINTER(D), P]
    lib.awg_pcg.restype = I
    lib.awg_get_array.argtypes = [P, I, P, S]
    lib.awg_get_array.restype = I
    lib.awg_profile.argtypes = [P, I]
    lib.awg_profile.restype = I
    lib.awg_profile_read.argtypes = [P, ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(D),
                                     ctypes.POINTER(ctypes.c_int64)]
    lib.awg_profile_read.restype = I
    lib.awg_profile_trace.argtypes = [P, I, P, P, P, ctypes.POINTER(I)]
    lib.awg_profile_trace.restype = I
    lib.awg_apply_block.argtypes = [P, I, I, P, P, I, I, P]
    lib.awg_apply_block.restype = I
    lib.awg_coarse_apply_block.argtypes = [P, I, I, I, P, P, I, P]
    lib.awg_coarse_apply_block.restype = I
    lib.awg_pcg_block.argtypes = [P, I, P, P, I, I, D, ctypes.POINTER(I), ctypes.POINTER(D), P]
    lib.awg_pcg_block.restype = I
    lib.awg_pcg_block_async.argtypes = [P, I, P, P, I, I, D, P, P, P, P]
    lib.awg_pcg_block_async.restype = I
    lib.awg_apply_hnn_noalloc.argtypes = [P, I, P, P, P]
    lib.awg_apply_hnn_noalloc.restype = I
    lib.awg_learned_data.argtypes = [P, P, P, P]
    lib.awg_learned_data.restype = I
    lib.awg_learned_forward.argtypes = [I, P, P, P, I, P]
    lib.awg_learned_forward.restype = I
    lib.awg_learned_grad.argtypes = [I, P, P, P, P, I, P]
    lib.awg_learned_grad.restype = I
    lib.awg_learned_train.argtypes = [I, P, P, P, I, D, I, P, P]
    lib.awg_learned_train.restype = I
    lib.awg_save.argtypes = [P, ctypes.c_char_p]
    lib.awg_save.restype = I
    lib.awg_load.argtypes = [ctypes.c_char_p, P, ctypes.POINTER(P)]
    lib.awg_load.restype = I
    _lib = lib
    return lib


def _check(st: int, where: str):
    if st != AWG_OK:
        raise AWGError(st, where)


def _stream_ptr(stream) -> ctypes.c_void_p:
    import torch
    s = torch.cuda.current_stream() if stream is None else stream
    return ctypes.c_void_p(s.cuda_stream)


def default_options(**kw) -> awg_options:
    """Defaults of the library with the given fields replaced.  A NumPy
    `learned_params` array is passed by pointer and kept alive on the
    returned structure."""
    o = awg_options()
    load_library().awg_default_options(ctypes.byref(o))
    for k, v in kw.items():
        if k == "learned_params" and v is not None and not isinstance(v, int):
            arr = np.ascontiguousarray(v, dtype=np.float64)
            if arr.size != LEARNED_NPARAM:
                raise ValueError(f"learned_params needs {LEARNED_NPARAM} values")
            o._learned_keep = arr
            v = arr.ctypes.data
        setattr(o, k, v)
    return o


# ----------------------------------------------------------- C-named entry points
def awg_setup(rowptr, colidx, val, partition, nparts: int, overlap: int, tau: float,
              options: Optional[awg_options] = None, stream=None) -> ctypes.c_void_p:
    """Build the preconditioner; all tensors on the same CUDA device."""
    lib = load_library()
    n = rowptr.numel() - 1
    h = ctypes.c_void_p()
    st = lib.awg_setup(n, colidx.numel(), rowptr.data_ptr(), colidx.data_ptr(), val.data_ptr(),
                       partition.data_ptr(), nparts, overlap, float(tau),
                       ctypes.byref(options) if options is not None else None,
                       _stream_ptr(stream), ctypes.byref(h))
    _check(st, "awg_setup")
    return h


def awg_destroy(h):
    load_library().awg_destroy(h)


def awg_save(h, path) -> None:
    """Write the set-up handle to the file `path` (awg_load reads it back)."""
    _check(load_library().awg_save(h, os.fsencode(path)), "awg_save")


def awg_load(path, stream=None) -> ctypes.c_void_p:
    """A new handle from a file written by awg_save, on the current device."""
    h = ctypes.c_void_p()
    _check(load_library().awg_load(os.fsencode(path), _stream_ptr(stream), ctypes.byref(h)), "awg_load")
    return h


def awg_get_info(h) -> dict:
    info = awg_info()
    _check(load_library().awg_get_info(h, ctypes.byref(info)), "awg_get_info")
    d = {k: getattr(info, k) for k, _ in awg_info._fields_}
    d["setup_ms"] = list(info.setup_ms)
    d["wt_blocks"] = list(info.wt_blocks)
    d["wd_blocks"] = list(info.wd_blocks)
    d["block_wt_ctas"] = list(info.block_wt_ctas)
    d["block_dense_bps"] = list(info.block_dense_bps)
    return d


def awg_apply(h, r, z, precision: int = FP64, stream=None):
    nrhs = 1 if r.dim() == 1 else r.shape[0]
    ld = r.shape[-1]
    _check(load_library().awg_apply(h, precision, r.data_ptr(), z.data_ptr(), nrhs, ld,
                                    _stream_ptr(stream)), "awg_apply")
    return z


def awg_apply_stage(h, which, x, y, precision: int = FP64, stream=None):
    w = STAGE[which] if isinstance(which, str) else int(which)
    _check(load_library().awg_apply_stage(h, w, precision, x.data_ptr(), y.data_ptr(),
                                          _stream_ptr(stream)), "awg_apply_stage")
    return y


def awg_pcg(h, b, x, rtol: float = 1e-8, precision: int = FP64, stream=None, check=True):
    nrhs = 1 if b.dim() == 1 else b.shape[0]
    ld = b.shape[-1]
    its = (ctypes.c_int * nrhs)()
    rel = (ctypes.c_double * nrhs)()
    st = load_library().awg_pcg(h, precision, b.data_ptr(), x.data_ptr(), nrhs, ld, float(rtol),
                                its, rel, _stream_ptr(stream))
    if check:
        _check(st, "awg_pcg")
    return st, list(its), list(rel)


def awg_apply_block(h, which, x, y, precision: int = FP64, stream=None):
    """y = stage(x) for the rows of x (nrhs x n, one right-hand side per row,
    nrhs <= 64) at once; `which` as awg_apply_stage, stages 0-6."""
    w = STAGE[which] if isinstance(which, str) else int(which)
    _check(load_library().awg_apply_block(h, w, precision, x.data_ptr(), y.data_ptr(), x.shape[0],
                                          x.shape[-1], _stream_ptr(stream)), "awg_apply_block")
    return y


COARSE = {"Einv": 0, "Finv": 1, "inex": 2}


def awg_coarse_apply_block(h, which, x, y, precision: int = FP64, engine: int = 1, stream=None):
    """y = M x for the rows of x (nrhs x dim, nrhs <= 64) with a dense coarse
    inverse M (which: "Einv", "Finv" or "inex"); engine 0 float64 CUDA cores,
    1 tensor-core slice products, 2 the same with short reduction splits."""
    w = COARSE[which] if isinstance(which, str) else int(which)
    _check(load_library().awg_coarse_apply_block(h, w, precision, int(engine), x.data_ptr(), y.data_ptr(),
                                                 x.shape[0], _stream_ptr(stream)), "awg_coarse_apply_block")
    return y


def awg_pcg_block(h, b, x, rtol: float = 1e-8, precision: int = FP64, stream=None, check=True):
    """PCG for the rows of b (nrhs x n) together: one pass over each
    operator per iteration for all of them, one recurrence per row."""
    nrhs = b.shape[0]
    its = (ctypes.c_int * nrhs)()
    rel = (ctypes.c_double * nrhs)()
    st = load_library().awg_pcg_block(h, precision, b.data_ptr(), x.data_ptr(), nrhs, b.shape[-1],
                                      float(rtol), its, rel, _stream_ptr(stream))
    if check:
        _check(st, "awg_pcg_block")
    return st, list(its), list(rel)


def awg_pcg_block_async(h, b, x, iters, relres, status, rtol: float = 1e-8, precision: int = FP64,
                        stream=None):
    """Enqueue a graph-driven block PCG for the rows of b (nrhs <= 128):
    iters (int32[nrhs]), relres (float64[nrhs]) and status (int32[1]) are
    CUDA tensors filled when the work completes."""
    ptr = lambda t: None if t is None else t.data_ptr()
    _check(load_library().awg_pcg_block_async(h, precision, b.data_ptr(), x.data_ptr(), b.shape[0], b.shape[-1],
                                              float(rtol), ptr(iters), ptr(relres), ptr(status),
                                              _stream_ptr(stream)), "awg_pcg_block_async")


def awg_get_array(h, what: str, size: int) -> np.ndarray:
    code, dt = ARRAY[what]
    out = np.zeros(max(size, 1), dtype=dt)
    _check(load_library().awg_get_array(h, code, out.ctypes.data_as(ctypes.c_void_p), size),
           f"awg_get_array({what})")
    return out[:size]


def awg_apply_hnn_noalloc(h, x, y, precision: int = FP64, stream=None):
    """y = H^NN x with the library's static scratch: no device allocation
    (for callers that cannot allocate while applying the preconditioner)."""
    _check(load_library().awg_apply_hnn_noalloc(h, precision, x.data_ptr(), y.data_ptr(),
                                                _stream_ptr(stream)), "awg_apply_hnn_noalloc")
    return y


def awg_learned_data(h, features=None, targets=None, stream=None):
    """Per-node features (sum_ns x 5) and leverage targets (sum_ns) of a
    built handle into caller-owned float64 CUDA tensors (either may be None)."""
    _check(load_library().awg_learned_data(
        h, None if features is None else features.data_ptr(),
        None if targets is None else targets.data_ptr(), _stream_ptr(stream)), "awg_learned_data")


def awg_learned_forward(features, params, out, precision: int = FP64, stream=None):
    _check(load_library().awg_learned_forward(features.shape[0], features.data_ptr(),
                                              params.data_ptr(), out.data_ptr(), precision,
                                              _stream_ptr(stream)), "awg_learned_forward")
    return out


def awg_learned_grad(features, targets, params, grad, precision: int = FP64, stream=None):
    """grad (NPARAM + 1 float64 on the device): gradient of the mean squared
    error, then the loss."""
    _check(load_library().awg_learned_grad(features.shape[0], features.data_ptr(),
                                           targets.data_ptr(), params.data_ptr(), grad.data_ptr(),
                                           precision, _stream_ptr(stream)), "awg_learned_grad")
    return grad


def awg_learned_train(features, targets, params: np.ndarray, steps: int, lr: float = 1e-2,
                      precision: int = FP64, stream=None):
    """Full-batch Adam on the device; returns (new params, loss per step)."""
    th = np.array(params, dtype=np.float64, copy=True)
    loss = np.zeros(max(steps, 1))
    _check(load_library().awg_learned_train(features.shape[0], features.data_ptr(),
                                            targets.data_ptr(), th.ctypes.data, int(steps),
                                            float(lr), precision, loss.ctypes.data,
                                            _stream_ptr(stream)), "awg_learned_train")
    return th, loss[:steps]


def awg_profile(h, mask: int):
    """Start (mask = bit set of kernel classes to time, 0xFF all; with
    PROF_SERIAL the apply's side stream is folded into the main stream;
    PROF_COUNT alone counts launches) or stop (0)."""
    _check(load_library().awg_profile(h, int(mask)), "awg_profile")


def awg_profile_read(h) -> dict:
    """Launch count and per-kernel-class event time (ms) and launch counts."""
    n = len(PROF_NAMES)
    launches = ctypes.c_int64()
    ms = (ctypes.c_double * n)()
    cnt = (ctypes.c_int64 * n)()
    _check(load_library().awg_profile_read(h, ctypes.byref(launches), ms, cnt), "awg_profile_read")
    return {"launches": launches.value,
            "ms": {k: ms[i] for i, k in enumerate(PROF_NAMES)},
            "count": {k: cnt[i] for i, k in enumerate(PROF_NAMES)}}


def awg_profile_trace(h, cap: int = 65536):
    """(class names, start ms, end ms) of the launches timed so far, on the
    device clock shared by all streams."""
    cls = np.zeros(cap, dtype=np.int32)
    t0 = np.zeros(cap)
    t1 = np.zeros(cap)
    cnt = ctypes.c_int()
    _check(load_library().awg_profile_trace(h, cap, cls.ctypes.data, t0.ctypes.data, t1.ctypes.data,
                                            ctypes.byref(cnt)), "awg_profile_trace")
    k = cnt.value
    return [PROF_NAMES[c] for c in cls[:k]], t0[:k], t1[:k]


# ------------------------------------------------------------- convenience class
class AWGSolver:
    """Owns one libawg handle built from host (NumPy) or device CSR arrays."""

    def __init__(self, rowptr, colidx, val, partition, nparts: int, overlap: int, tau: float,
                 device="cuda", **opts):
        import torch
        t = lambda a, dt: (a if isinstance(a, torch.Tensor) else torch.from_numpy(
            np.ascontiguousarray(a))).to(device=device, dtype=dt).contiguous()
        self.rowptr = t(rowptr, torch.int32)
        self.colidx = t(colidx, torch.int32)
        self.val = t(val, torch.float64)
        part = t(partition, torch.int32)
        self.n = self.rowptr.numel() - 1
        self.device = device
        self.h = awg_setup(self.rowptr, self.colidx, self.val, part, nparts, overlap, tau,
                           default_options(**opts))
        self.info = awg_get_info(self.h)

    @classmethod
    def load(cls, path, device="cuda"):
        """A solver on the handle stored in `path` by ``save`` (no setup)."""
        self = cls.__new__(cls)
        self.device = device
        self.h = awg_load(path)
        self.info = awg_get_info(self.h)
        self.n = self.info["n"]
        return self

    def save(self, path):
        awg_save(self.h, path)

    def close(self):
        if self.h is not None:
            awg_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def apply(self, r, precision: int = FP64, stage: Optional[str] = None):
        import torch
        z = torch.empty_like(r)
        if stage is None:
            return awg_apply(self.h, r, z, precision)
        return awg_apply_stage(self.h, stage, r, z, precision)

    def pcg(self, b, rtol: float = 1e-8, precision: int = FP64, check=True):
        import torch
        x = torch.zeros_like(b)
        st, its, rel = awg_pcg(self.h, b, x, rtol, precision, check=check)
        return x, its, rel, st

    def array(self, what: str) -> np.ndarray:
        i = self.info
        if what == "Z_blocks":  # sum_s n^s m^s
            size = int(np.dot(self.array("ns").astype(np.int64), self.array("modes").astype(np.int64)))
        else:
            size = {"ns": i["nparts"], "sub_idx": i["sum_ns"], "n_minus": i["nparts"],
                    "n_strict": i["nparts"], "modes": i["nparts"], "lam_minus": i["n_minus_all"],
                    "mmu": i["nnz"], "dvec": i["n"], "E": i["n0"] ** 2, "F": i["n_minus"] ** 2,
                    "W": i["n"] * i["n_minus"], "Z": i["n"] * i["n0"]}[what]
        return awg_get_array(self.h, what, size)
