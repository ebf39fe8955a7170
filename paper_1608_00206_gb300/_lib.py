"""ctypes binding of libhc.so: the C ABI of include/hc.h, one Python function
per C function, same names, argument marshalling only.  Pointers are plain
integers (device addresses) and streams are raw cudaStream_t handles."""
from __future__ import annotations

import ctypes
import os
import threading

_PKG = os.path.dirname(os.path.abspath(__file__))
SO_PATH = os.path.join(_PKG, "libhc.so")

HC_INT64, HC_FP64, HC_FP32, HC_FP32_MIXED, HC_FP32_FF = 0, 1, 2, 3, 4
HC_OK, HC_ERR_ARG, HC_ERR_DTYPE, HC_ERR_ALIGN, HC_ERR_ALIAS = 0, 1, 2, 3, 4
HC_ERR_WORKSPACE, HC_ERR_CUDA, HC_ERR_TIMEOUT = 5, 6, 7
HC_MAX_D = 24

# Every symbol include/hc.h declares, with (restype, argtypes).
_vp, _i, _sz, _cp = ctypes.c_void_p, ctypes.c_int, ctypes.c_size_t, ctypes.c_char_p


HC_SCHED_DEFAULT, HC_SCHED_PASSES, HC_SCHED_CHUNKED, HC_SCHED_CHUNKED_BULK = 0, 1, 2, 3
HC_SCHED_HYBRID, HC_SCHED_LOWMEM, HC_SCHED_PADDED = 4, 5, 6


class hc_schedule(ctypes.Structure):
    _fields_ = [("kind", _i), ("c", _i), ("k", _i), ("cols", _i), ("cols_outer", _i),
                ("top", _i)]

    def as_dict(self):
        return {"kind": self.kind, "c": self.c, "k": self.k, "cols": self.cols,
                "cols_outer": self.cols_outer, "top": self.top}


class hc_instance(ctypes.Structure):
    _fields_ = [("x", _vp), ("y", _vp), ("z", _vp), ("D", _i)]


SIGNATURES = {
    "hc_version": (_i, []),
    "hc_status_string": (_cp, [_i]),
    "hc_last_cuda_error": (_cp, []),
    "hc_workspace_size": (_sz, [_i, _i]),
    "hc_convolve": (_i, [_vp, _vp, _vp, _i, _i, _vp, _sz, _vp]),
    "hc_workspace_size_schedule": (_sz, [_i, _i, ctypes.c_void_p]),
    "hc_convolve_schedule": (_i, [_vp, _vp, _vp, _i, _i, ctypes.c_void_p, _vp, _sz, _vp]),
    "hc_set_default_schedule": (_i, [_i, _i, ctypes.c_void_p]),
    "hc_get_default_schedule": (_i, [_i, _i, ctypes.c_void_p]),
    "hc_autotune_workspace_size": (_sz, [_i, _i]),
    "hc_autotune": (_i, [_vp, _vp, _vp, _i, _i, _vp, _sz, _i, _vp, ctypes.c_void_p,
                         ctypes.POINTER(ctypes.c_double)]),
    "hc_convolve_noalloc": (_i, [_vp, _vp, _vp, _i, _i, _vp]),
    "hc_carryfree_workspace_size": (_sz, [_sz, _i]),
    "hc_carryfree": (_i, [_vp, _vp, _vp, _sz, _i, _vp, _sz, _vp]),
    "hc_backward_workspace_size": (_sz, [_i, _i]),
    "hc_convolve_backward": (_i, [_vp, _vp, _vp, _vp, _vp, _i, _i, _vp, _sz, _vp]),
    "hc_batched_workspace_size": (_sz, [ctypes.POINTER(hc_instance), _i, _i]),
    "hc_convolve_batched": (_i, [ctypes.POINTER(hc_instance), _i, _i, _vp, _sz, _vp]),
    "hc_batched_prepare": (_i, [ctypes.POINTER(hc_instance), _i, _i, _vp, _sz, _vp]),
    "hc_batched_launch": (_i, [_vp, _sz, _vp]),
    "hc_batched_inject_stall": (_i, [_vp, _i]),
    "hc_convolve_out": (_i, [_vp, _vp, _vp, _vp, _i, _i, _vp, _sz, _vp]),
    "hc_batched_prepare_split": (_i, [ctypes.POINTER(hc_instance), _i, _i, _i, _vp, _sz, _vp]),
    "hc_batched_autotune": (_i, [ctypes.POINTER(hc_instance), _i, _i, _vp, _sz, _i, _vp,
                                 ctypes.POINTER(_i), ctypes.POINTER(ctypes.c_double)]),
    "hc_maxconv_plan": (_i, [_i, ctypes.c_int64, ctypes.POINTER(_i), ctypes.POINTER(_i),
                             ctypes.POINTER(_i), ctypes.POINTER(_i)]),
    "hc_maxconv_workspace_size": (_sz, [_i, ctypes.c_int64]),
    "hc_maxconv": (_i, [_vp, _vp, _vp, _i, ctypes.c_int64, _vp, _sz, _vp]),
    "hc_device_status": (_i, [_vp, _vp]),
    "hc_probe_alu_rate": (_i, [_i, ctypes.POINTER(ctypes.c_double), _vp]),
    "hc_profile_enable": (_i, [_i]),
    "hc_profile_collect": (_i, [_cp, _i, ctypes.POINTER(ctypes.c_double),
                                ctypes.POINTER(ctypes.c_int), _i]),
}

_LOCK = threading.Lock()
_LIB = None


class HCError(RuntimeError):
    def __init__(self, status: int, what: str = ""):
        self.status = status
        msg = lib().hc_status_string(status).decode()
        if status == HC_ERR_CUDA:
            msg += f" ({lib().hc_last_cuda_error().decode()})"
        super().__init__(f"{what}: {msg}" if what else msg)


def lib():
    """Load libhc.so (raises if it has not been built: there is no fallback)."""
    global _LIB
    with _LOCK:
        if _LIB is None:
            if not os.path.exists(SO_PATH):
                raise RuntimeError(
                    f"{SO_PATH} is missing; build it with `python -m paper_1608_00206_gb300.build` "
                    "(or __graft_entry__.build()).  There is no CPU fallback.")
            l = ctypes.CDLL(SO_PATH)
            for name, (res, args) in SIGNATURES.items():
                f = getattr(l, name, None)
                if f is None:
                    continue  # reported by missing_symbols()
                f.restype = res
                f.argtypes = args
            _LIB = l
    return _LIB


def missing_symbols():
    """Names declared in include/hc.h that libhc.so does not export."""
    l = lib()
    return [n for n in SIGNATURES if getattr(l, n, None) is None]


def check(status: int, what: str = "") -> None:
    if status != HC_OK:
        raise HCError(status, what)


def profile_collect(max_kernels: int = 32):
    """{kernel name: (launches, total device ms)} since the last collect."""
    names = ctypes.create_string_buffer(64 * max_kernels)
    ms = (ctypes.c_double * max_kernels)()
    cnt = (ctypes.c_int * max_kernels)()
    n = lib().hc_profile_collect(names, 64, ms, cnt, max_kernels)
    return {names.raw[64 * i:64 * (i + 1)].split(b"\0")[0].decode(): (int(cnt[i]), float(ms[i]))
            for i in range(n)}


def __getattr__(name):
    if name in SIGNATURES:
        return getattr(lib(), name)
    raise AttributeError(name)
