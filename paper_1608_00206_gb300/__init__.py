"""GB300-native exact convolution of D-dimensional hypercubes (arXiv 1608.00206).

The compute path is libhc.so (hand-written sm_103a CUDA behind the C ABI of
``include/hc.h``).  This package is a thin layer over it: ``_lib`` is the
ctypes binding (same names as the C functions), ``api`` marshals torch
tensors (device memory, streams) into those calls.  There is no CPU fallback:
every entry point raises if the library is missing or a tensor is not on a
CUDA device (host tensors are copied to the device and back explicitly).
"""
from . import inputs  # noqa: F401  (numpy-only input generators)

__all__ = ["inputs", "convolve", "convolve_backward", "convolve_batched", "BatchedConv",
           "hypercube_conv", "HypercubeConv", "workspace_size", "carry_free_convolve", "packed_offsets",
           "maxconv", "maxconv_plan", "maxconv_workspace_size", "device_status", "build"]


def __getattr__(name):
    if name in ("convolve", "convolve_backward", "convolve_batched", "BatchedConv",
                "hypercube_conv", "HypercubeConv", "workspace_size", "backward_workspace_size",
                "dim_of", "HCError", "carry_free_convolve", "packed_offsets", "maxconv",
                "maxconv_plan", "maxconv_workspace_size", "device_status"):
        from . import api
        return getattr(api, name)
    if name == "build":
        from .build import build
        return build
    raise AttributeError(name)
