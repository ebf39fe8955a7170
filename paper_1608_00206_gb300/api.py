"""torch-facing API over libhc (argument marshalling only).

Tensors supply device memory and the current CUDA stream; every arithmetic
step runs in libhc's kernels.  Shapes: a hypercube over {0,1}^D is any
contiguous tensor of 2^D elements (flat or shaped (2,)*D); results have 3^D
elements, shaped (3,)*D when the input was shaped (2,)*D, flat otherwise.
"""
from __future__ import annotations

import ctypes

import torch

from . import _lib
from ._lib import HCError, check

_DT = {torch.int64: _lib.HC_INT64, torch.float64: _lib.HC_FP64, torch.float32: _lib.HC_FP32}


def dim_of(t: torch.Tensor) -> int:
    n = t.numel()
    D = n.bit_length() - 1
    if n < 1 or (1 << D) != n:
        raise ValueError(f"a hypercube has 2^D elements; got {n}")
    return D


def _code(dtype: torch.dtype, mixed: bool) -> int:
    if dtype not in _DT:
        raise TypeError(f"unsupported dtype {dtype}; use int64, float64 or float32")
    if mixed:
        if dtype != torch.float32:
            raise TypeError("mixed precision takes float32 inputs")
        return _lib.HC_FP32_MIXED
    return _DT[dtype]


def _stream(device: torch.device, stream=None) -> int:
    s = stream if stream is not None else torch.cuda.current_stream(device)
    return s.cuda_stream


def _ptr(t) -> int | None:
    return None if t is None else t.data_ptr()


def _out_shape(x: torch.Tensor, D: int):
    return (3,) * D if (x.dim() == D and all(s == 2 for s in x.shape) and D > 0) else (3 ** D,)


def workspace_size(D: int, dtype: torch.dtype = torch.float32, mixed: bool = False,
                   c: int = 0, kmax: int = 0) -> int:
    code = _code(dtype, mixed)
    if c or kmax:
        return int(_lib.lib().hc_workspace_size_config(D, code, c, kmax))
    return int(_lib.lib().hc_workspace_size(D, code))


def backward_workspace_size(D: int, dtype: torch.dtype = torch.float32) -> int:
    return int(_lib.lib().hc_backward_workspace_size(D, _code(dtype, False)))


def _workspace(nbytes: int, device, workspace):
    if nbytes == 0:
        return None
    if workspace is not None:
        if workspace.numel() * workspace.element_size() < nbytes:
            raise ValueError(f"workspace has {workspace.numel() * workspace.element_size()} "
                             f"bytes; {nbytes} needed")
        return workspace
    return torch.empty(nbytes, dtype=torch.uint8, device=device)


def _device_convolve(x, y, z, D, code, workspace, stream, c, kmax):
    lib = _lib.lib()
    if c or kmax:
        nbytes = int(lib.hc_workspace_size_config(D, code, c, kmax))
    else:
        nbytes = int(lib.hc_workspace_size(D, code))
    ws = _workspace(nbytes, x.device, workspace)
    st = _stream(x.device, stream)
    if c or kmax:
        s = lib.hc_convolve_config(_ptr(x), _ptr(y), _ptr(z), D, code, c, kmax, _ptr(ws),
                                   nbytes, st)
    else:
        s = lib.hc_convolve(_ptr(x), _ptr(y), _ptr(z), D, code, _ptr(ws), nbytes, st)
    check(s, "hc_convolve")


def convolve(x: torch.Tensor, y: torch.Tensor, out: torch.Tensor | None = None, *,
             mixed: bool = False, workspace: torch.Tensor | None = None, stream=None,
             c: int = 0, kmax: int = 0) -> torch.Tensor:
    """z = x * y over {0,1,2}^D.

    CUDA tensors: runs on their device and the current (or given) stream,
    asynchronously.  CPU tensors (the end-to-end path): x and y are copied to
    the current CUDA device, convolved there, and z is copied back into `out`
    (or a new CPU tensor, pinned if x is pinned); the call returns once z is
    on the host.
    """
    if x.dtype != y.dtype or x.numel() != y.numel():
        raise ValueError("x and y must have the same dtype and size")
    D = dim_of(x)
    code = _code(x.dtype, mixed)
    if x.is_cuda:
        if not y.is_cuda or y.device != x.device:
            raise ValueError("x and y must be on the same CUDA device")
        x = x.contiguous()
        y = y.contiguous()
        if out is None:
            out = torch.empty(_out_shape(x, D), dtype=x.dtype, device=x.device)
        elif not (out.is_cuda and out.is_contiguous() and out.numel() == 3 ** D and
                  out.dtype == x.dtype):
            raise ValueError("out must be a contiguous CUDA tensor of 3^D elements, same dtype")
        _device_convolve(x, y, out, D, code, workspace, stream, c, kmax)
        return out
    # host buffers: explicit copies around the device call
    dev = torch.device("cuda", torch.cuda.current_device())
    xd = x.contiguous().to(dev, non_blocking=True)
    yd = y.contiguous().to(dev, non_blocking=True)
    zd = torch.empty(3 ** D, dtype=x.dtype, device=dev)
    _device_convolve(xd, yd, zd, D, code, workspace, stream, c, kmax)
    if out is None:
        out = torch.empty(_out_shape(x, D), dtype=x.dtype, pin_memory=x.is_pinned())
    out.view(-1).copy_(zd, non_blocking=out.is_pinned())
    torch.cuda.current_stream(dev).synchronize()
    return out
