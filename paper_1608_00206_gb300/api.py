"""torch-facing API over libhc (argument marshalling only).

Tensors supply device memory and the current CUDA stream; every arithmetic
step runs in libhc's kernels.  Shapes: a hypercube over {0,1}^D is any
contiguous tensor of 2^D elements (flat or shaped (2,)*D); results have 3^D
elements, shaped (3,)*D when the input was shaped (2,)*D, flat otherwise.
"""
from __future__ import annotations

import ctypes

import torch

from . import _lib, tuning
from ._lib import HCError, check

_DT = {torch.int64: _lib.HC_INT64, torch.float64: _lib.HC_FP64, torch.float32: _lib.HC_FP32}


def dim_of(t: torch.Tensor) -> int:
    n = t.numel()
    D = n.bit_length() - 1
    if n < 1 or (1 << D) != n:
        raise ValueError(f"a hypercube has 2^D elements; got {n}")
    return D


def _code(dtype: torch.dtype, mixed) -> int:
    """Library dtype code.  mixed: False (the tensor's own arithmetic), True
    (float32 evaluation and products, float-float interpolation) or "ff"
    (every value in float-float); the last two take float32 tensors."""
    if dtype not in _DT:
        raise TypeError(f"unsupported dtype {dtype}; use int64, float64 or float32")
    if mixed:
        if dtype != torch.float32:
            raise TypeError("mixed precision takes float32 inputs")
        if mixed == "ff":
            return _lib.HC_FP32_FF
        if mixed is not True:
            raise ValueError(f"mixed is False, True or 'ff'; got {mixed!r}")
        return _lib.HC_FP32_MIXED
    return _DT[dtype]


def _stream(device: torch.device, stream=None) -> int:
    s = stream if stream is not None else torch.cuda.current_stream(device)
    return s.cuda_stream


def _ptr(t) -> int | None:
    return None if t is None else t.data_ptr()


def _out_shape(x: torch.Tensor, D: int):
    return (3,) * D if (x.dim() == D and all(s == 2 for s in x.shape) and D > 0) else (3 ** D,)


def _schedule(c: int = 0, kmax: int = 0, m: int = 0, cols: int = 0, cols_outer: int = 0,
              bulk: bool = False, top: int = 0, lowmem: bool = False, padded: bool = False):
    """None for the default schedule; else an hc_schedule: top > 0 selects the
    hybrid schedule (direct form on the top axes, c tile axes, kmax axes per
    pass); m > 0 the chunked schedule (c tile axes, m middle axes; bulk=True
    its chunked-bulk variant); otherwise c or kmax the whole-array-pass
    schedule; cols alone keeps the default kind."""
    if top:
        kind = _lib.HC_SCHED_LOWMEM if lowmem else _lib.HC_SCHED_HYBRID
        return _lib.hc_schedule(kind, c, kmax, cols, cols_outer, top)
    if m:
        kind = _lib.HC_SCHED_CHUNKED_BULK if bulk else _lib.HC_SCHED_CHUNKED
        return _lib.hc_schedule(kind, c, m, cols, cols_outer)
    if c or kmax:
        kind = _lib.HC_SCHED_PADDED if padded else _lib.HC_SCHED_PASSES
        return _lib.hc_schedule(kind, c, kmax, cols, cols_outer)
    if cols or cols_outer:
        return _lib.hc_schedule(_lib.HC_SCHED_DEFAULT, 0, 0, cols, cols_outer)
    return None


def workspace_size(D: int, dtype: torch.dtype = torch.float32, mixed: bool = False,
                   c: int = 0, kmax: int = 0, m: int = 0, cols: int = 0,
                   cols_outer: int = 0, bulk: bool = False, top: int = 0,
                   lowmem: bool = False, padded: bool = False) -> int:
    code = _code(dtype, mixed)
    s = _schedule(c, kmax, m, cols, cols_outer, bulk, top, lowmem, padded)
    if s is None:
        # the default schedule is the tuned one once the table is installed
        if torch.cuda.is_available():
            tuning.ensure_installed(torch.device("cuda", torch.cuda.current_device()))
        return int(_lib.lib().hc_workspace_size(D, code))
    return int(_lib.lib().hc_workspace_size_schedule(D, code, ctypes.byref(s)))


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


def _device_convolve(x, y, z, D, code, workspace, stream, sched):
    lib = _lib.lib()
    tuning.ensure_installed(x.device)
    if sched is None:
        nbytes = int(lib.hc_workspace_size(D, code))
    else:
        nbytes = int(lib.hc_workspace_size_schedule(D, code, ctypes.byref(sched)))
    ws = _workspace(nbytes, x.device, workspace)
    st = _stream(x.device, stream)
    if sched is None:
        s = lib.hc_convolve(_ptr(x), _ptr(y), _ptr(z), D, code, _ptr(ws), nbytes, st)
    else:
        s = lib.hc_convolve_schedule(_ptr(x), _ptr(y), _ptr(z), D, code, ctypes.byref(sched),
                                     _ptr(ws), nbytes, st)
    check(s, "hc_convolve")


# Outputs above this size are stored into a page-locked host `out` by the
# final pass instead of being copied after the computation: measured on
# GB300, a 28 GB result (D = 20 int64) reaches the host 5% sooner that way,
# while up to a few GB the copy engine's single copy is faster.
_DIRECT_HOST_BYTES = 8 << 30


def convolve(x: torch.Tensor, y: torch.Tensor, out: torch.Tensor | None = None, *,
             mixed: bool = False, workspace: torch.Tensor | None = None, stream=None,
             c: int = 0, kmax: int = 0, m: int = 0, cols: int = 0,
             cols_outer: int = 0, bulk: bool = False, top: int = 0,
             lowmem: bool = False, padded: bool = False) -> torch.Tensor:
    """z = x * y over {0,1,2}^D.

    mixed: False (the inputs' own arithmetic), True (float32 evaluation and
    products, float-float interpolation) or "ff" (every value in
    float-float, one rounding at the end); the last two take float32.

    CUDA tensors: runs on their device and the current (or given) stream,
    asynchronously.  Schedules: default (hc_convolve); m > 0 selects the
    chunked schedule with m middle axes and c tile axes (bulk=True: the
    chunked-bulk variant); top > 0 the hybrid schedule with that many
    direct-form top axes (with lowmem=True: the low-workspace schedule
    splitting that many top axes leaf by leaf); otherwise c or kmax
    (padded=True: the whole-array passes over a padded, aligned intermediate)
    select the whole-array-pass schedule; cols sets the interpolation tile
    width (cols_outer: that of the pass over the outermost axes).  CPU
    tensors (the end-to-end path): x and y are copied to
    the current CUDA device and convolved there; z is computed on the device
    and copied back into `out` (a new CPU tensor, pinned when x is), except
    that an output above 8 GiB going to a page-locked `out` is stored
    straight into it by the final pass (hc_convolve_out); the call returns
    once z is on the host.
    """
    if x.dtype != y.dtype or x.numel() != y.numel():
        raise ValueError("x and y must have the same dtype and size")
    D = dim_of(x)
    code = _code(x.dtype, mixed)
    sched = _schedule(c, kmax, m, cols, cols_outer, bulk, top, lowmem, padded)
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
        _device_convolve(x, y, out, D, code, workspace, stream, sched)
        return out
    # host buffers: x, y copied to the device; z either stored straight into a
    # page-locked `out` by the final pass (hc_convolve_out, the intermediate
    # in a device array), or computed on the device and copied back
    dev = torch.device("cuda", torch.cuda.current_device())
    xd = x.contiguous().to(dev, non_blocking=True)
    yd = y.contiguous().to(dev, non_blocking=True)
    if out is None:
        out = torch.empty(_out_shape(x, D), dtype=x.dtype, pin_memory=x.is_pinned())
    elif out.numel() != 3 ** D or out.dtype != x.dtype:
        raise ValueError("out must hold 3^D elements of the input dtype")
    zbytes = 3 ** D * x.element_size()
    if sched is None and out.is_pinned() and out.is_contiguous() and zbytes > _DIRECT_HOST_BYTES:
        lib = _lib.lib()
        tuning.ensure_installed(dev)
        nbytes = int(lib.hc_workspace_size(D, code))
        ws = _workspace(nbytes, dev, workspace)
        w = None if mixed else torch.empty(3 ** D, dtype=x.dtype, device=dev)
        check(lib.hc_convolve_out(_ptr(xd), _ptr(yd), _ptr(w), out.data_ptr(), D, code, _ptr(ws),
                                  nbytes, _stream(dev, stream)), "hc_convolve_out")
        torch.cuda.current_stream(dev).synchronize()
        return out
    zd = torch.empty(3 ** D, dtype=x.dtype, device=dev)
    _device_convolve(xd, yd, zd, D, code, workspace, stream, sched)
    out.view(-1).copy_(zd, non_blocking=out.is_pinned())
    torch.cuda.current_stream(dev).synchronize()
    return out


def convolve_backward(dz: torch.Tensor, x: torch.Tensor, y: torch.Tensor, *,
                      need_dx: bool = True, need_dy: bool = True,
                      workspace: torch.Tensor | None = None, stream=None):
    """(dx, dy) for z = x * y and upstream gradient dz (3^D elements), by the
    transposed recurrence; either may be skipped (returned as None)."""
    D = dim_of(x)
    code = _code(x.dtype, False)
    if not (x.is_cuda and y.is_cuda and dz.is_cuda):
        raise ValueError("convolve_backward takes CUDA tensors")
    if dz.numel() != 3 ** D or dz.dtype != x.dtype or y.dtype != x.dtype or y.numel() != x.numel():
        raise ValueError("dz must have 3^D elements and all dtypes must match")
    if not (need_dx or need_dy):
        return None, None
    dz, x, y = dz.contiguous(), x.contiguous(), y.contiguous()
    dx = torch.empty_like(x) if need_dx else None
    dy = torch.empty_like(y) if need_dy else None
    lib = _lib.lib()
    nbytes = int(lib.hc_backward_workspace_size(D, code))
    ws = _workspace(nbytes, x.device, workspace)
    s = lib.hc_convolve_backward(_ptr(dz), _ptr(x), _ptr(y), _ptr(dx), _ptr(dy), D, code,
                                 _ptr(ws), nbytes, _stream(x.device, stream))
    check(s, "hc_convolve_backward")
    return dx, dy


class HypercubeConv(torch.autograd.Function):
    """z = x * y with the hand-written adjoint as its backward.  Only x and y
    are saved; the evaluated operands are recomputed inside the backward
    kernels."""

    @staticmethod
    def forward(ctx, x, y):
        ctx.save_for_backward(x, y)
        return convolve(x, y)

    @staticmethod
    def backward(ctx, gz):
        x, y = ctx.saved_tensors
        dx, dy = convolve_backward(gz.reshape(-1), x, y, need_dx=ctx.needs_input_grad[0],
                                   need_dy=ctx.needs_input_grad[1])
        return dx, dy


def hypercube_conv(x: torch.Tensor, y: torch.Tensor) -> torch.Tensor:
    """Differentiable z = x * y (float32 or float64 CUDA tensors)."""
    return HypercubeConv.apply(x, y)


def packed_offsets(dims, dtype: torch.dtype, base: int = 2):
    """Offsets (elements) of the instances in a packed array of ``base``^D_i
    elements per instance (2: inputs, 3: outputs).  Each offset is rounded up
    to a multiple of 16 bytes, so that every instance's array is 16-byte
    aligned (the library's rule) when the packed array is; returns
    (offsets, total elements)."""
    es = torch.empty((), dtype=dtype).element_size()
    align = max(1, 16 // es)
    offs, o = [], 0
    for D in dims:
        offs.append(o)
        o += -(-(base ** int(D)) // align) * align
    return offs, o


class BatchedConv:
    """A prepared batch of independent convolutions (the batching form).

    ``xs``, ``ys``: sequences of CUDA tensors (2^D_i elements each, one dtype,
    D_i <= 14, or 15 for float32).  The work list is built once
    (hc_batched_prepare); :meth:`launch` runs the whole batch -- instances
    with D <= ``fused_max_d`` in one persistent kernel, the others as
    per-D grouped passes -- and can be captured in a CUDA graph
    (:meth:`capture`), whose replays recompute the batch from the current
    contents of xs, ys.  ``fused_max_d``: None = the library's default,
    "tune" = the batched autotuner's choice (:attr:`fused_max_d` holds it).
    """

    def __init__(self, xs, ys, outs=None, *, mixed: bool = False, stream=None,
                 fused_max_d=None):
        if len(xs) != len(ys):
            raise ValueError("xs and ys differ in length")
        self.n = len(xs)
        dtype = xs[0].dtype if self.n else torch.float32
        self.code = _code(dtype, mixed)
        self.device = xs[0].device if self.n else torch.device("cuda", torch.cuda.current_device())
        self.xs = [x.contiguous() for x in xs]
        self.ys = [y.contiguous() for y in ys]
        self.dims = []
        for x, y in zip(self.xs, self.ys):
            if not (x.is_cuda and y.is_cuda) or x.dtype != dtype or y.dtype != dtype:
                raise ValueError("batched inputs must be CUDA tensors of one dtype")
            if x.numel() != y.numel():
                raise ValueError("x and y of an instance differ in size")
            self.dims.append(dim_of(x))
        if outs is None:
            outs = [torch.empty(_out_shape(x, D), dtype=dtype, device=self.device)
                    for x, D in zip(self.xs, self.dims)]
        self.outs = outs
        arr = (_lib.hc_instance * max(1, self.n))()
        for i, (x, y, z, D) in enumerate(zip(self.xs, self.ys, self.outs, self.dims)):
            arr[i] = _lib.hc_instance(x.data_ptr(), y.data_ptr(), z.data_ptr(), D)
        self._arr = arr
        lib = _lib.lib()
        self.ws_bytes = int(lib.hc_batched_workspace_size(arr, self.n, self.code))
        if self.n and self.ws_bytes == 0:
            raise ValueError("batch rejected (an instance has D out of range or bad buffers)")
        self.workspace = torch.empty(max(self.ws_bytes, 256), dtype=torch.uint8,
                                     device=self.device)
        st = _stream(self.device, stream)
        self.fused_max_d = fused_max_d
        if fused_max_d is None:
            check(lib.hc_batched_prepare(arr, self.n, self.code, self.workspace.data_ptr(),
                                         self.ws_bytes, st), "hc_batched_prepare")
        elif fused_max_d == "tune":
            best, ms = ctypes.c_int(), ctypes.c_double()
            check(lib.hc_batched_autotune(arr, self.n, self.code, self.workspace.data_ptr(),
                                          self.ws_bytes, 3, st, ctypes.byref(best),
                                          ctypes.byref(ms)), "hc_batched_autotune")
            self.fused_max_d, self.tuned_ms = int(best.value), float(ms.value)
        else:
            check(lib.hc_batched_prepare_split(arr, self.n, self.code, int(fused_max_d),
                                               self.workspace.data_ptr(), self.ws_bytes, st),
                  "hc_batched_prepare_split")
        self.graph = None

    def launch(self, stream=None):
        check(_lib.lib().hc_batched_launch(self.workspace.data_ptr(), self.ws_bytes,
                                           _stream(self.device, stream)), "hc_batched_launch")
        return self.outs

    def capture(self):
        """Capture one launch in a CUDA graph (after one eager warm-up launch)."""
        self.launch()
        torch.cuda.synchronize(self.device)
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, capture_error_mode="thread_local"):
            self.launch()
        self.graph = g
        return g

    def replay(self):
        if self.graph is None:
            self.capture()
        self.graph.replay()
        return self.outs

    @classmethod
    def from_packed(cls, x_all: torch.Tensor, y_all: torch.Tensor, dims, *, mixed: bool = False,
                    stream=None, fused_max_d=None):
        """A batch whose instances live back to back in three arrays: x_all and
        y_all (CUDA, 1-D, ``packed_offsets(dims, dtype, 2)`` layout) and the
        outputs in ``self.z_all`` (``packed_offsets(dims, dtype, 3)``), so that
        a whole batch moves between host and device in one copy per array
        (:meth:`run_host`)."""
        dims = [int(D) for D in dims]
        dtype = x_all.dtype
        xo, nx = packed_offsets(dims, dtype, 2)
        zo, nz = packed_offsets(dims, dtype, 3)
        if x_all.dim() != 1 or y_all.shape != x_all.shape or y_all.dtype != dtype \
                or x_all.numel() < nx:
            raise ValueError("x_all, y_all must be 1-D arrays of one dtype in the packed layout")
        xs = [x_all[o:o + (1 << D)] for o, D in zip(xo, dims)]
        ys = [y_all[o:o + (1 << D)] for o, D in zip(xo, dims)]
        z_all = torch.empty(max(nz, 1), dtype=dtype, device=x_all.device)
        outs = [z_all[o:o + 3 ** D] for o, D in zip(zo, dims)]
        self = cls(xs, ys, outs, mixed=mixed, stream=stream, fused_max_d=fused_max_d)
        self.x_all, self.y_all, self.z_all = x_all, y_all, z_all
        return self

    def run_host(self, xh: torch.Tensor, yh: torch.Tensor, zh: torch.Tensor) -> torch.Tensor:
        """One batch from page-locked host arrays in the packed layout of a
        :meth:`from_packed` batch: copy x and y in, replay the captured batch,
        copy z out (one copy each, on the current stream), then synchronise."""
        if not hasattr(self, "z_all"):
            raise ValueError("run_host needs a batch made by BatchedConv.from_packed")
        if xh.shape != self.x_all.shape or yh.shape != self.y_all.shape or \
                zh.shape != self.z_all.shape:
            raise ValueError("host arrays must have the packed shapes of x_all, y_all, z_all")
        self.x_all.copy_(xh, non_blocking=True)
        self.y_all.copy_(yh, non_blocking=True)
        self.replay()
        zh.copy_(self.z_all, non_blocking=True)
        torch.cuda.current_stream(self.device).synchronize()
        return zh

    def status(self) -> int:
        """Synchronises and returns the workspace status word (0 = HC_OK)."""
        return int(_lib.lib().hc_device_status(self.workspace.data_ptr(),
                                               _stream(self.device, None)))

    def inject_stall(self, instance: int):
        check(_lib.lib().hc_batched_inject_stall(self.workspace.data_ptr(), instance),
              "hc_batched_inject_stall")


def convolve_batched(xs, ys, outs=None, *, mixed: bool = False, stream=None, fused_max_d=None):
    """All instances in one batched launch sequence; returns the list of outputs."""
    b = BatchedConv(xs, ys, outs, mixed=mixed, stream=stream, fused_max_d=fused_max_d)
    return b.launch(stream)


def carry_free_convolve(x: torch.Tensor, y: torch.Tensor, *, mixed: bool = False,
                        workspace: torch.Tensor | None = None, stream=None) -> torch.Tensor:
    """1D carry-free convolution of two length-N CUDA vectors (paper,
    Discussion; hc_carryfree): z[k] = sum of x[i] * y[j] over the pairs whose
    bitwise, carry-free sum is k, i.e. the base-3 digits of k are
    bit_d(i) + bit_d(j), with D = ceil(log2 N) digits.  N need not be a power
    of two: the library zero-pads both vectors to 2^D on the device.  z has
    3^D entries.  Example: i = 7 = (1,1,1), j = 5 = (1,0,1) lands in
    (2,1,2) = 23."""
    if x.dim() != 1 or y.dim() != 1:
        raise ValueError("carry-free convolution takes 1D vectors")
    if x.dtype != y.dtype or x.numel() != y.numel() or x.numel() < 1:
        raise ValueError("x and y must be non-empty and have the same dtype and length")
    if not (x.is_cuda and y.is_cuda and x.device == y.device):
        raise ValueError("carry-free convolution takes CUDA tensors on one device")
    N = x.numel()
    D = (N - 1).bit_length()
    code = _code(x.dtype, mixed)
    x, y = x.contiguous(), y.contiguous()
    z = torch.empty(3 ** D, dtype=x.dtype, device=x.device)
    lib = _lib.lib()
    tuning.ensure_installed(x.device)
    nbytes = int(lib.hc_carryfree_workspace_size(N, code))
    ws = _workspace(nbytes, x.device, workspace)
    check(lib.hc_carryfree(_ptr(x), _ptr(y), _ptr(z), N, code, _ptr(ws), nbytes,
                           _stream(x.device, stream)), "hc_carryfree")
    return z


def maxconv_plan(D: int, vmax: int) -> dict:
    """The library's plan for max-convolution of (D, vmax) (hc_maxconv_plan):
    p, limb width b, limb axes e and limb count L.  Raises HCError when no
    plan exists."""
    p, b, e, L = (ctypes.c_int() for _ in range(4))
    check(_lib.lib().hc_maxconv_plan(int(D), int(vmax), ctypes.byref(p), ctypes.byref(b),
                                     ctypes.byref(e), ctypes.byref(L)), "hc_maxconv_plan")
    return {"p": p.value, "b": b.value, "e": e.value, "L": L.value}


def maxconv_workspace_size(D: int, vmax: int) -> int:
    """Bytes of workspace hc_maxconv needs for (D, vmax) with the default
    (tuned, once installed) int64 schedule; 0 when no plan exists."""
    if torch.cuda.is_available():
        tuning.ensure_installed(torch.device("cuda", torch.cuda.current_device()))
    return int(_lib.lib().hc_maxconv_workspace_size(int(D), int(vmax)))


def maxconv(x: torch.Tensor, y: torch.Tensor, vmax: int, out: torch.Tensor | None = None, *,
            workspace: torch.Tensor | None = None, stream=None) -> torch.Tensor:
    """Max-convolution of int64 CUDA hypercubes with entries in [0, vmax]
    (paper, Discussion; hc_maxconv): z[k] = max of x[i] * y[j] over the pairs
    i + j = k, exact, through the p-norm ring (sums of p-th powers in limbs,
    one int64 convolution of D + e axes, nearest integer p-th roots).  Entries
    outside [0, vmax] are reported by :func:`device_status` on the workspace
    (HC_ERR_ARG) when a workspace is passed in, and make z unspecified."""
    if x.dtype != torch.int64 or y.dtype != torch.int64:
        raise TypeError("max-convolution takes int64 tensors")
    if not (x.is_cuda and y.is_cuda and x.device == y.device):
        raise ValueError("max-convolution takes CUDA tensors on one device")
    if x.numel() != y.numel():
        raise ValueError("x and y differ in length")
    D = dim_of(x)
    x, y = x.contiguous(), y.contiguous()
    if out is None:
        out = torch.empty(_out_shape(x, D), dtype=torch.int64, device=x.device)
    lib = _lib.lib()
    tuning.ensure_installed(x.device)
    nbytes = int(lib.hc_maxconv_workspace_size(D, int(vmax)))
    if nbytes == 0:
        raise _lib.HCError(_lib.HC_ERR_ARG, f"hc_maxconv: no plan for D={D}, vmax={vmax}")
    ws = _workspace(nbytes, x.device, workspace)
    check(lib.hc_maxconv(_ptr(x), _ptr(y), _ptr(out), D, int(vmax), _ptr(ws), nbytes,
                         _stream(x.device, stream)), "hc_maxconv")
    return out


def device_status(workspace: torch.Tensor, stream=None) -> int:
    """The status word a kernel recorded in `workspace` (hc_device_status;
    synchronises the stream)."""
    return int(_lib.lib().hc_device_status(_ptr(workspace), _stream(workspace.device, stream)))
