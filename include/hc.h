/*
 * hc.h -- C ABI of libhc, exact convolution of D-dimensional hypercubes on
 * NVIDIA GB300 (sm_103a).
 *
 * The operation (Introduction of Serang, arXiv 1608.00206):
 *     (x * y)[k] = sum over i + j = k of x[i] * y[j],
 * for x, y over {0,1}^D and z = x * y over {0,1,2}^D.  It is computed with the
 * Methods-section recurrence -- per axis, z[0] = x[0]*y[0], z[2] = x[1]*y[1],
 * z[1] = ((x[0]+x[1])*(y[0]+y[1]) - z[0]) - z[2] -- in O(D 3^D) operations
 * instead of the O(4^D) of Algorithm 1.
 *
 * Layout (Methods, "tensors are stored in row-major format"):
 *   x, y : 2^D elements, row-major, axis 1 slowest (x[i_1] is the first or
 *          second half of the flat array).
 *   z    : 3^D elements, row-major, axis 1 slowest: digit k_d of axis d has
 *          weight 3^(D-d).  The carry-free example of the Discussion --
 *          bits (1,1,1) + (1,0,1) -> digits (2,1,2) -- is flat index 23.
 *
 * Arithmetic:
 *   HC_INT64      int64 in and out, computed in Z/2^64 (two's-complement
 *                 wrap).  Exact whenever the true result fits in int64; the
 *                 paper calls the method exact when (a + b) - a = b.
 *   HC_FP64       float64 in and out.
 *   HC_FP32       float32 in and out.
 *   HC_FP32_MIXED float32 in and out; evaluation (sums) and products in
 *                 float32, the cancelling interpolation (t - z[0]) - z[2] in
 *                 float-float (error-free two-sum), one rounding at the end.
 *   HC_FP32_FF    float32 in and out; every value of the recurrence in
 *                 float-float: evaluation by two-sum, products by the FMA
 *                 two-product (the exact error of the binary32 product)
 *                 plus the cross terms, interpolation by two-sum; one
 *                 rounding to float32 at the end.  On integer-valued inputs
 *                 whose intermediates stay within float-float's 48 bits this
 *                 is the exact result rounded once.  Plain and
 *                 differentiation-free: hc_convolve, its schedules,
 *                 hc_convolve_out (w NULL), hc_convolve_noalloc and
 *                 hc_carryfree take it; the batched and differentiation
 *                 forms return HC_ERR_DTYPE.
 *   For every floating-point dtype the library applies the per-axis
 *   operations in the recurrence's own order (evaluation axis 1 first,
 *   interpolation axis D first) with no fused multiply-add, so results are
 *   bitwise identical to the recurrence evaluated sequentially in the same
 *   precision.  The forward error of each output is bounded by
 *   gamma_{3D+1} * zabs, zabs being the recurrence on |x|, |y| with every
 *   subtraction turned into an addition.
 *
 * Conventions common to every call:
 *   - All data pointers are DEVICE memory owned by the caller, 16-byte
 *     aligned (HC_ERR_ALIGN otherwise).  The library allocates nothing.
 *   - Inputs (x, y, dz) are const and never modified (unlike the paper's
 *     in-place listing, whose caption warns that x and y are overwritten).
 *   - Outputs are fully overwritten and must not overlap any input or the
 *     workspace (HC_ERR_ALIAS).
 *   - 0 <= D <= HC_MAX_D (HC_ERR_ARG otherwise).  D = 0 gives z[0] = x[0]*y[0].
 *   - workspace: device memory of at least the queried size, 256-byte
 *     aligned; NULL is allowed when the queried size is 0.  It holds
 *     intermediates and a status word; its contents need no initialisation.
 *   - Calls are asynchronous on `stream` (NULL = the legacy default stream):
 *     they validate arguments, enqueue kernels and return without a host
 *     synchronisation.  HC_ERR_CUDA reports a launch failure;
 *     hc_last_cuda_error() gives CUDA's message.
 *   - Calls with different workspaces may run concurrently on different
 *     streams.  Calls sharing a workspace must be stream-ordered.
 */
#ifndef HC_H_
#define HC_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Same type as cudaStream_t; declared here so this header needs no CUDA header. */
typedef struct CUstream_st* hc_stream_t;

typedef enum {
  HC_INT64 = 0,
  HC_FP64 = 1,
  HC_FP32 = 2,
  HC_FP32_MIXED = 3,
  HC_FP32_FF = 4
} hc_dtype;

typedef enum {
  HC_OK = 0,
  HC_ERR_ARG = 1,       /* bad D, NULL pointer, n < 0, unknown flag          */
  HC_ERR_DTYPE = 2,     /* unknown or unsupported dtype for this call        */
  HC_ERR_ALIGN = 3,     /* pointer not 16-byte (workspace: 256-byte) aligned */
  HC_ERR_ALIAS = 4,     /* an output overlaps an input or the workspace      */
  HC_ERR_WORKSPACE = 5, /* workspace smaller than the queried size           */
  HC_ERR_CUDA = 6,      /* a CUDA call failed; see hc_last_cuda_error()      */
  HC_ERR_TIMEOUT = 7    /* a bounded device-side wait gave up (batched form) */
} hc_status;

#define HC_MAX_D 24

/* Library version, (major << 16) | (minor << 8) | patch. */
int hc_version(void);

const char* hc_status_string(hc_status s);

/* CUDA's message for the most recent HC_ERR_CUDA on the calling thread. */
const char* hc_last_cuda_error(void);

/* ------------------------------------------------------------------------
 * Plain form.
 *
 * hc_workspace_size: bytes of workspace hc_convolve needs for (D, dtype);
 * returns 0 for an invalid (D, dtype) as well as when none is needed.
 *
 * hc_convolve: z = x * y.  x, y: 2^D elements; z: 3^D elements; all of the
 * dtype's element type (int64, double or float; float for HC_FP32_MIXED).
 * z may be a plain device allocation or managed memory: the call asks the
 * runtime (cudaPointerGetAttributes) which one it is, and only into a plain
 * device allocation are whole tiles stored with bulk (TMA engine) copies;
 * the results are the same bits either way.
 */
size_t hc_workspace_size(int D, hc_dtype dtype);

hc_status hc_convolve(const void* x, const void* y, void* z, int D, hc_dtype dtype,
                      void* workspace, size_t ws_bytes, hc_stream_t stream);

/* ------------------------------------------------------------------------
 * Schedules.  Every schedule computes the same bits; they differ in how the
 * D axes are split between shared-memory tiles and passes over HBM.
 *   HC_SCHED_PASSES  : whole-array passes evaluate the D - c outer axes, one
 *                      tile kernel handles the c inner axes (evaluation,
 *                      products, interpolation), whole-array passes
 *                      interpolate the outer axes, at most k per pass.
 *   HC_SCHED_CHUNKED : one persistent launch convolves chunks of c + k axes
 *                      (tiles of c axes, then the k middle axes interpolated
 *                      while the chunk is in L2); the D - c - k outer axes go
 *                      through whole-array passes.  D <= c + k: one launch.
 *   HC_SCHED_CHUNKED_BULK : CHUNKED with every middle axis evaluated by the
 *                      whole-array passes (workspace as for PASSES with c + k
 *                      tile axes), so that the persistent launch reads plain
 *                      rows; each tile leaves shared memory in one bulk (TMA
 *                      engine) copy that L2 keeps (evict_last priority) until
 *                      the chunk's middle axes are interpolated, and finished
 *                      columns are stored with evict_first priority.  An
 *                      intermediate in managed or host-mapped memory, or c
 *                      other than 7 or 8, runs the CHUNKED kernel on the
 *                      same plan (same bits).
 *   HC_SCHED_HYBRID  : the 4-way direct form on the top `top` axes (1..6):
 *                      for each digit string of those axes the tile sums the
 *                      products of the x and y sub-cube pairs that add up to
 *                      it (Methods: z[1] = x[0]*y[1] + x[1]*y[0], no
 *                      interpolation on that axis), then the Karatsuba form
 *                      on the D - top axes below (c tile axes, at most 8; the
 *                      middle axes in whole-array passes of at most k).
 *                      (4/3)^top times the evaluation and product work of
 *                      the other schedules, `top` fewer axes to interpolate
 *                      over HBM.  HC_INT64, HC_FP64 and HC_FP32 only.  Its
 *                      floating-point results are bitwise those of this
 *                      hybrid form (pairs summed in increasing x index),
 *                      which differ from the plain recurrence's rounding;
 *                      int64 results are Algorithm 1's.  HC_ERR_ARG when
 *                      D - top < 4.  Because its rounding differs, the
 *                      autotuner considers it for HC_INT64 only, and a
 *                      floating-point default schedule is never hybrid.
 *   HC_SCHED_LOWMEM  : the low-workspace form of the paper's recursion: the
 *                      top `top` axes (1..6) are split one leaf at a time --
 *                      for each of their 3^top digit strings a small kernel
 *                      sums the input sub-cubes that the digits select (the
 *                      leaf's evaluated inputs, 2^(D - top) elements each)
 *                      and the leaf, a convolution of D - top axes, runs
 *                      the PASSES schedule (c, k, per-element row copies)
 *                      into z's slice -- then passes of at most k axes
 *                      (width cols_outer) interpolate the top axes.
 *                      Workspace: the two leaf inputs (2^(D - top) each)
 *                      and one leaf's own workspace (its operands evaluated
 *                      on its D - top - c outer axes) -- a few MB at D = 20
 *                      with top = 6, against the gigabytes of the other
 *                      schedules.  Same bits as every other schedule;
 *                      3^top leaves of about five launches each.  HC_INT64,
 *                      HC_FP64 and HC_FP32 only; HC_ERR_ARG when D <= top.
 *   HC_SCHED_PADDED  : PASSES with the intermediate kept in the workspace
 *                      with each tile's 3^c outputs padded to a multiple of
 *                      128 bytes, so that every row the passes read and write
 *                      starts on a 128-byte boundary (z's own rows, 3^n
 *                      elements apart, start at every 8-byte offset); the
 *                      pass over the outermost axes writes z's layout.  The
 *                      workspace then holds 3^(D-c) padded tiles (about the
 *                      size of z) besides the PASSES operands.  Same bits.
 *                      Measured on GB300 it loses to PASSES (the aligned
 *                      inner pass gains 15%, the last pass, out of place
 *                      into z's unaligned rows, takes more than twice as
 *                      long), so the autotuner does not offer it.
 *   HC_SCHED_DEFAULT : the per-(D, dtype) default (built in: CHUNKED with
 *                      default sizes; replaced by hc_set_default_schedule,
 *                      typically with hc_autotune's winner).
 * Fields: c in 0..9 for HC_FP32, 0..8 otherwise (0 = the largest; clamped to
 * D); k in 0..6 (0 = 6); cols = columns per whole-array interpolation tile,
 * 8, 16 or 32, each element copied on its own (0 = 32 for 4-byte and 16 for
 * 8-byte intermediates), or -16 / -32: 16 or 32 columns whose rows are copied
 * in 16-byte pieces (each row widened to 16-byte boundaries).  cols_outer:
 * the same choice for the whole-array pass over the outermost axes alone
 * (its rows are the farthest apart; 0 = cols).  The adjoint's transposed
 * passes take the default schedule's widths for the same (D, dtype).
 * HC_ERR_ARG for fields out of range. */
#define HC_SCHED_DEFAULT 0
#define HC_SCHED_PASSES 1
#define HC_SCHED_CHUNKED 2
#define HC_SCHED_CHUNKED_BULK 3
#define HC_SCHED_HYBRID 4
#define HC_SCHED_LOWMEM 5
#define HC_SCHED_PADDED 6

typedef struct {
  int kind;
  int c;
  int k;
  int cols;
  int cols_outer;  /* width of the pass over the outermost axes; 0 = cols */
  int top;         /* HC_SCHED_HYBRID: direct-form top axes; HC_SCHED_LOWMEM:
                      top axes split leaf by leaf; 0 for the other kinds */
} hc_schedule;

size_t hc_workspace_size_schedule(int D, hc_dtype dtype, const hc_schedule* s);

hc_status hc_convolve_schedule(const void* x, const void* y, void* z, int D, hc_dtype dtype,
                               const hc_schedule* s, void* workspace, size_t ws_bytes,
                               hc_stream_t stream);

/* The schedule hc_convolve and hc_workspace_size use for (D, dtype);
 * s = NULL restores the built-in choice.  Process-wide, thread-safe; a
 * workspace sized before a change may no longer be large enough.
 * HC_ERR_ARG for a hybrid schedule with a floating-point dtype (a default
 * never changes the recurrence's rounding). */
hc_status hc_set_default_schedule(int D, hc_dtype dtype, const hc_schedule* s);

hc_status hc_get_default_schedule(int D, hc_dtype dtype, hc_schedule* s);

/* Autotuner: runs every candidate schedule for (D, dtype) on the caller's
 * buffers (x, y inputs; z output, overwritten; workspace of at least
 * hc_autotune_workspace_size bytes), `reps` timed runs each after one
 * warm-up, on `stream` with CUDA events (synchronising), and returns the
 * fastest in *best and its best time in *best_ms.  It does not install the
 * winner (see hc_set_default_schedule). */
size_t hc_autotune_workspace_size(int D, hc_dtype dtype);

hc_status hc_autotune(const void* x, const void* y, void* z, int D, hc_dtype dtype,
                      void* workspace, size_t ws_bytes, int reps, hc_stream_t stream,
                      hc_schedule* best, double* best_ms);

/* ------------------------------------------------------------------------
 * Separate output.  hc_convolve interpolates in place in z, so every pass
 * reads and writes it.  hc_convolve_out keeps that 3^D intermediate in `w`
 * (device memory, 3^D elements of the dtype, 16-byte aligned, overlapping
 * nothing else; NULL and unused for HC_FP32_MIXED, whose intermediate is in
 * the workspace) and writes z once, with the final stores: z may then be
 * any memory the device can store to, e.g. page-locked host memory, so the
 * result leaves the GPU while it is being computed, without a separate
 * copy.  Same schedule, workspace and bits as hc_convolve.  HC_ERR_ARG if w
 * is NULL for an exact or float dtype, or given for HC_FP32_MIXED;
 * HC_ERR_ALIAS if w overlaps x, y, z or the workspace; HC_ERR_ARG, before
 * anything is launched, if z is not device, managed or page-locked host
 * memory mapped at its own address, or w is not device or managed memory
 * (checked with cudaPointerGetAttributes, so the pointers must be known to
 * the CUDA runtime). */
hc_status hc_convolve_out(const void* x, const void* y, void* w, void* z, int D, hc_dtype dtype,
                          void* workspace, size_t ws_bytes, hc_stream_t stream);

/* ------------------------------------------------------------------------
 * Carry-free 1D convolution (Discussion: "carry-free convolution" solved by
 * embedding into a hypercube).  For vectors x, y of N >= 1 elements:
 *     z[k] = sum of x[i] * y[j] over the pairs (i, j) whose bits, added
 *            position by position without carries, give the base-3 digits
 *            of k,
 * with D = ceil(log2 N) digits (D = 0 for N = 1), most significant first.
 * Example (Discussion): i = 7 = (1,1,1), j = 5 = (1,0,1) contribute to
 * digits (2,1,2), z[23], not to the carried sum 12.  Reading bit d of an
 * index as axis d, this is hc_convolve of x and y zero-padded to 2^D
 * elements, which is how it is computed: a library kernel writes the padded
 * copies into the workspace, then the plain form runs on them (same
 * schedule, kernels and bits as hc_convolve).
 *   x, y : N elements of the dtype's type, device memory, 16-byte aligned;
 *          const.
 *   z    : 3^D elements, fully overwritten; entries whose digits no pair
 *          reaches (possible when N < 2^D) are zero.
 *   workspace: hc_carryfree_workspace_size(N, dtype) bytes, 256-byte aligned
 *          (for N a power of two this is hc_workspace_size(D, dtype) and no
 *          copy is made).
 * Errors: HC_ERR_ARG for N = 0, D > HC_MAX_D or a NULL pointer; the plain
 * form's alignment, aliasing and workspace rules otherwise.
 * hc_carryfree_workspace_size returns 0 for an invalid (N, dtype). */
size_t hc_carryfree_workspace_size(size_t N, hc_dtype dtype);

hc_status hc_carryfree(const void* x, const void* y, void* z, size_t N, hc_dtype dtype,
                       void* workspace, size_t ws_bytes, hc_stream_t stream);

/* ------------------------------------------------------------------------
 * Max-convolution of bounded non-negative integers (Discussion: p-norm rings
 * make max-convolution on hypercubes of integers with bounded dynamic range
 * exact once p is large enough and the p-norm estimates are rounded to the
 * nearest integer).  For x, y over {0,1}^D with every entry in [0, vmax]:
 *     z[k] = max of x[i] * y[j] over the pairs i + j = k,
 * all int64, same layouts as hc_convolve.  Method: with M = vmax^2 and p the
 * smallest integer for which M (2^(D/p) - 1) < 7/16 (the paper's error
 * bound below 1/2, kept 1/16 away from it for the floating-point root),
 * s[k] = sum over the pairs of (x[i] y[j])^p is computed exactly -- v^p in
 * limbs of b bits, the limb index on e extra axes, one HC_INT64 convolution
 * of D + e axes (every entry below 2^63) -- and z[k] is the integer nearest
 * s[k]^(1/p), which the bound makes the maximum.
 *   hc_maxconv_plan: p, the limb width b, the limb axes e and the limb count
 *     L for (D, vmax); HC_ERR_ARG when no plan exists: D or vmax out of range
 *     (vmax in 0 .. 2^31 - 1, and at most 2^19 unless p = 1, since for p > 1
 *     the root is taken in double precision), p above 2^24, more than 12
 *     limb axes, or D + e > HC_MAX_D.  Any output pointer may be NULL.
 *   hc_maxconv_workspace_size: bytes of workspace (0 when no plan exists):
 *     the power table, the two limb cubes (2^(D+e) int64 each), the
 *     3^(D+e) int64 convolution and that convolution's own workspace (the
 *     default HC_INT64 schedule's, so a schedule installed with
 *     hc_set_default_schedule changes it).
 *   hc_maxconv: x, y (2^D int64, const), z (3^D int64, overwritten); the
 *     plain form's alignment, aliasing and workspace rules.  The call clears
 *     the workspace status word on `stream`; an entry outside [0, vmax] is
 *     recorded there as HC_ERR_ARG (read it with hc_device_status), and z is
 *     then unspecified.  Cost: 3^(D+e) outputs of the int64 convolution for
 *     3^D results -- the price of exactness beyond 64 bits.
 */
hc_status hc_maxconv_plan(int D, int64_t vmax, int* p, int* limb_bits, int* limb_axes,
                          int* limbs);

size_t hc_maxconv_workspace_size(int D, int64_t vmax);

hc_status hc_maxconv(const int64_t* x, const int64_t* y, int64_t* z, int D, int64_t vmax,
                     void* workspace, size_t ws_bytes, hc_stream_t stream);

/* ------------------------------------------------------------------------
 * No-allocation form.  The paper has no counterpart: this entry point exists
 * for callers that must not allocate device memory at the call site -- code
 * running while another framework owns the device's memory pool,
 * latency-critical loops that cannot afford the device-wide synchronisation
 * that cudaMalloc and cudaFree imply, or plugin hosts that forbid allocation
 * once set up.  It computes exactly what hc_convolve computes, under the same
 * argument rules, but takes no workspace: it works in a fixed array of
 * HC_NOALLOC_SCRATCH_BYTES in the library's own device memory and calls no
 * allocating routine.
 *   - It always uses the built-in chunked schedule (whatever default schedule
 *     is installed).  Limit: a problem whose workspace for that schedule
 *     exceeds the array is refused with HC_ERR_WORKSPACE.  With 16 MiB that allows D <= 16 for HC_INT64
 *     and HC_FP64, D <= 17 for HC_FP32 and D <= 13 for HC_FP32_MIXED and
 *     HC_FP32_FF.
 *   - Set-up happens in the first call on each device (in each CUDA
 *     context): that call loads the library's device code for this entry
 *     point onto the GPU, which allocates the array there, and looks up the
 *     array's device address with that device current.  Make this first call
 *     during set-up -- before any stream capture and before any region in
 *     which allocation is forbidden; every later call in the same context
 *     allocates nothing.  The GPU then holds the array until the process
 *     exits.  After a device reset (cudaDeviceReset, or a primary context
 *     released and created again) the next call does the set-up again.
 *   - All calls on one device share the array, which keeps whatever the last
 *     call left there; the counters that must start at zero are cleared by
 *     each call itself, on its stream, before its kernels run.  Calls whose work
 *     overlaps on the GPU -- issued on different streams or from different
 *     threads without ordering between them -- race on it and produce wrong
 *     results; order them on one stream or with events.
 */
#define HC_NOALLOC_SCRATCH_BYTES ((size_t)16 << 20)

hc_status hc_convolve_noalloc(const void* x, const void* y, void* z, int D, hc_dtype dtype,
                              hc_stream_t stream);

/* ------------------------------------------------------------------------
 * Differentiation form.  For z = x * y and an upstream gradient dz = dL/dz
 * (3^D elements):
 *     dx[i] = sum_j dz[i + j] * y[j],     dy[j] = sum_i dz[i + j] * x[i],
 * computed as the transpose of the recurrence, dx = E^T (I^T dz (.) E y),
 * with per-axis I^T: (g0, g1, g2) -> (g0 - g1, g1, g2 - g1) and
 * E^T: (h0, h1, h2) -> (h0 + h1, h1 + h2).  The evaluated operands E x and
 * E y are recomputed tile by tile, never stored.  Either dx or dy may be
 * NULL to skip it.  HC_FP32_MIXED is not supported here (HC_ERR_DTYPE).
 */
size_t hc_backward_workspace_size(int D, hc_dtype dtype);

hc_status hc_convolve_backward(const void* dz, const void* x, const void* y, void* dx,
                               void* dy, int D, hc_dtype dtype, void* workspace,
                               size_t ws_bytes, hc_stream_t stream);

/* ------------------------------------------------------------------------
 * Batching form: n independent convolutions of possibly different D, one
 * persistent kernel launch.  The instance array is HOST memory; its device
 * pointers follow the plain-form rules, and no output may overlap another
 * instance's buffers (not checked across instances).
 *
 * Each instance has 0 <= D <= 14 (15 for HC_FP32): the tile axes plus at
 * most six outer axes (HC_ERR_ARG otherwise; larger D go to hc_convolve).
 *
 * hc_convolve_batched = hc_batched_prepare + hc_batched_launch.
 * hc_batched_prepare builds the work list on the host, copies it into the
 * workspace and synchronises `stream` (so it cannot be captured; the host
 * array may be reused on return).  It remembers the plan under the workspace
 * address for later launches.  It also asks the runtime once per instance
 * whether its output (its intermediate, for the grouped form) is a plain
 * device allocation; the groups whose arrays all are store their tiles with
 * bulk copies.
 * That choice is fixed in the prepared plan: between hc_batched_prepare and
 * every later hc_batched_launch, each instance's output (and intermediate)
 * must stay the same kind of memory at the same address -- a buffer freed
 * and replaced by managed or host-mapped memory at that address needs a new
 * hc_batched_prepare.
 * hc_batched_launch only resets counters and launches, so it can be captured
 * in a CUDA graph and replayed; every replay recomputes the prepared batch.
 * Device-side waits are bounded: a wait that gives up records HC_ERR_TIMEOUT
 * in the workspace status word (read it with hc_device_status).
 *
 * Fusion depth.  An instance with D <= fused_max_d runs fused: all such
 * instances share one persistent launch, each convolved in one piece (tiles,
 * then its outer axes interpolated while it is in L2).  The others run
 * grouped: per D, whole passes over all instances of that D (evaluation of
 * the outer axes, one tile launch, one interpolation pass), a few launches
 * per distinct D.  Both give the same bits.  hc_batched_prepare uses the
 * built-in depth; hc_batched_prepare_split takes it explicitly (-1: every
 * instance grouped except D = 0; >= 14, or 15 for HC_FP32: every instance
 * fused; HC_ERR_ARG below -1); hc_batched_autotune times every depth that
 * splits the batch differently, `reps` launches each after a warm-up, on
 * `stream` with CUDA events (synchronising; the outputs are overwritten),
 * returns the fastest in *best_fused_max_d (and its time in *best_ms unless
 * NULL) and leaves the workspace prepared with it.
 * hc_batched_workspace_size covers every depth.
 */
typedef struct {
  const void* x;
  const void* y;
  void* z;
  int D;
} hc_instance;

size_t hc_batched_workspace_size(const hc_instance* inst, int n, hc_dtype dtype);

hc_status hc_convolve_batched(const hc_instance* inst, int n, hc_dtype dtype, void* workspace,
                              size_t ws_bytes, hc_stream_t stream);

hc_status hc_batched_prepare(const hc_instance* inst, int n, hc_dtype dtype, void* workspace,
                             size_t ws_bytes, hc_stream_t stream);

hc_status hc_batched_launch(void* workspace, size_t ws_bytes, hc_stream_t stream);

hc_status hc_batched_prepare_split(const hc_instance* inst, int n, hc_dtype dtype, int fused_max_d,
                                   void* workspace, size_t ws_bytes, hc_stream_t stream);

hc_status hc_batched_autotune(const hc_instance* inst, int n, hc_dtype dtype, void* workspace,
                              size_t ws_bytes, int reps, hc_stream_t stream,
                              int* best_fused_max_d, double* best_ms);

/* Testing aid for the bounded waits (failure detection without a GPU fault):
 * rewrites the prepared work list in `workspace` so that the interpolation
 * tickets of `instance` wait for one more finished tile than the instance
 * has.  The next hc_batched_launch then records HC_ERR_TIMEOUT in the status
 * word after about a second, skips those tickets (their outputs are left
 * incomplete) and finishes every other instance.  hc_batched_prepare undoes
 * it.  Synchronous.  HC_ERR_ARG if the workspace was not prepared or the
 * instance is out of range.  Instances with D <= the tile axes (8; 9 for
 * HC_FP32) and instances run grouped have no waits, so the call has no
 * effect on them. */
hc_status hc_batched_inject_stall(void* workspace, int instance);

/* ------------------------------------------------------------------------
 * Tracing.  hc_profile_enable(1) makes every later kernel launch of the
 * library (any thread, any stream) record a pair of CUDA events on its own
 * stream around the kernel; hc_profile_enable(0) stops recording.
 * hc_profile_collect waits for the recorded events, then writes per kernel
 * name (NUL-terminated, name_len bytes per entry, in `names`) the number of
 * launches and their total device time in milliseconds, for at most
 * max_kernels names, clears the records and returns the number of names
 * written.  Any output array may be NULL.  Tracing adds two event records per
 * launch and is off by default. */
hc_status hc_profile_enable(int on);

int hc_profile_collect(char* names, int name_len, double* total_ms, int* counts,
                       int max_kernels);

/* ------------------------------------------------------------------------
 * Measurement aid (no counterpart in the paper): the device's rate of the
 * dtype's round-to-nearest add and multiply instructions, the operations of
 * the recurrence, for the roofline of the arithmetic-bound float64 path.  A
 * kernel of 8 independent add/multiply chains per thread, 8 CTAs of 256
 * threads per SM, is timed with CUDA events on `stream` (best of three after
 * a warm-up; synchronises); *ops_per_s receives the operations per second.
 * It allocates and frees its own small output array, so it is not for
 * allocation-free regions.  HC_FP64 and HC_FP32 only (HC_ERR_DTYPE
 * otherwise); HC_ERR_ARG for a NULL result pointer. */
hc_status hc_probe_alu_rate(hc_dtype dtype, double* ops_per_s, hc_stream_t stream);

/* ------------------------------------------------------------------------
 * Status word kept in the first bytes of every workspace.  Synchronises
 * `stream`, then returns HC_OK or the error a kernel recorded there
 * (HC_ERR_TIMEOUT).  HC_ERR_ARG for a NULL workspace.
 */
hc_status hc_device_status(const void* workspace, hc_stream_t stream);

#ifdef __cplusplus
}
#endif

#endif /* HC_H_ */
