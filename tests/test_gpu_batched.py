"""GPU parity of the batching form (many convolutions of uneven D; fused
instances in one persistent launch, the others as per-D grouped passes):
every instance bitwise equal to the oracle's recurrence in the same
precision at every fusion depth, the full 4096-instance workload equal to a
per-instance loop of the plain kernel, the batched autotuner, CUDA-graph
replay, and the bounded device-side wait that reports HC_ERR_TIMEOUT instead
of hanging."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle  # noqa: E402
from paper_1608_00206_gb300 import _lib, inputs  # noqa: E402

pytestmark = pytest.mark.gpu
DEV = "cuda:0"


@pytest.fixture(scope="module")
def hc():
    from paper_1608_00206_gb300.build import build
    build()
    import paper_1608_00206_gb300 as hc
    return hc


def T(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to(DEV)


def bits(a):
    return a.view(np.uint64) if a.dtype.itemsize == 8 else a.view(np.uint32)


@pytest.mark.parametrize("split", [None, -1, 5, 15])
@pytest.mark.parametrize("kind", ["int64", "float64", "float32", "mixed"])
def test_batched_every_dim_bit_exact(hc, kind, split):
    """Every D from 0 to the limit, repeated D included, at the default fusion
    depth, all grouped (-1), a split in the middle (5) and all fused (15)."""
    dims = list(range(0, 15)) + [14, 3, 9, 0, 12]
    if kind == "float32":
        dims.append(15)
    pairs = []
    for i, D in enumerate(dims):
        if kind == "int64":
            pairs.append(inputs.uniform_int_pair(D, -1000, 1000, seed=i))
        elif kind == "float64":
            pairs.append(inputs.prob_exponential_pair(D, seed=i))
        else:
            pairs.append(inputs.uniform01_pair(D, seed=i))
    outs = hc.convolve_batched([T(x) for x, _ in pairs], [T(y) for _, y in pairs],
                               mixed=(kind == "mixed"), fused_max_d=split)
    torch.cuda.synchronize()
    for (x, y), z, D in zip(pairs, outs, dims):
        want = oracle.convolve_mixed(x, y) if kind == "mixed" else oracle.convolve(x, y, threads=8)
        got = z.cpu().numpy().reshape(-1)
        assert np.array_equal(bits(got), bits(want)), f"D={D}"


def _workload(n=4096, seed=4096):
    dims = inputs.batched_dims(n, 6, 14, seed)
    return dims, inputs.batched_uniform01(dims, seed + 1)


def test_batched_4096_float32_workload(hc):
    """4096 instances, D ~ U{6..14}, float32 U[0,1): the persistent launch and
    its CUDA-graph replay equal a per-instance loop of hc_convolve bitwise, and
    a seeded subset covering every D equals the oracle bitwise."""
    dims, pairs = _workload()
    xs = [T(x) for x, _ in pairs]
    ys = [T(y) for _, y in pairs]
    b = hc.BatchedConv(xs, ys)
    outs = [o.clone() for o in b.launch()]
    assert b.status() == 0
    loop = [hc.convolve(x, y) for x, y in zip(xs, ys)]
    torch.cuda.synchronize()
    for o, l in zip(outs, loop):
        assert torch.equal(o.view(torch.int32), l.view(torch.int32))
    g = np.random.default_rng(0)
    subset = sorted({int(np.flatnonzero(dims == D)[0]) for D in range(6, 15)} |
                    set(g.choice(len(dims), 48, replace=False).tolist()))
    for i in subset:
        want = oracle.convolve(pairs[i][0], pairs[i][1], threads=16)
        assert np.array_equal(bits(outs[i].cpu().numpy().reshape(-1)), bits(want)), i
    # graph replay recomputes from the current inputs
    for o in b.outs:
        o.zero_()
    b.replay()
    torch.cuda.synchronize()
    for o, ref in zip(b.outs, outs):
        assert torch.equal(o.view(torch.int32), ref.view(torch.int32))
    xs[5].mul_(2.0)
    b.replay()
    torch.cuda.synchronize()
    assert torch.equal(b.outs[5].view(torch.int32), hc.convolve(xs[5], ys[5]).view(torch.int32))
    assert b.status() == 0


def test_batched_autotune_picks_a_depth(hc):
    """The batched autotuner tries every fusion depth that splits the batch,
    leaves the winner prepared, and the result is bitwise the same."""
    dims, pairs = _workload(n=256, seed=77)
    xs = [T(x) for x, _ in pairs]
    ys = [T(y) for _, y in pairs]
    b = hc.BatchedConv(xs, ys, fused_max_d="tune")
    assert -1 <= b.fused_max_d <= 15 and b.tuned_ms > 0
    outs = [o.clone() for o in b.launch()]
    ref = hc.BatchedConv(xs, ys, fused_max_d=15)
    for o, r in zip(outs, ref.launch()):
        assert torch.equal(o.view(torch.int32), r.view(torch.int32))
    assert b.status() == 0
    # and the tuned batch against the oracle on a subset covering every D
    seen = set()
    for o, (x, y), d in zip(outs, pairs, dims):
        if d not in seen:
            seen.add(d)
            want = oracle.convolve(x, y)
            assert np.array_equal(o.cpu().numpy().reshape(-1).view(np.uint32), want.view(np.uint32))


def test_bounded_wait_reports_timeout(hc):
    """A stall injected on the host (an instance's interpolation tickets wait
    for a tile that does not exist) ends in HC_ERR_TIMEOUT after about a
    second; every other instance is still computed and the context stays
    usable."""
    dims = [10, 11, 7, 12]
    pairs = [inputs.uniform_int_pair(D, -1000, 1000, seed=D) for D in dims]
    # all fused: only the persistent launch has waits
    b = hc.BatchedConv([T(x) for x, _ in pairs], [T(y) for _, y in pairs], fused_max_d=15)
    b.inject_stall(1)
    b.launch()
    assert b.status() == _lib.HC_ERR_TIMEOUT
    for i in (0, 2, 3):
        want = oracle.convolve(*pairs[i])
        assert np.array_equal(b.outs[i].cpu().numpy().reshape(-1), want)
    # the same workspace prepared again runs clean
    b2 = hc.BatchedConv([T(x) for x, _ in pairs], [T(y) for _, y in pairs], fused_max_d=15)
    b2.launch()
    assert b2.status() == 0
    assert np.array_equal(b2.outs[1].cpu().numpy().reshape(-1), oracle.convolve(*pairs[1]))


def test_batched_rejects_bad_instances(hc):
    x = T(np.zeros(1 << 16, np.int64))
    with pytest.raises(ValueError):
        hc.BatchedConv([x], [x])  # D = 16 int64 exceeds the batched limit


@pytest.mark.parametrize("kind", ["int64", "float32", "mixed"])
def test_packed_batch_from_host(hc, kind):
    """BatchedConv.from_packed + run_host: every instance's array sits at a
    16-byte-aligned offset of one packed array (odd sizes, so most offsets
    carry padding), the batch moves in one copy per array, and every
    instance is bitwise the oracle's result, twice in a row (graph replay on
    new host inputs)."""
    dims = [0, 1, 2, 3, 5, 7, 9, 11, 12, 13, 3, 1]
    dt = np.int64 if kind == "int64" else np.float32
    tdt = torch.int64 if kind == "int64" else torch.float32
    xo, nx = hc.packed_offsets(dims, tdt, 2)
    zo, nz = hc.packed_offsets(dims, tdt, 3)
    xh = torch.zeros(nx, dtype=tdt).pin_memory()
    yh = torch.zeros(nx, dtype=tdt).pin_memory()
    zh = torch.empty(nz, dtype=tdt).pin_memory()
    b = hc.BatchedConv.from_packed(torch.zeros(nx, dtype=tdt, device=DEV),
                                   torch.zeros(nx, dtype=tdt, device=DEV), dims,
                                   mixed=(kind == "mixed"))
    for rep in range(2):
        pairs = []
        for i, D in enumerate(dims):
            if kind == "int64":
                x, y = inputs.uniform_int_pair(D, -1000, 1000, seed=100 * rep + i)
            else:
                x, y = inputs.uniform01_pair(D, seed=100 * rep + i)
            pairs.append((x, y))
            xh[xo[i]:xo[i] + (1 << D)] = torch.from_numpy(x.astype(dt))
            yh[xo[i]:xo[i] + (1 << D)] = torch.from_numpy(y.astype(dt))
        b.run_host(xh, yh, zh)
        z = zh.numpy()
        for i, ((x, y), D) in enumerate(zip(pairs, dims)):
            want = oracle.convolve_mixed(x, y) if kind == "mixed" else oracle.convolve(x, y)
            got = z[zo[i]:zo[i] + 3 ** D]
            assert np.array_equal(bits(got.copy()), bits(want)), f"rep {rep} D={D}"
    with pytest.raises(ValueError):
        b.run_host(xh[:-1], yh, zh)
