"""Host logic of the packed batch layout (no GPU): every instance starts on
a 16-byte boundary, instances do not overlap, and the total covers the last
one."""
import pytest

torch = pytest.importorskip("torch")

from paper_1608_00206_gb300.api import packed_offsets  # noqa: E402


@pytest.mark.parametrize("dtype,es", [(torch.float32, 4), (torch.float64, 8), (torch.int64, 8)])
@pytest.mark.parametrize("base", [2, 3])
def test_offsets_aligned_disjoint_and_covering(dtype, es, base):
    dims = [0, 1, 2, 3, 4, 5, 7, 0, 13, 1, 6]
    offs, total = packed_offsets(dims, dtype, base)
    assert len(offs) == len(dims) and offs[0] == 0
    for i, (o, D) in enumerate(zip(offs, dims)):
        assert (o * es) % 16 == 0
        end = o + base ** D
        nxt = offs[i + 1] if i + 1 < len(offs) else total
        assert end <= nxt and nxt - end < 16 // es
    assert packed_offsets([], dtype, base) == ([], 0)
