"""Host block layout of the transfer pipeline (host logic, no GPU): one step's float32
attributes travel as one block of FLOATS_PER_GAUSSIAN * n floats, the arrays one after the
other in the attribute order of the C structure."""
import torch

from paper_2504_17954_gb300.hostio import FLOATS_PER_GAUSSIAN, HOST_LAYOUT, block_views
from paper_2504_17954_gb300.rasterizer import ATTRS, WIDTH


def test_layout_is_the_attribute_order_with_its_widths():
    assert [k for k, _ in HOST_LAYOUT] == list(ATTRS)
    assert [w for _, w in HOST_LAYOUT] == [3, 3, 4, 1, 3, 3, 4]
    assert FLOATS_PER_GAUSSIAN == 21 == sum(WIDTH.values())


def test_block_views_tile_the_block_exactly():
    n = 37
    blk = torch.arange(FLOATS_PER_GAUSSIAN * n, dtype=torch.float32)
    views = block_views(blk, n)
    assert len(views) == len(ATTRS)
    off = 0
    for (k, w), t in zip(HOST_LAYOUT, views):
        assert t.shape == ((n, w) if w > 1 else (n,)), k
        assert t.is_contiguous() and t.data_ptr() == blk.data_ptr() + 4 * off, k  # views, not copies
        assert float(t.reshape(-1)[0]) == off and float(t.reshape(-1)[-1]) == off + w * n - 1, k
        off += w * n
    assert off == blk.numel()
    views[3][5] = -1.0  # writes go to the block
    assert float(blk[(3 + 3 + 4) * n + 5]) == -1.0
