"""The binding rejects distance buffers the Bellman-Ford kernels would write out of
bounds, before any device work (these run on the CPU: the checks come first)."""
import pytest
import torch

import paper_1512_00066_b300 as stc


def _graph(n=8, device="cpu"):
    return stc.DeviceCsr(n, n, torch.zeros(n + 1, dtype=torch.int64, device=device),
                         torch.zeros(0, dtype=torch.int32, device=device), None)


@pytest.mark.parametrize("alg,bad_dtype", [(stc.MIN_PLUS_I32, torch.int64), (stc.MIN_PLUS_I32, torch.float32),
                                           (stc.MIN_PLUS_F32, torch.float64), (stc.MIN_PLUS_F32, torch.int32)])
def test_wrong_dtype_is_rejected(alg, bad_dtype):
    G = _graph()
    with pytest.raises(ValueError, match="dtype"):
        stc.bellman_ford_noalloc(alg, G, 0, torch.empty(8, dtype=bad_dtype))


def test_short_buffer_is_rejected():
    G = _graph()
    with pytest.raises(ValueError, match="elements"):
        stc.bellman_ford_noalloc(stc.MIN_PLUS_I32, G, 0, torch.empty(7, dtype=torch.int32))


def test_non_contiguous_buffer_is_rejected():
    G = _graph()
    d = torch.empty(16, dtype=torch.float32)[::2]
    assert d.numel() == 8
    with pytest.raises(ValueError, match="contiguous"):
        stc.bellman_ford_noalloc(stc.MIN_PLUS_F32, G, 0, d)


def test_buffer_off_the_graphs_device_is_rejected():
    G = _graph()
    with pytest.raises(ValueError, match="device|graph"):
        stc.bellman_ford_noalloc(stc.MIN_PLUS_I32, G, 0, torch.empty(8, dtype=torch.int32))


def test_algebra_without_bellman_ford_is_rejected():
    G = _graph()
    with pytest.raises(ValueError, match="algebra"):
        stc._check_dist(stc.PLUS_TIMES_F32, G, torch.empty(8, dtype=torch.float32), "bellman_ford")


def test_descriptor_follows_field_assignment():
    """The cached C descriptor (and its bytes, used by batched calls) is rebuilt
    after any field is assigned."""
    G = _graph()
    c0 = G._c()
    assert (c0.nrows, c0.ncols, c0.nnz) == (8, 8, 0)
    assert G._c() is c0 and G._c_bytes() == bytes(c0)
    G.col = torch.zeros(5, dtype=torch.int32)
    G.rowptr = torch.tensor([0, 5, 5, 5, 5, 5, 5, 5, 5], dtype=torch.int64)
    c1 = G._c()
    assert c1 is not c0 and c1.nnz == 5 and c1.col == G.col.data_ptr() and c1.rowptr == G.rowptr.data_ptr()
    assert G._c_bytes() == bytes(c1)
    G.nrows = 3
    assert G._c().nrows == 3 and bytes(G._c()) == G._c_bytes()
