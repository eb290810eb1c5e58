"""The allocation-free Bellman-Ford entry point against the ordinary one.

stc_bellman_ford_noalloc is for callers that cannot allocate device memory while
they run (host callbacks, real-time loops, processes that only hand out memory
from fixed pools): its working memory is a fixed array compiled into the
library, shared by every call on a device.  This file is collected last so that
a run stopping at the first failure has already run every other test.
"""
import numpy as np
import pytest
import torch

import oracle as O
import workloads as W
from gpu_util import need_gpu, to_dev

pytestmark = pytest.mark.gpu


def test_noalloc_matches_bellman_ford_on_two_calls_in_a_row():
    need_gpu()
    import paper_1512_00066_b300 as stc
    H = stc.Handle()
    G = W.rmat(14, seed=41)
    cases = [(stc.MIN_PLUS_I32, W.weights_int(G.nnz, 1, 1000, 42), torch.int32),
             (stc.MIN_PLUS_F32, W.weights_unit01(G.nnz, 43).astype(np.float32), torch.float32)]
    for alg, w, dt in cases:
        dG = to_dev(G.with_val(w))
        ref, _ = H.bellman_ford(alg, dG, 0, persistent=True)
        ref = ref.cpu().numpy()
        # the frontier method's round count depends on the order of atomic updates
        # inside a round; it is bounded by the full-relaxation round count
        _, jacobi_rounds = O.bellman_ford(O.MP_I32 if alg == stc.MIN_PLUS_I32 else O.MP_F32,
                                          G.with_val(w), 0)
        for source in (0, 0):  # two calls in a row share the same scratch array
            out = torch.full((G.nrows,), 7, dtype=dt, device="cuda")
            rounds = stc.bellman_ford_noalloc(alg, dG, source, out)
            got = out.cpu().numpy()
            # Bellman-Ford distances are exact: bit-for-bit equality is the tolerance
            assert got.tobytes() == ref.tobytes()
            assert 1 <= rounds <= jacobi_rounds
        # a different source right after, compared with the ordinary entry point
        src = int(W.sample_sources(G, 1, 5)[0])
        out = torch.empty(G.nrows, dtype=dt, device="cuda")
        stc.bellman_ford_noalloc(alg, dG, src, out)
        ref2, _ = H.bellman_ford(alg, dG, src)
        assert out.cpu().numpy().tobytes() == ref2.cpu().numpy().tobytes()


def test_noalloc_rejects_graphs_above_its_capacity():
    need_gpu()
    import paper_1512_00066_b300 as stc
    n = stc.NOALLOC_BF_MAX_VERTICES + 1
    big = stc.DeviceCsr(n, n, torch.zeros(n + 1, dtype=torch.int64, device="cuda"),
                        torch.zeros(0, dtype=torch.int32, device="cuda"),
                        torch.zeros(0, dtype=torch.int32, device="cuda"))
    out = torch.empty(n, dtype=torch.int32, device="cuda")
    with pytest.raises(stc.StcError) as e:
        stc.bellman_ford_noalloc(stc.MIN_PLUS_I32, big, 0, out)
    assert e.value.status == 9
