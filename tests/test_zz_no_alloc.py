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


def test_noalloc_matches_the_oracle_and_the_ordinary_entry_point_on_two_calls_in_a_row():
    need_gpu()
    import paper_1512_00066_b300 as stc
    H = stc.Handle()
    G = W.rmat(14, seed=41)
    src2 = int(W.sample_sources(G, 1, 5)[0])
    cases = [(stc.MIN_PLUS_I32, O.MP_I32, W.weights_int(G.nnz, 1, 1000, 42), torch.int32),
             (stc.MIN_PLUS_F32, O.MP_F32, W.weights_unit01(G.nnz, 43).astype(np.float32), torch.float32)]
    for alg, oalg, w, dt in cases:
        Gw = G.with_val(w)
        dG = to_dev(Gw)
        # the oracle: plain full relaxation (Section 4.2), which also bounds the
        # frontier method's round count (that count depends on the order of atomic
        # updates inside a round)
        ref, jacobi_rounds = O.bellman_ford(oalg, Gw, 0)
        for _ in range(2):  # two calls in a row share the same scratch array
            out = torch.full((G.nrows,), 7, dtype=dt, device="cuda")
            rounds = stc.bellman_ford_noalloc(alg, dG, 0, out)
            got = out.cpu().numpy()
            # Bellman-Ford distances are exact: bit-for-bit equality is the tolerance
            assert got.tobytes() == ref.tobytes()
            assert 1 <= rounds <= jacobi_rounds
            # and the same bits as the ordinary entry point
            ordinary, _ = H.bellman_ford(alg, dG, 0, persistent=True)
            assert got.tobytes() == ordinary.cpu().numpy().tobytes()
        # a different source right after, against the oracle
        ref2, _ = O.bellman_ford(oalg, Gw, src2)
        out = torch.empty(G.nrows, dtype=dt, device="cuda")
        stc.bellman_ford_noalloc(alg, dG, src2, out)
        assert out.cpu().numpy().tobytes() == ref2.tobytes()


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
