"""The allocation-free forward sweep (nk_sssp_noalloc).

nk_sssp_noalloc serves callers that cannot allocate device memory when they call in (code
under an allocator that forbids cudaMalloc/cudaFree, or a host library whose device
footprint must not grow after start-up); its scratch is a static device array.  Two calls
in a row (the array keeps the previous call's contents) must each give exactly what the
oracle's BFS gives on the oracle's own copy of the graph, and what the allocating nk_sssp
gives; the second call must make no allocation call and leave the device's free memory
unchanged; sizes beyond the array's limit must be refused.  This file sorts last so that a
run stopping at the first failure has run every other test first; it also passes alone in
a fresh process.
"""
from __future__ import annotations

import numpy as np
import pytest

import oracle

pytestmark = pytest.mark.gpu


def test_noalloc_sweep_matches_oracle_and_allocating_sweep_twice():
    import torch
    torch.cuda.set_device(0)
    from paper_1403_3005_gb300 import nk
    stream = torch.cuda.current_stream()
    n, rp, col = oracle.generate("rmat", 14, 21)     # hubs, isolated vertices, ~8 levels
    g = nk.graph_from_csr(rp, col)
    d_rp = torch.from_numpy(rp).cuda()
    d_col = torch.from_numpy(col).cuda()
    dist = torch.full((n,), -7, dtype=torch.int32, device="cuda")
    sigma = torch.full((n,), 12345, dtype=torch.int64, device="cuda")
    deg = np.diff(rp)
    for call, s in enumerate((int(np.argmax(deg)), int(np.flatnonzero(deg == 1)[0]))):  # a hub, then a leaf
        torch.cuda.synchronize()
        allocs, free0 = nk.alloc_count(), torch.cuda.mem_get_info()[0]
        nk.sssp_noalloc(d_rp, d_col, s, dist, sigma, stream)
        torch.cuda.synchronize()
        if call == 1:  # the first call may load the module that holds the static array
            assert nk.alloc_count() == allocs
            assert torch.cuda.mem_get_info()[0] == free0
        got_d, got_s = dist.cpu().numpy(), sigma.cpu().numpy().view(np.uint64)
        want_d, want_s = oracle.bfs(rp, col, s)
        assert np.array_equal(got_d, want_d)
        assert np.array_equal(got_s, want_s)
        gpu_d, gpu_s = nk.sssp(g, s)
        assert np.array_equal(got_d, gpu_d) and np.array_equal(got_s, gpu_s)
    g.free()


def test_noalloc_refuses_sizes_beyond_its_scratch():
    import torch
    from paper_1403_3005_gb300 import nk
    n = (1 << 20) + 1
    rp = torch.zeros(n + 1, dtype=torch.int32, device="cuda")
    col = torch.zeros(1, dtype=torch.int32, device="cuda")
    out = torch.empty(n, dtype=torch.int64, device="cuda")
    with pytest.raises(nk.NkError) as e:
        nk.sssp_noalloc(rp, col[:0], 0, out.view(torch.int32)[:n], out)
    assert e.value.rc == nk.ERR_ARG and "1048576" in str(e.value)
