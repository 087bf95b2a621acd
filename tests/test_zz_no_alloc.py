"""The allocation-free forward sweep (nk_sssp_noalloc) against the allocating one.

nk_sssp_noalloc is for callers that cannot allocate device memory when they call in;
its scratch is a static device array.  Two calls in a row (the array keeps the previous
call's contents) must each give exactly what nk_sssp gives, and sizes beyond the array's
limit must be refused.  This file sorts last so that a run stopping at the first failure
has run every other test first; it also passes alone in a fresh process.
"""
from __future__ import annotations

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def test_noalloc_sweep_matches_allocating_sweep_twice():
    import torch
    torch.cuda.set_device(0)
    from paper_1403_3005_gb300 import nk
    stream = torch.cuda.current_stream()
    g = nk.graph_generate("rmat", 14, 21)          # hubs, isolated vertices, ~8 levels
    rp, col = g.export_csr()
    n = len(rp) - 1
    d_rp = torch.from_numpy(rp).cuda()
    d_col = torch.from_numpy(col).cuda()
    dist = torch.full((n,), -7, dtype=torch.int32, device="cuda")
    sigma = torch.full((n,), 12345, dtype=torch.int64, device="cuda")
    deg = np.diff(rp)
    for s in (int(np.argmax(deg)), int(np.flatnonzero(deg == 1)[0])):   # a hub, then a leaf
        nk.sssp_noalloc(d_rp, d_col, s, dist, sigma, stream)
        torch.cuda.synchronize()
        want_d, want_s = nk.sssp(g, s)
        assert np.array_equal(dist.cpu().numpy(), want_d)
        assert np.array_equal(sigma.cpu().numpy().view(np.uint64), want_s)


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
