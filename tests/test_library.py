"""CPU-side checks of the C ABI library: it builds, loads, exports every function that
include/nk.h declares, the binding covers them, and argument checks fail cleanly
without touching a GPU.  Also the multi-rank sharding of sources (gloo, 2 ranks)."""
from __future__ import annotations

import ctypes
import os
import re
import subprocess

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "nk.h")


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    names = re.findall(r"^\s*(?:const\s+)?[A-Za-z_][\w\s\*]*?\b(nk_\w+)\s*\(", text, flags=re.M)
    return sorted(set(names))


@pytest.fixture(scope="module")
def libpath():
    from paper_1403_3005_gb300 import build
    return build.build()


def test_header_parses():
    names = declared_functions()
    assert "nk_betweenness_sampled" in names and "nk_serve_submit" in names
    assert len(names) >= 20


def test_library_exports_every_declared_symbol(libpath):
    out = subprocess.run(["nm", "-D", "--defined-only", libpath], capture_output=True, text=True,
                         check=True).stdout
    exported = set(re.findall(r"\bT\s+(nk_\w+)", out))
    missing = [n for n in declared_functions() if n not in exported]
    assert not missing, missing


def test_binding_covers_header(libpath):
    from paper_1403_3005_gb300 import nk
    assert set(declared_functions()) == set(nk.SIGNATURES)
    L = nk.lib()
    for name in declared_functions():
        assert hasattr(L, name)


def test_argument_errors_without_gpu(libpath):
    from paper_1403_3005_gb300 import nk
    L = nk.lib()
    assert L.nk_betweenness_sampled(None, 1, 5, None) == nk.ERR_ARG
    assert b"null" in L.nk_last_error()
    assert L.nk_betweenness_exact(None, None) == nk.ERR_ARG
    assert L.nk_sssp(None, 0, None, None) == nk.ERR_ARG
    out = ctypes.c_void_p()
    assert L.nk_graph_from_csr(0, None, None, 0, 0, ctypes.byref(out)) == nk.ERR_ARG
    assert L.nk_graph_generate(99, (ctypes.c_double * 1)(1.0), 10, 1, ctypes.byref(out)) in (nk.ERR_ARG,)
    assert L.nk_sample_sources(10, 1, 11, None, 0) == nk.ERR_ARG
    assert L.nk_set_wait_limit_ns(0) == nk.ERR_ARG
    assert L.nk_graph_free(None) == nk.OK
    assert nk.version().startswith("nk-gb300")


def test_product_path_does_not_import_oracle():
    pkg = os.path.join(ROOT, "paper_1403_3005_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".h", ".cuh")):
                text = open(os.path.join(dirpath, f)).read()
                assert "oracle" not in text.replace("oracle-free", ""), f


def test_noalloc_refuses_bad_buffers_before_any_launch(libpath):
    """The allocation-free sweep's binding checks dtype, size, contiguity and device of
    every buffer before anything reaches the library (CPU tensors never get that far)."""
    import torch
    from paper_1403_3005_gb300 import nk
    n = 10
    rp = torch.zeros(n + 1, dtype=torch.int32)
    col = torch.zeros(4, dtype=torch.int32)
    dist = torch.zeros(n, dtype=torch.int32)
    sigma = torch.zeros(n, dtype=torch.int64)
    launches = nk.launch_count()
    bad = [
        ((rp.long(), col, dist, sigma), "row_ptr must be torch.int32"),
        ((rp, col.long(), dist, sigma), "col must be torch.int32"),
        ((rp, col, dist.long(), sigma), "dist must be torch.int32"),
        ((rp, col, dist, sigma.int()), "sigma must be torch.int64"),
        ((rp, col, dist[:n - 1], sigma), "need n = 10 entries"),
        ((rp, col, dist, sigma[:n - 1]), "need n = 10 entries"),
        ((rp, col, dist, torch.zeros(2 * n, dtype=torch.int64)[::2]), "contiguous"),
        ((rp, col, dist, sigma), "must be a CUDA tensor"),
        ((np.zeros(n + 1, np.int32), col, dist, sigma), "must be a torch tensor"),
    ]
    for args, msg in bad:
        with pytest.raises(ValueError, match=msg):
            nk.sssp_noalloc(args[0], args[1], 0, args[2], args[3])
    assert nk.launch_count() == launches


# ---------------------------------------------------------------- multi-rank sharding
def test_source_shard_partitions_the_set():
    from paper_1403_3005_gb300 import nk
    for k in (1, 5, 8192, 8193):
        src = np.arange(k)
        for world in (1, 2, 3, 8):
            parts = [nk.source_shard(src, r, world) for r in range(world)]
            assert np.array_equal(np.concatenate(parts), src)
            assert max(map(len, parts)) - min(map(len, parts)) <= 1


def _shard_worker(rank, world, port, n, rp, col, src, q):
    import torch.distributed as dist
    import oracle
    from paper_1403_3005_gb300 import nk
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import torch
    # the product's partition-and-reduce helper, with the oracle as the per-rank compute
    got = nk.sharded_betweenness(n, src, rank, world,
                                 lambda part: torch.from_numpy(oracle.betweenness_sources(rp, col, part, 1.0)))
    if rank == 0:
        q.put(got.numpy())
    dist.barrier()
    dist.destroy_process_group()


def test_source_sharding_over_two_gloo_ranks():
    """Sources are independent (Section 3.2): a contiguous slice of one source set per rank
    and one sum all-reduce of the n-vector give the unsharded sampled estimate."""
    import multiprocessing as mp
    import socket

    import oracle
    n, rp, col = oracle.generate("ba", 3000, 4, m0=3)
    src = oracle.sample_sources(n, 9, 200)
    want = oracle.betweenness_sampled(rp, col, 9, 200)
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        port = s.getsockname()[1]
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_shard_worker, args=(r, 2, port, n, rp, col, src, q)) for r in range(2)]
    for p in procs:
        p.start()
    got = q.get(timeout=120)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert np.allclose(got, want, rtol=1e-12, atol=1e-12)
