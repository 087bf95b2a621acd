"""GB300-native betweenness centrality (exact Brandes and the source-sampled estimate)
behind a C ABI (include/nk.h, libnk.so), with a thin ctypes binding (``nk``)."""
from . import nk  # noqa: F401
from .nk import (Graph, NkError, RunOpts, Server, autotune, betweenness_exact,  # noqa: F401
                 betweenness_sampled, betweenness_sources, graph_from_csr, graph_from_edges,
                 graph_generate, last_run_stats, sample_sources, set_stream, sssp)
