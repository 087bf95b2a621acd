"""The oracle's pins catch plausible mistakes.

Each case copies the oracle's C source, plants one mistake of the kind a restatement of the
paper could make (a dropped term, a wrong index or endpoint, a wrong scale, an off-by-one),
builds the copy in a temporary directory and runs the pins that guard that part of the
oracle against it: at least one must fail.  The oracle under oracle/ is never modified.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import pytest

import oracle
import test_oracle as T

SRC = os.path.join(os.path.dirname(oracle.__file__), "nk_oracle.c")

# (what is wrong, text in the source, replacement, pins that must notice)
MUTATIONS = [
    ("Brandes' recurrence without the 1 + delta term",
     "delta[v] += ((double)sigma[v] / (double)sigma[w]) * (1.0 + delta[w]);",
     "delta[v] += ((double)sigma[v] / (double)sigma[w]) * (delta[w]);",
     [(T.test_path, (10,)), (T.test_star, (7,))]),
    ("exact scores not halved (ordered pairs)",
     "or_betweenness(n, row_ptr, col, n, src, 0.5, scores)",
     "or_betweenness(n, row_ptr, col, n, src, 1.0, scores)",
     [(T.test_path, (10,))]),
    ("sampled scale n/k instead of n/(2k)",
     "(double)n / (2.0 * (double)k), scores)",
     "(double)n / (double)k, scores)",
     [(T.test_sampled_k_equals_n_is_exact, ())]),
    ("path counts added from the wrong endpoint",
     "sigma[w], sigma[v], &sigma[w]",
     "sigma[w], sigma[w], &sigma[w]",
     [(T.test_sigma_grid_binomials, ())]),
    ("edge score without its reverse arc",
     "out[j] = scale * (arc[j] + arc[r]);",
     "out[j] = scale * (arc[j] + arc[j]);",
     [(T.test_edge_betweenness_closed_forms, ()), (T.test_edge_betweenness_single_source_bruteforce, ())]),
    ("closeness distances off by one",
     "far[w] += (double)dist[w];",
     "far[w] += (double)(dist[w] - 1);",
     [(T.test_closeness_closed_forms, ())]),
    ("path walk picks the run boundary one too late",
     "if (t < run) { z = c; break; }",
     "if (t <= run) { z = c; break; }",
     [(T.test_rk_pair_and_path_laws, ())]),
    ("weighted predecessors found by hop count",
     "dist[v] + (int64_t)w[j] == dist[x]",
     "dist[v] + 1 == dist[x]",
     [(T.test_weighted_cycle_with_a_heavy_edge, ()), (T.test_weighted_bruteforce_small, (1,))]),
    ("vertex-diameter bound 2 ecc instead of 2 ecc + 1",
     "int64_t bound = 2 * (int64_t)ecc + 1;",
     "int64_t bound = 2 * (int64_t)ecc;",
     [(T.test_vertex_diameter_estimate_closed_forms, ())]),
    ("BFS distances off by one level",
     "                dist[w] = dist[v] + 1;\n                queue[tail++] = w;",
     "                dist[w] = dist[v] + 2;\n                queue[tail++] = w;",
     [(T.test_distance_closed_forms, ()), (T.test_bfs_distances_match_floyd_warshall, (T.G.grid(6, 7),))]),
    ("CSR build keeps duplicate arcs",
     "if (i > 0 && arc[i] == arc[i - 1]) continue;",
     "if (0 && i > 0 && arc[i] == arc[i - 1]) continue;",
     [(T.test_csr_canonical_form, ())]),
    ("sampler takes the largest keys",
     "for (int32_t i = 0; i < k; ++i) src[i] = kv[i].v;",
     "for (int32_t i = 0; i < k; ++i) src[i] = kv[n - 1 - i].v;",
     [(T.test_sampler_properties, ())]),
    ("R-MAT quadrants b and c swapped",
     "else if (x < t2) { ru = 0; rv = 1; }\n            else if (x < t3) { ru = 1; rv = 0; }",
     "else if (x < t2) { ru = 1; rv = 0; }\n            else if (x < t3) { ru = 0; rv = 1; }",
     [(T.test_rmat_quadrant_frequencies, ())]),
    ("Dijkstra resets path counts on equal lengths",
     "if (dist[x] < 0 || nd < dist[x]) {",
     "if (dist[x] < 0 || nd <= dist[x]) {",
     [(T.test_weighted_bruteforce_small, (1,)), (T.test_weighted_bruteforce_small, (2,)),
      (T.test_weighted_reduces_to_unweighted, (T.G.grid(6, 7),))]),
    ("pair draw lets the target equal the source",
     "    if (v >= u) ++v;",
     "    if (v > u) ++v;",
     [(T.test_rk_pair_and_path_laws, ())]),
    ("ER skipping one pair too many",
     "t = t + 1 + (int64_t)q;",
     "t = t + 2 + (int64_t)q;",
     [(T.test_er_edge_count_and_canonical, ()), (T.test_er_pair_inclusion_uniform, ())]),
    ("BA draws its partner slot from [0, 2e) instead of [0, 2e]",
     "(uint64_t)(2 * e + 1));\n        M[2 * e + 1] = M[r];",
     "(uint64_t)(2 * e + (e == 0)));\n        M[2 * e + 1] = M[r];",
     [(T.test_ba_attachment_distribution, ())]),
    ("closeness reach counted twice",
     "reach[w] += 1.0;",
     "reach[w] += 2.0;",
     [(T.test_closeness_closed_forms, ())]),
    ("estimate scaled by n (n - 1) / r (ordered pairs)",
     "const double scale = (double)n * (double)(n - 1) / (2.0 * (double)r);",
     "const double scale = (double)n * (double)(n - 1) / ((double)r);",
     [(T.test_rk_counts_in_ranges_add_up_to_the_estimate, ()), (T.test_rk_unbiased_and_within_epsilon, ())]),
    ("sample count without its + 1 term",
     "(double)lg + 1.0 + log(1.0 / delta)",
     "(double)lg + log(1.0 / delta)",
     [(T.test_rk_sample_count_hand_values, ())]),
]


@pytest.mark.parametrize("what,old,new,pins", MUTATIONS, ids=[m[0] for m in MUTATIONS])
def test_pins_catch_planted_mistake(what, old, new, pins, tmp_path, monkeypatch):
    src = open(SRC).read()
    assert old in src, "mutation point not found"
    mutated = tmp_path / "nk_oracle_mutant.c"
    mutated.write_text(src.replace(old, new))
    so = tmp_path / "libmutant.so"
    subprocess.check_call(["gcc", "-O2", "-ffp-contract=off", "-fPIC", "-shared", "-o", str(so),
                           str(mutated), "-lm"])
    monkeypatch.setattr(oracle, "_lib", oracle._bind(ctypes.CDLL(str(so))))
    caught = []
    for fn, args in pins:
        try:
            fn(*args)
        except Exception:  # a failed assertion, an oracle error or a crash of the pin
            caught.append(fn.__name__)
    assert caught, f"no pin noticed: {what}"
