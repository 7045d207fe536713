"""Mutation tests: plant plausible mistakes in a copy of the oracle (on the CPU) and check that
the pins fail for every one of them. The oracle itself is never modified. Each mutant runs in a
child process: a mutant that writes outside its table may crash, which also counts as caught."""
import math
import os
import subprocess
import sys

import numpy as np
import pytest

import oracle
from paper_1110_2561_gb300 import workloads as w
from closed_forms import brute_force_g_range, free_spin_moments, free_spins, kaufman_logz, ring_logz

# (name, original text, planted mistake); each original must occur exactly once.
MUTANTS = [
    ("edges: energy sign", "E -= bJ[b] * spin[bi[b]] * spin[bj[b]];", "E += bJ[b] * spin[bi[b]] * spin[bj[b]];"),
    ("edges: last bond dropped", "for (int b = 0; b < nb; ++b) E -=", "for (int b = 0; b + 1 < nb; ++b) E -="),
    ("edges: spin from wrong bit", "spin[i] = ((s >> i) & 1u) ? +1 : -1;", "spin[i] = ((s >> (n - 1 - i)) & 1u) ? +1 : -1;"),
    ("edges: bins transposed", "g[e * (n + 1) + m] += 1;", "g[(n - m) * 0 + e * (n + 1) + (n - m) * ((e % 2) == 1) + m * ((e % 2) == 0)] += 1;"),
    ("masks: NOT dropped", "uint64_t agree = ~(s ^ spread) & grp[t].mask;", "uint64_t agree = (s ^ spread) & grp[t].mask;"),
    ("masks: both directions", "for (int j = k + 1; j < n; ++j) {\n            int64_t v = K[k * n + j];",
     "for (int j = 0; j < n; ++j) {\n            int64_t v = K[k * n + j];"),
    ("masks: M from down spins", "g[((E + S) / 2) * (n + 1) + up] += 1;", "g[((E + S) / 2) * (n + 1) + (n - up) * (E != 0) + up * (E == 0)] += 1;"),
    ("frontier: energy sign", "dE -= Kuv * Su * Sv;", "dE += Kuv * Su * Sv;"),
    ("frontier: up count lost", "t1[(a1 * ne1 + e + de) * nm1 + m + sv] += c;", "t1[(a1 * ne1 + e + de) * nm1 + m + (sv && (v & 1))] += c;"),
    ("frontier cut: field sign", "int64_t dE = -f[v] * Sv;", "int64_t dE = +f[v] * Sv;"),
    ("frontier cut: cut's up count dropped", "if (cnt) gt[(e_cut + er) * (n + 1) + up + mr] += cnt;",
     "if (cnt) gt[(e_cut + er) * (n + 1) + mr] += cnt;"),
    ("frontier cut: bonds inside the cut dropped", "E_cut -= K[cut[a] * n + cut[b]] * spin[cut[a]] * spin[cut[b]];",
     "E_cut -= 0 * K[cut[a] * n + cut[b]] * spin[cut[a]] * spin[cut[b]];"),
    ("frontier cut: field of the last cut spin lost", "for (int a = 0; a < k; ++a) f[v] += K[v * n + cut[a]] * spin[cut[a]];",
     "for (int a = 0; a + 1 < k; ++a) f[v] += K[v * n + cut[a]] * spin[cut[a]];"),
    ("thermo: field sign", "long double H = E - f * M;\n                    long double w = expl(logl((long double)c) - H / t - Lmax);\n                    Z += w;",
     "long double H = E + f * M;\n                    long double w = expl(logl((long double)c) - H / t - Lmax);\n                    Z += w;"),
    ("thermo: C over T", "C[p] = (double)(vH / (t * t));", "C[p] = (double)(vH / t);"),
    ("thermo: chi over T^2", "chi[p] = (double)(vM / t);", "chi[p] = (double)(vM / (t * t));"),
    ("thermo: weights without g", "long double w = expl(logl((long double)c) - H / t - Lmax);\n                    Z += w;",
     "long double w = expl(0.0L * logl((long double)c) - H / t - Lmax);\n                    Z += w;"),
    ("thermo: variance not centred", "vH += w * (H - mH) * (H - mH);", "vH += w * H * H;"),
    ("thermo: energy mean uses M", "Z += w; sH += w * H; sM += w * M;", "Z += w; sH += w * E; sM += w * M;"),
    ("magnetisation: |M| dropped", "sA += w * fabsl(M);", "sA += w * M;"),
    ("magnetisation: cube for fourth", "s4 += w * M * M * M * M;", "s4 += w * M * M * M * fabsl(M) / (fabsl(M) + 1);"),
    # (a flipped field sign is an equivalent mutant here: every full table is symmetric in M, so
    # |M| and the even moments are even in h)
    ("magnetisation: field not over T", "long double w = expl(logl((long double)c) - (E - f * M) / t - Lmax);",
     "long double w = expl(logl((long double)c) - E / t + f * M - Lmax);"),
    ("magnetisation: Binder factor", "1.0L - m4 / (3.0L * m2 * m2)", "1.0L - m4 / (2.0L * m2 * m2)"),
]


def table1(path_rows):
    return {(E, M): nc for nc, M, E in path_rows}


def pins_pass(lib, table1_triples) -> bool:
    """A compact run of the pins; False as soon as one fails."""
    try:
        lat = w.square(4, 4, True)
        want = table1(table1_triples)
        for fn in (oracle.g_edges, oracle.g_masks, oracle.g_frontier):
            g = fn(lat.n, lat.edges, lib=lib)
            e_min, _, _ = oracle.bins(lat.n, lat.edges, lib=lib)
            got = {(e_min + 2 * int(e), -lat.n + 2 * int(m)): int(g[e, m]) for e, m in zip(*np.nonzero(g))}
            if got != want:
                return False
        # a free lattice (not in Table 1) through each method: ground states and binomial columns
        fl = w.square(3, 4, False)
        for fn in (oracle.g_edges, oracle.g_masks, oracle.g_frontier):
            g = fn(fl.n, fl.edges, lib=lib)
            if g[0, 0] != 1 or g[0, fl.n] != 1 or any(int(g[:, m].sum()) != math.comb(fl.n, m) for m in range(fl.n + 1)):
                return False
        # the programme conditioned on a cut: Table 1 with one row cut, and a signed random graph
        for cut in (0xF, 0xA5A5):
            g = oracle.g_frontier_cut(lat.n, lat.edges, cut, lib=lib)
            e_min, _, _ = oracle.bins(lat.n, lat.edges, lib=lib)
            got = {(e_min + 2 * int(e), -lat.n + 2 * int(m)): int(g[e, m]) for e, m in zip(*np.nonzero(g))}
            if got != want:
                return False
        cg = w.random_graph(10, 18, w.SplitMix64(12))
        want_c = brute_force_g_range(cg.n, [tuple(int(x) for x in r) for r in cg.edges], 0, 1 << cg.n)
        g = oracle.g_frontier_cut(cg.n, cg.edges, 0b1001101001, lib=lib)
        e_min, _, _ = oracle.bins(cg.n, cg.edges, lib=lib)
        if {(e_min + 2 * int(e), -cg.n + 2 * int(m)): int(g[e, m]) for e, m in zip(*np.nonzero(g))} != want_c:
            return False
        # configuration ranges: which words a range holds (spin i is bit i)
        rg = w.random_graph(9, 14, w.SplitMix64(11))
        edges = [tuple(int(x) for x in r) for r in rg.edges]
        want_r = brute_force_g_range(rg.n, edges, 37, 301)
        for fn in (oracle.g_edges, oracle.g_masks):
            g = fn(rg.n, rg.edges, 37, 301, lib=lib)
            e_min, _, _ = oracle.bins(rg.n, rg.edges, lib=lib)
            got = {(e_min + 2 * int(e), -rg.n + 2 * int(m)): int(g[e, m]) for e, m in zip(*np.nonzero(g))}
            if got != want_r:
                return False
        # thermodynamics: Kaufman, ring in a field, free spins
        e_min, _, _ = oracle.bins(lat.n, lat.edges, lib=lib)
        g = oracle.g_edges(lat.n, lat.edges, lib=lib)
        for t in (0.7, 2.2, 4.0):
            if abs(oracle.thermo(lat.n, e_min, g, [t], [0.0], lib=lib)[0][0, 0] - kaufman_logz(4, 4, t)) > 1e-10:
                return False
        r = w.ring(7)
        gr = oracle.g_edges(r.n, r.edges, lib=lib)
        er, _, _ = oracle.bins(r.n, r.edges, lib=lib)
        for t, f in ((0.9, 0.4), (2.0, -1.1)):
            if abs(oracle.thermo(r.n, er, gr, [t], [f], lib=lib)[0][0, 0] - ring_logz(7, t, f)) > 1e-10:
                return False
        n = 5
        g0 = oracle.g_edges(n, np.zeros((0, 3), dtype=np.int64), lib=lib)
        for t, f in ((0.6, 0.8), (2.5, -0.3)):
            lz, E, M, C, chi = (x[0, 0] for x in oracle.thermo(n, 0, g0, [t], [f], lib=lib))
            l0, m0, x0 = free_spins(n, t, f)
            if not (np.isclose(lz, l0, rtol=1e-12) and np.isclose(M, m0, rtol=1e-12) and np.isclose(chi, x0, rtol=1e-12)
                    and np.isclose(E, -f * m0, rtol=1e-12) and np.isclose(C, f * f * x0 / t, rtol=1e-12)):
                return False
            a, m2, m4, u = (x[0, 0] for x in oracle.magnetisation(n, 0, g0, [t], [f], lib=lib))
            a0, m20, m40 = free_spin_moments(n, t, f)
            if not (np.isclose(a, a0, rtol=1e-12) and np.isclose(m2, m20, rtol=1e-12) and np.isclose(m4, m40, rtol=1e-12)
                    and np.isclose(u, 1 - m40 / (3 * m20 * m20), rtol=1e-12)):
                return False
    except ValueError:
        return False
    return True


def run_child(index: int, workdir: str) -> int:
    """Exit status of a child that compiles mutant `index` (-1: no mutation) and runs the pins:
    0 = every pin passed, 1 = a pin failed, anything else = the child crashed."""
    here = os.path.dirname(os.path.abspath(__file__))
    env = dict(os.environ, PYTHONPATH=os.pathsep.join([os.path.dirname(here), here]))
    r = subprocess.run([sys.executable, os.path.abspath(__file__), str(index), workdir], env=env,
                       capture_output=True, text=True, timeout=300)
    return r.returncode


def test_unmutated_copy_passes(tmp_path):
    assert run_child(-1, str(tmp_path)) == 0


@pytest.mark.parametrize("index", range(len(MUTANTS)), ids=[m[0] for m in MUTANTS])
def test_mutant_is_caught(tmp_path, index):
    name, orig, bad = MUTANTS[index]
    assert oracle.source().count(orig) == 1, f"mutation anchor for {name!r} not found exactly once"
    assert run_child(index, str(tmp_path)) != 0, f"planted mistake {name!r} passed every pin"


def _table1_from_golden():
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "table1_4x4_periodic.txt")
    rows = []
    with open(path) as f:
        for line in f:
            line = line.strip()
            if line and not line.startswith("#"):
                rows.append(tuple(int(x) for x in line.split()))
    return rows


if __name__ == "__main__":
    idx, work = int(sys.argv[1]), sys.argv[2]
    src = oracle.source()
    if idx >= 0:
        src = src.replace(MUTANTS[idx][1], MUTANTS[idx][2])
    sys.exit(0 if pins_pass(oracle.load_variant(src, work), _table1_from_golden()) else 1)
