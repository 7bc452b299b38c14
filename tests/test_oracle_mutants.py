"""The oracle's pins catch plausible mistakes.

Each case plants one mistake in a copy of the oracle's C source (a dropped
term, a wrong sign, transposed operands, lost exponent bookkeeping, a wrong
incidence rule, an odometer off by one), compiles it on the CPU, and checks
that at least one of the pins (nested sum, renormalised Ising, exponent-
spread slices) rejects it.  The oracle itself is never modified.
"""
import math
import os
import shutil
import subprocess
import tempfile

import numpy as np
import pytest

from oracle import brute, tree
from paper_2002_01935_gb300 import inputs, planner

SRC = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "oracle",
                   "tn_oracle.c")

MUTANTS = [
    ("dropped -Im*Im term", "acc_re += ar * br - ai * bi;", "acc_re += ar * br;"),
    ("wrong sign in Im part", "acc_im += ar * bi + ai * br;", "acc_im += ar * bi - ai * br;"),
    ("operands read transposed", "for (int i = t->rank - 1; i >= 0; --i) {\n        stride[t->lab[i]] = s;",
     "for (int i = 0; i < t->rank; ++i) {\n        stride[t->lab[i]] = s;"),
    ("renormalisation exponent lost", "t->exp2 += e;", "t->exp2 += 0;"),
    ("slices summed without exponent alignment",
     "f_new = ldexp(1.0, (int)(e_new - acc_exp));", "f_new = 1.0;"),
    ("hyperedge contracted too early", "if (is_open[l] || c < total[l]) outl[r++] = l;\n            }\n            for",
     "if (is_open[l] || c < 2) outl[r++] = l;\n            }\n            for"),
    ("odometer drops the last term", "for (i64 s = 0; s < n_sum_entries; ++s) {",
     "for (i64 s = 0; s + 1 < n_sum_entries; ++s) {"),
]


def _pins_pass(lib) -> bool:
    """True iff every pin accepts the library."""
    # nested sum on random complex networks with hyperedges and open labels
    for seed in range(6):
        net = inputs.random_network(7, 12, 500 + seed, n_open=seed % 3, max_dim=3)
        pairs = planner.greedy_tree(net.labels, net.dims, net.open)
        ref = brute.nested_sum(net.tensors, net.labels, net.dims, net.open)
        scale = brute.nested_sum([np.abs(t) for t in net.tensors], net.labels, net.dims, net.open)
        try:
            m, e = tree.contract(net.tensors, net.labels, net.dims, net.open, pairs, lib=lib)
        except ValueError:
            return False
        if not np.all(np.abs(m * 2.0 ** e - ref) <= 1e-12 * np.abs(scale) + 1e-300):
            return False
    # values far outside the double range: exponent bookkeeping
    net = inputs.random_ising(30, seed=1)
    pairs = planner.greedy_tree(net.labels, net.dims, net.open)
    scaled = [t if i < 30 else t * 2.0 ** 700 for i, t in enumerate(net.tensors)]
    m0, e0 = tree.contract(net.tensors, net.labels, net.dims, net.open, pairs, lib=lib)
    m1, e1 = tree.contract(scaled, net.labels, net.dims, net.open, pairs, lib=lib)
    if not (float(m0) > 0 and float(m1) > 0):
        return False
    if abs((math.log2(float(m1)) + e1) - (math.log2(float(m0)) + e0) - 700 * 45) > 1e-8:
        return False
    # slices whose values differ by 2^k, growing and shrinking: the slice sum
    # must align exponents in both directions
    a = np.array([[1.0, 2.0], [3.0, 4.0]])
    dims = {0: 2, 1: 2}
    for b in (np.array([1.0, 2.0 ** 200]), np.array([2.0 ** 30, 1.0])):
        m, e = tree.contract([a, b], [[0, 1], [1]], dims, [], [(0, 1)], [1], lib=lib)
        ref = (1 + 3) * b[0] + (2 + 4) * b[1]
        if abs(float(m) * 2.0 ** e - ref) > 1e-12 * ref:
            return False
    return True


def test_unmodified_oracle_passes_pins():
    assert _pins_pass(tree._load())


@pytest.mark.parametrize("name,orig,mutated", MUTANTS, ids=[m[0] for m in MUTANTS])
def test_planted_mistake_is_caught(name, orig, mutated, tmp_path):
    if shutil.which("gcc") is None:
        pytest.skip("gcc not available")
    src = open(SRC).read()
    assert src.count(orig) >= 1, f"mutation anchor not found: {name}"
    bad = src.replace(orig, mutated, 1)
    c = tmp_path / "mutant.c"
    so = tmp_path / "libmutant.so"
    c.write_text(bad)
    subprocess.run(["gcc", "-O1", "-fopenmp", "-fPIC", "-shared", "-o", str(so), str(c), "-lm"],
                   check=True)
    lib = tree.load_library(str(so))
    assert not _pins_pass(lib), f"pins did not catch: {name}"
