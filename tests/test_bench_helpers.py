"""The benchmark's host-side bookkeeping (no GPU): algorithmic bytes per apply,
eigenvalue matching, and the error report against the oracle's stored solve."""
import importlib.util
import os

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _bench():
    spec = importlib.util.spec_from_file_location("bench_mod", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def test_step_bytes_counts_real_and_pair_passes():
    b = _bench()
    n, nnz_p, ns = 1000, 5000, 32
    roots = np.array([2.0, 1 + 1j, 1 - 1j, 3.0])
    tot, launches = b._step_bytes(n, nnz_p, ns, roots, vbytes=8, ibytes=2)
    mat = nnz_p * 10 + 4 * (ns + 1)
    assert launches == 4
    assert tot == 2 * (mat + 2 * n * 8) + (mat + 2 * n * 8) + (mat + 3 * n * 8)


def test_match_errors_pairs_each_value_once():
    b = _bench()
    a = np.array([1.0, 1.0 + 1e-9, 5.0])
    ref = np.array([5.0, 1.0, 1.0])
    e = b._match_errors(a, ref)
    assert e[0] == 0.0 and abs(e[1] - 1e-9) < 1e-15 and e[2] == 0.0


def test_oracle_errors_read_the_stored_solve():
    b = _bench()
    ref = []
    for line in open(os.path.join(ROOT, "tests", "golden", "plain_large_oracle.txt")):
        f = line.split()
        if f and f[0].startswith("lam") and f[0][3:].isdigit():
            ref.append(complex(float(f[1]), float(f[2])))
    assert len(ref) == 21
    assert b._oracle_errors(np.array(ref)) == [0.0] * 21
    e = b._oracle_errors(np.array(ref[:3]) * (1 + 1e-6))
    assert all(abs(x - 1e-6) < 1e-8 for x in e)
