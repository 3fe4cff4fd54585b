"""Input generator checks (no GPU): shape, cleaning, determinism, R-MAT statistics."""
import os
import subprocess
import sys

import numpy as np

import graphgen

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _check_clean_symmetric(ro, col):
    n = len(ro) - 1
    assert ro[0] == 0 and ro[-1] == len(col)
    assert np.all(np.diff(ro) >= 0)
    assert col.min() >= 0 and col.max() < n
    src = np.repeat(np.arange(n, dtype=np.int64), np.diff(ro))
    assert not np.any(src == col), "self-loop left in"
    key = src * n + col
    assert np.all(np.diff(key) > 0), "rows not strictly sorted (duplicate or unsorted)"
    rkey = col.astype(np.int64) * n + src
    assert np.array_equal(np.sort(rkey), key), "not symmetric"


def test_kronecker_clean_and_symmetric():
    ro, col = graphgen.kronecker(12, 16, 5)
    assert len(ro) == 4097
    _check_clean_symmetric(ro, col)
    # 2^12*16 tuples -> at most twice that many directed entries after cleaning
    assert 0.5 * 2 * 65536 < len(col) <= 2 * 65536


def test_erdos_renyi_clean_and_symmetric():
    ro, col = graphgen.erdos_renyi(12, 16, 5)
    _check_clean_symmetric(ro, col)
    deg = np.diff(ro)
    # uniform endpoints: low skew, nearly every vertex has edges
    assert deg.max() < 80 and (deg == 0).sum() < 5


def test_deterministic_and_seed_sensitive():
    a = graphgen.kronecker(11, 16, 9)
    b = graphgen.kronecker(11, 16, 9)
    c = graphgen.kronecker(11, 16, 10)
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])
    assert not np.array_equal(a[1][:1000], c[1][:1000])


def test_thread_count_does_not_change_the_graph():
    code = ("import sys, hashlib; sys.path.insert(0, %r); import graphgen;"
            "ro, col = graphgen.kronecker(13, 16, 4);"
            "print(hashlib.sha256(ro.tobytes() + col.tobytes()).hexdigest())" % ROOT)
    out = []
    for t in ("1", "3"):
        env = dict(os.environ, OMP_NUM_THREADS=t)
        out.append(subprocess.run([sys.executable, "-c", code], env=env, check=True,
                                  capture_output=True, text=True).stdout.strip())
    assert out[0] == out[1]


def test_rmat_quadrant_frequencies():
    # before permutation the top bit of (src, dst) follows the initiator:
    # P(src bit 0) = A + B = 0.76, P(dst bit 0) = A + C = 0.76, P(both 1) = D = 0.05
    src, dst = graphgen.rmat_tuples(14, 16, 2)
    top = 1 << 13
    s1 = (src & top) != 0
    d1 = (dst & top) != 0
    assert abs((~s1).mean() - 0.76) < 0.005
    assert abs((~d1).mean() - 0.76) < 0.005
    assert abs((s1 & d1).mean() - 0.05) < 0.003
    assert abs((~s1 & ~d1).mean() - 0.57) < 0.005


def test_permutation_is_a_permutation():
    p = graphgen.permutation(1000, 3)
    assert np.array_equal(np.sort(p), np.arange(1000))
    assert not np.array_equal(p, np.arange(1000))


def test_pick_roots():
    ro, col = graphgen.kronecker(10, 16, 1)
    r = graphgen.pick_roots(ro, 64, 1)
    assert len(r) == 64 and len(set(r.tolist())) == 64
    assert np.all(np.diff(ro)[r] >= 1)
    r2 = graphgen.pick_roots(ro, 5000, 1, distinct=False)
    assert len(r2) == 5000 and np.all(np.diff(ro)[r2] >= 1)
    assert np.array_equal(graphgen.pick_roots(ro, 64, 1), r)


def test_directed_build_keeps_direction():
    ro, col = graphgen.csr_from_tuples(4, np.array([0, 1, 1], np.int32),
                                       np.array([1, 2, 2], np.int32), symmetrize=False)
    assert ro.tolist() == [0, 1, 2, 2, 2] and col.tolist() == [1, 2]
