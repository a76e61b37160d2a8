"""Pins of the oracle's exact kNN (CPU only).

The C brute force is checked against an independent numpy brute force (full
distance matrix, lexicographic sort), and against properties the definition
fixes: symmetric canonical distances, equivariance under relabelling, exact
scaling by powers of two, tie-breaking by index, duplicates.
"""
import numpy as np
import pytest

from oracle import knn as K


def _lattice(n_side=6):
    g = np.stack(np.meshgrid(np.arange(n_side), np.arange(n_side), indexing="ij"), -1).reshape(-1, 2)
    return g.astype(np.float32) * 0.5


@pytest.mark.parametrize("m,k", [(2, 7), (3, 12), (5, 20), (17, 9)])
def test_c_matches_numpy_bruteforce_random(m, k):
    x = np.random.default_rng(10 + m).standard_normal((150, m)).astype(np.float32)
    a = K.knn(x, k)
    b = K.knn_dense(x, k)
    assert np.array_equal(a[0], b[0])
    assert np.array_equal(a[1], b[1])


def test_ties_break_by_index_on_lattice():
    # a square lattice has many exactly equal distances: ties must go to the smaller index
    x = _lattice(6)
    nbr, d2 = K.knn(x, 8)
    ref_nbr, ref_d2 = K.knn_dense(x, 8)
    assert np.array_equal(nbr, ref_nbr) and np.array_equal(d2, ref_d2)
    # interior point 14 = (2, 2): four neighbours at d2 = 0.25, ordered by index
    assert list(nbr[14, :4]) == [8, 13, 15, 20]
    assert np.all(d2[14, :4] == 0.25) and np.all(d2[14, 4:8] == 0.5)


def test_duplicates_are_neighbours_at_zero():
    x = np.random.default_rng(3).standard_normal((60, 3)).astype(np.float32)
    x[10] = x[20] = x[30]
    nbr, d2 = K.knn(x, 4)
    assert list(nbr[10, :2]) == [20, 30] and np.all(d2[10, :2] == 0.0)
    assert list(nbr[30, :2]) == [10, 20]


def test_canonical_distance_symmetric_bitwise():
    x = np.random.default_rng(4).standard_normal((80, 6)).astype(np.float32) * 3
    D = K.dense_d2(x)
    assert np.array_equal(D, D.T)
    a = np.repeat(np.arange(80), 80)
    b = np.tile(np.arange(80), 80)
    assert np.array_equal(K.pair_d2(x, a, b).reshape(80, 80), D)


def test_relabelling_equivariance():
    x = np.random.default_rng(5).standard_normal((200, 3)).astype(np.float32)
    perm = np.random.default_rng(6).permutation(200)
    nbr, d2 = K.knn(x, 10)
    nbr_p, d2_p = K.knn(x[perm], 10)
    inv = np.argsort(perm)
    # row i of the permuted problem is row perm[i] of the original, with indices mapped
    assert np.array_equal(perm[nbr_p], nbr[perm])
    assert np.array_equal(d2_p, d2[perm])
    assert inv[perm[0]] == 0


def test_power_of_two_scaling_is_exact():
    x = np.random.default_rng(7).standard_normal((120, 4)).astype(np.float32)
    nbr, d2 = K.knn(x, 15)
    nbr4, d24 = K.knn(x * np.float32(4.0), 15)
    assert np.array_equal(nbr, nbr4)
    assert np.array_equal(d2 * 16.0, d24)


def test_row_ranges_and_errors():
    x = np.random.default_rng(8).standard_normal((90, 2)).astype(np.float32)
    full = K.knn(x, 6)
    part = K.knn(x, 6, rows=(30, 55))
    assert np.array_equal(part[0], full[0][30:55]) and np.array_equal(part[1], full[1][30:55])
    with pytest.raises(ValueError):
        K.knn(x, 90)
    with pytest.raises(ValueError):
        K.knn(x, 0)
    rows = np.array([5, 77, 5, 0])
    r_nbr, r_d2 = K.knn_rows(x, 6, rows)
    assert np.array_equal(r_nbr, full[0][rows]) and np.array_equal(r_d2, full[1][rows])
    # k = n - 1 returns every other point
    nbr, _ = K.knn(x[:12], 11)
    assert all(sorted(nbr[i]) == [j for j in range(12) if j != i] for i in range(12))


@pytest.mark.parametrize("case", ["torus", "gauss100", "lattice_ties", "duplicates", "tiny"])
def test_large_n_path_equals_bruteforce(case):
    # the candidate-and-certificate path (k-d tree for m <= 8, FP64 matrix products for m > 8)
    # must return the brute force's lists bit for bit, ties and duplicates included
    from paper_2104_15124_gb300 import workloads as W
    if case == "torus":
        x, k = W.torus4(6000, 0.01, 3), 64
    elif case == "gauss100":
        x, k = W.gauss_embedded(3000, 5, 100, 1e-3, 4).x, 128
    elif case == "lattice_ties":
        g = np.stack(np.meshgrid(np.arange(30), np.arange(30), indexing="ij"), -1).reshape(-1, 2)
        x, k = g.astype(np.float32), 12
    elif case == "duplicates":
        b = np.random.default_rng(4).standard_normal((400, 12)).astype(np.float32)
        x, k = np.concatenate([b, b[:50], b[:50]]), 20
    else:
        x, k = np.random.default_rng(5).standard_normal((30, 3)).astype(np.float32), 29
    nbr, d2 = K.knn(x, k)
    a, b, _ = K.knn_large(x, k)
    assert np.array_equal(a, nbr) and np.array_equal(b, d2)
