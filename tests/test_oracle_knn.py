"""Pins of the oracle's kNN (reading R1: exact float32 key, ties to the
lower index, self included) against a scalar brute force and invariances."""
import numpy as np
import pytest

import oracle as O


def scalar_knn(P, k):
    """Brute force, one scalar at a time: every operation rounded to float32,
    then the first k of the (key, index) order."""
    P = np.asarray(P, dtype=np.float32)
    out = []
    for q in range(len(P)):
        keys = []
        for j in range(len(P)):
            dx = np.float32(P[q, 0]) - np.float32(P[j, 0])
            dy = np.float32(P[q, 1]) - np.float32(P[j, 1])
            dz = np.float32(P[q, 2]) - np.float32(P[j, 2])
            key = np.float32(np.float32(np.float32(dx * dx) + np.float32(dy * dy)) + np.float32(dz * dz))
            keys.append((float(key), j))
        keys.sort()
        out.append([j for _, j in keys[:k]])
    return np.array(out, dtype=np.int32)


def test_knn_matches_scalar_bruteforce_random():
    rng = np.random.default_rng(7)
    P = rng.normal(size=(70, 3)).astype(np.float32)
    np.testing.assert_array_equal(O.knn(P, 16), scalar_knn(P, 16))


def test_knn_ties_go_to_lower_index():
    # integer grid: many exactly equal keys; duplicates too
    g = np.array([[x, y, z] for x in range(4) for y in range(3) for z in range(3)], dtype=np.float32)
    P = np.concatenate([g, g[:5]])          # rows 36..40 duplicate rows 0..4
    ref = scalar_knn(P, 9)
    got = O.knn(P, 9)
    np.testing.assert_array_equal(got, ref)
    # a duplicate's first neighbour is the lower-index copy (key 0, lower index)
    assert got[36, 0] == 0 and got[36, 1] == 36
    # among the 6 face neighbours of an interior grid point at key 1 the order is by index
    q = 1 * 9 + 1 * 3 + 1   # (1, 1, 1)
    ones = [j for j in got[q] if j != q and j < 36]
    assert ones[:6] == sorted(ones[:6])


def test_knn_self_first_for_distinct_points():
    rng = np.random.default_rng(3)
    P = rng.uniform(-1, 1, size=(200, 3)).astype(np.float32)
    nb = O.knn(P, 16)
    np.testing.assert_array_equal(nb[:, 0], np.arange(200))


def test_knn_invariant_under_exact_shift():
    rng = np.random.default_rng(11)
    P = rng.integers(-8, 8, size=(150, 3)).astype(np.float32)
    Q = P + np.float32(64.0)        # exact: small integers + 2^6
    np.testing.assert_array_equal(O.knn(P, 16), O.knn(Q, 16))


def test_knn_rejects_k_above_n():
    with pytest.raises(ValueError):
        O.knn(np.zeros((3, 3), np.float32), 4)


def test_nearest_matches_scalar_bruteforce():
    rng = np.random.default_rng(8)
    X = rng.integers(-3, 3, size=(40, 3)).astype(np.float32)    # integer grid: exact ties
    Q = rng.integers(-3, 3, size=(25, 3)).astype(np.float32) + np.float32(0.5)
    idx, key = O.nearest(Q, X)
    for i in range(len(Q)):
        cands = []
        for j in range(len(X)):
            dx = np.float32(Q[i, 0]) - np.float32(X[j, 0])
            dy = np.float32(Q[i, 1]) - np.float32(X[j, 1])
            dz = np.float32(Q[i, 2]) - np.float32(X[j, 2])
            k = np.float32(np.float32(np.float32(dx * dx) + np.float32(dy * dy)) + np.float32(dz * dz))
            cands.append((float(k), j))
        cands.sort()
        assert (int(idx[i]), float(key[i])) == (cands[0][1], cands[0][0])
    mask, dist = O.change_mask(Q, X, 0.9)
    np.testing.assert_array_equal(mask, (key > np.float32(0.81)).astype(np.uint8))


def _per_op_key(q, p):
    dx = np.float32(q[0]) - np.float32(p[0])
    dy = np.float32(q[1]) - np.float32(p[1])
    dz = np.float32(q[2]) - np.float32(p[2])
    return np.float32(np.float32(np.float32(dx * dx) + np.float32(dy * dy)) + np.float32(dz * dz))


def test_knn_key_is_rounded_per_operation():
    """(a, b, c) and (c, a, b) are equally far from the origin, but the float32
    key (dx*dx + dy*dy) + dz*dz rounds differently for them; the order must
    follow the rounded keys (R1), not the exact distances."""
    rng = np.random.default_rng(123)
    q = np.zeros(3, np.float32)
    for _ in range(10000):
        a, b, c = rng.uniform(0.5, 1.0, 3).astype(np.float32)
        p_lo, p_hi = np.array([c, a, b], np.float32), np.array([a, b, c], np.float32)
        if _per_op_key(q, p_hi) < _per_op_key(q, p_lo):     # the higher index must come first
            break
    else:
        pytest.skip("no distinguishing case found")
    far = rng.uniform(5.0, 6.0, size=(6, 3)).astype(np.float32)
    P = np.concatenate([q[None], p_lo[None], p_hi[None], far])
    nb = O.knn(P, 3)
    assert list(nb[0]) == [0, 2, 1]
