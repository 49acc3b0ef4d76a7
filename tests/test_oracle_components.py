"""Pins of the oracle's small-component removal (Section 4.2, Fig. 20-21,
Algorithm 4.1) against an independent flood fill and hand-built grids.

The oracle labels by the row-major two-pass method with an equivalence table;
the brute force here is a breadth-first flood fill over the 6 periodic face
neighbours, so a mistake in the pass order, the equivalence merge or the
periodic faces shows up as a different partition."""
from collections import deque

import numpy as np
import pytest

import oracle


def flood_labels(dims, S, phase):
    """components by breadth-first search, numbered in order of first
    appearance (x fastest), -1 for the other phase"""
    nx, ny, nz = dims
    S = np.asarray(S, np.uint8).reshape(nz, ny, nx)
    lab = -np.ones((nz, ny, nx), np.int64)
    n = 0
    for z in range(nz):
        for y in range(ny):
            for x in range(nx):
                if S[z, y, x] != phase or lab[z, y, x] >= 0:
                    continue
                lab[z, y, x] = n
                q = deque([(z, y, x)])
                while q:
                    c, b, a = q.popleft()
                    for dz, dy, dx in ((1, 0, 0), (-1, 0, 0), (0, 1, 0), (0, -1, 0),
                                       (0, 0, 1), (0, 0, -1)):
                        t = ((c + dz) % nz, (b + dy) % ny, (a + dx) % nx)
                        if S[t] == phase and lab[t] < 0:
                            lab[t] = n
                            q.append(t)
                n += 1
    return lab.ravel(), n


def flood_remove(dims, S, m):
    S = np.array(S, np.uint8).ravel()
    flipped = 0
    for phase in (0, 1):
        lab, n = flood_labels(dims, S, phase)
        size = np.bincount(lab[lab >= 0], minlength=max(n, 1))
        small = (lab >= 0) & (size[np.maximum(lab, 0)] < m)
        S[small] = 1 - phase
        flipped += int(small.sum())
    return S, flipped


def grid(dims, fill=1):
    return np.full(dims[0] * dims[1] * dims[2], fill, np.uint8)


def at(dims, x, y, z):
    return x + dims[0] * (y + dims[1] * z)


@pytest.mark.parametrize("dims", [(7, 5, 6), (1, 6, 5), (2, 3, 9), (8, 8, 1), (1, 1, 7), (4, 4, 4)])
@pytest.mark.parametrize("p", [0.25, 0.45, 0.6])
def test_labels_match_flood_fill(dims, p):
    rng = np.random.default_rng(hash((dims, p)) % 2**32)
    S = (rng.random(dims[0] * dims[1] * dims[2]) >= p).astype(np.uint8)   # P(liquid) = p
    for phase in (0, 1):
        lab, n = oracle.label_components(dims, S, phase)
        ref, nref = flood_labels(dims, S, phase)
        assert n == nref
        assert np.array_equal(lab, ref)


@pytest.mark.parametrize("m", [1, 2, 5, 9])
def test_removal_matches_flood_fill(m):
    rng = np.random.default_rng(100 + m)
    for dims in ((9, 7, 8), (6, 6, 12), (3, 10, 4)):
        for p in (0.3, 0.5, 0.7):
            S = (rng.random(dims[0] * dims[1] * dims[2]) >= p).astype(np.uint8)
            out, fl = oracle.remove_small_components(dims, S, m)
            ref, fref = flood_remove(dims, S, m)
            assert fl == fref
            assert np.array_equal(out, ref)
            if m == 1:          # every component has at least one voxel
                assert fl == 0 and np.array_equal(out, S)


def test_threshold_is_strict():
    # components smaller than the threshold go, equal ones stay
    d = (10, 10, 10)
    S = grid(d)
    for x, y in ((1, 1), (2, 1), (1, 2), (2, 2)):            # 4 voxels
        S[at(d, x, y, 2)] = 0
    for x, y in ((6, 6), (5, 6), (7, 6), (6, 5), (6, 7)):    # 5 voxels (a plus)
        S[at(d, x, y, 6)] = 0
    out, fl = oracle.remove_small_components(d, S, 5)
    assert fl == 4
    assert out[at(d, 1, 1, 2)] == 1 and out[at(d, 6, 6, 6)] == 0
    assert int((out == 0).sum()) == 5


def test_components_join_across_periodic_faces():
    d = (8, 6, 6)
    S = grid(d)
    for x in (0, 7):                     # one component of 2 x 2 voxels through x = 0 / 7
        for y in (2, 3):
            S[at(d, x, y, 3)] = 0
    lab, n = oracle.label_components(d, S, 0)
    assert n == 1
    out, fl = oracle.remove_small_components(d, S, 5)
    assert fl == 4 and np.all(out == 1)
    out, fl = oracle.remove_small_components(d, S, 4)
    assert fl == 0
    # moved off the face, the halves are two components of 2
    S2 = grid(d)
    for x in (1, 6):
        for y in (2, 3):
            S2[at(d, x, y, 3)] = 0
    assert oracle.label_components(d, S2, 0)[1] == 2
    assert oracle.remove_small_components(d, S2, 3)[1] == 4
    # the same through the y and z faces
    for ax in (1, 2):
        S3 = grid(d)
        for k in (0, d[ax] - 1):
            c = [3, 3, 3]
            c[ax] = k
            S3[at(d, *c)] = 0
        assert oracle.label_components(d, S3, 0)[1] == 1


def test_edge_and_corner_contacts_do_not_connect():
    d = (6, 6, 6)
    S = grid(d)
    S[at(d, 1, 1, 1)] = 0
    S[at(d, 2, 2, 1)] = 0          # shares an edge
    S[at(d, 3, 3, 2)] = 0          # shares a corner with the one before
    lab, n = oracle.label_components(d, S, 0)
    assert n == 3


def test_liquid_components_go_before_vapor_ones():
    # a liquid 3x3x3 shell (26 voxels) around a one-voxel vapor cavity, with
    # threshold 27: liquid first removes the shell (26 < 27), after which the
    # cavity is part of the surrounding vapor; vapor first would fill the
    # cavity and keep a 27-voxel liquid cube
    d = (9, 9, 9)
    S = grid(d)
    for z in range(3, 6):
        for y in range(3, 6):
            for x in range(3, 6):
                S[at(d, x, y, z)] = 0
    S[at(d, 4, 4, 4)] = 1
    out, fl = oracle.remove_small_components(d, S, 27)
    assert fl == 26 and np.all(out == 1)
    # threshold 26: the shell stays and the cavity (1 < 26) is filled
    out, fl = oracle.remove_small_components(d, S, 26)
    assert fl == 1 and int((out == 0).sum()) == 27


def test_slab_with_specks_recovers_the_planes():
    # a flat liquid slab z in [4, 10) with isolated liquid specks in the
    # vapor and vapor specks in the liquid: removal restores the two planes
    d = (12, 10, 16)
    S = grid(d)
    for z in range(4, 10):
        S[d[0] * d[1] * z: d[0] * d[1] * (z + 1)] = 0
    clean = S.copy()
    rng = np.random.default_rng(3)
    for _ in range(12):
        x, y = rng.integers(0, 12), rng.integers(0, 10)
        S[at(d, x, y, int(rng.choice([1, 13, 14])))] = 0        # vapor rows
        S[at(d, x, y, int(rng.choice([6, 7])))] = 1             # liquid rows
    out, fl = oracle.remove_small_components(d, S, 5)
    assert np.array_equal(out, clean)
    assert fl == int((S != clean).sum())


def test_no_threshold_changes_nothing():
    rng = np.random.default_rng(9)
    d = (5, 6, 7)
    S = (rng.random(210) < 0.5).astype(np.uint8)
    for m in (0, -3):
        out, fl = oracle.remove_small_components(d, S, m)
        assert fl == 0 and np.array_equal(out, S)
