"""Pins of the oracle's two-phase Mumford-Shah segmentation (Eq. 13) with the
densities fixed: the relaxed primal-dual solver against exhaustive
enumeration of every labelling on 12-voxel grids, the nu = 0 limit (the
pointwise threshold of the K-means rule, Eq. 11-12), and a noisy slab whose
two planes the perimeter term restores."""
import itertools

import numpy as np
import pytest

import oracle

ALL12 = [np.array(b, np.uint8) for b in itertools.product([0, 1], repeat=12)]


def energy_by_hand(dims, rho, c_l, c_v, nu, S):
    # Eq. 13 written out: data terms plus nu x the liquid/vapor faces of the
    # periodic grid (each voxel's three upper faces)
    nx, ny, nz = dims
    s = np.asarray(S).reshape(nz, ny, nx)
    r = np.asarray(rho).reshape(nz, ny, nx)
    data = np.where(s == 0, (r - c_l) ** 2, (r - c_v) ** 2).sum()
    faces = 0
    for ax, n in zip((2, 1, 0), (nx, ny, nz)):
        if n > 1:
            faces += int((s != np.roll(s, -1, axis=ax)).sum())
    return data + nu * faces


@pytest.mark.parametrize("dims", [(2, 2, 3), (3, 2, 2), (1, 3, 4)])
@pytest.mark.parametrize("nu", [0.02, 0.1, 0.3])
def test_relaxation_reaches_the_exhaustive_minimum(dims, nu):
    rng = np.random.default_rng(int(100 * nu) + dims[0])
    for _ in range(3):
        rho = rng.random(12)
        S, u = oracle.ms_segment(dims, rho, 0.8, 0.1, nu, 4000)
        best = min(energy_by_hand(dims, rho, 0.8, 0.1, nu, b) for b in ALL12)
        e = oracle.ms_energy(dims, rho, 0.8, 0.1, nu, S)
        assert e == pytest.approx(energy_by_hand(dims, rho, 0.8, 0.1, nu, S), rel=1e-12)
        assert e == pytest.approx(best, rel=1e-9, abs=1e-12)


def test_no_perimeter_term_is_the_threshold_rule():
    # nu = 0: each voxel independently takes the nearer density, i.e. liquid
    # iff rho > (c_l + c_v)/2 -- the K-means labelling rule
    rng = np.random.default_rng(7)
    dims = (6, 5, 9)
    rho = rng.random(270)
    S, _ = oracle.ms_segment(dims, rho, 0.7, 0.2, 0.0, 200)
    assert np.array_equal(S, np.where(rho > 0.45, 0, 1).astype(np.uint8))


def test_noisy_slab_recovers_its_planes():
    dims = (8, 8, 24)
    z = np.repeat(np.arange(24), 64)
    clean = np.where((z >= 8) & (z < 16), 0, 1).astype(np.uint8)
    rng = np.random.default_rng(5)
    rho = np.where(clean == 0, 0.8, 0.05) + rng.uniform(-0.5, 0.5, clean.size)
    S0, _ = oracle.ms_segment(dims, rho, 0.8, 0.05, 0.0, 3000)
    assert (S0 != clean).sum() > 100                        # the threshold alone is noisy
    S, u = oracle.ms_segment(dims, rho, 0.8, 0.05, 0.2, 3000)
    assert np.array_equal(S, clean)
    assert oracle.ms_energy(dims, rho, 0.8, 0.05, 0.2, S) < oracle.ms_energy(dims, rho, 0.8, 0.05,
                                                                              0.2, S0)
    assert np.all((u == 0.0) | (u == 1.0))                   # the relaxed minimiser is binary here


def test_larger_nu_never_lengthens_the_perimeter():
    # minimisers of data + nu x perimeter have a perimeter non-increasing in nu
    rng = np.random.default_rng(11)
    dims = (2, 2, 3)
    rho = rng.random(12)
    per = []
    for nu in (0.0, 0.01, 0.03, 0.1, 0.3, 1.0):
        S, _ = oracle.ms_segment(dims, rho, 0.8, 0.1, nu, 4000)
        per.append(energy_by_hand(dims, rho, 0.8, 0.1, 1.0, S) - energy_by_hand(dims, rho, 0.8, 0.1,
                                                                                 0.0, S))
    assert all(a >= b for a, b in zip(per, per[1:]))


def test_alternation_without_perimeter_is_kmeans():
    # nu = 0: segmenting with fixed densities is the nearest-centre rule and
    # the density update the centre update, so alternating from (max, min)
    # is Lloyd's K-means (Eq. 14) -- same labels, same centres
    rng = np.random.default_rng(21)
    dims = (7, 6, 10)
    rho = np.concatenate([rng.normal(0.8, 0.15, 200), rng.normal(0.1, 0.15, 220)])
    rng.shuffle(rho)
    Sk, cl_k, cv_k, _ = oracle.kmeans(rho)
    S, cl, cv, rounds = oracle.ms_alternate(dims, rho, 0.0, 100, 50, rho.max(), rho.min())
    assert np.array_equal(S, Sk)
    assert cl == pytest.approx(cl_k, rel=1e-12) and cv == pytest.approx(cv_k, rel=1e-12)
    assert rounds >= 2


def test_alternation_lowers_the_energy():
    dims = (8, 8, 24)
    z = np.repeat(np.arange(24), 64)
    clean = np.where((z >= 8) & (z < 16), 0, 1).astype(np.uint8)
    rng = np.random.default_rng(6)
    rho = np.where(clean == 0, 0.8, 0.05) + rng.uniform(-0.5, 0.5, clean.size)
    c0 = (rho.max(), rho.min())
    S1, _ = oracle.ms_segment(dims, rho, c0[0], c0[1], 0.2, 3000)
    S, cl, cv, rounds = oracle.ms_alternate(dims, rho, 0.2, 3000, 20, *c0)
    assert oracle.ms_energy(dims, rho, cl, cv, 0.2, S) <= oracle.ms_energy(dims, rho, *c0, 0.2, S1)
    assert np.array_equal(S, clean)
    assert cl == pytest.approx(rho[clean == 0].mean(), rel=1e-12)
    assert cv == pytest.approx(rho[clean == 1].mean(), rel=1e-12)

