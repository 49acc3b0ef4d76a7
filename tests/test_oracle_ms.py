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



def _relaxed_energy(dims, r, nu, u):
    # the convex relaxation's objective: sum u r + nu x total variation over
    # the periodic faces (each voxel's three upper faces)
    nx, ny, nz = dims
    uu = np.asarray(u).reshape(nz, ny, nx)
    tv = 0.0
    for ax, n in zip((2, 1, 0), (nx, ny, nz)):
        if n > 1:
            tv += np.abs(uu - np.roll(uu, -1, axis=ax)).sum()
    return float((np.asarray(u) * np.asarray(r)).sum() + nu * tv)


def test_primal_gap_shrinks_with_the_iterations():
    # the relaxation's minimum equals Eq. 13's (coarea): the primal gap of
    # the relaxed u after k iterations against the exhaustive minimum of
    # Eq. 13 (both written relative to the all-vapor labelling) shrinks
    # with k and is tiny at the iteration count the pins use
    rng = np.random.default_rng(31)
    dims = (2, 2, 3)
    rho = rng.random(12)
    cl, cv, nu = 0.8, 0.1, 0.1
    r = (rho - cl) ** 2 - (rho - cv) ** 2
    e_vapor = ((rho - cv) ** 2).sum()
    best = min(energy_by_hand(dims, rho, cl, cv, nu, b) for b in ALL12) - e_vapor
    gaps = []
    for k in (10, 50, 200, 1000, 4000):
        _, u = oracle.ms_segment(dims, rho, cl, cv, nu, k)
        gaps.append(_relaxed_energy(dims, r, nu, u) - best)
    print("primal gap after 10/50/200/1000/4000 iterations:", ["%.2e" % g for g in gaps])
    assert all(g >= -1e-12 for g in gaps)
    assert gaps[-1] < 1e-9 and gaps[-1] <= gaps[0]


# ---- Eq. 13 as the detection's segmentation step (orc_ms_detect) ---------------
def _slab_counts(dims, lo, hi, rng, specks):
    # an integer density image (counts per voxel): a slab of 4s in [lo, hi)
    # along z, 0 elsewhere, with specks of the other phase at least two
    # voxels from the planes and from each other (each has 6 neighbours of
    # its surroundings' phase)
    nx, ny, nz = dims
    z = np.repeat(np.arange(nz), nx * ny)
    clean = np.where((z >= lo) & (z < hi), 0, 1).astype(np.uint8)
    B = np.where(clean == 0, 4.0, 0.0)
    ok = (np.abs(z - lo) >= 2) & (np.abs(z - (hi - 1)) >= 2) & (np.abs(z - lo + 1) >= 2) & \
        (np.abs(z - hi) >= 2)
    cand = rng.permutation(np.nonzero(ok)[0])
    taken = []
    for v in cand:
        x, y, zz = v % nx, (v // nx) % ny, v // (nx * ny)
        if all(max(abs(x - t[0]) % (nx - 1), abs(y - t[1]) % (ny - 1), abs(zz - t[2])) >= 2
               for t in taken):
            taken.append((x, y, zz))
            B[v] = 4.0 - B[v]
        if len(taken) == specks:
            break
    return B, clean


def test_detection_step_removes_specks_kmeans_keeps():
    dims = (8, 8, 24)
    rng = np.random.default_rng(41)
    B, clean = _slab_counts(dims, 8, 16, rng, 30)
    Sk, *_ = oracle.kmeans(B)
    assert (Sk != clean).sum() == 30                        # the threshold keeps every speck
    # the means are exactly 4 and 0: a speck keeps its own phase for a data
    # gain of 16 against 6 faces of perimeter, so nu above 16/6 removes it
    S, rounds = oracle.ms_detect(dims, B, 1.0, 3.0, 2000, 6, Sk)
    assert np.array_equal(S, clean)
    assert 1 <= rounds <= 6
    # small nu keeps them
    S0, _ = oracle.ms_detect(dims, B, 1.0, 2.0, 2000, 6, Sk)
    assert np.array_equal(S0, Sk)


def test_detection_step_is_a_fixed_point_and_lowers_the_energy():
    dims = (6, 7, 20)
    rng = np.random.default_rng(42)
    z = np.repeat(np.arange(20), 42)
    B = np.where((z >= 6) & (z < 14), 3.0, 0.0) + rng.integers(0, 3, z.size)
    Sk, *_ = oracle.kmeans(B)
    inv = 0.5
    S, rounds = oracle.ms_detect(dims, B, inv, 1.2, 1500, 10, Sk)
    assert rounds < 10                                      # stopped because the labels repeat
    again, r2 = oracle.ms_detect(dims, B, inv, 1.2, 1500, 1, S)
    assert np.array_equal(again, S) and r2 == 1

    def means(T):
        return (B[T == 0].sum() / (T == 0).sum() * inv, B[T == 1].sum() / (T == 1).sum() * inv)

    rho = B * inv
    e_k = oracle.ms_energy(dims, rho, *means(Sk), 1.2, Sk)
    e_s = oracle.ms_energy(dims, rho, *means(S), 1.2, S)
    assert e_s <= e_k


def test_detection_step_without_perimeter_is_the_threshold_of_its_means():
    dims = (5, 6, 14)
    rng = np.random.default_rng(43)
    B = rng.integers(0, 7, 420).astype(float)
    Sk, *_ = oracle.kmeans(B)
    S, _ = oracle.ms_detect(dims, B, 0.25, 0.0, 200, 8, Sk)
    cl = B[S == 0].sum() / (S == 0).sum() * 0.25
    cv = B[S == 1].sum() / (S == 1).sum() * 0.25
    assert np.array_equal(S, np.where(B * 0.25 > 0.5 * (cl + cv), 0, 1).astype(np.uint8)) or \
        np.array_equal(S, Sk)


def test_detection_step_leaves_a_single_phase_alone():
    dims = (4, 4, 4)
    B = np.full(64, 2.0)
    S = np.zeros(64, np.uint8)
    out, rounds = oracle.ms_detect(dims, B, 1.0, 0.1, 50, 4, S)
    assert rounds == 0 and np.array_equal(out, S)


def test_detect_with_eq13_recovers_the_slab_planes():
    from paper_1502_03234_gb300 import slabgen

    s = slabgen.make_slab(16000, seed=7)
    pk = oracle.DetectParams()
    pm = oracle.DetectParams(segmentation=1)
    dk = oracle.detect(s.x, s.box, pk)
    dm = oracle.detect(s.x, s.box, pm)
    nx, ny, nz = dm.dims
    hz = s.box[2] / nz
    zc = (np.arange(nz) + 0.5) * hz
    z0, z1 = s.z_planes
    far = (np.abs(zc - z0) > 2 * hz) & (np.abs(zc - z1) > 2 * hz)
    want = np.where((zc > z0) & (zc < z1), 0, 1)
    S = dm.S.reshape(nz, ny, nx)
    assert np.all(S[far] == want[far][:, None, None])
    # Eq. 13 moves only voxels next to the K-means interface
    changed = dm.S != dk.S
    print("voxels Eq. 13 changed against K-means:", int(changed.sum()))
    zc_changed = zc[np.nonzero(changed.reshape(nz, ny, nx))[0]]
    assert np.all(np.minimum(np.abs(zc_changed - z0), np.abs(zc_changed - z1)) < 4 * hz)
    assert np.all(dm.rc >= 3.0) and np.all(dm.rc <= 6.0)
