"""Pins of the oracle's interface detection (Section 4): density image,
smoothing, two-class K-means, Godunov/FSM/CFSM distances, trilinear lookup."""
import math
import os

import numpy as np
import pytest

from paper_1502_03234_gb300 import slabgen

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# ---- Eq. 9 -------------------------------------------------------------------
def test_density_counts_every_particle_once(orc):
    L = (10.0, 9.0, 30.0)
    x, _ = slabgen.make_gas(500, L, seed=1)
    dims = orc.grid_dims(L, 1.0)
    assert dims == (10, 9, 30)
    B = orc.density(x, L, dims)
    assert B.sum() == 500 and B.min() >= 0
    # brute force: voxel index of each particle from its coordinates
    ref = np.zeros(int(np.prod(dims)), np.int64)
    for p in x:
        ix = [orc.bin_index(p[a], dims[a], L[a]) for a in range(3)]
        ref[ix[0] + dims[0] * (ix[1] + dims[1] * ix[2])] += 1
    assert np.array_equal(B, ref)


def test_grid_dims_reading_of_eq10(orc):
    # N_x = max(3, floor(L_x / b)), so b_x = L_x / N_x >= b
    assert orc.grid_dims((23.94, 23.94, 95.76), 1.0) == (23, 23, 95)
    assert orc.grid_dims((2.0, 5.5, 7.9), 2.6) == (3, 3, 3)


# ---- smoothing --------------------------------------------------------------
def test_smoothing_of_a_delta_is_the_binomial_kernel(orc):
    dims = (15, 13, 17)
    B = np.zeros(int(np.prod(dims)), np.int32)
    c = (7, 6, 8)
    B[c[0] + dims[0] * (c[1] + dims[1] * c[2])] = 1
    Bs = orc.smooth(dims, B, 8).reshape(dims[2], dims[1], dims[0])
    for dz in range(-5, 6):
        for dy in range(-5, 6):
            for dx in range(-5, 6):
                w = 1
                for d in (dx, dy, dz):
                    w *= math.comb(8, d + 4) if abs(d) <= 4 else 0
                assert Bs[c[2] + dz, c[1] + dy, c[0] + dx] == w


def test_smoothing_conserves_mass_and_constants(orc):
    rng = np.random.default_rng(2)
    dims = (9, 11, 12)
    B = rng.integers(0, 6, int(np.prod(dims))).astype(np.int32)
    Bs = orc.smooth(dims, B, 8)
    assert Bs.sum() == 256 ** 3 * B.sum()                 # exact integers
    assert np.all(Bs == np.round(Bs))
    const = np.full(int(np.prod(dims)), 3, np.int32)
    assert np.all(orc.smooth(dims, const, 8) == 3 * 256 ** 3)
    assert np.array_equal(orc.smooth(dims, B, 0), B.astype(np.float64))


def test_smoothing_wraps_periodically_on_tiny_grids(orc):
    # a kernel wider than the grid wraps more than once; mass still conserved
    dims = (3, 3, 4)
    rng = np.random.default_rng(3)
    B = rng.integers(0, 4, 36).astype(np.int32)
    Bs = orc.smooth(dims, B, 8)
    assert Bs.sum() == 256 ** 3 * B.sum()


# ---- Eq. 14 (K = 2) -------------------------------------------------------------
def _global_two_means(values):
    """brute force over every threshold split of the sorted values"""
    v = np.sort(values)
    best = None
    for k in range(1, len(v)):
        if v[k] == v[k - 1]:
            continue
        lo, hi = v[:k], v[k:]
        e = ((lo - lo.mean()) ** 2).sum() + ((hi - hi.mean()) ** 2).sum()
        if best is None or e < best[0] - 1e-9:
            best = (e, v[k])
    return best[1]


def test_kmeans_two_levels_exact(orc):
    v = np.array([2.0] * 30 + [10.0] * 70)
    S, cl, cv, it = orc.kmeans(v)
    assert cl == 10.0 and cv == 2.0
    assert np.array_equal(S, (v < 6).astype(np.uint8))


@pytest.mark.parametrize("seed", range(6))
def test_kmeans_reaches_the_global_optimum_on_bimodal_data(orc, seed):
    rng = np.random.default_rng(seed)
    a = np.round(rng.normal(20, 4, 400))
    b = np.round(rng.normal(200, 30, 300))
    v = np.concatenate([a, b])
    rng.shuffle(v)
    S, cl, cv, it = orc.kmeans(v)
    thr = _global_two_means(v)
    assert np.array_equal(S == 0, v >= thr)
    assert cl == pytest.approx(v[v >= thr].mean(), rel=1e-15)
    assert cv == pytest.approx(v[v < thr].mean(), rel=1e-15)


def test_kmeans_constant_image_is_all_liquid(orc):
    S, cl, cv, it = orc.kmeans(np.full(50, 7.0))
    assert np.all(S == 0)


# ---- Eq. 16-19 --------------------------------------------------------------
def _golden_godunov():
    rows = []
    with open(os.path.join(GOLDEN, "godunov_hand.txt")) as fh:
        for line in fh:
            line = line.split("#")[0].strip()
            if line:
                rows.append([float(t) for t in line.split()])
    return rows


def test_godunov_hand_solved_values(orc):
    for a0, a1, a2, h0, h1, h2, expect in _golden_godunov():
        got = orc.godunov([a0, a1, a2], [h0, h1, h2])
        assert got == pytest.approx(expect, rel=1e-14, abs=1e-14)


def test_godunov_solution_satisfies_eq16(orc):
    rng = np.random.default_rng(4)
    for _ in range(2000):
        a = rng.uniform(0, 3, 3)
        h = rng.uniform(0.5, 1.5, 3)
        d = orc.godunov(a, h)
        s = sum(max(d - ak, 0.0) ** 2 / hk ** 2 for ak, hk in zip(a, h))
        assert s == pytest.approx(1.0, rel=1e-12)
        assert d > min(a)


def _point_source(dims):
    S = np.zeros(int(np.prod(dims)), np.uint8)
    S[0] = 1  # vapor voxel at the origin (periodic)
    return S


def test_fsm_point_source_hand_values(orc):
    dims = (21, 21, 21)
    h = 1.0
    D, rounds = orc.fsm(dims, (h, h, h), _point_source(dims))
    D = D.reshape(dims[2], dims[1], dims[0])
    for k in range(1, 8):
        assert D[0, 0, k] == pytest.approx(k * h, abs=1e-14)
        assert D[0, k, 0] == pytest.approx(k * h, abs=1e-14)
    assert D[0, 1, 1] == pytest.approx(h * (1 + 1 / math.sqrt(2)), abs=1e-14)
    assert D[1, 1, 1] == pytest.approx(h * (1 + 1 / math.sqrt(2) + 1 / math.sqrt(3)), abs=1e-14)
    # symmetric under the periodic reflections
    assert D[0, 0, 3] == D[0, 0, dims[0] - 3]
    assert D[2, 1, 3] == pytest.approx(D[3, 2, 1], abs=1e-14)


def test_fsm_anisotropic_hand_value(orc):
    dims = (15, 15, 15)
    D, _ = orc.fsm(dims, (1.0, 2.0, 1.0), _point_source(dims))
    D = D.reshape(dims[2], dims[1], dims[0])
    assert D[0, 1, 0] == pytest.approx(2.0, abs=1e-14)     # one step along y (h_y = 2)
    assert D[0, 1, 1] == pytest.approx(2.6, abs=1e-14)     # 0.25 e^2 + (e-1)^2 = 1, e = 1.6


def test_fsm_flat_slab_is_exact(orc):
    # liquid voxels k steps from the nearest vapor layer sit at k*h_z
    dims = (6, 5, 40)
    hz = 0.8
    z = np.arange(dims[2])
    S3 = np.ones((dims[2], dims[1], dims[0]), np.uint8)
    S3[10:30] = 0
    D, _ = orc.fsm(dims, (1.0, 1.0, hz), S3.ravel())
    D = D.reshape(S3.shape)
    expect = np.where((z >= 10) & (z < 30), np.minimum(z - 9, 30 - z) * hz, 0.0)
    np.testing.assert_allclose(D[:, 2, 3], expect, atol=1e-12)


def test_fsm_upper_bounds_euclidean_distance(orc):
    # the first-order upwind distance to a point source is never below the
    # Euclidean distance and converges to it away from the axes
    dims = (31, 31, 31)
    D, _ = orc.fsm(dims, (1.0, 1.0, 1.0), _point_source(dims))
    D = D.reshape(dims[2], dims[1], dims[0])
    for (z, y, x) in [(0, 0, 5), (0, 3, 4), (2, 3, 6), (5, 5, 5), (1, 7, 9)]:
        e = math.sqrt(x * x + y * y + z * z)
        assert e - 1e-12 <= D[z, y, x] <= e * 1.25


def test_fsm_cap(orc):
    dims = (31, 4, 4)
    D, _ = orc.fsm(dims, (1.0, 1.0, 1.0), _point_source(dims), cap=4.5)
    assert D.max() == 4.5


@pytest.mark.parametrize("seed,frac", [(0, 0.0), (1, 0.01), (2, 0.05)])
def test_cfsm_equals_fsm_inside_the_band(orc, seed, frac):
    # Section 4.3.2: CFSM and FSM agree for the grid points within the cutoff
    rng = np.random.default_rng(seed)
    dims = (24, 20, 28)
    S3 = np.ones((dims[2], dims[1], dims[0]), np.uint8)
    S3[8:20] = 0                                     # slab_x-like input
    S = S3.ravel().copy()
    S[rng.random(S.size) < frac] = 1                 # x_y-like random interfacial points
    h = (1.0, 1.1, 0.9)
    r_grid = 4.0 + max(h)
    Df, _ = orc.fsm(dims, h, S, cap=r_grid)
    Dc, it = orc.cfsm(dims, h, S, r_grid)
    assert it > 0
    np.testing.assert_allclose(Dc, Df, atol=1e-12, rtol=0)


def test_cfsm_reports_non_convergence(orc):
    dims = (30, 4, 4)
    D, it = orc.cfsm(dims, (1, 1, 1), _point_source(dims), r_grid=20.0, iter_max=3)
    assert it == -1


# ---- Algorithm 3.1 -------------------------------------------------------------
def test_trilinear_reproduces_linear_fields(orc):
    # trilinear interpolation is exact for a field linear in each coordinate;
    # sample away from the periodic seam where the field would jump
    L = (12.0, 10.0, 14.0)
    dims = (12, 10, 14)
    b = np.asarray(L) / np.asarray(dims)
    zc, yc, xc = np.meshgrid(*(((np.arange(n) + 0.5) * bb) for n, bb in zip(dims[::-1], b[::-1])),
                             indexing="ij")
    coef = np.array([0.3, -0.7, 1.1])
    D = (coef[0] * xc + coef[1] * yc + coef[2] * zc + 2.0).ravel()
    rng = np.random.default_rng(5)
    x = rng.uniform(np.array(b) * 0.5, np.asarray(L) - np.array(b) * 0.5, size=(300, 3))
    d = orc.particle_distance(x, L, dims, D)
    np.testing.assert_allclose(d, x @ coef + 2.0, rtol=1e-12, atol=1e-12)


def test_trilinear_hits_box_centres_and_wraps(orc):
    L = (6.0, 6.0, 6.0)
    dims = (6, 6, 6)
    rng = np.random.default_rng(6)
    D = rng.random(216)
    centres = np.array([[0.5, 0.5, 0.5], [5.5, 2.5, 0.5], [3.5, 4.5, 5.5]])
    d = orc.particle_distance(centres, L, dims, D)
    idx = [0, 5 + 6 * 2, 3 + 6 * (4 + 6 * 5)]
    np.testing.assert_allclose(d, D[idx], atol=1e-15)
    # on the seam between the last and the first box: the mean of the two
    d = orc.particle_distance(np.array([[0.0, 0.5, 0.5]]), L, dims, D)
    assert d[0] == pytest.approx(0.5 * (D[0] + D[5]))


# ---- the whole chain on a synthetic slab --------------------------------------
def test_detection_recovers_the_slab_planes(orc):
    s = slabgen.make_slab(16000, seed=11)
    p = orc.DetectParams(rc_min=3.0, rc_max=6.0, voxel=1.0)
    det = orc.detect(s.x, s.box, p)
    dims = det.dims
    bz = s.box[2] / dims[2]
    zc = (np.arange(dims[2]) + 0.5) * bz
    z_lo, z_hi = s.z_planes
    S3 = det.S.reshape(dims[2], dims[1], dims[0])
    far_liquid = (zc > z_lo + 3 * bz) & (zc < z_hi - 3 * bz)
    far_vapor = (zc < z_lo - 3 * bz) | (zc > z_hi + 3 * bz)
    assert np.all(S3[far_liquid] == 0)
    assert np.all(S3[far_vapor] == 1)
    # every column crosses the interface exactly twice (periodic in z)
    trans = np.sum(S3 != np.roll(S3, 1, axis=0), axis=0)
    assert np.all(trans == 2)
    # particles deep in the liquid get r_c,min; vapor particles get r_c,max
    z = s.x[:, 2]
    deep = (z > z_lo + 8) & (z < z_hi - 8)
    assert np.all(det.rc[deep] == 3.0) and np.all(det.cls[deep] == 0)
    vap = (z < z_lo - 3) | (z > z_hi + 3)
    assert np.all(det.rc[vap] == 6.0)
    assert det.cfsm_iters > 0
