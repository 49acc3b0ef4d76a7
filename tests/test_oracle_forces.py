"""Pins of the oracle's link-cell list and DCM force sum (Algorithm 3.2)."""
import numpy as np
import pytest

from paper_1502_03234_gb300 import slabgen


def _gas(n, L, seed):
    x, _ = slabgen.make_gas(n, L, seed=seed, min_sep=0.85)
    return x


def test_cell_list_is_a_valid_counting_sort(orc):
    L = (13.0, 11.0, 17.0)
    x = _gas(700, L, 1)
    nc = orc.cell_dims(L, 1.5)
    cell_of, start, sid = orc.cell_list(x, L, nc)
    assert start[0] == 0 and start[-1] == len(x)
    assert np.all(np.diff(start) >= 0)
    assert sorted(sid.tolist()) == list(range(len(x)))          # a permutation
    for c in range(len(start) - 1):
        members = sid[start[c]:start[c + 1]]
        assert np.all(np.diff(members) > 0)                     # ascending id
        assert np.all(cell_of[members] == c)
    # each particle lies geometrically inside its cell
    edge = np.asarray(L) / np.asarray(nc)
    cx = cell_of % nc[0]
    cy = (cell_of // nc[0]) % nc[1]
    cz = cell_of // (nc[0] * nc[1])
    idx = np.stack([cx, cy, cz], 1)
    assert np.all(idx * edge <= x + 1e-12) and np.all(x < (idx + 1) * edge + 1e-12)


@pytest.mark.parametrize("cell", [1.0, 1.5, 3.0, 7.0])
def test_cell_list_force_equals_brute_force(orc, cell):
    # the O(N^2) minimum-image sum is the definition; the cell list must find
    # exactly the same pairs (counts bit-equal, forces to rounding)
    L = (14.0, 13.0, 16.0)
    x = _gas(900, L, 2)
    rng = np.random.default_rng(5)
    rc = rng.uniform(2.5, 6.0, len(x))
    nc = orc.cell_dims(L, cell)
    a = orc.forces(x, rc, L, nc)
    b = orc.forces(x, rc, L, None, brute=True)
    assert np.array_equal(a.npair, b.npair)
    np.testing.assert_allclose(a.f, b.f, rtol=1e-12, atol=1e-12)
    np.testing.assert_allclose(a.pe, b.pe, rtol=1e-12, atol=1e-13)
    np.testing.assert_allclose(a.vir, b.vir, rtol=1e-12, atol=1e-11)


def test_pair_rule_is_strict_and_one_sided(orc):
    # Algorithm 3.2: j acts on i iff |r_ij| < r_c[i]; i's own cutoff only
    L = (20.0, 20.0, 20.0)
    x = np.array([[5.0, 5.0, 5.0], [7.5, 5.0, 5.0]])
    r = orc.forces(x, [3.0, 2.0], L, orc.cell_dims(L, 1.5))
    assert r.npair.tolist() == [1, 0]
    _, fr = orc.lj(2.5)
    assert r.f[0, 0] == pytest.approx(fr * (-2.5))
    assert np.all(r.f[1] == 0.0)
    # exactly at the cutoff: not counted
    r = orc.forces(x, [2.5, 2.5], L, orc.cell_dims(L, 1.5))
    assert r.npair.tolist() == [0, 0]


def test_minimum_image_across_the_boundary(orc):
    L = (12.0, 12.0, 12.0)
    x = np.array([[0.2, 6.0, 6.0], [11.5, 6.0, 6.0]])   # 0.7 apart through x = 0
    r = orc.forces(x, [3.0, 3.0], L, orc.cell_dims(L, 1.5))
    _, fr = orc.lj(0.7)
    assert r.f[0, 0] == pytest.approx(fr * 0.7)
    assert r.f[1, 0] == pytest.approx(-fr * 0.7)


def test_static_limit_matches_half_list_and_newton3(orc):
    # r_c,min == r_c,max: DCM reduces to the static cutoff (Section 6.1.2:
    # "exactly the same results"); the half list of Algorithm 2.1 applies
    # Newton's third law, so the total force vanishes
    L = (12.0, 12.0, 15.0)
    x = _gas(600, L, 3)
    rc = 3.0
    full = orc.forces(x, np.full(len(x), rc), L, orc.cell_dims(L, 1.5))
    f_half, pe_half = orc.forces_static_half(x, rc, L)
    np.testing.assert_allclose(full.f, f_half, rtol=1e-11, atol=1e-11)
    np.testing.assert_allclose(full.pe, pe_half, rtol=1e-11, atol=1e-12)
    total = full.f.sum(axis=0)
    assert np.all(np.abs(total) <= 1e-10 * np.abs(full.f).sum())


def test_dcm_forces_are_not_newton3(orc):
    # with per-particle cutoffs the interaction is asymmetric (Section 3)
    L = (12.0, 12.0, 12.0)
    x = _gas(400, L, 4)
    rc = np.where(x[:, 2] < 6.0, 3.0, 5.0)
    r = orc.forces(x, rc, L, orc.cell_dims(L, 1.5))
    assert np.abs(r.f.sum(axis=0)).max() > 1e-6


def test_energy_is_the_potential_of_the_force(orc):
    # static limit: F_i = -dU/dx_i with U = sum over pairs of V (central
    # differences of the oracle's own total energy)
    L = (11.0, 11.0, 11.0)
    x = _gas(250, L, 6)
    rc = np.full(len(x), 3.0)
    nc = orc.cell_dims(L, 1.5)
    base = orc.forces(x, rc, L, nc)
    rng = np.random.default_rng(7)
    for i in rng.choice(len(x), 8, replace=False):
        for a in range(3):
            h = 1e-6
            xp = x.copy()
            xp[i, a] += h
            xm = x.copy()
            xm[i, a] -= h
            up = orc.forces(xp, rc, L, nc).pe.sum()
            um = orc.forces(xm, rc, L, nc).pe.sum()
            if (orc.forces(xp, rc, L, nc).npair != base.npair).any():
                continue   # a pair crossed the cutoff: not differentiable
            assert base.f[i, a] == pytest.approx(-(up - um) / (2 * h), rel=2e-5, abs=2e-6)


def test_virial_single_sum_identity(orc):
    # for an isolated cluster (no periodic image within range) and pair forces
    # obeying Newton 3, W_ab = sum_i x_i,a F_i,b
    L = (40.0, 40.0, 40.0)
    rng = np.random.default_rng(8)
    x = _gas(120, (8.0, 8.0, 8.0), 9) + 16.0
    r = orc.forces(x, np.full(len(x), 3.5), L, orc.cell_dims(L, 2.0))
    W = np.einsum("ia,ib->ab", x, r.f)
    got = np.array([[r.vir[0], r.vir[3], r.vir[4]],
                    [r.vir[3], r.vir[1], r.vir[5]],
                    [r.vir[4], r.vir[5], r.vir[2]]])
    np.testing.assert_allclose(got, W, rtol=1e-9, atol=1e-9)
    del rng


def test_rejects_cutoff_beyond_half_box(orc):
    L = (10.0, 10.0, 10.0)
    x = _gas(50, L, 10)
    with pytest.raises(ValueError):
        orc.forces(x, np.full(len(x), 5.0), L, orc.cell_dims(L, 1.5))


def test_forces_equal_an_independent_numpy_statement(orc):
    # Algorithm 3.2 restated in numpy (shares no code with the oracle's pair
    # routine): minimum image, j counted for i iff 0 < |r_ij| < r_c[i],
    # F_i += 24 eps (2 (s/r)^12 - (s/r)^6) / r^2 * r_ij, PE_i += 2 eps ((s/r)^12 - (s/r)^6)
    L = np.array([12.0, 13.0, 15.0])
    x = _gas(600, tuple(L), 9)
    rng = np.random.default_rng(17)
    rc = rng.uniform(2.5, 5.5, len(x))
    ref = orc.forces(x, rc, tuple(L), orc.cell_dims(tuple(L), 1.5))
    d = x[:, None, :] - x[None, :, :]
    d -= L * np.round(d / L)
    r2 = (d * d).sum(-1)
    np.fill_diagonal(r2, np.inf)
    inside = r2 < (rc * rc)[:, None]
    s6 = np.where(inside, 1.0 / r2 ** 3, 0.0)
    fr = np.where(inside, 24.0 * (2.0 * s6 * s6 - s6) / np.where(inside, r2, 1.0), 0.0)
    f = (fr[:, :, None] * d).sum(1)
    pe = (2.0 * (s6 * s6 - s6)).sum(1)
    assert np.array_equal(ref.npair, inside.sum(1))
    assert np.max(np.abs(ref.f - f)) < 1e-10 * max(1.0, np.abs(f).max())
    assert np.max(np.abs(ref.pe - pe)) < 1e-10 * max(1.0, np.abs(pe).max())
