"""Pins of the oracle's pair physics and cutoff function against facts other
than the oracle itself (closed forms, identities, numerical differentiation).
"""
import math

import numpy as np
import pytest


# ---- Eq. 4: textbook facts of the Lennard-Jones potential ------------------
def test_lj_zero_crossing_and_minimum(orc):
    for eps, sigma in [(1.0, 1.0), (0.7, 1.3)]:
        V, _ = orc.lj(sigma, eps, sigma)
        assert abs(V) < 1e-15                      # V(sigma) = 0
        rmin = 2.0 ** (1.0 / 6.0) * sigma
        V, fr = orc.lj(rmin, eps, sigma)
        assert V == pytest.approx(-eps, rel=1e-14)  # well depth -eps at 2^(1/6) sigma
        assert abs(fr) < 1e-13                      # zero force at the minimum


def test_lj_force_is_minus_gradient(orc):
    # F_i<-j = fr * r_vec must equal -dV/dr * r_hat: check by central differences
    for r in [0.95, 1.05, 1.3, 1.5, 2.2, 2.99, 5.5]:
        h = 1e-6 * r
        vp, _ = orc.lj(r + h)
        vm, _ = orc.lj(r - h)
        dvdr = (vp - vm) / (2 * h)
        _, fr = orc.lj(r)
        assert fr * r == pytest.approx(-dvdr, rel=1e-7, abs=1e-10)


def test_lj_repulsive_inside_attractive_outside(orc):
    rmin = 2.0 ** (1.0 / 6.0)
    assert orc.lj(0.9 * rmin)[1] > 0     # pushes i away from j
    assert orc.lj(1.1 * rmin)[1] < 0     # pulls i towards j


def test_lj_long_range_tail(orc):
    # far away the r^-6 dispersion term dominates: V ~ -4 eps (sigma/r)^6
    r = 40.0
    V, _ = orc.lj(r)
    assert V == pytest.approx(-4.0 * r ** -6, rel=1e-8)


# ---- Eq. 7-8: the exponential cutoff function ---------------------------------
@pytest.mark.parametrize("rcmin,rcmax,alpha", [(3.0, 6.0, -0.5), (3.0, 7.0, -0.5),
                                               (4.5, 9.0, -0.5), (3.0, 6.0, -2.0)])
def test_cutoff_endpoints_and_continuity(orc, rcmin, rcmax, alpha):
    # Eq. 8 is chosen so that Eq. 7 is continuous at both ends
    assert orc.cutoff(0.0, rcmin, rcmax, alpha) == rcmax
    assert orc.cutoff(-3.0, rcmin, rcmax, alpha) == rcmax
    assert orc.cutoff(1e-12, rcmin, rcmax, alpha) == pytest.approx(rcmax, abs=1e-10)
    assert orc.cutoff(rcmax - 1e-12, rcmin, rcmax, alpha) == pytest.approx(rcmin, abs=1e-10)
    assert orc.cutoff(rcmax, rcmin, rcmax, alpha) == rcmin
    assert orc.cutoff(rcmax + 5, rcmin, rcmax, alpha) == rcmin


def test_cutoff_monotone_and_exponential_shape(orc):
    rcmin, rcmax, alpha = 3.0, 6.0, -0.5
    ds = np.linspace(0.01, rcmax - 0.01, 200)
    r = np.array([orc.cutoff(d, rcmin, rcmax, alpha) for d in ds])
    assert np.all(np.diff(r) < 0)                      # larger cutoff nearer the interface
    # r_c(d) - b is a * 2^(alpha (rc_max - d)): one unit of d multiplies it
    # by 2^(-alpha).  b is where the exponential would settle; recover it from three equally
    # spaced points (Aitken), independent of how the oracle computes it
    r0, r1, r2 = (orc.cutoff(d, rcmin, rcmax, alpha) for d in (1.0, 2.0, 3.0))
    b_est = (r0 * r2 - r1 * r1) / (r0 + r2 - 2 * r1)
    ratio = (r2 - b_est) / (r1 - b_est)
    assert ratio == pytest.approx(2.0 ** (-alpha), rel=1e-9)
    # and the limits fix a and b: continuity at d = rcmax gives a + b = rcmin
    a_est = r1 - b_est
    a_est /= 2.0 ** (alpha * (rcmax - 2.0))
    assert a_est + b_est == pytest.approx(rcmin, rel=1e-10)


def test_cutoff_static_limit(orc):
    # rc_min == rc_max: every distance gets the same cutoff (DCM = static)
    for d in [-1, 0, 0.5, 2.0, 3.0, 10.0]:
        assert orc.cutoff(d, 4.0, 4.0, -0.5) == 4.0


def test_cutoff_steeper_alpha_is_more_step_like(orc):
    # a more negative alpha makes Eq. 7 closer to a step function; the step
    # sits at d = rc_max (a -> -(rc_max - rc_min), b -> rc_max)
    mid = [orc.cutoff(3.0, 3.0, 6.0, a) for a in (-0.25, -0.5, -1.0, -4.0)]
    assert all(x < y for x, y in zip(mid, mid[1:]))
    assert 6.0 - mid[-1] < 1e-3


def test_cutoff_classes(orc):
    rcmin, rcmax, alpha, K = 3.0, 6.0, -0.5, 4
    thr = orc.class_thresholds(rcmin, rcmax, alpha, K)
    assert len(thr) == K - 2 and np.all(np.diff(thr) < 0)
    # the thresholds are where the cutoff crosses the class edges
    for k, t in enumerate(thr, start=1):
        edge = rcmin + (rcmax - rcmin) * k / (K - 1)
        assert orc.cutoff(t, rcmin, rcmax, alpha) == pytest.approx(edge, rel=1e-12)
    assert orc.cutoff_class(rcmax, rcmax, K, thr) == 0
    assert orc.cutoff_class(100.0, rcmax, K, thr) == 0
    assert orc.cutoff_class(0.0, rcmax, K, thr) == K - 1
    assert orc.cutoff_class(-2.0, rcmax, K, thr) == K - 1
    # every class's cutoffs lie inside its edges
    for d in np.linspace(0.001, rcmax - 0.001, 500):
        c = orc.cutoff_class(d, rcmax, K, thr)
        r = orc.cutoff(d, rcmin, rcmax, alpha)
        lo = rcmin + (rcmax - rcmin) * (c - 1) / (K - 1)
        hi = rcmin + (rcmax - rcmin) * c / (K - 1)
        assert lo - 1e-9 <= r <= hi + 1e-9


def test_linear_cutoff_closed_forms(orc):
    # Section 3.1 / Fig. 12 (r_c 4.5 / 9): the line from (0, r_c,max) to
    # (r_c,max, r_c,min) -- halfway in d is halfway in r_c
    assert orc.cutoff_linear(4.5, 4.5, 9.0) == 6.75
    assert orc.cutoff_linear(0.0, 4.5, 9.0) == 9.0
    assert orc.cutoff_linear(-3.0, 4.5, 9.0) == 9.0
    assert orc.cutoff_linear(9.0, 4.5, 9.0) == 4.5
    assert orc.cutoff_linear(20.0, 4.5, 9.0) == 4.5
    assert orc.cutoff_linear(1.5, 3.0, 6.0) == pytest.approx(5.25, abs=1e-15)
    # a straight line: zero second differences, slope -(max - min)/max
    d = np.linspace(0.3, 5.7, 19)
    r = np.array([orc.cutoff_linear(x, 3.0, 6.0) for x in d])
    np.testing.assert_allclose(np.diff(r, 2), 0.0, atol=1e-13)
    np.testing.assert_allclose(np.diff(r) / np.diff(d), -0.5, rtol=1e-12)
    # the static limit
    assert orc.cutoff_linear(2.0, 4.0, 4.0) == 4.0


def test_exponential_cutoff_lies_above_the_linear_one(orc):
    # Eq. 7 with alpha < 0 is concave in d, so it lies above its chord, which
    # is the linear function: the reason the thesis gives for the
    # exponential function's higher accuracy (it assigns larger cutoffs)
    for rcmin, rcmax in ((3.0, 6.0), (4.5, 9.0), (3.0, 7.0)):
        for alpha in (-0.25, -0.5, -1.0):
            for d in np.linspace(0.01, rcmax - 0.01, 60):
                assert orc.cutoff(d, rcmin, rcmax, alpha) > orc.cutoff_linear(d, rcmin, rcmax)


def test_linear_cutoff_classes(orc):
    rcmin, rcmax, K = 3.0, 6.0, 4
    thr = orc.class_thresholds_linear(rcmin, rcmax, K)
    # edges 4 and 5 are crossed at d = 4 and 2
    np.testing.assert_allclose(thr, [2.0, 4.0][::-1], rtol=1e-15)
    for k, t in enumerate(thr, start=1):
        edge = rcmin + (rcmax - rcmin) * k / (K - 1)
        assert orc.cutoff_linear(t, rcmin, rcmax) == pytest.approx(edge, rel=1e-14)
    for d in np.linspace(0.001, rcmax - 0.001, 300):
        c = orc.cutoff_class(d, rcmax, K, thr)
        r = orc.cutoff_linear(d, rcmin, rcmax)
        assert rcmin + (rcmax - rcmin) * (c - 1) / (K - 1) - 1e-12 <= r
        assert r <= rcmin + (rcmax - rcmin) * c / (K - 1) + 1e-12


def test_detection_with_the_linear_function(orc):
    from paper_1502_03234_gb300 import slabgen
    s = slabgen.make_slab(5000, seed=4)
    ex = orc.detect(s.x, s.box, orc.DetectParams())
    li = orc.detect(s.x, s.box, orc.DetectParams(cutoff_fn=1))
    assert np.array_equal(ex.S, li.S) and np.array_equal(ex.d, li.d)
    ref = np.array([orc.cutoff_linear(x, 3.0, 6.0) for x in li.d])
    assert np.array_equal(li.rc, ref)
    assert np.all(li.rc <= ex.rc)
    thr = orc.class_thresholds_linear(3.0, 6.0, 4)
    assert np.array_equal(li.cls, [orc.cutoff_class(x, 6.0, 4, thr) for x in li.d])


def test_bin_index_geometry(orc):
    L, n = 23.94, 17
    rng = np.random.default_rng(3)
    for x in rng.random(2000) * L:
        k = orc.bin_index(x, n, L)
        edge = L / n
        assert k * edge - 1e-12 <= x < (k + 1) * edge + 1e-12
    assert orc.bin_index(L * (1 - 1e-17), n, L) == n - 1
    assert orc.wrap(-1e-18, L) in (0.0,) or orc.wrap(-1e-18, L) < L
    assert 0.0 <= orc.wrap(L, L) < L
    assert orc.wrap(-0.5, L) == pytest.approx(L - 0.5)


def test_lj_printed_values(orc):
    # Eq. 4's closed form evaluated to ten digits (epsilon = sigma = 1): V(r)
    # and the radial force F . r_hat = fr * r (negative: attractive)
    for r, V_ref, F_ref in [(1.5, -0.3203365943, -1.1580288310),
                            (3.0, -0.0054794417, -0.0109438301),
                            (2.0 ** (1.0 / 6.0), -1.0, 0.0)]:
        V, fr = orc.lj(r)
        assert V == pytest.approx(V_ref, abs=5e-11)
        assert fr * r == pytest.approx(F_ref, abs=5e-11)


def test_cutoff_printed_values(orc):
    # Eq. 7's closed form to twelve digits: (3, 6) gives a = -3.428571428571,
    # b = 6.428571428571 (r_c(0) = 6, r_c(6) = 3); (3, 7) a = -4.387833338551
    for d, ref in [(1.0, 5.822479901840), (2.0, 5.571428571429), (3.0, 5.216388375109),
                   (4.5, 4.389930659995)]:
        assert orc.cutoff(d, 3.0, 6.0, -0.5) == pytest.approx(ref, abs=5e-12)
    assert orc.cutoff(3.0, 3.0, 7.0, -0.5) == pytest.approx(6.290875003913, abs=5e-12)
    # a from the endpoints: r_c(d) - b = a 2^(alpha (r_max - d)) with b = r_min - a
    a = -3.428571428571
    assert orc.cutoff(1e-9, 3.0, 6.0, -0.5) == pytest.approx(a * 2 ** (-0.5 * 6.0) + (3.0 - a),
                                                           abs=1e-9)
