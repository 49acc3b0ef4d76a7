"""Pins of the oracle's velocity-Verlet loop (Eq. 1-2) against an independent
ODE integration, time reversibility and second-order energy error."""
import numpy as np
import pytest

from paper_1502_03234_gb300 import slabgen


def _static_params(orc, rc=3.0, dt=0.005, detect_every=2):
    det = orc.DetectParams(rc_min=rc, rc_max=rc, voxel=1.0)
    return orc.RunParams(det=det, dt=dt, cell_min=1.5, detect_every=detect_every)


def test_two_body_matches_independent_ode_solution(orc):
    from scipy.integrate import solve_ivp

    L = (20.0, 20.0, 20.0)
    r0 = 1.35
    x0 = np.array([[10.0 - r0 / 2, 10.0, 10.0], [10.0 + r0 / 2, 10.0, 10.0]])
    v0 = np.zeros((2, 3))
    v0[0, 0], v0[1, 0] = 0.3, -0.3
    T = 2.0

    def rhs(t, y):
        r, u = y
        # mu r'' = F(r), mu = m/2, with F(r) = 24 (2 r^-13 - r^-7) written out
        return [u, 2.0 * 24.0 * (2.0 * r ** -13 - r ** -7)]

    sol = solve_ivp(rhs, (0, T), [r0, -0.6], method="DOP853", rtol=1e-12, atol=1e-12)
    r_exact = sol.y[0, -1]
    errs = []
    for dt in (0.004, 0.002):
        p = _static_params(orc, dt=dt)
        x, v, f, rc, ep, ek = orc.run(x0, v0, L, p, int(round(T / dt)))
        r = x[1, 0] - x[0, 0]
        errs.append(abs(r - r_exact))
        assert abs(r - r_exact) < 2e-4
        # centre of mass at rest and motion stays on the x axis
        assert x[:, 1] == pytest.approx([10.0, 10.0], abs=1e-14)
    # second-order method: halving dt cuts the error by about 4
    assert 3.0 < errs[0] / errs[1] < 5.0


def test_time_reversibility(orc):
    L = (12.0, 12.0, 12.0)
    x0, v0 = slabgen.make_gas(300, L, seed=3, temperature=0.5)
    p = _static_params(orc, rc=3.0, dt=0.002)
    x1, v1, *_ = orc.run(x0, v0, L, p, 50)
    x2, v2, *_ = orc.run(x1, -v1, L, p, 50, step0=50)
    d = x2 - x0
    d -= np.round(d / np.asarray(L)) * np.asarray(L)
    assert np.abs(d).max() < 1e-9
    np.testing.assert_allclose(-v2, v0, atol=1e-9)


def test_energy_error_is_second_order(orc):
    # a dilute cluster in a big box: no pair reaches the cutoff, so the
    # truncation never jumps and the energy error is the integrator's own
    L = (30.0, 30.0, 30.0)
    x0, v0 = slabgen.make_gas(60, (6.0, 6.0, 6.0), seed=4, temperature=0.4, min_sep=1.0)
    x0 = x0 + 12.0
    drift = []
    for dt in (0.004, 0.002):
        p = _static_params(orc, rc=14.0, dt=dt)
        _, _, _, _, ep, ek = orc.run(x0, v0, L, p, int(round(0.4 / dt)))
        e = ep + ek
        drift.append(np.abs(e - e[0]).max() / abs(e[0]))
    assert drift[0] < 5e-4
    assert 3.0 < drift[0] / drift[1] < 5.0


def test_run_cadence_redetects(orc):
    # with detect_every = 1 the cutoffs in use follow the final positions
    s = slabgen.make_slab(16000, seed=12)
    det = orc.DetectParams(rc_min=3.0, rc_max=6.0, voxel=1.0)
    p = orc.RunParams(det=det, dt=0.005, cell_min=1.5, detect_every=1)
    x, v, f, rc, ep, ek = orc.run(s.x, s.v, s.box, p, 2)
    d = orc.detect(x, s.box, det)
    np.testing.assert_array_equal(rc, d.rc)
