"""Wetting walls in the oracle: free-slip walls (Sec. 2.5: diagonal populations
sent on along the wall) and the static contact angle (Sec. "Adjustment of the
color gradient for static contact angles").  Pins:
  * free slip: a body-forced single-phase channel stays a uniform plug,
    u = g (t + 1/2) at every node, exactly (no-slip walls give a profile);
  * the adjusted colour gradient at a wall node keeps |F| and makes the angle
    theta with the wall normal (n . n^s = cos theta);
  * a drop on the wall relaxes to a circular cap whose contact angle, measured
    through the blue phase from its area and base, follows the prescribed one.
The contact angle is measured through the blue phase: F points towards red and
n^1, n^2 make theta with the wall normal."""
import math

import numpy as np
import pytest

from oracle import oracle as O


def test_free_slip_channel_is_a_uniform_plug():
    g = 1e-5
    for slip in (1, 0):
        o = O.Oracle(O.OracleParams(nx=8, ny=16, gx=g, bc_y=O.WALL, wall_slip=slip, sigma=0.0))
        ones, z = np.ones((16, 8)), np.zeros((16, 8))
        o.init_fields(ones, z, z, z)
        o.step(200)
        ux = o.fields()["ux"]
        if slip:
            assert np.abs(ux - g * 200.5).max() < 1e-15
        else:
            assert ux[8].mean() - ux[0].mean() > 0.1 * g * 200     # no-slip: sheared profile


def cap_angle(area: float, base: float) -> float:
    """Contact angle of a circular cap of the given area and base width."""
    a = base / 2.0
    f = lambda th: (th - math.sin(th) * math.cos(th)) / math.sin(th) ** 2 - area / a ** 2
    lo, hi = 1e-3, math.pi - 1e-3                     # f increases with theta
    for _ in range(80):
        mid = 0.5 * (lo + hi)
        if f(mid) < 0:
            lo = mid
        else:
            hi = mid
    return 0.5 * (lo + hi)


def drop(theta_deg: float, nx=80, ny=40, steps=6000):
    """Blue drop (a 26 x 13 rectangle, the paper's 0.33 x 0.165 aspect) on the
    bottom wall of an nx x ny box, gamma = 1, sigma = 0.01."""
    o = O.Oracle(O.OracleParams(nx=nx, ny=ny, bc_y=O.WALL, sigma=0.01, beta=0.7, tau_r=1.0, tau_b=1.0,
                                contact_angle=math.radians(theta_deg)))
    rb = np.zeros((ny, nx))
    rb[:13, nx // 2 - 13:nx // 2 + 13] = 1.0
    rr = 1.0 - rb
    z = np.zeros((ny, nx))
    o.init_fields(rr, rb, z, z)
    return o


def test_adjusted_gradient_makes_theta_with_the_wall():
    th = math.radians(60.0)
    o = drop(60.0)
    o.step(50)
    Fx, Fy, _ = O.gradient_fields(o)
    for y, nsy in ((0, 1.0),):
        F = np.hypot(Fx[y], Fy[y])
        m = F > 1e-6
        assert m.sum() >= 2
        assert np.allclose(Fy[y][m] / F[m] * nsy, math.cos(th), atol=1e-12)


def measured_angle(o, nx):
    f = o.fields()
    blue = (1.0 - f["psi"]) / 2.0
    return math.degrees(cap_angle(blue.sum(), blue[0].sum()))


@pytest.mark.parametrize("theta", [60.0, 90.0, 120.0])
def test_drop_relaxes_to_the_prescribed_angle(theta):
    o = drop(theta)
    o.step(6000)
    got = measured_angle(o, 80)
    assert abs(got - theta) < 8.0, (theta, got)


def test_wetting_walls_conserve_each_colour_exactly():
    """Free-slip links deliver every population to exactly one node and the
    contact-angle turn only rotates F, so per-colour mass is conserved to round-off
    (here with gravity along the wall and a drop touching both walls)."""
    o = O.Oracle(O.OracleParams(nx=48, ny=20, bc_y=O.WALL, wall_slip=1, sigma=0.01, beta=0.7,
                                gamma=3.0, tau_r=0.7, tau_b=0.9, gx=1e-5,
                                contact_angle=math.radians(70.0)))
    rb = np.zeros((20, 48))
    rb[:, 16:32] = 1.0
    o.init_fields(3.0 * (1.0 - rb), rb, np.zeros((20, 48)), np.zeros((20, 48)))
    f0 = o.fields()
    o.step(400)
    f1 = o.fields()
    for k in ("rho_r", "rho_b"):
        assert abs(f1[k].sum() - f0[k].sum()) <= 1e-12 * f0[k].sum()
