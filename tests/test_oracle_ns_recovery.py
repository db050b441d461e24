"""Pins of the collision step against the hydrodynamics it is built to recover
(Sec. 2.1, "Proper recovery of Navier-Stokes equations"), and of the recolouring
operator against its closed-form colour flux (Eq. (eq:recoloringOperator)).

Closed forms (Chapman-Enskog expansion of Eq. (eq:singleCollisionMRT); a single
pure phase k at rest density rho_0, small plane waves of wave number k):

* Third moment.  The standard equilibrium Eq. (eq:equilibrium) has the lattice's
  third moment, sum N c_a c_b c_g = (rho/3)(u_a d_bg + u_b d_ag + u_g d_ab).  The
  Hermite term of Eq. (eq:equilibrium_hermite) lifts the mixed components
  (xxy, xyy) to those of a Maxwellian at temperature (c_s^k)^2, rho c_s^2 u; the
  diagonal ones (xxx, yyy) cannot change on D2Q9 (c_x^3 = c_x) and keep rho u_x, an
  excess of (1 - 3 c_s^2) rho u_x = (1.8 alpha_k - 0.8) rho u_x = Q^k_x over the
  Maxwellian's 3 rho c_s^2 u_x.
* Shear viscosity.  The xy momentum flux relaxes with s_8 = omega and is driven by
  the mixed third moment: nu = c^2 (1/omega - 1/2) with c^2 = 1/3 for the standard
  equilibrium and c^2 = (c_s^k)^2 for the Hermite one.
* Source U^k = M^-1 C^k.  The excess Q^k enters the first-order moments
  e = sum (3|c|^2 - 4) N (row 1 of M) as 3 (d_x Q_x + d_y Q_y) and
  p_xx = sum (c_x^2 - c_y^2) N (row 7) as (d_x Q_x - d_y Q_y).  A source C added
  after collision cancels an excess E of a moment relaxed at rate s exactly when
  C = (1 - s/2) E, so C_1 = 3 (1 - s_1/2)(d_x Q_x + d_y Q_y), as printed, and
  C_7 = (1 - s_7/2)(d_x Q_x - d_y Q_y): factor 1 and a minus sign, where the
  paper prints 3 (...)(d_x Q_x + d_y Q_y) (the reading of C^k_7).
* Sound.  With that source the momentum flux is exactly the Maxwellian one,
  sigma = rho_0 c_s^2 [(1/s_nu - 1/2)(grad u + grad u^T - I div u)
  + (1/s_e - 1/2) I div u], so a sound wave travels at c_s and decays at
  Gamma = k^2 D / 2 with D = c_s^2 [(1/s_nu - 1/2) + (1/s_e - 1/2)], in every
  direction.  With the standard equilibrium (no source),
  D = (1/3)(1/s_nu - 1/2) + (2/3 - c_s^2)(1/s_e - 1/2).
  s_nu = s_7 = s_8 = omega_eff and s_e = s_1 = lambda omega_eff (MRT); both are
  omega for BGK.

The rates are measured from the oracle's own time series (Prony's method on the
wave's Fourier coefficient) and held to 2 % of the closed forms.  A planted
mistake in any of these terms (C_1's factor or rate, C_7's factor or sign, the
Q^k factor, the Hermite factor) misses them by 13 % or more, or breaks the
mirror symmetry; `test_planted_mistakes_fail_a_pin` builds the oracle with each
mistake and checks that.
"""
import math
import os
import re

import numpy as np
import pytest

from oracle import oracle as O

C = np.array([(0, 0), (1, 0), (0, 1), (-1, 0), (0, -1), (1, 1), (-1, 1), (-1, -1), (1, -1)],
             dtype=np.float64)
CX, CY = C[:, 0], C[:, 1]
TOL = 0.02
LAMBDA = 0.8


def _phase(colour, gamma):
    """(rest density, alpha, c_s^2) of a pure phase (Eq. (eq:gammaAlphaBeta),
    Eq. (eq:pressureRelation))."""
    alpha = O.derived(O.OracleParams(gamma=gamma))["alpha_r"] if colour == 0 else 0.2
    return (gamma if colour == 0 else 1.0), alpha, 3.0 * (1.0 - alpha) / 5.0


def _prony2(sig):
    """Decay rate and angular frequency of a sequence made of two complex
    exponentials (one recurrence s[t+2] = a s[t+1] + b s[t] fitted by least squares)."""
    A = np.stack([sig[1:-1], sig[:-2]], 1)
    coef = np.linalg.lstsq(A, sig[2:], rcond=None)[0]
    z = np.roots([1.0, -coef[0], -coef[1]])
    return float(np.mean(-np.log(np.abs(z)))), float(np.mean(np.abs(np.angle(z))))


def sound_wave(colour, gamma, tau, direction, L, eq=O.EQ_HERMITE, coll=O.MRT, periods=2.5,
               skip=30, **kw):
    """Gamma / k^2, phase speed, and the largest |u_x - u_y| / |u| (diagonal waves)
    of a standing sound wave rho = rho_0 (1 + 1e-4 cos(k.x)) in one pure phase.
    Along x the lattice is L x 1; along the diagonal L x L with k = 2 pi (1, 1)/L."""
    rho0, _, cs2 = _phase(colour, gamma)
    ny = 1 if direction == "x" else L
    p = O.OracleParams(nx=L, ny=ny, gamma=gamma, tau_r=tau, tau_b=tau, sigma=0.0,
                       collision=coll, equilibrium=eq, mrt_lambda=LAMBDA, **kw)
    y, x = np.mgrid[0:ny, 0:L].astype(np.float64)
    ph = 2.0 * np.pi * (x if direction == "x" else x + y) / L
    k = 2.0 * np.pi / L * (1.0 if direction == "x" else math.sqrt(2.0))
    rho = rho0 * (1.0 + 1e-4 * np.cos(ph))
    z = np.zeros_like(rho)
    o = O.Oracle(p)
    o.init_fields(*((rho, z) if colour == 0 else (z, rho)), z, z)
    steps = skip + int(periods * 2.0 * math.pi / (math.sqrt(cs2) * k))
    basis = np.exp(-1j * ph)
    sig, mirror = [], 0.0
    key = "rho_r" if colour == 0 else "rho_b"
    for t in range(steps):
        f = o.fields()
        sig.append((f[key] * basis).sum() / f[key].size)
        if direction == "d" and t % 10 == 9:
            umax = np.abs(f["ux"]).max()
            mirror = max(mirror, float(np.abs(f["ux"] - f["uy"]).max() / umax))
        o.step(1)
    G, w = _prony2(np.array(sig[skip:]))
    return G / k ** 2, w / k, mirror


def shear_wave_nu(colour, gamma, tau, eq, coll, L=64, steps=400):
    """Kinematic viscosity from the decay of u_x = 1e-4 sin(2 pi y / L)."""
    rho0, _, _ = _phase(colour, gamma)
    p = O.OracleParams(nx=1, ny=L, gamma=gamma, tau_r=tau, tau_b=tau, sigma=0.0, collision=coll,
                       equilibrium=eq, mrt_lambda=LAMBDA)
    s = np.sin(2.0 * np.pi * np.arange(L) / L)[:, None]
    one, z = rho0 * np.ones((L, 1)), np.zeros((L, 1))
    o = O.Oracle(p)
    o.init_fields(*((one, z) if colour == 0 else (z, one)), 1e-4 * s, z)
    o.step(50)
    a0 = (o.fields()["ux"] * s).sum()
    o.step(steps)
    a1 = (o.fields()["ux"] * s).sum()
    if not a1 / a0 > 0.0:          # the mode changed sign or blew up: no viscosity
        return math.inf
    return -math.log(a1 / a0) / steps / (2.0 * math.pi / L) ** 2


def _d_sound(cs2, tau, eq, coll):
    """Closed-form D (Gamma = k^2 D / 2) of the module docstring."""
    w = 1.0 / tau
    s_nu, s_e = w, (LAMBDA * w if coll == O.MRT else w)
    if eq == O.EQ_HERMITE:
        return cs2 * ((1.0 / s_nu - 0.5) + (1.0 / s_e - 0.5))
    return (1.0 / 3.0) * (1.0 / s_nu - 0.5) + (2.0 / 3.0 - cs2) * (1.0 / s_e - 0.5)


# (colour, gamma, tau, L along x): the light phase (alpha_b = 0.2) and the heavy
# phase of a gamma = 10 pair (alpha_r = 0.92), both far from alpha = 4/9.
X_CASES = [(1, 1.0, 0.6, 128), (0, 10.0, 0.6, 256)]


def check_shear(eq_coll=((O.EQ_STD, O.BGK), (O.EQ_STD, O.MRT), (O.EQ_HERMITE, O.BGK),
                         (O.EQ_HERMITE, O.MRT))):
    """Worst relative miss of the shear viscosity over both phases."""
    worst = 0.0
    for colour, gamma in ((1, 1.0), (0, 10.0)):
        _, _, cs2 = _phase(colour, gamma)
        for eq, coll in eq_coll:
            c2 = cs2 if eq == O.EQ_HERMITE else 1.0 / 3.0
            nu = shear_wave_nu(colour, gamma, 0.8, eq, coll)
            worst = max(worst, abs(nu / (c2 * 0.3) - 1.0))
    return worst


def check_sound_x(eq=O.EQ_HERMITE, coll=O.MRT, **kw):
    """Worst relative miss of Gamma/k^2 and of the sound speed along x."""
    worst = 0.0
    for colour, gamma, tau, L in X_CASES:
        _, _, cs2 = _phase(colour, gamma)
        g, c, _ = sound_wave(colour, gamma, tau, "x", L, eq=eq, coll=coll, **kw)
        worst = max(worst, abs(g / (0.5 * _d_sound(cs2, tau, eq, coll)) - 1.0),
                    abs(c / math.sqrt(cs2) - 1.0))
    return worst


def check_sound_diagonal(**kw):
    """(relative miss of Gamma/k^2, mirror error) of a diagonal wave, light phase."""
    _, _, cs2 = _phase(1, 1.0)
    g, c, mirror = sound_wave(1, 1.0, 0.6, "d", 48, **kw)
    return abs(g / (0.5 * _d_sound(cs2, 0.6, O.EQ_HERMITE, O.MRT)) - 1.0), mirror


# ------------------------------------------------------------------------ pins

def test_shear_wave_viscosity():
    """nu = (1/3)(1/omega - 1/2) with the standard equilibrium and
    nu = (c_s^k)^2 (1/omega - 1/2) with the Hermite one, BGK and MRT, in the light
    phase and the heavy phase of gamma = 10 (c_s^2 = 0.48 and 0.048)."""
    assert check_shear() < TOL


@pytest.mark.parametrize("eq,coll", [(O.EQ_STD, O.BGK), (O.EQ_STD, O.MRT)])
def test_sound_wave_standard_equilibrium(eq, coll):
    """Sound speed c_s = sqrt(3 (1 - alpha)/5) (Eq. (eq:pressureRelation)) and the
    standard equilibrium's damping D = (1/3)(1/s_nu - 1/2) + (2/3 - c_s^2)(1/s_e - 1/2),
    which pins s_e = lambda omega_eff (Sec. 2.1, MRT operator)."""
    assert check_sound_x(eq=eq, coll=coll) < TOL


def test_sound_wave_hermite_source_along_x():
    """MRT + Hermite equilibrium + U^k: along x the wave decays as the Maxwellian
    fluid's, D = c_s^2 [(1/s_nu - 1/2) + (1/s_e - 1/2)].  This fixes C_1 (factor 3,
    rate s_1, the Q^k factor) and the factor of C_7."""
    assert check_sound_x() < TOL


def test_sound_wave_hermite_source_along_the_diagonal():
    """The same closed form along the diagonal, where d_x Q_x = d_y Q_y: the decay
    is isotropic, and u_x = u_y holds exactly (the x <-> y mirror maps the wave on
    itself and changes the sign of m_7 = p_xx - p_yy, so C_7 must be odd under
    it: d_x Q_x - d_y Q_y).  The printed + sign breaks the mirror symmetry."""
    miss, mirror = check_sound_diagonal()
    assert miss < TOL and mirror < 1e-8
    _, mirror_plus = check_sound_diagonal(c7_sign=1.0)
    assert mirror_plus > 1e-3


def test_printed_c7_destabilises_the_heavy_phase():
    """With C_7 as printed (factor 3) a sound wave along x in the gamma = 10 heavy
    phase is amplified (negative damping): the printed term over-corrects the
    longitudinal stress by twice the Q^k error, which exceeds the phase's own
    viscous damping when c_s^2 = 0.048."""
    g, _, _ = sound_wave(0, 10.0, 0.6, "x", 128, c7_factor=3.0, c7_sign=1.0)
    assert g < 0.0


# ---------------------------------------------------------------- recolouring

def test_recolouring_flux_closed_form():
    """Eq. (eq:recoloringOperator): the red flux gained by recolouring is
    sum_i N^r_i c_i - (rho_r/rho) sum_i N_i c_i
      = beta rho_r rho_b / rho^2 (2 R_1 + 2 sqrt(2) R_5) n,  n = F/|F|,
    with R_i = rho_r phi^r_i + rho_b phi^b_i (sum_{axis} (c.n) c = 2 n and
    sum_{diag} (c.n) c / sqrt(2) = 2 sqrt(2) n), and each colour keeps its mass."""
    rng = np.random.default_rng(11)
    for _ in range(50):
        gamma = rng.uniform(1.0, 50.0)
        beta = rng.uniform(0.1, 1.0)
        p = O.OracleParams(gamma=gamma, beta=beta)
        ar = O.derived(p)["alpha_r"]
        N = rng.uniform(0.01, 0.5, 9)
        rho = N.sum()
        fr = rng.uniform(0.02, 0.98)
        rho_r, rho_b = fr * rho, (1.0 - fr) * rho
        F = rng.normal(size=2) * rng.uniform(1e-3, 1.0)
        n = F / np.linalg.norm(F)
        Nr, Nb = O.recolour(p, rho_r, rho_b, F[0], F[1], N)
        flux = np.array([(Nr * CX).sum(), (Nr * CY).sum()]) - rho_r / rho * np.array(
            [(N * CX).sum(), (N * CY).sum()])
        R1 = rho_r * (1 - ar) / 5 + rho_b * (1 - 0.2) / 5
        R5 = rho_r * (1 - ar) / 20 + rho_b * (1 - 0.2) / 20
        expect = beta * rho_r * rho_b / rho ** 2 * (2 * R1 + 2 * math.sqrt(2.0) * R5) * n
        assert np.abs(flux - expect).max() < 1e-14 * max(1.0, np.abs(expect).max()) + 1e-16
        assert abs(Nr.sum() - rho_r) < 1e-14 and np.allclose(Nr + Nb, N, rtol=0, atol=1e-15)


# ------------------------------------------------------------ planted mistakes

def _recolour_miss():
    try:
        test_recolouring_flux_closed_form()
    except AssertionError:
        return 1.0
    return 0.0


# (name, regex on lbm_oracle.c, replacement, check that must then fail)
MISTAKES = [
    ("C_1 factor 1 instead of 3", r"real C1 = 3\.0 \*", "real C1 = 1.0 *", "x"),
    ("C_1 rate omega instead of s_1", r"\(1\.0 - 0\.5 \* s\[1\]\)", "(1.0 - 0.5 * w)", "x"),
    ("Q^k factor sign", r"\(1\.8 \* (a[rb]) - 0\.8\)", r"(0.8 - 1.8 * \1)", "x"),
    ("Q^k factor 1.8 alpha - 0.4", r"\(1\.8 \* (a[rb]) - 0\.8\)", r"(1.8 * \1 - 0.4)", "x"),
    ("Hermite factor (3|c_i| - 4)", r"\(3\.0 \* c2\(i\) - 4\.0\)", "(3.0 * sqrt((real)c2(i)) - 4.0)",
     "shear"),
    ("Hermite factor (3 c_s^2 + 1)", r"\(3\.0 \* cs2 - 1\.0\)", "(3.0 * cs2 + 1.0)", "shear"),
    ("recolouring rho_r rho_b / rho", r"rho_r \* rho_b / \(rho \* rho\)", "rho_r * rho_b / rho", "recolour"),
    ("recolouring without 1/|c_i|", r"\(sqrt\(\(real\)c2\(i\)\) \* sqrt\(F2\)\)", "sqrt(F2)", "recolour"),
    ("recolouring beta twice", r"term = \(real\)p->beta \*", "term = (real)p->beta * (real)p->beta *",
     "recolour"),
]


def test_planted_mistakes_fail_a_pin(tmp_path, monkeypatch):
    """Each plausible transcription mistake, planted in a copy of the oracle,
    fails one of the pins above; so does C_7 with the printed factor or sign."""
    src = open(os.path.join(os.path.dirname(O.__file__), "lbm_oracle.c")).read()
    for j, (name, pat, rep, check) in enumerate(MISTAKES):
        mutated, n = re.subn(pat, rep, src)
        assert n >= 1, name
        d = tmp_path / f"m{j}"
        d.mkdir()
        monkeypatch.setattr(O, "_lib", O.bind(O.compile_variant(mutated, str(d))))
        if check == "x":
            miss = check_sound_x()
        elif check == "shear":
            miss = check_shear(((O.EQ_HERMITE, O.MRT),))
        else:
            miss = _recolour_miss()
        assert miss > 0.1, (name, miss)
        monkeypatch.undo()
    assert check_sound_x(c7_factor=3.0) > 0.1
    assert check_sound_diagonal(c7_sign=1.0)[1] > 1e-3
