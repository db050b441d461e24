"""Seeded synthetic workloads shaped like the paper's LBM cases.

Only geometry, parameter choices and random numbers live here: no lattice
Boltzmann arithmetic (no equilibrium, no moments).  Both the CUDA path and the
FP64 oracle consume these fields and parameter sets, each building its own
initial populations from them.

Shapes follow arXiv 1903.01168:
  * static bubble / Laplace test (Sec. 4, Eq. (laplaceslaw)): a light circular
    bubble in a heavy periodic box;
  * gravity-driven periodic slug (Sec. 5.1, Table tab:physprop): elongated light
    bubbles in a heavy liquid between no-slip walls, Poiseuille start profile
    V(y) = g / (2 nu_l) * y (H - y);
  * open channel (Sec. 5.2): velocity inlet with alternating liquid / gas
    segments and a pressure outlet.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field, asdict

import numpy as np

DEFAULT_SEED = 1234


def tau_of_nu(nu: float) -> float:
    """Relaxation time of a kinematic viscosity, tau = 3 nu + 1/2 (Sec. 2.1)."""
    return 3.0 * nu + 0.5


def bubble_fields(nx: int, ny: int, cx: float, cy: float, R: float, gamma: float):
    """Sharp-interface static bubble: light (blue, rho_b^0 = 1) inside the
    circle (x - cx)^2 + (y - cy)^2 < R^2 (periodic distance), heavy (red,
    rho_r^0 = gamma) outside, fluid at rest."""
    y, x = np.mgrid[0:ny, 0:nx].astype(np.float64)
    dx = np.abs(x - cx)
    dx = np.minimum(dx, nx - dx)
    dy = np.abs(y - cy)
    dy = np.minimum(dy, ny - dy)
    inside = dx * dx + dy * dy < R * R
    rho_r = np.where(inside, 0.0, gamma)
    rho_b = np.where(inside, 1.0, 0.0)
    zero = np.zeros((ny, nx))
    return rho_r, rho_b, zero, zero.copy()


def stadium_mask(nx: int, ny: int, x0: float, length: float, height: float, yc: float):
    """Stadium (rectangle with semicircular caps) of total length `length`
    starting at x0 (periodic in x), height `height`, centred on row yc."""
    y, x = np.mgrid[0:ny, 0:nx].astype(np.float64)
    r = height / 2.0
    xs = (x - x0) % nx          # distance downstream of the bubble tail
    core = (xs >= r) & (xs <= length - r) & (np.abs(y - yc) < r)
    c1 = (xs - r) ** 2 + (y - yc) ** 2 < r * r
    c2 = (xs - (length - r)) ** 2 + (y - yc) ** 2 < r * r
    return core | ((xs <= length) & (c1 | c2))


def slug_fields(nx: int, ny: int, gamma: float, n_bubbles: int, bubble_len: float,
                bubble_h: float, g: float = 0.0, nu_l: float = 0.1, poiseuille: bool = True):
    """Periodic slug train between no-slip walls at y = -1/2 and y = ny - 1/2:
    n_bubbles evenly spaced light stadium bubbles in heavy liquid.  With
    poiseuille=True the start velocity is V(y) = g/(2 nu_l) * Y (H - Y),
    Y = y + 1/2, H = ny (Sec. 5.1)."""
    gas = np.zeros((ny, nx), dtype=bool)
    pitch = nx / max(n_bubbles, 1)
    for b in range(n_bubbles):
        gas |= stadium_mask(nx, ny, b * pitch + (pitch - bubble_len) / 2.0, bubble_len,
                            bubble_h, (ny - 1) / 2.0)
    rho_r = np.where(gas, 0.0, gamma)
    rho_b = np.where(gas, 1.0, 0.0)
    ux = np.zeros((ny, nx))
    if poiseuille and g != 0.0:
        Y = np.arange(ny) + 0.5
        ux[:] = (g / (2.0 * nu_l) * Y * (ny - Y))[:, None]
    return rho_r, rho_b, ux, np.zeros((ny, nx))


def random_fields(nx: int, ny: int, seed: int, gamma: float = 1.0, n_bubbles: int = 3,
                  u_amp: float = 0.02, rmin: float = 3.0, rmax: float | None = None,
                  walls_y: bool = False):
    """Seeded random two-phase state for parity tests: a few light circular
    bubbles (radii in [rmin, rmax]) in a heavy fluid plus a smooth divergence-
    free-ish velocity field of amplitude u_amp built from low Fourier modes.
    With walls_y the velocity vanishes toward y = -1/2 and ny - 1/2."""
    rng = np.random.default_rng(seed)
    rmax = rmax if rmax is not None else max(rmin + 1.0, min(nx, ny) / 5.0)
    y, x = np.mgrid[0:ny, 0:nx].astype(np.float64)
    gas = np.zeros((ny, nx), dtype=bool)
    for _ in range(n_bubbles):
        cx, cy = rng.uniform(0, nx), rng.uniform(0, ny)
        R = rng.uniform(rmin, rmax)
        dx = np.abs(x - cx)
        dx = np.minimum(dx, nx - dx)
        dy = np.abs(y - cy)
        dy = np.minimum(dy, ny - dy)
        gas |= dx * dx + dy * dy < R * R
    rho_r = np.where(gas, 0.0, gamma)
    rho_b = np.where(gas, 1.0, 0.0)
    # stream function of a few low modes -> (d_y s, -d_x s)
    ux = np.zeros((ny, nx))
    uy = np.zeros((ny, nx))
    for _ in range(4):
        kx = rng.integers(1, 3)
        ky = rng.integers(1, 3)
        a = rng.normal()
        ph1, ph2 = rng.uniform(0, 2 * np.pi, 2)
        sx = 2 * np.pi * kx / nx
        sy = 2 * np.pi * ky / ny
        ux += a * sy * np.sin(sx * x + ph1) * np.cos(sy * y + ph2)
        uy -= a * sx * np.cos(sx * x + ph1) * np.sin(sy * y + ph2)
    if walls_y:
        Y = (y + 0.5) / ny
        env = np.sin(np.pi * Y)
        ux *= env
        uy *= env
    scale = u_amp / max(np.abs(ux).max(), np.abs(uy).max(), 1e-30)
    return rho_r, rho_b, ux * scale, uy * scale


# ----------------------------------------------------------- parameter sets

@dataclass
class SimSpec:
    """One simulation of a workload: lattice, physical parameters and geometry."""
    nx: int
    ny: int
    gamma: float = 1.0
    tau_r: float = 1.0
    tau_b: float = 1.0
    sigma: float = 0.005
    beta: float = 0.7
    gx: float = 0.0
    gy: float = 0.0
    bc_x: int = 0          # 0 periodic, 1 wall, 2 inlet/outlet
    bc_y: int = 0
    geometry: str = "bubble"   # "bubble" | "slug" | "inout" | "rayleigh_taylor" | "square"
    bubble: tuple = ()         # (cx, cy, R)
    slug: tuple = ()           # (n_bubbles, length, height)
    steps: int = 0
    storage: int = 0           # 0 f32, 1 f16 deviation, 2 bf16 deviation
    u_in_r: float = 0.0
    u_in_b: float = 0.0
    p_out: float = 0.0
    inlet_period_r: int = 0
    inlet_period_b: int = 0
    collision: int = 0         # 0 BGK, 1 MRT
    equilibrium: int = 0       # 0 standard, 1 Hermite (with the U^k source under MRT)
    extra: dict = field(default_factory=dict)

    def as_dict(self) -> dict:
        return asdict(self)


def static_bubble_64() -> SimSpec:
    """64 x 64 periodic static bubble, R = 16, gamma = 1, tau = 1, sigma = 0.005,
    beta = 0.7, no gravity, 2000 steps (Laplace test of Sec. 4)."""
    return SimSpec(nx=64, ny=64, gamma=1.0, tau_r=1.0, tau_b=1.0, sigma=0.005, beta=0.7,
                   geometry="bubble", bubble=(32.0, 32.0, 16.0), steps=2000)


def laplace_sweep(n: int = 256, steps: int = 20000) -> list[SimSpec]:
    """The 40-run Laplace sweep on a periodic n x n lattice: radii
    {20,30,40,50,60} x density ratio {1,10} x viscosity ratio {1,10} x sigma
    {0.001, 0.01}, beta = 0.7.  The smaller kinematic viscosity is 0.1; the
    other follows from nu_b / nu_r = gamma / M with M = mu_r / mu_b."""
    out = []
    for R in (20, 30, 40, 50, 60):
        for gamma in (1.0, 10.0):
            for M in (1.0, 10.0):
                for sigma in (0.001, 0.01):
                    ratio = gamma / M                # nu_b / nu_r
                    if ratio >= 1.0:
                        nu_r, nu_b = 0.1, 0.1 * ratio
                    else:
                        nu_b, nu_r = 0.1, 0.1 / ratio
                    out.append(SimSpec(nx=n, ny=n, gamma=gamma, tau_r=tau_of_nu(nu_r),
                                       tau_b=tau_of_nu(nu_b), sigma=sigma, beta=0.7,
                                       geometry="bubble", bubble=(n / 2.0, n / 2.0, float(R)),
                                       steps=steps))
    return out


def slug_channel(Re: float = 50.0, M: float = 1.0, nx: int = 2048, ny: int = 128,
                 storage: int = 0, steps: int = 100000) -> SimSpec:
    """Gravity-driven periodic slug between no-slip walls: gamma = 10, tau_l = 0.55,
    g = 8 Re nu_l^2 / H^3, sigma from Bo = (rho_l - rho_g) g H^2 / sigma = 0.7848
    (Table tab:adim_cases2), two light stadium bubbles of length nx/4 and height
    0.6 H."""
    gamma = 10.0
    nu_l = (0.55 - 0.5) / 3.0
    g = 8.0 * Re * nu_l ** 2 / ny ** 3
    sigma = (gamma - 1.0) * g * ny ** 2 / 0.7848
    mu_l = gamma * nu_l
    nu_g = mu_l / M / 1.0                         # mu_g = mu_l / M, rho_g = 1
    return SimSpec(nx=nx, ny=ny, gamma=gamma, tau_r=0.55, tau_b=tau_of_nu(nu_g), sigma=sigma,
                   beta=0.7, gx=g, bc_x=0, bc_y=1, geometry="slug",
                   slug=(2, nx / 4.0, 0.6 * ny), steps=steps, storage=storage,
                   extra={"Re": Re, "M": M, "nu_l": nu_l})


def ensemble(seed: int = DEFAULT_SEED, n_sims: int = 256, steps: int = 10000) -> list[SimSpec]:
    """Uneven batched ensemble: lattices uniform in {64..512} x {64..1024}
    (multiples of 32), half static bubbles (R in [8, min(nx, ny)/4]) and half
    periodic slugs, density ratio in {1, 10}, FP16-deviation storage."""
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(n_sims):
        nx = int(rng.integers(2, 17)) * 32
        ny = int(rng.integers(2, 33)) * 32
        gamma = float(rng.choice([1.0, 10.0]))
        if rng.random() < 0.5:
            R = float(rng.uniform(8.0, min(nx, ny) / 4.0))
            out.append(SimSpec(nx=nx, ny=ny, gamma=gamma, tau_r=0.8, tau_b=0.8, sigma=0.005,
                               beta=0.7, geometry="bubble", bubble=(nx / 2.0, ny / 2.0, R),
                               steps=steps, storage=1))
        else:
            # body force for a centreline start speed of 0.01: g = 8 nu u_max / H^2, nu = 0.1
            g = 8.0 * 0.1 * 0.01 / ny ** 2
            out.append(SimSpec(nx=nx, ny=ny, gamma=gamma, tau_r=0.8, tau_b=0.8, sigma=0.005,
                               beta=0.7, gx=g, bc_y=1, geometry="slug",
                               slug=(1, nx / 2.0, 0.5 * ny), steps=steps, storage=1,
                               extra={"nu_l": 0.1}))
    return out


def serving_trace(seed: int = DEFAULT_SEED, n_requests: int = 32, rate_hz: float = 4.0,
                  steps_range=(5000, 50000)) -> list[tuple[float, SimSpec]]:
    """Poisson-arrival inlet/outlet slug requests: lattices nx in [512, 8192],
    ny in [64, 256] (multiples of 32), 5k-50k steps, storage uniform over
    {f32, f16-dev, bf16-dev}; a Zou-He velocity inlet alternating liquid (red)
    and gas (blue) segments (inlet speeds 1.25e-2 / 7.5e-2 as in Sec. 5.2) and a
    pressure outlet; no-slip walls top and bottom.  Returns (arrival_s, spec)."""
    rng = np.random.default_rng(seed)
    t = 0.0
    out = []
    for _ in range(n_requests):
        t += float(rng.exponential(1.0 / rate_hz))
        nx = int(rng.integers(16, 257)) * 32
        ny = int(rng.integers(2, 9)) * 32
        steps = int(rng.integers(steps_range[0] // 100, steps_range[1] // 100 + 1)) * 100
        storage = int(rng.integers(0, 3))
        out.append((t, SimSpec(nx=nx, ny=ny, gamma=5.0, tau_r=0.6, tau_b=0.6, sigma=1e-3,
                               beta=0.7, bc_x=2, bc_y=1, geometry="inout", steps=steps,
                               storage=storage, u_in_r=1.25e-2, u_in_b=7.5e-2,
                               p_out=0.48, inlet_period_r=400, inlet_period_b=200)))
    return out


def rayleigh_taylor(L: int = 140, amp: float = 0.15, storage: int = 0) -> SimSpec:
    """Rayleigh-Taylor instability as in the paper's two-phase cases: an L x 2L box
    (about 40 000 nodes), heavy fluid (red, gamma = 1.8) above light fluid,
    viscosity ratio 1, no surface tension, gravity 1e-4 l.u. downwards.  The
    viscosity follows from Re = sqrt((H/2)^3 g) / nu = 420 with H = 2L.  The
    interface is y = H/2 - amp L sin(2 pi x / L).  The printed amplitude of that
    formula (1, in units of L) would reach both walls; 0.15 L is the cited setup's
    value.  No-slip walls at the bottom and top.  The lattice has walls in y only,
    so x is periodic.  Time unit t_g = sqrt(H / g)."""
    H = 2 * L
    g = 1e-4
    nu = math.sqrt((H / 2.0) ** 3 * g) / 420.0
    tau = tau_of_nu(nu)
    t_g = math.sqrt(H / g)
    return SimSpec(nx=L, ny=H, gamma=1.8, tau_r=tau, tau_b=tau, sigma=0.0, beta=0.7, gx=0.0, gy=-g,
                   bc_x=0, bc_y=1, geometry="rayleigh_taylor", steps=int(round(5 * t_g)), storage=storage,
                   extra={"amp": amp, "t_g": t_g, "nu": nu})


def rayleigh_taylor_fields(nx: int, ny: int, gamma: float, amp: float):
    """Sharp interface y = ny/2 - amp nx sin(2 pi (x + 1/2) / nx) (node centres at
    x + 1/2, so the field is mirror-symmetric about x = nx/4 for even nx): heavy
    (red, rho = gamma) above, light (blue, rho = 1) below, at rest."""
    x = np.arange(nx) + 0.5
    y = np.arange(ny)[:, None] + 0.5
    yi = ny / 2.0 - amp * nx * np.sin(2.0 * np.pi * x / nx)[None, :]
    heavy = y >= yi
    rr = np.where(heavy, gamma, 0.0)
    rb = np.where(heavy, 0.0, 1.0)
    z = np.zeros((ny, nx))
    return rr, rb, z, z.copy()


# Density and viscosity ratios (heavy / light) of the square-to-droplet study and the
# relaxation times chosen for them (the paper gives no viscosities): the heavy
# phase relaxes with tau_h; the light phase's tau follows from the viscosity
# ratio mu_h / mu_l = (rho_h nu_h) / (rho_l nu_l).  (1, 100) takes tau_h = 1.5
# (tau_l = 0.51): with tau_h = 5.5 its error did not fall with resolution.
# (1000, 1000) has equal kinematic viscosities, tau = 0.8 for both phases.
SQUARE_TO_DROPLET_CASES = {(1, 1): 1.0, (5, 2): 1.0, (1000, 1000): 0.8, (1, 100): 1.5}


def square_to_droplet(n: int, ratios=(1, 1), sigma: float = 0.01) -> SimSpec:
    """The paper's square-to-droplet resolution study (Sec. 4, "Square-to-droplet
    case"): an n x n periodic box, a light square of side a = 0.33 n centred,
    sigma = 0.01 l.u., beta = 0.99 (60 / n)^(5/8) (the resolution scaling the paper
    takes from its reference), run for 10 t_sigma with t_sigma = sqrt(rho a^3 / sigma)
    (rho of the heavy phase).  The side is 0.33 n rounded to whole nodes, and that
    side is the a of Laplace's reference.  `ratios` = (rho_h / rho_l, mu_h / mu_l)."""
    gamma, M = ratios
    tau_h = SQUARE_TO_DROPLET_CASES[tuple(ratios)]
    nu_h = (tau_h - 0.5) / 3.0
    nu_l = gamma * nu_h / M            # mu_h / mu_l = M with rho_l = 1, rho_h = gamma
    a = float(round(0.33 * n))
    t_sigma = math.sqrt(gamma * a ** 3 / sigma)
    return SimSpec(nx=n, ny=n, gamma=float(gamma), tau_r=tau_h, tau_b=tau_of_nu(nu_l), sigma=sigma,
                   beta=0.99 * (60.0 / n) ** 0.625, geometry="square", steps=int(round(10 * t_sigma)),
                   extra={"a": a, "t_sigma": t_sigma, "ratios": (gamma, M)})


def square_fields(n: int, a: float, gamma: float):
    """Light (blue) square of a (whole) nodes a side, centred in an n x n box,
    heavy (red) around, at rest."""
    side = int(round(a))
    lo = (n - side) // 2
    inside = np.zeros(n, dtype=bool)
    inside[lo:lo + side] = True
    sq = inside[None, :] & inside[:, None]
    rr = np.where(sq, 0.0, gamma)
    rb = np.where(sq, 1.0, 0.0)
    z = np.zeros((n, n))
    return rr, rb, z, z.copy()


def centreline_laplace_error(p: np.ndarray, n: int, a: float, sigma: float) -> float:
    """L2 error of the pressure along the horizontal centreline inside the drop
    (0.4 n < x < 0.6 n), against Laplace's jump sigma / R = sigma sqrt(pi) / a
    above the far-field pressure (mean over the box's outer rim of width n/10),
    relative to that jump."""
    dp_ref = sigma * math.sqrt(math.pi) / a
    w = max(1, n // 10)
    rim = np.concatenate([p[:w].ravel(), p[-w:].ravel(), p[w:-w, :w].ravel(), p[w:-w, -w:].ravel()])
    p_out = rim.mean()
    row = 0.5 * (p[n // 2 - 1] + p[n // 2]) if n % 2 == 0 else p[n // 2]
    x = np.arange(n) + 0.5
    sel = (x > 0.4 * n) & (x < 0.6 * n)
    err = (row[sel] - p_out) - dp_ref
    return float(np.sqrt(np.mean(err ** 2)) / dp_ref)


def poiseuille_profile(ny: int, g: float, nu: float) -> np.ndarray:
    """Closed-form plane Poiseuille profile between halfway walls:
    u(y) = g / (2 nu) * Y (H - Y), Y = y + 1/2, H = ny."""
    Y = np.arange(ny) + 0.5
    return g / (2.0 * nu) * Y * (ny - Y)


def layered_poiseuille_profile(ny: int, h: float, g: float, rho_low: float, mu_low: float,
                               rho_high: float, mu_high: float) -> np.ndarray:
    """Closed-form two-layer channel flow: layer 'low' for Y < h, 'high' above,
    body acceleration g along x, no slip at Y = 0 and Y = H, continuity of u and
    of mu du/dY at Y = h.  Each layer solves mu_k u'' = -rho_k g."""
    H = float(ny)
    # u_low = -A1/2 Y^2 + a1 Y ; u_high = -A2/2 Y^2 + a2 Y + b2, A_k = rho_k g / mu_k
    A1 = rho_low * g / mu_low
    A2 = rho_high * g / mu_high
    # unknowns a1, a2, b2
    mat = np.array([
        [0.0, H, 1.0],                   # u_high(H) = 0
        [h, -h, -1.0],                   # u_low(h) - u_high(h) = 0
        [mu_low, -mu_high, 0.0],         # mu_low u_low'(h) - mu_high u_high'(h) = 0
    ])
    rhs = np.array([A2 / 2.0 * H * H,
                    A1 / 2.0 * h * h - A2 / 2.0 * h * h,
                    mu_low * A1 * h - mu_high * A2 * h])
    a1, a2, b2 = np.linalg.solve(mat, rhs)
    Y = np.arange(ny) + 0.5
    low = -A1 / 2.0 * Y ** 2 + a1 * Y
    high = -A2 / 2.0 * Y ** 2 + a2 * Y + b2
    return np.where(Y < h, low, high)


def laplace_pressure_jump(p: np.ndarray, psi: np.ndarray, cx: float, cy: float):
    """Laplace measurement on a periodic lattice: R_eff from the light-phase area
    sum((1 - psi)/2) = pi R_eff^2; dp = mean p over r < R_eff/2 minus mean p over
    r > R_eff + 8 (periodic distance from (cx, cy)).  Returns (dp, R_eff)."""
    ny, nx = p.shape
    y, x = np.mgrid[0:ny, 0:nx].astype(np.float64)
    dx = np.abs(x - cx)
    dx = np.minimum(dx, nx - dx)
    dy = np.abs(y - cy)
    dy = np.minimum(dy, ny - dy)
    r = np.sqrt(dx * dx + dy * dy)
    area = ((1.0 - psi) / 2.0).sum()
    Reff = math.sqrt(area / math.pi)
    return p[r < Reff / 2].mean() - p[r > Reff + 8].mean(), Reff


def slug_geometry(psi: np.ndarray, periodic: bool = True) -> dict:
    """Geometry of a train of light bubbles moving along x (Sec. 5.1 measures),
    from a colour field psi (ny, nx): the centreline profile psi_c (middle row, or
    the mean of the two middle rows for even ny) and its zeros on the linear
    interpolant between nodes (tail: psi_c from >= 0 to < 0 in +x; nose: from < 0
    to >= 0); bubble length nose - tail; slug length from a nose to the next
    tail; film thickness (ny - g(x_mid)) / 2 with g(x) = sum_y (1 - psi)/2 linear
    between columns and x_mid the bubble's middle.  Returns a dict with
    n_bubbles, n_slugs, bubble_len, slug_len, film (means), x_tail, x_nose, gas."""
    ny, nx = psi.shape
    ya, yb = (ny - 1) // 2, ny // 2
    pc = 0.5 * (psi[ya] + psi[yb])
    gas = ((1.0 - psi) / 2.0).sum(axis=0)
    nxt = np.roll(pc, -1)
    idx = np.nonzero((pc >= 0.0) != (nxt >= 0.0))[0]
    if not periodic:
        idx = idx[idx < nx - 1]
    pos = (idx + pc[idx] / (pc[idx] - nxt[idx])) % nx
    is_tail = pc[idx] >= 0.0
    out = {"n_bubbles": 0, "n_slugs": 0, "bubble_len": 0.0, "slug_len": 0.0, "film": 0.0,
           "x_tail": [], "x_nose": [], "gas": gas}
    if not is_tail.any():
        return out
    first = int(np.argmax(is_tail))
    order = np.arange(first, first + len(idx)) % len(idx) if periodic else np.arange(first, len(idx))
    seq = [(pos[k], is_tail[k]) for k in order]
    pairs = [(a[0], b[0]) for a, b in zip(seq, seq[1:] + (seq[:1] if periodic else [])) if a[1] and not b[1]]
    if not pairs:
        return out
    tails = np.array([a for a, _ in pairs])
    noses = np.array([b for _, b in pairs])
    blen = noses - tails
    if periodic:
        blen = np.where(blen < 0, blen + nx, blen)
    xm = tails + blen / 2.0
    cols = np.arange(nx + 1)
    gext = np.append(gas, gas[0] if periodic else gas[-1])
    xm = xm % nx if periodic else np.clip(xm, 0, nx - 1)
    film = (ny - np.interp(xm, cols, gext)) / 2.0
    nxt_tail = np.roll(tails, -1)
    slug = nxt_tail - noses
    if periodic:
        slug = np.where(slug < 0, slug + nx, slug)
    else:
        slug = slug[:-1]
    out.update(n_bubbles=len(tails), n_slugs=len(slug), bubble_len=float(blen.mean()),
               slug_len=float(slug.mean()) if len(slug) else 0.0, film=float(film.mean()),
               x_tail=list(tails), x_nose=list(noses))
    return out
