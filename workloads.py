"""Seeded synthetic inputs shared by the oracle checks, the CUDA tests and the
benchmark.

This module only produces input data: parameter sets and initial height
fields / population arrays drawn from seeded generators. It holds none of the
arithmetic of the lattice Boltzmann step (no pressures, friction, equilibria
or streaming), so it can feed both the oracle and the CUDA path.

Parameter dicts use the layout both bindings accept:
    n, lattice (1 = D1Q3, 2 = D2Q9), nx, ny, tau,
    gamma[n]     gamma_{i,i+1} for i = 1..n (n+1 is the gas),
    S[i][k-1]    spreading coefficient S_{ik}, i = 0..n-1, k = 1..n-i,
    mu[n], beta[n], nw, mw, hstar.

Workload recipes (the paper fixes no grid sizes or values for its timed
runs; these stand in for its two- and three-layer spinodal set-ups):
  * two-layer pseudo-2D film: D1Q3, 512 periodic cells, h1 = h2 = 1 plus
    seeded uniform noise of +-1e-3, gamma 0.01 / 0.01, mu = 1/6, slip 1,
    exponents (3, 2), h* = 0.1, contact angle 20 degrees;
  * three-layer pseudo-3D spinodal film: D2Q9, 1024 x 1024 periodic cells,
    means 1.0 / 0.8 / 0.6 plus seeded Gaussian noise sigma = 1e-3, gamma
    0.01 / 0.008 / 0.006, mu = (1, 2, 4) / 6, slip 1, (3, 2), h* = 0.07,
    contact angle 20 degrees.
A contact angle theta is turned into the one-layer spreading coefficients by
Young's law, cos(theta) = 1 + S_{i1} / gamma_{i+1,i+2}; multi-layer
coefficients S_{ik}, k >= 2, are zero as in the paper's three-layer runs.

Batched stability sweep (many uneven instances in one batch; the paper runs
its linear-stability checks one film at a time):
  * 512 instances, n uniform in 2..5, square sides from {64, 128, 256, 512},
    tensions gamma_{i,i+1} log-uniform in [0.002, 0.02], viscosities
    mu_1 = 1/16 and mu_i / mu_1 log-uniform in [0.25, 4], slip 1, (3, 2),
    h* = 0.07, contact angle 20 degrees, layer means uniform in [0.6, 1.1];
    every layer perturbed by 1e-4 a_i cos(2 pi (kx x + ky y) / side), a_i
    uniform in [-1, 1] and (kx, ky) a random wavenumber with components in
    0..8 (not both zero); seed 3.

Long dewetting run (compared with the oracle by statistics): two layers of
0.25 plus seeded Gaussian noise 1e-3 (seed 9) on D2Q9 64 x 64, gamma 0.01,
S_01 = S_11 = gamma (cos 20 deg - 1), h* = 0.05; the film ruptures after
about 8000 steps and coarsens into drops.

Droplet and lens equilibria (section "Droplet equilibria"; the paper gives
no grid sizes, so these are stand-ins):
  * sessile ridge, D1Q3: one layer, precursor h*, a circular-arc ridge of
    base half-width a at contact angle theta0; S_01 = gamma (cos thetaY - 1)
    so that Young's law gives thetaY;
  * symmetric liquid lens, D1Q3: liquid one flat at thickness T1, liquid two
    a lens of two equal arcs (opening angle theta0 above and below the far
    level of the liquid-one surface) on its precursor h*; gamma_12 =
    gamma_23 = gamma and S_11 = 2 gamma (cos thetaN - 1), every other S
    zero, so that Neumann's law gives thetaN on both sides;
  * three-layer lens field, D2Q9: layer 1 flat at 1.0, layer 2 flat at
    0.3 r (deep enough for the lens to float), layer 3 four seeded lenses of
    base radius r (12.5 cells at 128 x 128, 200 at 2048 x 2048) on its
    precursor h* = 0.05; one tension gamma for all three liquids and
    S_21 = 2 gamma (cos thetaN - 1), every other S zero (the substrate and
    the lower liquids fully wet, so layers 1 and 2 stay flat films). The
    tension is gamma = 0.125 / r (0.01 at r = 12.5): films a few tens of
    cells thick with gamma = 0.01 carry capillary waves that the explicit
    step does not damp, and scaling gamma with 1 / r keeps thickness times
    tension, and so the step's stability, the same at every size; the
    Neumann angles depend on tension ratios only.
"""
import math

import numpy as np

DEG = math.pi / 180.0


def _young_spreading(gamma, theta_deg, n):
    c = math.cos(theta_deg * DEG) - 1.0
    S = []
    for i in range(n):
        row = [0.0] * (n - i)
        row[0] = gamma[i] * c
        S.append(row)
    return S


def film2_d1q3_params(nx=512):
    """Two-layer pseudo-2D film on a D1Q3 lattice."""
    n = 2
    gamma = [0.01, 0.01]
    return dict(n=n, lattice=1, nx=int(nx), ny=1, tau=1.0, gamma=gamma,
                S=_young_spreading(gamma, 20.0, n), mu=[1 / 6, 1 / 6],
                beta=[1.0, 1.0], nw=3, mw=2, hstar=0.1)


def film2_d1q3_heights(nx=512, seed=1):
    rng = np.random.default_rng(seed)
    return 1.0 + rng.uniform(-1e-3, 1e-3, size=(2, 1, int(nx)))


def film3_d2q9_params(nx=1024, ny=1024):
    """Three-layer pseudo-3D spinodal film on a D2Q9 lattice."""
    n = 3
    gamma = [0.01, 0.008, 0.006]
    return dict(n=n, lattice=2, nx=int(nx), ny=int(ny), tau=1.0, gamma=gamma,
                S=_young_spreading(gamma, 20.0, n),
                mu=[1 / 6, 2 / 6, 4 / 6], beta=[1.0, 1.0, 1.0], nw=3, mw=2,
                hstar=0.07)


def film3_d2q9_heights(nx=1024, ny=1024, seed=2):
    rng = np.random.default_rng(seed)
    means = np.array([1.0, 0.8, 0.6]).reshape(3, 1, 1)
    return means + rng.normal(0.0, 1e-3, size=(3, int(ny), int(nx)))


def random_params(seed, n, lattice, nx, ny=1, tau=1.0, multilayer_S=True):
    """Seeded random parameter set, with all S_{ik} populated when asked.

    Tensions and viscosities are drawn log-uniformly, slips uniformly;
    exponents come from a few integer pairs with nw > mw. The ranges
    (mu in [0.03, 0.25], beta in [0.8, 1.5]) keep the explicit friction
    update contractive down to the precursor thickness, so every draw
    passes the solver's create-time stability check.
    """
    rng = np.random.default_rng(seed)
    gamma = list(np.exp(rng.uniform(np.log(2e-3), np.log(2e-2), n)))
    mu = list(np.exp(rng.uniform(np.log(0.03), np.log(0.25), n)))
    beta = list(rng.uniform(0.8, 1.5, n))
    S = []
    for i in range(n):
        row = []
        for k in range(1, n - i + 1):
            if k == 1 or multilayer_S:
                row.append(float(rng.uniform(-1.0, 0.5) * 1e-3))
            else:
                row.append(0.0)
        S.append(row)
    nw, mw = [(3, 2), (4, 3), (9, 3), (6, 2)][int(rng.integers(0, 4))]
    return dict(n=n, lattice=lattice, nx=int(nx), ny=int(ny), tau=float(tau),
                gamma=[float(g) for g in gamma], S=S,
                mu=[float(m) for m in mu], beta=[float(b) for b in beta],
                nw=nw, mw=mw, hstar=float(rng.uniform(0.05, 0.1)))


def random_heights(seed, p, lo=0.3, hi=1.2, noise=1e-2):
    """Layer means in [lo, hi] plus seeded uniform noise of +-noise."""
    rng = np.random.default_rng(seed)
    n, ny, nx = int(p["n"]), int(p["ny"]), int(p["nx"])
    means = rng.uniform(lo, hi, size=(n, 1, 1))
    return means + rng.uniform(-noise, noise, size=(n, ny, nx))


def random_populations(seed, p, h_lo=0.3, h_hi=1.2, amp=2e-3):
    """A seeded non-equilibrium population array f[n][Q][ny][nx].

    The rest population carries a random layer thickness in [h_lo, h_hi];
    moving populations carry independent uniform values in [-amp, amp].
    Used as a generic state for single-step comparisons.
    """
    rng = np.random.default_rng(seed)
    n, ny, nx = int(p["n"]), int(p["ny"]), int(p["nx"])
    q = 3 if int(p["lattice"]) == 1 else 9
    f = rng.uniform(-amp, amp, size=(n, q, ny, nx))
    f[:, 0] = rng.uniform(h_lo, h_hi, size=(n, ny, nx))
    return f


def single_mode_heights(p, h0, amps, mode, eps):
    """h_i = h0_i + eps * amps_i * cos(2 pi (mx x / nx + my y / ny)).

    A single Fourier mode used by the linear-stability checks.
    """
    n, ny, nx = int(p["n"]), int(p["ny"]), int(p["nx"])
    mx, my = mode
    y, x = np.meshgrid(np.arange(ny), np.arange(nx), indexing="ij")
    ph = 2 * np.pi * (mx * x / nx + my * y / ny)
    h = np.empty((n, ny, nx))
    for i in range(n):
        h[i] = h0[i] + eps * amps[i] * np.cos(ph)
    return h


def cap_profile(dist, peak, base, theta):
    """Height of a circular arc (a spherical cap in 2-D) of contact angle
    theta (radians) whose top is `peak` above a flat `base` at distance
    dist = 0; `base` outside the contact line."""
    rc = (peak - base) / (1.0 - math.cos(theta))
    inside = np.sqrt(np.maximum(rc * rc - np.asarray(dist, dtype=float) ** 2, 0.0))
    return base + np.maximum(0.0, inside - rc * math.cos(theta))


def drop1d_params(nx=128, theta_y_deg=20.0, gamma=0.01, hstar=0.1):
    """One layer on D1Q3 whose Young angle is theta_y_deg."""
    return dict(n=1, lattice=1, nx=int(nx), ny=1, tau=1.0, gamma=[gamma],
                S=[[gamma * (math.cos(math.radians(theta_y_deg)) - 1.0)]],
                mu=[1.0 / 6.0], beta=[1.0], nw=3, mw=2, hstar=hstar)


def drop1d_heights(nx=128, theta0_deg=20.0, area=None, half_width=20.0, hstar=0.1):
    """A circular-arc ridge centred in the box on the precursor h*. Either
    its base half-width or its cross-section `area` (above h*) is given."""
    th = math.radians(theta0_deg)
    if area is not None:
        rc = math.sqrt(area / (th - math.sin(th) * math.cos(th)))
    else:
        rc = half_width / math.sin(th)
    x = np.arange(nx, dtype=float)
    h = cap_profile(x - nx / 2.0, hstar + rc * (1.0 - math.cos(th)), hstar, th)
    return h.reshape(1, 1, nx)


def lens1d_params(nx=160, theta_n_deg=20.0, gamma=0.01, hstar=0.1):
    """Two layers on D1Q3: liquid two forms a symmetric lens on liquid one."""
    s11 = 2.0 * gamma * (math.cos(math.radians(theta_n_deg)) - 1.0)
    return dict(n=2, lattice=1, nx=int(nx), ny=1, tau=1.0, gamma=[gamma, gamma],
                S=[[0.0, 0.0], [s11]], mu=[1.0 / 6.0, 1.0 / 6.0], beta=[1.0, 1.0],
                nw=3, mw=2, hstar=hstar)


def lens1d_heights(nx=160, theta0_deg=20.0, half_width=20.0, t1=6.0, hstar=0.1):
    """Liquid one flat at t1 with the lower arc carved out, liquid two the
    lens (both arcs) on its precursor."""
    th = math.radians(theta0_deg)
    rc = half_width / math.sin(th)
    x = np.arange(nx, dtype=float)
    arc = cap_profile(x - nx / 2.0, rc * (1.0 - math.cos(th)), 0.0, th)
    return np.stack([t1 - arc, hstar + 2.0 * arc]).reshape(2, 1, nx)


def lens3_params(nx=128, ny=128, radius=12.5, theta_n_deg=20.0, hstar=0.05):
    """Three layers on D2Q9: liquid three forms symmetric lenses of base
    radius `radius` on liquid two; only S_21 is non-zero."""
    gamma = 0.125 / radius
    s21 = 2.0 * gamma * (math.cos(math.radians(theta_n_deg)) - 1.0)
    return dict(n=3, lattice=2, nx=int(nx), ny=int(ny), tau=1.0,
                gamma=[gamma, gamma, gamma], S=[[0.0, 0.0, 0.0], [0.0, 0.0], [s21]],
                mu=[1.0 / 6.0, 2.0 / 6.0, 4.0 / 6.0], beta=[1.0, 1.0, 1.0],
                nw=3, mw=2, hstar=hstar)


def lens3_centres(nx, ny, radius, count=4, seed=4):
    """Seeded lens centres at least 2.6 radii apart (periodic distance)."""
    rng = np.random.default_rng(seed)
    centres = []
    for _ in range(10000):
        if len(centres) == count:
            break
        c = rng.uniform(0.0, 1.0, 2) * (nx, ny)
        ok = True
        for d in centres:
            dx = abs(c[0] - d[0]); dx = min(dx, nx - dx)
            dy = abs(c[1] - d[1]); dy = min(dy, ny - dy)
            ok = ok and math.hypot(dx, dy) >= 2.6 * radius
        if ok:
            centres.append(c)
    if len(centres) < count:
        raise ValueError("lenses do not fit the box")
    return np.array(centres)


def lens3_heights(nx=128, ny=128, radius=12.5, theta0_deg=20.0, hstar=0.05, seed=4):
    """Layer 1 flat at 1, layer 2 flat at 0.3 r minus the lower arcs, layer 3
    the lenses (both arcs) on the precursor h*; heights [3][ny][nx]."""
    th = math.radians(theta0_deg)
    rc = radius / math.sin(th)
    depth = rc * (1.0 - math.cos(th))
    x = np.arange(nx, dtype=float)[None, :]
    y = np.arange(ny, dtype=float)[:, None]
    arc = np.zeros((ny, nx))
    for cx, cy in lens3_centres(nx, ny, radius, seed=seed):
        dx = np.abs(x - cx); dx = np.minimum(dx, nx - dx)
        dy = np.abs(y - cy); dy = np.minimum(dy, ny - dy)
        arc = np.maximum(arc, cap_profile(np.hypot(dx, dy), depth, 0.0, th))
    t2 = 0.3 * radius
    return np.stack([np.ones((ny, nx)), t2 - arc, hstar + 2.0 * arc])


def sweep_instances(count=512, seed=3, sides=(64, 128, 256, 512), eps=1e-4):
    """The batched stability sweep: a list of (params, heights [n][side][side]
    float32, (kx, ky), amps) per instance."""
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(count):
        n = int(rng.integers(2, 6))
        side = int(rng.choice(sides))
        gamma = [float(g) for g in np.exp(rng.uniform(np.log(2e-3), np.log(2e-2), n))]
        mu1 = 1.0 / 16.0
        mu = [mu1] + [float(mu1 * r) for r in np.exp(rng.uniform(np.log(0.25), np.log(4.0), n - 1))]
        p = dict(n=n, lattice=2, nx=side, ny=side, tau=1.0, gamma=gamma,
                 S=_young_spreading(gamma, 20.0, n), mu=mu, beta=[1.0] * n, nw=3, mw=2,
                 hstar=0.07)
        means = rng.uniform(0.6, 1.1, n)
        amps = rng.uniform(-1.0, 1.0, n)
        while True:
            kx, ky = (int(v) for v in rng.integers(0, 9, 2))
            if kx or ky:
                break
        x = np.arange(side, dtype=np.float64)
        ph = 2.0 * np.pi * (kx * x[None, :] + ky * x[:, None]) / side
        mode = np.cos(ph)
        h = np.empty((n, side, side), dtype=np.float32)
        for i in range(n):
            h[i] = means[i] + eps * amps[i] * mode
        out.append((p, h, (kx, ky), amps))
    return out


def dewet2_params(side=64, theta_deg=20.0):
    """Two thin layers on D2Q9 that dewet: gamma 0.01 / 0.01, S_01 = S_11 =
    gamma (cos theta - 1), mu = 1/6, slip 1, (3, 2), h* = 0.05."""
    g = 0.01
    s = g * (math.cos(math.radians(theta_deg)) - 1.0)
    return dict(n=2, lattice=2, nx=int(side), ny=int(side), tau=1.0, gamma=[g, g],
                S=[[s, 0.0], [s]], mu=[1.0 / 6.0, 1.0 / 6.0], beta=[1.0, 1.0], nw=3, mw=2,
                hstar=0.05)


def dewet2_heights(side=64, seed=9):
    """Both layers 0.25 plus seeded Gaussian noise sigma = 1e-3."""
    rng = np.random.default_rng(seed)
    return 0.25 + 1e-3 * rng.standard_normal((2, side, side))


def film3_d2q9_heights_device(nx, ny, count, seed):
    """`count` three-layer films of the same recipe (means 1.0 / 0.8 / 0.6,
    Gaussian noise sigma 1e-3), drawn on the GPU from a generator seeded
    with `seed`: a float32 CUDA tensor [count][3][ny][nx]. Used where many
    thousand seeded films are needed at once."""
    import torch
    g = torch.Generator(device="cuda")
    g.manual_seed(int(seed))
    means = torch.tensor([1.0, 0.8, 0.6], device="cuda").view(1, 3, 1, 1)
    return (means + 1e-3 * torch.randn((int(count), 3, int(ny), int(nx)), generator=g,
                                       device="cuda")).float().contiguous()


def film3_unet_planes(p):
    """Constant input planes of the U-Net surrogate for a three-layer film:
    the tensions relative to 0.01 and the viscosity ratios mu_2 / mu_1 and
    mu_3 / mu_1 over 4."""
    return [g / 0.01 for g in p["gamma"]] + [m / p["mu"][0] / 4.0 for m in p["mu"][1:]]
