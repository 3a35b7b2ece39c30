"""Contact-angle measurement of relaxed droplets and lenses, as in the
paper's droplet-equilibrium section: a circular arc H_theta that shares the
peak position and height of the measured profile is fitted by minimising
the relative volume difference

    E(theta) = sum |h - H_theta| / sum (h - base),

and Young's law (sessile drops) or Neumann's law (lenses) gives the
expected angle. In 2-D the profile is the azimuthal average around the
drop's peak and the sums carry the ring area 2 pi r. Test helpers only.
"""
import math

import numpy as np

import workloads


def _scan_min(err, lo_deg=0.5, hi_deg=60.0):
    """Minimum of err(theta) by a 0.01-degree scan refined by golden section."""
    ths = np.radians(np.arange(lo_deg, hi_deg, 0.05))
    es = np.array([err(t) for t in ths])
    j = int(np.argmin(es))
    a = ths[max(j - 1, 0)]
    b = ths[min(j + 1, len(ths) - 1)]
    g = (math.sqrt(5.0) - 1.0) / 2.0
    c, d = b - g * (b - a), a + g * (b - a)
    for _ in range(40):
        if err(c) < err(d):
            b = d
        else:
            a = c
        c, d = b - g * (b - a), a + g * (b - a)
    t = 0.5 * (a + b)
    return t, err(t)


def arc_error(dist, h, weight, base, theta):
    """E(theta) of a profile h(dist) against the arc through its peak."""
    i = int(np.argmax(h))
    arc = workloads.cap_profile(dist - dist[i], h[i], base, theta)
    return float((weight * np.abs(h - arc)).sum() / (weight * (h - base)).sum())


def fit_angle_1d(h, base, centre=None):
    """Fitted contact angle (degrees) and E of a periodic 1-D profile; the
    distance is taken from the profile's peak (or `centre`)."""
    h = np.asarray(h, dtype=float).ravel()
    nx = h.size
    c = int(np.argmax(h)) if centre is None else int(centre)
    # unwrap the periodic box around the peak
    order = (np.arange(nx) + c - nx // 2) % nx
    hh = h[order]
    dist = np.arange(nx, dtype=float) - nx // 2
    w = np.ones(nx)
    t, e = _scan_min(lambda th: arc_error(dist, hh, w, base, th))
    return math.degrees(t), e


def error_at_angle_1d(h, base, theta_deg):
    h = np.asarray(h, dtype=float).ravel()
    nx = h.size
    c = int(np.argmax(h))
    hh = h[(np.arange(nx) + c - nx // 2) % nx]
    dist = np.arange(nx, dtype=float) - nx // 2
    return arc_error(dist, hh, np.ones(nx), base, math.radians(theta_deg))


def radial_profile(field, centre, rmax):
    """Azimuthal average of a periodic 2-D field in unit-width rings around
    centre (x, y); returns ring radii, means and ring areas."""
    ny, nx = field.shape
    x = np.arange(nx, dtype=float)[None, :]
    y = np.arange(ny, dtype=float)[:, None]
    dx = x - centre[0]
    dx -= nx * np.round(dx / nx)
    dy = y - centre[1]
    dy -= ny * np.round(dy / ny)
    r = np.hypot(dx, dy)
    k = np.floor(r).astype(int)
    nb = int(rmax)
    sums = np.bincount(k.ravel(), weights=field.ravel(), minlength=nb + 1)[:nb]
    cnts = np.bincount(k.ravel(), minlength=nb + 1)[:nb]
    rad = np.arange(nb) + 0.5
    return rad, sums / np.maximum(cnts, 1), cnts.astype(float)


def fit_angle_radial(field, centre, rmax, base):
    """Fitted angle (degrees) and E of an axisymmetric cap in a 2-D field."""
    rad, prof, area = radial_profile(field, centre, rmax)
    # the profile is a function of r >= 0 with its peak at r = 0
    t, e = _scan_min(lambda th: _radial_err(rad, prof, area, base, th))
    return math.degrees(t), e


def _radial_err(rad, prof, area, base, theta):
    arc = workloads.cap_profile(rad, prof[0], base, theta)
    return float((area * np.abs(prof - arc)).sum() / (area * (prof - base)).sum())


def peak_centre(field, guess, window):
    """Centroid of the excess above the window's minimum near `guess`
    (periodic), which locates a drop to sub-cell accuracy."""
    ny, nx = field.shape
    gx, gy = int(round(guess[0])), int(round(guess[1]))
    xs = (np.arange(gx - window, gx + window + 1)) % nx
    ys = (np.arange(gy - window, gy + window + 1)) % ny
    sub = field[np.ix_(ys, xs)]
    ex = sub - sub.min()
    w = ex.sum()
    cx = (ex.sum(axis=0) * np.arange(-window, window + 1)).sum() / w + gx
    cy = (ex.sum(axis=1) * np.arange(-window, window + 1)).sum() / w + gy
    return cx % nx, cy % ny


def lens_angles_1d(h, hstar, far=10):
    """Upper and lower opening angles (degrees) and their E for a 1-D lens
    of layer 2 on layer 1 (heights [2][nx]): the upper arc is z2 above its
    far level, the lower one z1 below its far level."""
    h = np.asarray(h, dtype=float).reshape(2, -1)
    z1, z2 = h[0], h[0] + h[1]
    c = int(np.argmax(h[1]))
    nx = z1.size
    farx = (np.arange(far) + c + nx // 2 - far // 2) % nx
    up = z2 - z2[farx].mean()
    lo = z1[farx].mean() - z1
    tu, eu = fit_angle_1d(up, 0.0, centre=c)
    tl, el = fit_angle_1d(lo, 0.0, centre=c)
    return (tu, eu), (tl, el)


def lens3_angles(h, centres, radius):
    """Upper and lower opening angles of every lens in a three-layer field
    (heights [3][ny][nx]): the upper surface z3 and the lower surface z2
    against their far levels, each from its azimuthal profile."""
    h = np.asarray(h, dtype=float)
    z2 = h[0] + h[1]
    z3 = z2 + h[2]
    out = []
    for c in centres:
        cc = peak_centre(h[2], c, int(radius))
        rmax = 1.6 * radius
        rad, p3, _ = radial_profile(z3, cc, rmax)
        rad, p2, _ = radial_profile(z2, cc, rmax)
        up = fit_angle_radial(z3 - p3[-3:].mean(), cc, rmax, 0.0)
        lo = fit_angle_radial(p2[-3:].mean() - z2, cc, rmax, 0.0)
        out.append((up, lo))
    return out


def free_energy(p, h):
    """Free energy of Eq. (free_energy_n_layer), long-wave form, from heights
    [n][ny][nx] with the lattice gradient of the step (isotropic stencil on
    D2Q9, central difference on D1Q3); S_ik phi_k for the wetting terms (the
    power law, or the exponential form when p["wet_kind"] == 1); the
    substrate z_0 of the parameters (sinusoidal, or flat)."""
    n = int(p["n"])
    ny, nx = int(p["ny"]), int(p["nx"])
    h = np.asarray(h, dtype=np.float64).reshape(n, ny, nx)
    y, x = np.meshgrid(np.arange(ny), np.arange(nx), indexing="ij")
    z0 = float(p.get("sub_amp", 0.0)) * np.cos(
        2 * np.pi * (int(p.get("sub_kx", 0)) * x / nx + int(p.get("sub_ky", 0)) * y / ny))
    z = np.concatenate([z0[None], z0[None] + np.cumsum(h, axis=0)])

    def sh(a, dx, dy):  # a(x + dx, y + dy), periodic
        return np.roll(np.roll(a, -dx, axis=-1), -dy, axis=-2)

    def grad2(a):
        if int(p["lattice"]) == 2:
            gx = (sh(a, 1, 0) - sh(a, -1, 0)) / 3.0 + ((sh(a, 1, 1) - sh(a, -1, 1))
                                                      + (sh(a, 1, -1) - sh(a, -1, -1))) / 12.0
            gy = (sh(a, 0, 1) - sh(a, 0, -1)) / 3.0 + ((sh(a, 1, 1) - sh(a, 1, -1))
                                                      + (sh(a, -1, 1) - sh(a, -1, -1))) / 12.0
            return gx * gx + gy * gy
        gx = 0.5 * (sh(a, 1, 0) - sh(a, -1, 0))
        return gx * gx

    g2 = [grad2(z[i]) for i in range(0, n + 1)]
    hs, nw, mw = float(p["hstar"]), int(p["nw"]), int(p["mw"])

    def phi(k, t):
        if int(p.get("wet_kind", 0)) == 1:  # charged surfaces: 2 a - a^2
            a = np.exp(-float(p["kappa"]) * (t - k * hs))
            return 2 * a - a * a
        r = k * hs / t
        return (nw * r ** mw - mw * r ** nw) / (nw - mw)

    F = 0.0
    for i in range(1, n + 1):
        F += (p["gamma"][i - 1] * (1.0 + 0.5 * g2[i])).sum()
    for i in range(0, n):
        for k in range(1, n - i + 1):
            F += (p["S"][i][k - 1] * phi(k, z[i + k] - z[i]) * (1.0 + 0.5 * g2[i])).sum()
    return float(F)


def radial_spectrum(field, nbins=None):
    """Azimuthally averaged power |hhat(q)|^2 of a periodic 2-D field
    (mean removed), in unit-width bins of |k| (integer wavenumbers)."""
    f = np.asarray(field, dtype=np.float64)
    ny, nx = f.shape
    P = np.abs(np.fft.fft2(f - f.mean())) ** 2
    ky = np.fft.fftfreq(ny) * ny
    kx = np.fft.fftfreq(nx) * nx
    k = np.hypot(kx[None, :], ky[:, None])
    b = np.rint(k).astype(int)
    nb = nbins or min(nx, ny) // 2
    s = np.bincount(b.ravel(), weights=P.ravel(), minlength=nb + 1)[:nb]
    c = np.bincount(b.ravel(), minlength=nb + 1)[:nb]
    return s / np.maximum(c, 1)


def rupture_step(sample, hstar, every, limit):
    """First multiple of `every` (up to `limit`) at which some layer of
    sample(t) -> heights falls below 1.5 h*, with the heights then."""
    for t in range(every, limit + 1, every):
        h = sample(t)
        if h.min() < 1.5 * hstar:
            return t, h
    return None, None
