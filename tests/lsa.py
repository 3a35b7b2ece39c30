"""Independent linearisation of the multilayer LBM step about a flat film.

Test helper (no CUDA, no oracle code). For a periodic lattice and one Fourier
mode exp(i q.x) the step is linear in the perturbation of the populations,
so one time step is a complex matrix G(q) of size (n Q) x (n Q). It is built
here straight from the definitions:

  * heights and fluxes are the zeroth and first population moments;
  * pressures: Eq. (Laplace_pressure) and Eq. (disjoining_pressure) expanded
    to first order about the flat interfaces Z_i (the |grad z|^2 terms are
    second order and drop); p_i = sum_{j >= i} (Lambda_j + Pi_j);
  * lattice gradient / Laplacian become their Fourier symbols
        grad -> (1/c_s^2) sum_k w_k c_k (e^{i q.c_k} - 1),
        lap  -> (2/c_s^2) sum_k w_k (e^{i q.c_k} - 1);
  * friction: R = K(h0) J with K taken from the shear-stress integration
    below (derived from Eqs. (u_ansatz)-(viscous_boundary) independently of
    the matrix D);
  * Eq. (equilibrium_distribution) to first order: f0 = h, f_k = w_k c_k.J/c_s^2;
  * Eq. (BGK) with Eq. (force), then streaming f_k(x + c_k) = f*_k(x), i.e.
    multiplication by e^{-i q.c_k}.

It also gives the continuum growth matrix of Eq. (linear_thin_film_equation)
with the mobility of Eq. (thin_film_equation_n) written as M = -K^-1 T.
"""
import numpy as np

CS2 = 1.0 / 3.0

D1Q3 = (np.array([0, 1, -1]), np.array([0, 0, 0]), np.array([2 / 3, 1 / 6, 1 / 6]))
D2Q9 = (np.array([0, 1, 1, 0, -1, -1, -1, 0, 1]),
        np.array([0, 0, 1, 1, 1, 0, -1, -1, -1]),
        np.array([4 / 9, 1 / 9, 1 / 36, 1 / 9, 1 / 36, 1 / 9, 1 / 36, 1 / 9, 1 / 36]))


def lattice(p):
    return D1Q3 if int(p["lattice"]) == 1 else D2Q9


def _exp_a(p, k, h):
    """a = e^{-kappa (h - k h*)} of the exponential (charged-surface) form
    phi_k = 2 a - a^2 (wet_kind 1)."""
    return np.exp(-p["kappa"] * (h - k * p["hstar"]))


def phi_k(p, k, h):
    if int(p.get("wet_kind", 0)) == 1:
        a = _exp_a(p, k, h)
        return 2 * a - a * a
    a = k * p["hstar"] / h
    n, m = p["nw"], p["mw"]
    return (n * a ** m - m * a ** n) / (n - m)


def dphi_k(p, k, h):
    if int(p.get("wet_kind", 0)) == 1:
        a = _exp_a(p, k, h)  # da/dh = -kappa a
        return 2 * p["kappa"] * a * (a - 1)
    a = k * p["hstar"] / h
    n, m = p["nw"], p["mw"]
    return n * m / (n - m) * (a ** n - a ** m) / h


def ddphi_k(p, k, h):
    if int(p.get("wet_kind", 0)) == 1:
        a = _exp_a(p, k, h)
        return 2 * p["kappa"] ** 2 * a * (1 - 2 * a)
    a = k * p["hstar"] / h
    n, m = p["nw"], p["mw"]
    return n * m / (n - m) * (-(n + 1) * a ** n + (m + 1) * a ** m) / h ** 2


def flux_of_gradients(h, mu, beta):
    """Matrix L with J = L G for per-layer pressure gradients G.

    Stokes layers: mu_i u'' = G_i. The shear stress in layer i, integrated
    down from the stress-free top, is G_i (z - z_i) - sum_{j>i} h_j G_j. The
    velocity is integrated upward from u = 0 at z_0 - beta_1; at each
    interface the upper layer's parabola, continued a distance beta_{i+1}
    below the interface, meets the lower layer's interface velocity
    (Eq. no_slip). Layer fluxes are the integrals of u over each layer.
    """
    n = len(h)
    L = np.zeros((n, n))
    for j in range(n):
        G = np.zeros(n)
        G[j] = 1.0
        ub = 0.0
        for i in range(n):
            s = -sum(h[q] * G[q] for q in range(i + 1, n))  # stress at z_i
            # slip zone below z_{i-1}: mean stress at z_{i-1} - beta_i / 2
            ub += beta[i] / mu[i] * (s - G[i] * (h[i] + beta[i] / 2))
            L[i, j] = h[i] * ub + (s * h[i] ** 2 / 2 - G[i] * h[i] ** 3 / 3) / mu[i]
            ub += (s * h[i] - G[i] * h[i] ** 2 / 2) / mu[i]
    return L


def friction_matrix(p, h):
    """K with friction R = K J: force balance R_i = h_i G_i, J = L G."""
    h = np.asarray(h, dtype=float)
    L = flux_of_gradients(h, p["mu"], p["beta"])
    return np.diag(h) @ np.linalg.inv(L)


def pressure_jump_jacobian(p, h0, lap_sym):
    """E[i, j] = d(Lambda_i + Pi_i) / d z_j at the flat state (0-based)."""
    n = int(p["n"])
    S = p["S"]
    Z = np.concatenate([[0.0], np.cumsum(h0)])
    E = np.zeros((n, n), dtype=complex)
    for i in range(1, n + 1):
        tension = p["gamma"][i - 1]
        for k in range(1, n - i + 1):
            tension += S[i][k - 1] * phi_k(p, k, Z[i + k] - Z[i])
        E[i - 1, i - 1] += -tension * lap_sym
        # - sum_k S_ik phi'_k(z_{i+k} - z_i)
        for k in range(1, n - i + 1):
            c = -S[i][k - 1] * ddphi_k(p, k, Z[i + k] - Z[i])
            E[i - 1, i + k - 1] += c
            E[i - 1, i - 1] -= c
        # + sum_l S_{l,i-l} phi'_{i-l}(z_i - z_l)
        for l in range(0, i):
            c = S[l][i - l - 1] * ddphi_k(p, i - l, Z[i] - Z[l])
            E[i - 1, i - 1] += c
            if l >= 1:
                E[i - 1, l - 1] -= c
    return E


def symbols(p, q):
    cx, cy, w = lattice(p)
    ph = np.exp(1j * (q[0] * cx + q[1] * cy))
    gx = np.sum(w * cx * (ph - 1)) / CS2
    gy = np.sum(w * cy * (ph - 1)) / CS2
    lap = 2 * np.sum(w * (ph - 1)) / CS2
    return gx, gy, lap


def step_matrix(p, h0, q):
    """G(q) acting on the population perturbation vector, index i*Q + k."""
    n = int(p["n"])
    tau = float(p["tau"])
    cx, cy, w = lattice(p)
    Qn = len(w)
    gx, gy, lap = symbols(p, q)
    E = pressure_jump_jacobian(p, h0, lap.real)
    Lz = np.tril(np.ones((n, n)))  # z = Lz h
    Up = np.triu(np.ones((n, n)))  # p = Up Delta
    P_of_h = Up @ E @ Lz           # p_i perturbation from h perturbation
    K = friction_matrix(p, h0)
    N = n * Qn
    Hm = np.zeros((n, N))
    Jx = np.zeros((n, N))
    Jy = np.zeros((n, N))
    for i in range(n):
        for k in range(Qn):
            Hm[i, i * Qn + k] = 1
            Jx[i, i * Qn + k] = cx[k]
            Jy[i, i * Qn + k] = cy[k]
    pm = P_of_h @ Hm
    Fx = -np.diag(h0) @ (gx * pm) + K @ Jx
    Fy = -np.diag(h0) @ (gy * pm) + K @ Jy
    C = (1 - 1 / tau) * np.eye(N, dtype=complex)
    for i in range(n):
        for k in range(Qn):
            r = i * Qn + k
            if k == 0:
                feq = Hm[i]
            else:
                feq = w[k] * (cx[k] * Jx[i] + cy[k] * Jy[i]) / CS2
            C[r] += feq / tau + w[k] * (cx[k] * Fx[i] + cy[k] * Fy[i]) / CS2
    shift = np.exp(-1j * (q[0] * np.tile(cx, n) + q[1] * np.tile(cy, n)))
    return shift[:, None] * C


def continuum_growth(p, h0, qmag):
    """Eigenvalues of A = -q^2 M E(q) with M = -K^-1 T, continuum symbols."""
    n = int(p["n"])
    h0 = np.asarray(h0, dtype=float)
    E = pressure_jump_jacobian(p, h0, -qmag ** 2).real
    Lz = np.tril(np.ones((n, n)))
    T = np.diag(h0) @ np.triu(np.ones((n, n)))
    M = -np.linalg.inv(friction_matrix(p, h0)) @ T
    A = -qmag ** 2 * M @ E @ Lz
    return np.linalg.eigvals(A)
