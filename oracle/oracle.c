/*
 * oracle.c -- FP64 CPU oracle of the multilayer shallow-water LBM step.
 *
 * TEST INFRASTRUCTURE ONLY (see oracle.h). Plain loops over cells and
 * layers, dense LU for the boundary-condition system, no blocking, no
 * fusion. One step follows this order for every cell, using time-t data only:
 *   1. moments h_i = sum_k f_ki, J_i = sum_k c_k f_ki        (section LBM)
 *   2. interfaces z_0 = 0, z_i = z_{i-1} + h_i               (section Model)
 *   3. grad z_i and lap z_i with the lattice stencils
 *   4. Lambda_i, Pi_i, p_i = sum_{j>=i} (Lambda_j + Pi_j)
 *   5. grad p_i
 *   6. D a = r for the friction 2 mu_i h_i a_i                (Eq. friction_force)
 *   7. F_i = -h_i grad p_i + 2 mu_i h_i a_i                    (Eq. force)
 *   8. f* = f - (f - f_eq)/tau + w_k c_k . F_i / c_s^2         (Eq. BGK)
 *   9. f_ki(x + c_k, t + 1) = f*_ki(x)
 *
 * Readings of passages that are garbled, ambiguous or silent (each is also
 * listed with its reasoning in the design notes):
 *   R1  D, first row: u_1(z_0 - beta_1) = 0 with z_0 = 0 gives
 *       [beta_1^2, -beta_1, 1] (Eq. no_slip); the printed +beta_1 is a sign slip.
 *   R2  right-hand side of Eq. (boundary_conditions): every flux row carries
 *       +h_i U_i = J_i (Eq. flux); the printed z_1 U_1 ... (z_{n-1}-z_n) U_n
 *       are misprints of the layer thickness.
 *   R3  stress rows use mu_{i+1}/mu_i (Eq. viscous_boundary); the last block
 *       printed mu_{n-1}/mu_n is read as mu_n/mu_{n-1}. z_n^2 - z_{n-1}^3 is
 *       read as z_n^2 - z_{n-1}^2.
 *   R4  S = (D^-1)_{3j+1, 3k+2} (1-based), the full n x n block that maps the
 *       flux rows to the a_j unknowns, so a = S J.
 *   R5  discrete derivatives: the isotropic lattice stencils
 *       grad phi = (1/c_s^2) sum_k w_k c_k (phi(x+c_k) - phi(x)),
 *       lap  phi = (2/c_s^2) sum_k w_k (phi(x+c_k) - phi(x)).
 *   R6  equilibrium: f_{k0} means the rest population of layer i; c_2^4 means
 *       c_s^4; there is no constant w_k h term (the scheme "lacks the
 *       dispersive term").
 *   R7  forcing: 1/c_2^2 means 1/c_s^2; the direction c_k is kept in the
 *       forcing term, w_k c_k . F_i / c_s^2. No velocity shift.
 *   R8  D2Q9 velocities are the integer vectors; sqrt(2) in the printed list is
 *       the length of the diagonal ones.
 *   R9  the substrate is flat (z_0 = 0) unless a sinusoidal z_0 is given
 *       (sub_amp, sub_kx, sub_ky); z_0 enters the interface heights and the
 *       (1 + |grad z_0|^2 / 2) factor of the substrate's wetting terms.
 */
#include "oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

/* ------------------------------------------------------------------ */
/* lattices (section LBM)                                              */
/* ------------------------------------------------------------------ */
static const int D1Q3_CX[3] = {0, 1, -1};
static const double D1Q3_W[3] = {2.0 / 3.0, 1.0 / 6.0, 1.0 / 6.0};

/* c_0 = 0, then counter-clockwise from +x */
static const int D2Q9_CX[9] = {0, 1, 1, 0, -1, -1, -1, 0, 1};
static const int D2Q9_CY[9] = {0, 0, 1, 1, 1, 0, -1, -1, -1};
static const double D2Q9_W[9] = {4.0 / 9.0,  1.0 / 9.0,  1.0 / 36.0,
                                 1.0 / 9.0,  1.0 / 36.0, 1.0 / 9.0,
                                 1.0 / 36.0, 1.0 / 9.0,  1.0 / 36.0};
static const double CS2 = 1.0 / 3.0; /* lattice speed of sound squared */

int orc_Q(const orc_params* P) { return P->lattice == 1 ? 3 : 9; }

void orc_lattice(const orc_params* P, int* cx, int* cy, double* w) {
  int Q = orc_Q(P);
  for (int k = 0; k < Q; ++k) {
    if (P->lattice == 1) {
      cx[k] = D1Q3_CX[k];
      cy[k] = 0;
      w[k] = D1Q3_W[k];
    } else {
      cx[k] = D2Q9_CX[k];
      cy[k] = D2Q9_CY[k];
      w[k] = D2Q9_W[k];
    }
  }
}

/* ------------------------------------------------------------------ */
/* wetting potential, Eq. (wetting_potential)                          */
/*   phi_k(h) = [nw r^mw - mw r^nw] / (nw - mw), r = k hstar / h        */
/* or, for charged surfaces (wet_kind 1), with a = e^{-kappa (h - k h*)} */
/*   phi_k(h) = 2 a - a^2                                               */
/* ------------------------------------------------------------------ */
double orc_phi(const orc_params* P, int k, double h) {
  if (P->wet_kind == 1) {
    double a = exp(-P->kappa * (h - (double)k * P->hstar));
    return 2.0 * a - a * a;
  }
  double r = (double)k * P->hstar / h;
  double n = (double)P->nw, m = (double)P->mw;
  return (n * pow(r, m) - m * pow(r, n)) / (n - m);
}

/* d/dh of the above: d(r^a)/dh = -a r^a / h; da/dh = -kappa a */
double orc_dphi(const orc_params* P, int k, double h) {
  if (P->wet_kind == 1) {
    double a = exp(-P->kappa * (h - (double)k * P->hstar));
    return (2.0 - 2.0 * a) * (-P->kappa * a);
  }
  double r = (double)k * P->hstar / h;
  double n = (double)P->nw, m = (double)P->mw;
  return (n * (-m * pow(r, m) / h) - m * (-n * pow(r, n) / h)) / (n - m);
}

/* ------------------------------------------------------------------ */
/* spreading coefficients, Eq. (spreading_parameters)                  */
/* ------------------------------------------------------------------ */
void orc_spreading_from_tensions(orc_params* P, const double* g) {
  int n = P->n, G = n + 2;
#define GAM(a, b) g[(a) * G + (b)]
  for (int i = 0; i < ORC_MAXN; ++i)
    for (int k = 0; k < ORC_MAXN; ++k) P->S[i][k] = 0.0;
  for (int i = 0; i < n; ++i) {
    for (int k = 1; k <= n - i; ++k) {
      double s;
      if (k == 1)
        s = GAM(i, i + 2) - GAM(i, i + 1) - GAM(i + 1, i + 2);
      else
        s = GAM(i, i + k + 1) + GAM(i + 1, i + k) - GAM(i, i + k) -
            GAM(i + 1, i + k + 1);
      P->S[i][k - 1] = s;
    }
  }
  for (int i = 1; i <= n; ++i) P->gamma[i - 1] = GAM(i, i + 1);
#undef GAM
}

/* ------------------------------------------------------------------ */
/* boundary-condition matrix D, Eq. (boundary_conditions)              */
/* unknowns ordered (a_1, b_1, c_1, ..., a_n, b_n, c_n); rows:          */
/*   row 0            : u_1(z_0 - beta_1) = 0                   (R1)    */
/*   row 1            : flux of layer 1                                */
/*   rows 3i-1..3i+1  : for interface i = 1..n-1: stress continuity,   */
/*                      velocity continuity with slip beta_{i+1},      */
/*                      flux of layer i+1                              */
/*   row 3n-1         : stress-free top, 2 a_n z_n + b_n = 0            */
/* ------------------------------------------------------------------ */
void orc_build_D(const orc_params* P, const double* h, double* D) {
  int n = P->n, N3 = 3 * n;
  double z[ORC_MAXN + 1];
  z[0] = 0.0;
  for (int i = 1; i <= n; ++i) z[i] = z[i - 1] + h[i - 1];
  for (int r = 0; r < N3 * N3; ++r) D[r] = 0.0;
#define DD(r, c) D[(r) * N3 + (c)]
  /* Eq. (no_slip) at the substrate, heights measured from z_0 (R1, R9) */
  double b1 = P->beta[0];
  double zb = z[0] - b1;
  DD(0, 0) = zb * zb;
  DD(0, 1) = zb;
  DD(0, 2) = 1.0;
  /* Eq. (flux) of layer 1 */
  DD(1, 0) = (z[1] * z[1] * z[1] - z[0] * z[0] * z[0]) / 3.0;
  DD(1, 1) = (z[1] * z[1] - z[0] * z[0]) / 2.0;
  DD(1, 2) = z[1] - z[0];
  int row = 2;
  for (int i = 1; i <= n - 1; ++i) {
    int cl = 3 * (i - 1), cu = 3 * i; /* columns of layers i and i+1 */
    double zi = z[i];
    double ratio = P->mu[i] / P->mu[i - 1]; /* mu_{i+1}/mu_i (R3) */
    /* Eq. (viscous_boundary): u_i'(z_i) = (mu_{i+1}/mu_i) u_{i+1}'(z_i) */
    DD(row, cl + 0) = 2.0 * zi;
    DD(row, cl + 1) = 1.0;
    DD(row, cu + 0) = -2.0 * ratio * zi;
    DD(row, cu + 1) = -ratio;
    ++row;
    /* Eq. (no_slip): u_{i+1}(z_i - beta_{i+1}) = u_i(z_i) */
    double zs = zi - P->beta[i];
    DD(row, cl + 0) = zi * zi;
    DD(row, cl + 1) = zi;
    DD(row, cl + 2) = 1.0;
    DD(row, cu + 0) = -zs * zs;
    DD(row, cu + 1) = -zs;
    DD(row, cu + 2) = -1.0;
    ++row;
    /* Eq. (flux) of layer i+1 */
    double zl = z[i], zu = z[i + 1];
    DD(row, cu + 0) = (zu * zu * zu - zl * zl * zl) / 3.0;
    DD(row, cu + 1) = (zu * zu - zl * zl) / 2.0;
    DD(row, cu + 2) = zu - zl;
    ++row;
  }
  /* stress-free top: mu_{n+1} = 0 in Eq. (viscous_boundary) */
  DD(row, 3 * (n - 1) + 0) = 2.0 * z[n];
  DD(row, 3 * (n - 1) + 1) = 1.0;
#undef DD
}

/* dense LU with partial pivoting, solves A x = b for nrhs right-hand sides
 * stored as columns of B (m x nrhs, row-major). A and B are overwritten. */
static int lu_solve(int m, double* A, int nrhs, double* B) {
  for (int c = 0; c < m; ++c) {
    int p = c;
    double best = fabs(A[c * m + c]);
    for (int r = c + 1; r < m; ++r)
      if (fabs(A[r * m + c]) > best) {
        best = fabs(A[r * m + c]);
        p = r;
      }
    if (best == 0.0) return -1;
    if (p != c) {
      for (int j = 0; j < m; ++j) {
        double t = A[c * m + j];
        A[c * m + j] = A[p * m + j];
        A[p * m + j] = t;
      }
      for (int j = 0; j < nrhs; ++j) {
        double t = B[c * nrhs + j];
        B[c * nrhs + j] = B[p * nrhs + j];
        B[p * nrhs + j] = t;
      }
    }
    for (int r = c + 1; r < m; ++r) {
      double l = A[r * m + c] / A[c * m + c];
      if (l == 0.0) continue;
      for (int j = c; j < m; ++j) A[r * m + j] -= l * A[c * m + j];
      for (int j = 0; j < nrhs; ++j) B[r * nrhs + j] -= l * B[c * nrhs + j];
    }
  }
  for (int c = m - 1; c >= 0; --c) {
    for (int j = 0; j < nrhs; ++j) {
      double s = B[c * nrhs + j];
      for (int k = c + 1; k < m; ++k) s -= A[c * m + k] * B[k * nrhs + j];
      B[c * nrhs + j] = s / A[c * m + c];
    }
  }
  return 0;
}

/* Eq. (friction_force): (2 mu_i h_i a_i) with a = S (h U) (R2, R4). The two
 * flux components share the same D, so they are two right-hand sides. */
int orc_friction(const orc_params* P, const double* h, const double* Jx,
                 const double* Jy, double* Rx, double* Ry) {
  int n = P->n, N3 = 3 * n;
  double D[9 * ORC_MAXN * ORC_MAXN];
  double B[3 * ORC_MAXN * 2];
  orc_build_D(P, h, D);
  for (int r = 0; r < N3 * 2; ++r) B[r] = 0.0;
  for (int i = 1; i <= n; ++i) {
    int flux_row = 3 * (i - 1) + 1; /* row 3k+2 (1-based) for layer k+1 */
    B[flux_row * 2 + 0] = Jx[i - 1];
    B[flux_row * 2 + 1] = Jy ? Jy[i - 1] : 0.0;
  }
  if (lu_solve(N3, D, 2, B) != 0) return -1;
  for (int i = 1; i <= n; ++i) {
    double ax = B[(3 * (i - 1)) * 2 + 0];
    double ay = B[(3 * (i - 1)) * 2 + 1];
    Rx[i - 1] = 2.0 * P->mu[i - 1] * h[i - 1] * ax;
    if (Ry) Ry[i - 1] = 2.0 * P->mu[i - 1] * h[i - 1] * ay;
  }
  return 0;
}

/* ------------------------------------------------------------------ */
/* pressures: Eq. (Laplace_pressure), Eq. (disjoining_pressure) and     */
/* p_i - p_atm = sum_{j=i}^{n} (Lambda_j + Pi_j)                       */
/* ------------------------------------------------------------------ */
void orc_pressures(const orc_params* P, const double* h, const double* gzx,
                   const double* gzy, const double* lz, double* Lambda,
                   double* Pi, double* p) {
  orc_pressures_sub(P, h, gzx, gzy, lz, 0.0, Lambda, Pi, p); /* flat (R9) */
}

void orc_pressures_sub(const orc_params* P, const double* h, const double* gzx,
                       const double* gzy, const double* lz, double g0sq,
                       double* Lambda, double* Pi, double* p) {
  int n = P->n;
  /* z relative to the substrate: only thicknesses z_m - z_l enter below */
  double z[ORC_MAXN + 1], g2[ORC_MAXN + 1];
  z[0] = 0.0;
  g2[0] = g0sq; /* |grad z_0|^2 of the substrate */
  for (int i = 1; i <= n; ++i) {
    z[i] = z[i - 1] + h[i - 1];
    double gx = gzx[i - 1], gy = gzy ? gzy[i - 1] : 0.0;
    g2[i] = gx * gx + gy * gy;
  }
  for (int i = 1; i <= n; ++i) {
    /* Laplace pressure with interpolated tension */
    double tension = P->gamma[i - 1];
    for (int k = 1; k <= n - i; ++k)
      tension += P->S[i][k - 1] * orc_phi(P, k, z[i + k] - z[i]);
    Lambda[i - 1] = -tension * lz[i - 1];
    /* disjoining pressure: pull of the layers above, push from below */
    double pi = 0.0;
    for (int k = 1; k <= n - i; ++k)
      pi -= P->S[i][k - 1] * orc_dphi(P, k, z[i + k] - z[i]) *
            (1.0 + g2[i] / 2.0);
    for (int l = 0; l <= i - 1; ++l)
      pi += P->S[l][i - l - 1] * orc_dphi(P, i - l, z[i] - z[l]) *
            (1.0 + g2[l] / 2.0);
    Pi[i - 1] = pi;
  }
  double acc = 0.0;
  for (int i = n; i >= 1; --i) {
    acc += Lambda[i - 1] + Pi[i - 1];
    p[i - 1] = acc;
  }
}

/* ------------------------------------------------------------------ */
/* equilibrium, Eq. (equilibrium_distribution) (R6)                    */
/* ------------------------------------------------------------------ */
void orc_equilibrium(const orc_params* P, double h, double Ux, double Uy,
                     double* feq) {
  int cx[9], cy[9];
  double w[9];
  orc_lattice(P, cx, cy, w);
  int Q = orc_Q(P);
  double U2 = Ux * Ux + Uy * Uy;
  feq[0] = h * (1.0 - w[0] * U2 / (2.0 * CS2));
  for (int k = 1; k < Q; ++k) {
    double cu = cx[k] * Ux + cy[k] * Uy;
    feq[k] = w[k] * h *
             (cu / CS2 + cu * cu / (2.0 * CS2 * CS2) - U2 / (2.0 * CS2));
  }
}

void orc_init(const orc_params* P, const double* h0, double* f) {
  int Q = orc_Q(P);
  long nc = (long)P->nx * P->ny;
  double feq[9];
  for (int i = 0; i < P->n; ++i)
    for (long c = 0; c < nc; ++c) {
      orc_equilibrium(P, h0[i * nc + c], 0.0, 0.0, feq);
      for (int k = 0; k < Q; ++k) f[((long)i * Q + k) * nc + c] = feq[k];
    }
}

void orc_moments(const orc_params* P, const double* f, double* h, double* Jx,
                 double* Jy) {
  int cx[9], cy[9];
  double w[9];
  orc_lattice(P, cx, cy, w);
  int Q = orc_Q(P);
  long nc = (long)P->nx * P->ny;
  for (int i = 0; i < P->n; ++i)
#pragma omp parallel for schedule(static)
    for (long c = 0; c < nc; ++c) {
      double s = 0.0, sx = 0.0, sy = 0.0;
      for (int k = 0; k < Q; ++k) {
        double v = f[((long)i * Q + k) * nc + c];
        s += v;
        sx += cx[k] * v;
        sy += cy[k] * v;
      }
      h[i * nc + c] = s;
      if (Jx) Jx[i * nc + c] = sx;
      if (Jy) Jy[i * nc + c] = sy;
    }
}

static const double ORC_PI = 3.14159265358979323846;

double orc_substrate(const orc_params* P, long x, long y) {
  if (P->sub_amp == 0.0) return 0.0;
  /* phase / (2 pi) = kx x / nx + ky y / ny, reduced exactly in integers */
  long nx = P->nx, ny = P->ny, nc = nx * ny;
  long m = (((long)P->sub_kx * x) % nx * ny + ((long)P->sub_ky * y) % ny * nx) % nc;
  if (m < 0) m += nc;
  return P->sub_amp * cos(2.0 * ORC_PI * (double)m / (double)nc);
}

static long wrap(long a, long m) {
  long r = a % m;
  return r < 0 ? r + m : r;
}

/* ------------------------------------------------------------------ */
/* one time step                                                       */
/* ------------------------------------------------------------------ */
int orc_step(const orc_params* P, const double* fin, double* fout) {
  const int n = P->n, Q = orc_Q(P);
  const long nx = P->nx, ny = P->ny, nc = nx * ny;
  int cx[9], cy[9];
  double w[9];
  orc_lattice(P, cx, cy, w);

  double* h = malloc(sizeof(double) * n * nc);
  double* Jx = malloc(sizeof(double) * n * nc);
  double* Jy = malloc(sizeof(double) * n * nc);
  double* z = malloc(sizeof(double) * n * nc);
  double* gzx = malloc(sizeof(double) * n * nc);
  double* gzy = malloc(sizeof(double) * n * nc);
  double* lz = malloc(sizeof(double) * n * nc);
  double* p = malloc(sizeof(double) * n * nc);
  double* z0 = malloc(sizeof(double) * nc);
  double* g0 = malloc(sizeof(double) * nc);
  if (!h || !Jx || !Jy || !z || !gzx || !gzy || !lz || !p || !z0 || !g0) {
    free(h); free(Jx); free(Jy); free(z); free(gzx); free(gzy); free(lz); free(p);
    free(z0); free(g0);
    return -1;
  }
  int status = 0;

  /* 1. moments */
  orc_moments(P, fin, h, Jx, Jy);

  /* Every cell of each stage below reads time-t fields and writes only its
     own entries, so the cells are split across OpenMP threads; the
     arithmetic and its order per cell do not depend on the thread count. */

  /* 2. substrate z_0 with its squared lattice gradient (R5), interface
     heights z_i = z_0 + sum_{j<=i} h_j */
#pragma omp parallel for schedule(static)
  for (long c = 0; c < nc; ++c) z0[c] = orc_substrate(P, c % nx, c / nx);
#pragma omp parallel for schedule(static)
  for (long c = 0; c < nc; ++c) {
    long x = c % nx, y = c / nx;
    double sx = 0.0, sy = 0.0;
    for (int k = 1; k < Q; ++k) {
      long nb = wrap(y + cy[k], ny) * nx + wrap(x + cx[k], nx);
      sx += w[k] * cx[k] * (z0[nb] - z0[c]);
      sy += w[k] * cy[k] * (z0[nb] - z0[c]);
    }
    g0[c] = (sx / CS2) * (sx / CS2) + (sy / CS2) * (sy / CS2);
  }
#pragma omp parallel for schedule(static)
  for (long c = 0; c < nc; ++c) {
    double acc = z0[c];
    for (int i = 0; i < n; ++i) {
      acc += h[i * nc + c];
      z[i * nc + c] = acc;
    }
  }

  /* 3. grad z, lap z (R5) */
  for (int i = 0; i < n; ++i)
#pragma omp parallel for schedule(static)
    for (long y = 0; y < ny; ++y)
      for (long x = 0; x < nx; ++x) {
        long c = y * nx + x;
        double z0 = z[i * nc + c], sx = 0.0, sy = 0.0, sl = 0.0;
        for (int k = 1; k < Q; ++k) {
          long nb = wrap(y + cy[k], ny) * nx + wrap(x + cx[k], nx);
          double d = z[i * nc + nb] - z0;
          sx += w[k] * cx[k] * d;
          sy += w[k] * cy[k] * d;
          sl += w[k] * d;
        }
        gzx[i * nc + c] = sx / CS2;
        gzy[i * nc + c] = sy / CS2;
        lz[i * nc + c] = 2.0 * sl / CS2;
      }

  /* 4. pressures */
#pragma omp parallel for schedule(static)
  for (long c = 0; c < nc; ++c) {
    double hc[ORC_MAXN], gx[ORC_MAXN], gy[ORC_MAXN], lc[ORC_MAXN];
    double La[ORC_MAXN], Pc[ORC_MAXN], pc[ORC_MAXN];
    for (int i = 0; i < n; ++i) {
      hc[i] = h[i * nc + c];
      gx[i] = gzx[i * nc + c];
      gy[i] = gzy[i * nc + c];
      lc[i] = lz[i * nc + c];
    }
    orc_pressures_sub(P, hc, gx, gy, lc, g0[c], La, Pc, pc);
    for (int i = 0; i < n; ++i) p[i * nc + c] = pc[i];
  }

  /* 5-9. grad p, friction, force, collision, streaming (each source cell
     writes its own nine destinations) */
#pragma omp parallel for schedule(static) reduction(min : status)
  for (long y = 0; y < ny; ++y)
    for (long x = 0; x < nx; ++x) {
      long c = y * nx + x;
      double hc[ORC_MAXN], jx[ORC_MAXN], jy[ORC_MAXN], Rx[ORC_MAXN],
          Ry[ORC_MAXN];
      for (int i = 0; i < n; ++i) {
        hc[i] = h[i * nc + c];
        jx[i] = Jx[i * nc + c];
        jy[i] = Jy[i * nc + c];
      }
      if (orc_friction(P, hc, jx, jy, Rx, Ry) != 0) status = -1;
      for (int i = 0; i < n; ++i) {
        /* 5. grad p_i (R5) */
        double p0 = p[i * nc + c], gpx = 0.0, gpy = 0.0;
        for (int k = 1; k < Q; ++k) {
          long nb = wrap(y + cy[k], ny) * nx + wrap(x + cx[k], nx);
          double d = p[i * nc + nb] - p0;
          gpx += w[k] * cx[k] * d;
          gpy += w[k] * cy[k] * d;
        }
        gpx /= CS2;
        gpy /= CS2;
        /* 7. Eq. (force) */
        double Fx = -hc[i] * gpx + Rx[i];
        double Fy = -hc[i] * gpy + Ry[i];
        /* 8. Eq. (BGK) with Eq. (equilibrium_distribution) */
        double Ux = jx[i] / hc[i], Uy = jy[i] / hc[i];
        double feq[9];
        orc_equilibrium(P, hc[i], Ux, Uy, feq);
        for (int k = 0; k < Q; ++k) {
          double fk = fin[((long)i * Q + k) * nc + c];
          double fstar = fk - (fk - feq[k]) / P->tau +
                         w[k] * (cx[k] * Fx + cy[k] * Fy) / CS2;
          /* 9. streaming to x + c_k */
          long dst = wrap(y + cy[k], ny) * nx + wrap(x + cx[k], nx);
          fout[((long)i * Q + k) * nc + dst] = fstar;
        }
      }
    }

  free(h); free(Jx); free(Jy); free(z); free(gzx); free(gzy); free(lz); free(p);
  free(z0); free(g0);
  return status;
}

int orc_run(const orc_params* P, double* f, long nsteps) {
  long len = (long)P->n * orc_Q(P) * P->nx * P->ny;
  double* g = malloc(sizeof(double) * len);
  if (!g) return -1;
  int status = 0;
  for (long s = 0; s < nsteps; ++s) {
    if (orc_step(P, f, g) != 0) status = -1;
    memcpy(f, g, sizeof(double) * len);
  }
  free(g);
  return status;
}

/* ------------------------------------------------------------------ */
/* threads of the cell loops (OpenMP; 1 when built without it)         */
/* ------------------------------------------------------------------ */
#ifdef _OPENMP
#include <omp.h>
void orc_set_threads(int n) { omp_set_num_threads(n > 0 ? n : 1); }
int orc_max_threads(void) { return omp_get_max_threads(); }
#else
void orc_set_threads(int n) { (void)n; }
int orc_max_threads(void) { return 1; }
#endif
