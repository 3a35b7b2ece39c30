/*
 * oracle.h -- plain FP64 CPU oracle of the multilayer shallow-water lattice
 * Boltzmann step for the n-layer thin-film equation (Richter, Malgaretti &
 * Harting, "Modeling of thin liquid films with arbitrary many layers").
 *
 * TEST INFRASTRUCTURE ONLY. This library is the independent checker of the
 * CUDA path. Only the tests, the smoke check and the CPU-baseline leg of the
 * benchmark may load it; the product library never does. It shares no code,
 * header, table or helper with the CUDA path.
 *
 * Everything here is written out step by step from the paper in double
 * precision, with dense linear algebra and no blocking or fusion:
 *   - wetting potential            : Eq. (wetting_potential)
 *   - spreading coefficients       : Eq. (spreading_parameters)
 *   - Laplace / disjoining pressure: Eqs. (Laplace_pressure),
 *                                    (disjoining_pressure), p_i - p_atm sum
 *   - friction force via D, S      : Eqs. (u_ansatz)-(friction_force)
 *   - equilibrium, BGK, force      : Eqs. (equilibrium_distribution), (BGK),
 *                                    (force)
 * Readings of garbled or silent passages are listed in oracle.c next to the
 * code they affect.
 *
 * Layout of distributions: f[((i * Q + k) * ny + y) * nx + x], layer i,
 * direction k (paper's order), row-major cell (x fastest). Heights: h[(i *
 * ny + y) * nx + x]. All grids are periodic.
 */
#ifndef MLSW_ORACLE_H
#define MLSW_ORACLE_H

#ifdef __cplusplus
extern "C" {
#endif

#define ORC_MAXN 8

typedef struct {
  int n;        /* number of liquid layers (1..ORC_MAXN)                     */
  int lattice;  /* 1 = D1Q3 (ny must be 1), 2 = D2Q9                        */
  int nx, ny;   /* periodic lattice size                                    */
  double tau;   /* BGK relaxation time                                      */
  double gamma[ORC_MAXN];        /* gamma[i-1] = gamma_{i,i+1}, i = 1..n     */
  double S[ORC_MAXN][ORC_MAXN];  /* S[i][k-1] = S_{ik}, i = 0..n-1, k<=n-i   */
  double mu[ORC_MAXN];           /* mu[i-1] = mu_i                          */
  double beta[ORC_MAXN];         /* beta[i-1] = beta_i                      */
  int nw, mw;                    /* wetting exponents, nw > mw              */
  double hstar;                  /* precursor thickness h*                  */
  /* substrate z_0(x, y) = sub_amp cos(2 pi (sub_kx x / nx + sub_ky y / ny));
     sub_amp = 0 is the flat substrate of the paper's runs */
  double sub_amp;
  int sub_kx, sub_ky;
  /* wetting potential: 0 = the power law of Eq. (wetting_potential) with
     exponents (nw, mw); 1 = the exponential decay the paper quotes for
     charged surfaces, phi_k(d) = 2 e^{-kappa (d - k h*)} - e^{-2 kappa (d - k h*)},
     with the same limits phi_k(k h*) = 1, phi_k'(k h*) = 0, phi_k -> 0 */
  int wet_kind;
  double kappa;
} orc_params;

/* wetting potential phi_k(h) and its derivative, Eq. (wetting_potential) */
double orc_phi(const orc_params* P, int k, double h);
double orc_dphi(const orc_params* P, int k, double h);

/* S_{ik} from the full tension table g[(a)*(n+2)+b] = gamma_{a,b},
 * a,b = 0..n+1 (0 = substrate, n+1 = gas). Also copies gamma_{i,i+1}. */
void orc_spreading_from_tensions(orc_params* P, const double* g);

/* lattice tables */
int orc_Q(const orc_params* P);
void orc_lattice(const orc_params* P, int* cx, int* cy, double* w);

/* substrate height z_0 at cell (x, y) */
double orc_substrate(const orc_params* P, long x, long y);

/* the 3n x 3n boundary-condition matrix D at one cell (row-major) */
void orc_build_D(const orc_params* P, const double* h, double* D);

/* friction force 2 mu_i h_i a_i for both flux components at one cell.
 * h[n], Jx[n], Jy[n] in; Rx[n], Ry[n] out. Returns 0, or -1 if D is
 * singular. */
int orc_friction(const orc_params* P, const double* h, const double* Jx,
                 const double* Jy, double* Rx, double* Ry);

/* pressure jumps and layer pressures at one cell from the interface data:
 * h[n]; gzx[n], gzy[n] = grad z_i; lz[n] = lap z_i (index i-1).
 * Lambda[n], Pi[n], p[n] out (p = p_i - p_atm). */
void orc_pressures(const orc_params* P, const double* h, const double* gzx,
                   const double* gzy, const double* lz, double* Lambda,
                   double* Pi, double* p);

/* the same on a corrugated substrate: g0sq = |grad z_0|^2 at the cell
 * (orc_pressures is this with g0sq = 0) */
void orc_pressures_sub(const orc_params* P, const double* h, const double* gzx,
                       const double* gzy, const double* lz, double g0sq,
                       double* Lambda, double* Pi, double* p);

/* equilibrium populations of one layer at one cell, Eq. (equilibrium_distribution) */
void orc_equilibrium(const orc_params* P, double h, double Ux, double Uy,
                     double* feq);

/* f = f_eq(h0, U = 0) on the whole grid */
void orc_init(const orc_params* P, const double* h0, double* f);

/* moments h_i, J_i on the whole grid (Jy may be NULL for D1Q3) */
void orc_moments(const orc_params* P, const double* f, double* h, double* Jx,
                 double* Jy);

/* one full time step fin -> fout (distinct buffers). Returns 0 or -1. */
int orc_step(const orc_params* P, const double* fin, double* fout);

/* nsteps steps in place on f (uses an internal second buffer) */
int orc_run(const orc_params* P, double* f, long nsteps);

/* Threads of the per-cell loops (OpenMP): the results do not depend on
   the count. orc_max_threads() is the count in use, 1 without OpenMP. */
void orc_set_threads(int n);
int orc_max_threads(void);

#ifdef __cplusplus
}
#endif
#endif
