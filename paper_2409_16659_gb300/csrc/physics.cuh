// physics.cuh -- per-cell device routines of the multilayer shallow-water
// LBM step (FP32): lattice tables, layer pressures, friction coupling,
// equilibrium/collision. Used by the step kernels and by
// mlswlbm_friction_eval.
#pragma once

#include <cuda_runtime.h>

namespace mlsw {

constexpr int kMaxLayers = 5;

// ---------------------------------------------------------------------------
// Bounds-checked build (compiled with -DMLSW_DEBUG). Index helpers check
// every padded-layout index, shared-memory access and global store of the
// step kernels; an access out of range is counted and redirected to a
// harmless cell (index 0 of a population buffer is the padding cell
// x = -4 of the first row, which no real cell reads) instead of faulting.
// Each translation unit keeps its own counter; the host reads and clears
// them through mlswlbm_debug_bounds_violations. Release builds compile
// none of this.
// ---------------------------------------------------------------------------
#ifdef MLSW_DEBUG
static __device__ unsigned int g_bounds_violations;
__device__ __forceinline__ void note_bounds_violation() { atomicAdd(&g_bounds_violations, 1u); }
#define MLSW_DEFINE_BOUNDS_READER(fn)                                                  \
  unsigned fn() {                                                                      \
    unsigned v = 0, z = 0;                                                             \
    if (cudaMemcpyFromSymbol(&v, g_bounds_violations, sizeof v) != cudaSuccess) return ~0u; \
    if (cudaMemcpyToSymbol(g_bounds_violations, &z, sizeof z) != cudaSuccess) return ~0u;   \
    return v;                                                                          \
  }
#else
#define MLSW_DEFINE_BOUNDS_READER(fn) \
  unsigned fn() { return 0; }
#endif

// Kernel-side copy of the problem statement, rounded to FP32 once.
//
// Shifted rest population: the device stores g_0 = f_0 - H_i for the rest
// population of layer i (H_i a per-layer constant near the film thickness)
// and g_k = f_k otherwise. Moments are then formed as deviations
// dh_i = sum_k g_k (h_i = H_i + dh_i), so the interface stencils work on
// O(1e-3) numbers instead of O(1) ones. In FP32 the long-wave curvature of
// an O(1) height field is comparable to its rounding (ulp(1) = 1.2e-7), so
// storing f_0 itself loses the capillary signal; the shift keeps ~1e-10.
// The arithmetic of the scheme is unchanged: only the representation of
// f_0 moves by a constant.
// Device layout of a population buffer: every plane (layer i, direction k,
// plane index i * Q + k) is a padded 2-D array of `rows` rows of `pitch`
// floats; the real cell (x, y) sits at row y + gy, column x + gx. The ring
// of ghost cells within two cells of the real domain (x in [-2, nx + 2),
// y in [-2, ny + 2) for D2Q9; x only for D1Q3) holds the periodic images of
// the real cells, so the step kernels read a tile plus its halo without
// any wrap-around arithmetic. gx = 4 keeps every tile's box 16-byte aligned
// for the tensor-memory-access unit; pitch and rows cover whole tiles.
struct Layout {
  int nx, ny;    // real lattice
  int gx, gy;    // padded position of the real cell (0, 0)
  int pitch;     // floats per padded row (multiple of 4)
  int rows;      // padded rows per plane
  long plane;    // pitch * rows
  int nplanes;   // planes of a buffer (0: not known, planes are then not checked)
  __host__ __device__ long at(int p, int x, int y) const {
#if defined(MLSW_DEBUG) && defined(__CUDA_ARCH__)
    if (x + gx < 0 || x + gx >= pitch || y + gy < 0 || y + gy >= rows || p < 0 ||
        (nplanes > 0 && p >= nplanes)) {
      note_bounds_violation();
      return 0;
    }
#endif
    return (long)p * plane + (long)(y + gy) * pitch + (x + gx);
  }
  // floats of one buffer (0 when the plane count is not known)
  __host__ __device__ long length() const { return (long)nplanes * plane; }
};

struct KParams {
  int n;
  int nx, ny;
  float omega;                       // 1 / tau
  float gamma[kMaxLayers];           // gamma_{i,i+1}
  float S[kMaxLayers][kMaxLayers];   // S[l][k-1] = S_{lk}
  float mu_inv[kMaxLayers];          // 1 / mu_i
  float beta[kMaxLayers];            // beta_i
  float hstar;
  int nw, mw;
  float c_phi;                       // 1 / (nw - mw)
  float c_dphi;                      // nw mw / (nw - mw)
  float H[kMaxLayers];               // rest-population shift of each layer
  // Hsum[l][m] = H_{l+1} + ... + H_m (1-based layers, 0 <= l < m <= n): the
  // reference part of the thickness z_m - z_l between interfaces l and m
  float Hsum[kMaxLayers + 1][kMaxLayers + 1];
  Layout L;                          // padded layout of both population buffers
  // periodic images: ghost column gcol[g] (g = 0..3 for x = -2, -1, nx,
  // nx + 1) holds real column gsrcx[g]; likewise rows
  int gsrcx[4], gsrcy[4];
  // 1 when a side of the lattice is shorter than 4 cells: a real column or
  // row can then have several ghost images
  int tiny;
  // substrate z_0(x, y) = sub_amp cos(2 pi (sub_kx x / nx + sub_ky y / ny));
  // sub_amp = 0 is the flat substrate
  float sub_amp;
  int sub_kx, sub_ky;
  // wetting potential: 0 the power law (nw, mw), 1 the charged-surface form
  // phi_k(d) = 2 a - a^2, a = e^{-kappa (d - k h*)}
  int wet_kind;
  float kappa;
  // L2 cache policy of the D2Q9 step (see d2q9_tile_loop): kL2None,
  // kL2Stream or kL2Resident
  int l2_policy;
};

// kL2None: no cache hints (batches, whose many lattices stream through);
// kL2Stream: a lattice larger than the L2, output kept as long as possible;
// kL2Resident: one population buffer fits in the L2 and stays there.
enum L2Policy { kL2None = 0, kL2Stream = 1, kL2Resident = 2 };

// Substrate height at lattice cell (x, y) (any integers: the cosine is
// periodic); the phase is reduced exactly in integers.
__device__ __forceinline__ float substrate_at(const KParams& P, int x, int y) {
  const long nx = P.nx, ny = P.ny, nc = nx * ny;
  long m = ((long)P.sub_kx * x % nx) * ny + ((long)P.sub_ky * y % ny) * nx;
  m %= nc;
  if (m < 0) m += nc;
  float s, c;
  sincospif(2.f * (float)((double)m / (double)nc), &s, &c);
  return P.sub_amp * c;
}

// ---------------------------------------------------------------------------
// lattices (section LBM): c_0 = 0, then the paper's order
// ---------------------------------------------------------------------------
template <int LAT> struct Lattice;

template <> struct Lattice<1> {  // D1Q3
  static constexpr int Q = 3;
  __host__ __device__ static constexpr int cx(int k) { return k == 1 ? 1 : (k == 2 ? -1 : 0); }
  __host__ __device__ static constexpr int cy(int) { return 0; }
  __host__ __device__ static constexpr float w(int k) { return k == 0 ? 2.f / 3.f : 1.f / 6.f; }
};

template <> struct Lattice<2> {  // D2Q9, counter-clockwise from +x
  static constexpr int Q = 9;
  __host__ __device__ static constexpr int cx(int k) {
    return (k == 1 || k == 2 || k == 8) ? 1 : ((k == 4 || k == 5 || k == 6) ? -1 : 0);
  }
  __host__ __device__ static constexpr int cy(int k) {
    return (k == 2 || k == 3 || k == 4) ? 1 : ((k == 6 || k == 7 || k == 8) ? -1 : 0);
  }
  __host__ __device__ static constexpr float w(int k) {
    return k == 0 ? 4.f / 9.f : ((k & 1) ? 1.f / 9.f : 1.f / 36.f);
  }
};

// ---------------------------------------------------------------------------
// Arithmetic on one cell (float) or on two cells at once (f2, a packed pair
// evaluated with the FP32x2 instructions of sm_100-class GPUs: one FFMA2 /
// FADD2 / FMUL2 does the work of two scalar ones). The per-cell routines
// below are written once over T in {float, f2}.
// ---------------------------------------------------------------------------
struct f2 {
  float2 v;
};
__device__ __forceinline__ f2 mk2(float a, float b) { return {make_float2(a, b)}; }
__device__ __forceinline__ f2 operator+(f2 a, f2 b) { return {__fadd2_rn(a.v, b.v)}; }
__device__ __forceinline__ f2 operator*(f2 a, f2 b) { return {__fmul2_rn(a.v, b.v)}; }
// a - b as one FFMA2: b * (-1) + a (exact product, one rounding)
__device__ __forceinline__ f2 operator-(f2 a, f2 b) {
  return {__ffma2_rn(b.v, make_float2(-1.f, -1.f), a.v)};
}
__device__ __forceinline__ f2 operator-(f2 a) { return {make_float2(-a.v.x, -a.v.y)}; }
__device__ __forceinline__ f2 operator+(f2 a, float b) { return a + mk2(b, b); }
__device__ __forceinline__ f2 operator+(float a, f2 b) { return mk2(a, a) + b; }
__device__ __forceinline__ f2 operator-(f2 a, float b) { return a - mk2(b, b); }
__device__ __forceinline__ f2 operator-(float a, f2 b) { return mk2(a, a) - b; }
__device__ __forceinline__ f2 operator*(f2 a, float b) { return a * mk2(b, b); }
__device__ __forceinline__ f2 operator*(float a, f2 b) { return mk2(a, a) * b; }
__device__ __forceinline__ f2& operator+=(f2& a, f2 b) { return a = a + b; }
__device__ __forceinline__ f2& operator-=(f2& a, f2 b) { return a = a - b; }

template <class T> struct Num;
template <> struct Num<float> {
  __device__ static float splat(float a) { return a; }
};
template <> struct Num<f2> {
  __device__ static f2 splat(float a) { return mk2(a, a); }
};

__device__ __forceinline__ float fmav(float a, float b, float c) { return fmaf(a, b, c); }
__device__ __forceinline__ f2 fmav(f2 a, f2 b, f2 c) { return {__ffma2_rn(a.v, b.v, c.v)}; }
__device__ __forceinline__ f2 fmav(f2 a, float b, f2 c) { return fmav(a, mk2(b, b), c); }
__device__ __forceinline__ f2 fmav(float a, f2 b, f2 c) { return fmav(mk2(a, a), b, c); }
__device__ __forceinline__ f2 fmav(f2 a, f2 b, float c) { return fmav(a, b, mk2(c, c)); }
__device__ __forceinline__ f2 fmav(f2 a, float b, float c) { return fmav(a, mk2(b, b), mk2(c, c)); }

// fast reciprocal: the __fdividef intrinsic (at most 2 ulp for the O(1e-2 ..
// 1e2) arguments used here: layer thicknesses, friction pivots)
__device__ __forceinline__ float rcp(float x) { return __fdividef(1.f, x); }
__device__ __forceinline__ f2 rcp(f2 x) { return mk2(rcp(x.v.x), rcp(x.v.y)); }
__device__ __forceinline__ float expv(float x) { return expf(x); }
__device__ __forceinline__ f2 expv(f2 x) { return mk2(expf(x.v.x), expf(x.v.y)); }

template <class T>
__device__ __forceinline__ T ipow(T r, int e) {
  T a = Num<T>::splat(1.f);
  for (int i = 0; i < e; ++i) a = a * r;
  return a;
}

// r^mw and r^nw: the common exponent pair (3, 2) at compile time (W32), any
// other pair with a run-time loop
template <bool W32, class T>
__device__ __forceinline__ void wet_powers(const KParams& P, T r, T& rm, T& rn) {
  if (W32) {
    rm = r * r;
    rn = rm * r;
  } else {
    rm = ipow(r, P.mw);
    rn = ipow(r, P.nw);
  }
}

// ---------------------------------------------------------------------------
// Layer pressures p_i - p_atm at one cell (Eqs. Laplace_pressure,
// disjoining_pressure; p_i = sum_{j>=i} (Lambda_j + Pi_j)).
// Every interface pair (l, m = l + k), 0 <= l < m <= N, enters once with
// the thickness d = z_m - z_l between them: E = S_lk phi'_k(d)
// (1 + |grad z_l|^2 / 2) is subtracted from Pi_l and added to Pi_m, and
// S_lk phi_k(d) raises the tension of interface l. l = 0 is the substrate
// (height z0, slope factor sg0; no pressure of its own).
// The inputs are the deviations of the interface heights, zd[i - 1] =
// z_i - (H_1 + ... + H_i), so d = Hsum[l][m] + (zd_m - zd_l) (zd_0 = 0): the
// deviations are O(1e-3) numbers and their differences carry the FP32
// round-off of the deviations, not of the O(1) heights.
// ---------------------------------------------------------------------------
// NN: only nearest-neighbour pairs (k = 1) carry a spreading coefficient
// (S_{lk} = 0 for k >= 2, as in the paper's three-layer runs); the pair loop
// is then branch-free.
// z0, sg0: the substrate height z_0 (on the scale of zd) and 1 + |grad z_0|^2 / 2
// at the cell; 0 and 1 for the flat substrate.
template <int N, bool W32, class T, bool NN = false>
__device__ __forceinline__ void layer_pressures_dev(const KParams& P, const T (&zd)[N],
                                                    const T (&gx)[N], const T (&gy)[N],
                                                    const T (&lz)[N], T (&p)[N],
                                                    T z0 = Num<T>::splat(0.f),
                                                    T sg0 = Num<T>::splat(1.f)) {
  T ten[N], pi[N], sg[N];
#pragma unroll
  for (int i = 0; i < N; ++i) {
    ten[i] = Num<T>::splat(P.gamma[i]);
    pi[i] = Num<T>::splat(0.f);
    sg[i] = fmav(0.5f, fmav(gx[i], gx[i], gy[i] * gy[i]), Num<T>::splat(1.f));
  }
#pragma unroll
  for (int l = 0; l < N; ++l) {
    const T sgl = (l == 0) ? sg0 : sg[l > 0 ? l - 1 : 0];
    const T zl = (l == 0) ? z0 : zd[l > 0 ? l - 1 : 0];
#pragma unroll
    for (int m = l + 1; m <= (NN ? l + 1 : N); ++m) {
      const int k = m - l;
      const float s = P.S[l][k - 1];
      if (NN || s != 0.f) {
        const T d = (zd[m - 1] - zl) + P.Hsum[l][m];
        T phi, dphi;
        if (!W32 && P.wet_kind == 1) {
          // charged surfaces: a = e^{-kappa (d - k h*)}, phi = 2 a - a^2,
          // phi' = 2 kappa a (a - 1)
          const T a = expv(fmav(d, -P.kappa, P.kappa * ((float)k * P.hstar)));
          phi = a * (2.f - a);
          dphi = (2.f * P.kappa) * (a * (a - 1.f));
        } else {
          const T inv_d = rcp(d);
          const T r = ((float)k * P.hstar) * inv_d;
          T rm, rn;
          wet_powers<W32>(P, r, rm, rn);
          phi = W32 ? fmav(rm, 3.f, -2.f * rn)
                    : (fmav(rm, (float)P.nw, -(float)P.mw * rn)) * P.c_phi;
          dphi = (P.c_dphi * (rn - rm)) * inv_d;
        }
        const T se = s * dphi;
        // explicit fused updates, so one cell and a packed pair of cells
        // round identically
        if (l >= 1) {
          ten[l > 0 ? l - 1 : 0] = fmav(s, phi, ten[l > 0 ? l - 1 : 0]);
          pi[l > 0 ? l - 1 : 0] = fmav(-se, sgl, pi[l > 0 ? l - 1 : 0]);
        }
        pi[m - 1] = fmav(se, sgl, pi[m - 1]);
      }
    }
  }
  T acc = Num<T>::splat(0.f);
#pragma unroll
  for (int i = N - 1; i >= 0; --i) {
    acc = acc + fmav(-ten[i], lz[i], pi[i]);
    p[i] = acc;
  }
}

// ---------------------------------------------------------------------------
// Friction 2 mu_i h_i a_i (Eq. friction_force) by shear-stress integration.
//
// In Stokes layers with pressure gradient G_i, mu_i u'' = G_i. Integrating
// the stress down from the stress-free top (Eq. viscous_boundary with
// mu_{n+1} = 0) gives, in layer i, sigma(z) = G_i (z - z_i) - sum_{j>i} h_j G_j.
// Integrating u = sigma / mu_i upward from the substrate, the slip condition
// of Eq. (no_slip) -- the parabola of layer i continued a distance beta_i
// below z_{i-1} meets u_{i-1}(z_{i-1}) -- adds the jump
// (beta_i / mu_i) sigma_i(z_{i-1} - beta_i / 2). Integrating u over each
// layer (Eq. flux) gives J = L G with an N x N matrix L built column by
// column in O(N^2). Force balance of the thin-sheet equation,
// 0 = -h_i G_i + 2 mu_i h_i a_i, then gives the friction R_i = h_i G_i with
// G = L^-1 J: one factorisation, two right-hand sides (x and y), by the
// adjugate for N <= 3 and by elimination with row pivoting for N = 4, 5 (L is
// not symmetric in general: the slip convention breaks reciprocity; the
// pivoted form is scalar only).
// ---------------------------------------------------------------------------
// Solves L G = J for two right-hand sides with the adjugate of L
// (N = 1, 2, 3). Unused for larger N.
template <int N, class T>
__device__ __forceinline__ void solve_small(const T (&L)[N][N], const T (&Jx)[N],
                                            const T (&Jy)[N], T (&Gx)[N], T (&Gy)[N]) {
  if constexpr (N == 1) {
    const T r = rcp(L[0][0]);
    Gx[0] = Jx[0] * r;
    Gy[0] = Jy[0] * r;
  } else if constexpr (N == 2) {
    const T r = rcp(fmav(L[0][0], L[1][1], -(L[0][1] * L[1][0])));
    Gx[0] = fmav(L[1][1], Jx[0], -(L[0][1] * Jx[1])) * r;
    Gx[1] = fmav(L[0][0], Jx[1], -(L[1][0] * Jx[0])) * r;
    Gy[0] = fmav(L[1][1], Jy[0], -(L[0][1] * Jy[1])) * r;
    Gy[1] = fmav(L[0][0], Jy[1], -(L[1][0] * Jy[0])) * r;
  } else if constexpr (N == 3) {
    const T a = L[0][0], b = L[0][1], c = L[0][2];
    const T d = L[1][0], e = L[1][1], f = L[1][2];
    const T g = L[2][0], hh = L[2][1], k = L[2][2];
    const T A00 = fmav(e, k, -(f * hh)), A01 = fmav(c, hh, -(b * k)), A02 = fmav(b, f, -(c * e));
    const T A10 = fmav(f, g, -(d * k)), A11 = fmav(a, k, -(c * g)), A12 = fmav(c, d, -(a * f));
    const T A20 = fmav(d, hh, -(e * g)), A21 = fmav(b, g, -(a * hh)), A22 = fmav(a, e, -(b * d));
    const T r = rcp(fmav(a, A00, fmav(b, A10, c * A20)));
    Gx[0] = fmav(A00, Jx[0], fmav(A01, Jx[1], A02 * Jx[2])) * r;
    Gx[1] = fmav(A10, Jx[0], fmav(A11, Jx[1], A12 * Jx[2])) * r;
    Gx[2] = fmav(A20, Jx[0], fmav(A21, Jx[1], A22 * Jx[2])) * r;
    Gy[0] = fmav(A00, Jy[0], fmav(A01, Jy[1], A02 * Jy[2])) * r;
    Gy[1] = fmav(A10, Jy[0], fmav(A11, Jy[1], A12 * Jy[2])) * r;
    Gy[2] = fmav(A20, Jy[0], fmav(A21, Jy[1], A22 * Jy[2])) * r;
  }
}

template <int N, class T>
__device__ __forceinline__ void friction(const KParams& P, const T (&h)[N], const T (&Jx)[N],
                                         const T (&Jy)[N], T (&Rx)[N], T (&Ry)[N]) {
  T L[N][N];
#pragma unroll
  for (int j = 0; j < N; ++j) {
    T ub = Num<T>::splat(0.f);  // velocity at the bottom of layer i for unit G_j
#pragma unroll
    for (int i = 0; i < N; ++i) {
      const float mi = P.mu_inv[i], bi = P.beta[i];
      const T hi = h[i];
      if (j > i) {
        // unit gradient in a layer above: only the stress s = -h_j acts
        const T s = -h[j];
        ub = fmav(s, bi * mi, ub);
        L[i][j] = fmav(hi, ub, (mi * 0.5f) * (hi * hi) * s);
        ub = fmav(mi * hi, s, ub);
      } else if (j == i) {
        // unit gradient in this layer (g = 1, s = 0)
        ub = fmav(-(bi * mi), hi + 0.5f * bi, ub);
        L[i][j] = fmav(hi, ub, (-mi / 3.f) * (hi * hi) * hi);
        ub = fmav(-0.5f * mi, hi * hi, ub);
      } else {
        L[i][j] = hi * ub;  // layers above the forced one move with it
      }
    }
  }
  if constexpr (N <= 3) {
    // adjugate (Cramer) solution of the 1x1 / 2x2 / 3x3 system
    T Gx[N], Gy[N];
    solve_small<N>(L, Jx, Jy, Gx, Gy);
#pragma unroll
    for (int i = 0; i < N; ++i) {
      Rx[i] = h[i] * Gx[i];
      Ry[i] = h[i] * Gy[i];
    }
    return;
  } else {
    static_assert(sizeof(T) == sizeof(float), "pivoted elimination is scalar");
    float bx[N], by[N];
#pragma unroll
    for (int i = 0; i < N; ++i) {
      bx[i] = Jx[i];
      by[i] = Jy[i];
    }
    float inv_piv[N];
#pragma unroll
    for (int c = 0; c < N; ++c) {
      int piv = c;
      float best = fabsf(L[c][c]);
#pragma unroll
      for (int r = c + 1; r < N; ++r) {
        const float a = fabsf(L[r][c]);
        if (a > best) {
          best = a;
          piv = r;
        }
      }
      // the row exchange as selects on fixed indices, so that the system
      // stays in registers
#pragma unroll
      for (int r = c + 1; r < N; ++r) {
        const bool sw = (piv == r);
#pragma unroll
        for (int q = c; q < N; ++q) {
          const float a = L[c][q], b = L[r][q];
          L[c][q] = sw ? b : a;
          L[r][q] = sw ? a : b;
        }
        const float ax = bx[c], bxr = bx[r], ay = by[c], byr = by[r];
        bx[c] = sw ? bxr : ax;
        bx[r] = sw ? ax : bxr;
        by[c] = sw ? byr : ay;
        by[r] = sw ? ay : byr;
      }
      inv_piv[c] = rcp(L[c][c]);
#pragma unroll
      for (int r = c + 1; r < N; ++r) {
        const float l = L[r][c] * inv_piv[c];
#pragma unroll
        for (int q = c + 1; q < N; ++q) L[r][q] -= l * L[c][q];
        bx[r] -= l * bx[c];
        by[r] -= l * by[c];
      }
    }
#pragma unroll
    for (int c = N - 1; c >= 0; --c) {
      float sx = bx[c], sy = by[c];
#pragma unroll
      for (int q = c + 1; q < N; ++q) {
        sx -= L[c][q] * bx[q];
        sy -= L[c][q] * by[q];
      }
      bx[c] = sx * inv_piv[c];
      by[c] = sy * inv_piv[c];
    }
#pragma unroll
    for (int i = 0; i < N; ++i) {
      Rx[i] = h[i] * bx[i];
      Ry[i] = h[i] * by[i];
    }
  }
}

}  // namespace mlsw
