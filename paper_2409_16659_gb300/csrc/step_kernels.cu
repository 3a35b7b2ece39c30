// step_kernels.cu -- the fused multilayer shallow-water LBM time step.
//
// One launch = one time step over the whole periodic lattice. Each CTA owns
// a tile of cells and, in one pass over the populations of its tile plus a
// two-cell halo:
//   A. loads f (post-streaming state of time t, rest population stored
//      shifted by H_i, see physics.cuh), forms h_i (tile + halo) and J_i
//      (tile) -- section LBM moments;
//   B. on tile + 1 ring: interfaces z_i, their lattice gradient and
//      Laplacian, and the layer pressures p_i (Eqs. Laplace_pressure,
//      disjoining_pressure);
//   C. on the tile: grad p_i, friction (Eq. friction_force), force
//      (Eq. force), equilibrium (Eq. equilibrium_distribution), BGK with
//      forcing (Eq. BGK) and push-streaming into the other buffer.
// Algorithmic traffic is one read and one write of every population; the
// halo re-reads are served from L2.
//
// Discrete derivatives are the isotropic lattice stencils, written as sums
// of differences from the centre so a constant field gives exactly zero:
//   grad phi = (1/c_s^2) sum_k w_k c_k (phi(x + c_k) - phi(x))
//   lap  phi = (2/c_s^2) sum_k w_k (phi(x + c_k) - phi(x)).
#include "kernels.h"
#include "physics.cuh"

namespace mlsw {

__device__ __forceinline__ int wrap(int v, int n) {
  v %= n;
  return v < 0 ? v + n : v;
}

// Collision with forcing and push-streaming of one layer at one cell.
// h = H + dh; f_old (only read when !TAU1) holds the pre-collision stored
// populations (rest population shifted by H).
template <int LAT, bool TAU1>
__device__ __forceinline__ void collide_store(const KParams& P, float h, float dh, float jx,
                                              float jy, float Fx, float Fy, const float* f_old,
                                              float* __restrict__ out_layer, long plane,
                                              int gx, int gy) {
  using Lt = Lattice<LAT>;
  const float inv_h = 1.f / h;
  const float ux = jx * inv_h, uy = jy * inv_h;
  const float u2 = ux * ux + uy * uy;
  float sum_eq = 0.f;
  float fs[Lt::Q];
#pragma unroll
  for (int k = 1; k < Lt::Q; ++k) {
    const float cu = (float)Lt::cx(k) * ux + (float)Lt::cy(k) * uy;
    // w_k h (c.U / cs^2 + (c.U)^2 / (2 cs^4) - U^2 / (2 cs^2)), cs^2 = 1/3
    const float feq = Lt::w(k) * h * (3.f * cu + 4.5f * cu * cu - 1.5f * u2);
    sum_eq += feq;
    float v = TAU1 ? feq : f_old[k] + P.omega * (feq - f_old[k]);
    v += 3.f * Lt::w(k) * ((float)Lt::cx(k) * Fx + (float)Lt::cy(k) * Fy);
    fs[k] = v;
  }
  // rest population: h - sum of the moving equilibria, which equals
  // h (1 - w_0 U^2 / (2 cs^2)) and keeps the cell's mass exact in the sum;
  // stored shifted by H, i.e. dh - sum_eq
  const float geq0 = dh - sum_eq;
  fs[0] = TAU1 ? geq0 : f_old[0] + P.omega * (geq0 - f_old[0]);
#pragma unroll
  for (int k = 0; k < Lt::Q; ++k) {
    int dx = gx + Lt::cx(k), dy = gy + Lt::cy(k);
    if (Lt::cx(k) > 0 && dx >= P.nx) dx -= P.nx;
    if (Lt::cx(k) < 0 && dx < 0) dx += P.nx;
    if (LAT == 2) {
      if (Lt::cy(k) > 0 && dy >= P.ny) dy -= P.ny;
      if (Lt::cy(k) < 0 && dy < 0) dy += P.ny;
    }
    out_layer[(long)k * plane + (long)dy * P.nx + dx] = fs[k];
  }
}

// ---------------------------------------------------------------------------
// D2Q9: tile TX x TY cells, blockDim = (32, BY), RPT rows per thread.
// ---------------------------------------------------------------------------
template <int N, int BY, int RPT, bool TAU1>
__global__ void __launch_bounds__(32 * BY)
    step_d2q9_kernel(const float* __restrict__ fin, float* __restrict__ fout, KParams P,
                     int* __restrict__ status) {
  using Lt = Lattice<2>;
  constexpr int Q = 9;
  constexpr int TX = 32, TY = BY * RPT, NT = 32 * BY;
  constexpr int RW = TX + 4, RH = TY + 4;  // moments region: tile + 2 rings
  constexpr int PW = TX + 2, PH = TY + 2;  // pressure region: tile + 1 ring
  constexpr int HALO = 4 * RW + 4 * TY;
  __shared__ float zs[N][RH][RW];
  __shared__ float hs[N][RH][RW];
  __shared__ float ps[N][PH][PW];

  const int nx = P.nx, ny = P.ny;
  const long plane = (long)nx * ny;
  const int x0 = blockIdx.x * TX, y0 = blockIdx.y * TY;
  const int tx = threadIdx.x, ty = threadIdx.y, tid = ty * 32 + tx;

  // ---- A. moments: own cells (kept in registers) -------------------------
  float hh[RPT][N], dd[RPT][N], jx[RPT][N], jy[RPT][N];
  const int gx = wrap(x0 + tx, nx);
#pragma unroll
  for (int r = 0; r < RPT; ++r) {
    const int row = ty + r * BY;
    const int gy = wrap(y0 + row, ny);
    const float* src = fin + (long)gy * nx + gx;
    float v[N][Q];
#pragma unroll
    for (int i = 0; i < N; ++i)
#pragma unroll
      for (int k = 0; k < Q; ++k) v[i][k] = __ldg(src + (long)(i * Q + k) * plane);
    float z = 0.f;
#pragma unroll
    for (int i = 0; i < N; ++i) {
      float s = 0.f, sx = 0.f, sy = 0.f;
#pragma unroll
      for (int k = 0; k < Q; ++k) {
        s += v[i][k];
        if (Lt::cx(k) > 0) sx += v[i][k];
        if (Lt::cx(k) < 0) sx -= v[i][k];
        if (Lt::cy(k) > 0) sy += v[i][k];
        if (Lt::cy(k) < 0) sy -= v[i][k];
      }
      dd[r][i] = s;
      hh[r][i] = P.H[i] + s;
      jx[r][i] = sx;
      jy[r][i] = sy;
      z += s;
      hs[i][row + 2][tx + 2] = hh[r][i];
      zs[i][row + 2][tx + 2] = z;
    }
  }
  // ---- A. moments: halo ring of width 2 (heights only) -------------------
  for (int idx = tid; idx < HALO; idx += NT) {
    int rr, rc;
    if (idx < 2 * RW) {
      rr = idx / RW;
      rc = idx % RW;
    } else if (idx < 4 * RW) {
      const int j = idx - 2 * RW;
      rr = RH - 2 + j / RW;
      rc = j % RW;
    } else {
      const int j = idx - 4 * RW;
      rr = 2 + (j >> 2);
      const int c4 = j & 3;
      rc = c4 < 2 ? c4 : RW - 4 + c4;
    }
    const int hx = wrap(x0 - 2 + rc, nx), hy = wrap(y0 - 2 + rr, ny);
    const float* src = fin + (long)hy * nx + hx;
    float v[N][Q];
#pragma unroll
    for (int i = 0; i < N; ++i)
#pragma unroll
      for (int k = 0; k < Q; ++k) v[i][k] = __ldg(src + (long)(i * Q + k) * plane);
    float z = 0.f;
#pragma unroll
    for (int i = 0; i < N; ++i) {
      float s = 0.f;
#pragma unroll
      for (int k = 0; k < Q; ++k) s += v[i][k];
      z += s;
      hs[i][rr][rc] = P.H[i] + s;
      zs[i][rr][rc] = z;
    }
  }
  __syncthreads();

  // ---- B. pressures on tile + 1 ring --------------------------------------
  for (int idx = tid; idx < PH * PW; idx += NT) {
    const int pr = idx / PW, pc = idx % PW;
    const int rr = pr + 1, rc = pc + 1;
    float h[N], gxz[N], gyz[N], lz[N], p[N];
#pragma unroll
    for (int i = 0; i < N; ++i) {
      const float c = zs[i][rr][rc];
      const float e = zs[i][rr][rc + 1] - c, wv = zs[i][rr][rc - 1] - c;
      const float n_ = zs[i][rr + 1][rc] - c, s_ = zs[i][rr - 1][rc] - c;
      const float ne = zs[i][rr + 1][rc + 1] - c, nw = zs[i][rr + 1][rc - 1] - c;
      const float se = zs[i][rr - 1][rc + 1] - c, sw = zs[i][rr - 1][rc - 1] - c;
      // (1/cs^2)(w_1 = 1/9, w_2 = 1/36) -> 1/3 and 1/12
      gxz[i] = (e - wv) * (1.f / 3.f) + ((ne - nw) + (se - sw)) * (1.f / 12.f);
      gyz[i] = (n_ - s_) * (1.f / 3.f) + ((ne - se) + (nw - sw)) * (1.f / 12.f);
      // (2/cs^2)(w_1, w_2) -> 2/3 and 1/6
      lz[i] = ((e + wv) + (n_ + s_)) * (2.f / 3.f) + ((ne + nw) + (se + sw)) * (1.f / 6.f);
      h[i] = hs[i][rr][rc];
    }
    layer_pressures<N>(P, h, gxz, gyz, lz, p);
#pragma unroll
    for (int i = 0; i < N; ++i) ps[i][pr][pc] = p[i];
  }
  __syncthreads();

  // ---- C. force, collision, streaming on the tile -------------------------
  bool bad = false;
#pragma unroll
  for (int r = 0; r < RPT; ++r) {
    const int row = ty + r * BY;
    if (x0 + tx >= nx || y0 + row >= ny) continue;
    const int gy = y0 + row;
    const int pr = row + 1, pc = tx + 1;
    float Rx[N], Ry[N];
    friction<N>(P, hh[r], jx[r], jy[r], Rx, Ry);
#pragma unroll
    for (int i = 0; i < N; ++i) {
      const float c = ps[i][pr][pc];
      const float e = ps[i][pr][pc + 1] - c, wv = ps[i][pr][pc - 1] - c;
      const float n_ = ps[i][pr + 1][pc] - c, s_ = ps[i][pr - 1][pc] - c;
      const float ne = ps[i][pr + 1][pc + 1] - c, nw = ps[i][pr + 1][pc - 1] - c;
      const float se = ps[i][pr - 1][pc + 1] - c, sw = ps[i][pr - 1][pc - 1] - c;
      const float gpx = (e - wv) * (1.f / 3.f) + ((ne - nw) + (se - sw)) * (1.f / 12.f);
      const float gpy = (n_ - s_) * (1.f / 3.f) + ((ne - se) + (nw - sw)) * (1.f / 12.f);
      const float h = hh[r][i];
      const float Fx = -h * gpx + Rx[i];
      const float Fy = -h * gpy + Ry[i];
      bad |= !(h > 0.f) || !isfinite(Fx) || !isfinite(Fy) || !isfinite(jx[r][i]) ||
             !isfinite(jy[r][i]);
      float fo[Q];
      if (!TAU1) {
        const float* src = fin + (long)gy * nx + (x0 + tx) + (long)(i * Q) * plane;
#pragma unroll
        for (int k = 0; k < Q; ++k) fo[k] = src[(long)k * plane];
      }
      collide_store<2, TAU1>(P, h, dd[r][i], jx[r][i], jy[r][i], Fx, Fy, fo,
                             fout + (long)(i * Q) * plane, plane, x0 + tx, gy);
    }
  }
  if (bad) atomicOr(status, 1);
}

// ---------------------------------------------------------------------------
// D1Q3: tile of TX cells, one cell per thread.
// ---------------------------------------------------------------------------
template <int N, int TX, bool TAU1>
__global__ void __launch_bounds__(TX)
    step_d1q3_kernel(const float* __restrict__ fin, float* __restrict__ fout, KParams P,
                     int* __restrict__ status) {
  constexpr int Q = 3;
  constexpr int RW = TX + 4, PW = TX + 2;
  __shared__ float zs[N][RW];
  __shared__ float hs[N][RW];
  __shared__ float ps[N][PW];
  const int nx = P.nx;
  const long plane = nx;
  const int x0 = blockIdx.x * TX, tx = threadIdx.x;

  float hh[N], dd[N], jx[N];
  {
    const int gx = wrap(x0 + tx, nx);
    float z = 0.f;
#pragma unroll
    for (int i = 0; i < N; ++i) {
      const float f0 = __ldg(fin + (long)(i * Q + 0) * plane + gx);
      const float f1 = __ldg(fin + (long)(i * Q + 1) * plane + gx);
      const float f2 = __ldg(fin + (long)(i * Q + 2) * plane + gx);
      const float s = f0 + (f1 + f2);
      dd[i] = s;
      hh[i] = P.H[i] + s;
      jx[i] = f1 - f2;
      z += s;
      hs[i][tx + 2] = hh[i];
      zs[i][tx + 2] = z;
    }
  }
  if (tx < 4) {
    const int rc = tx < 2 ? tx : RW - 4 + tx;
    const int gx = wrap(x0 - 2 + rc, nx);
    float z = 0.f;
#pragma unroll
    for (int i = 0; i < N; ++i) {
      const float s = __ldg(fin + (long)(i * Q + 0) * plane + gx) +
                      (__ldg(fin + (long)(i * Q + 1) * plane + gx) +
                       __ldg(fin + (long)(i * Q + 2) * plane + gx));
      z += s;
      hs[i][rc] = P.H[i] + s;
      zs[i][rc] = z;
    }
  }
  __syncthreads();
  for (int pc = tx; pc < PW; pc += TX) {
    const int rc = pc + 1;
    float h[N], gxz[N], gyz[N], lz[N], p[N];
#pragma unroll
    for (int i = 0; i < N; ++i) {
      const float c = zs[i][rc];
      const float e = zs[i][rc + 1] - c, wv = zs[i][rc - 1] - c;
      gxz[i] = 0.5f * (e - wv);  // (1/cs^2) w_1 = 1/2
      gyz[i] = 0.f;
      lz[i] = e + wv;            // (2/cs^2) w_1 = 1
      h[i] = hs[i][rc];
    }
    layer_pressures<N>(P, h, gxz, gyz, lz, p);
#pragma unroll
    for (int i = 0; i < N; ++i) ps[i][pc] = p[i];
  }
  __syncthreads();
  if (x0 + tx >= nx) return;
  float zero[N], Rx[N], Ry[N];
#pragma unroll
  for (int i = 0; i < N; ++i) zero[i] = 0.f;
  friction<N>(P, hh, jx, zero, Rx, Ry);
  bool bad = false;
#pragma unroll
  for (int i = 0; i < N; ++i) {
    const float c = ps[i][tx + 1];
    const float gpx = 0.5f * ((ps[i][tx + 2] - c) - (ps[i][tx] - c));
    const float h = hh[i];
    const float Fx = -h * gpx + Rx[i];
    bad |= !(h > 0.f) || !isfinite(Fx) || !isfinite(jx[i]);
    float fo[Q];
    if (!TAU1) {
#pragma unroll
      for (int k = 0; k < Q; ++k) fo[k] = fin[(long)(i * Q + k) * plane + x0 + tx];
    }
    collide_store<1, TAU1>(P, h, dd[i], jx[i], 0.f, Fx, 0.f, fo, fout + (long)(i * Q) * plane,
                           plane, x0 + tx, 0);
  }
  if (bad) atomicOr(status, 1);
}

// ---------------------------------------------------------------------------
// dispatch
// ---------------------------------------------------------------------------
constexpr int kD2BY = 8, kD2RPT = 2;  // D2Q9 tile 32 x 16, 256 threads
constexpr int kD1TX = 128;            // D1Q3 tile of 128 cells

template <int N, bool TAU1>
static cudaError_t launch_n(int lattice, const float* fin, float* fout, const KParams& P,
                            int* status, cudaStream_t st) {
  if (lattice == 2) {
    constexpr int TY = kD2BY * kD2RPT;
    dim3 grid((P.nx + 31) / 32, (P.ny + TY - 1) / TY);
    step_d2q9_kernel<N, kD2BY, kD2RPT, TAU1><<<grid, dim3(32, kD2BY), 0, st>>>(fin, fout, P, status);
  } else {
    dim3 grid((P.nx + kD1TX - 1) / kD1TX);
    step_d1q3_kernel<N, kD1TX, TAU1><<<grid, kD1TX, 0, st>>>(fin, fout, P, status);
  }
  return cudaGetLastError();
}

template <bool TAU1>
static cudaError_t launch_tau(int lattice, const float* fin, float* fout, const KParams& P,
                              int* status, cudaStream_t st) {
  switch (P.n) {
    case 1: return launch_n<1, TAU1>(lattice, fin, fout, P, status, st);
    case 2: return launch_n<2, TAU1>(lattice, fin, fout, P, status, st);
    case 3: return launch_n<3, TAU1>(lattice, fin, fout, P, status, st);
    case 4: return launch_n<4, TAU1>(lattice, fin, fout, P, status, st);
    case 5: return launch_n<5, TAU1>(lattice, fin, fout, P, status, st);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_step(int lattice, const float* fin, float* fout, const KParams& P, int* status,
                        cudaStream_t st) {
  if (P.omega == 1.f) return launch_tau<true>(lattice, fin, fout, P, status, st);
  return launch_tau<false>(lattice, fin, fout, P, status, st);
}

}  // namespace mlsw
