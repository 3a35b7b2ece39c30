// aux_kernels.cu -- initialisation, ghost images, height read-out,
// representation shifts, diagnostics reductions and the stand-alone friction
// evaluation. All population arrays use the padded Layout of physics.cuh
// (a dense caller array is the Layout with no ghosts).
#include <cfloat>
#include <cstdint>

#include "kernels.h"
#include "tma.cuh"
#include "physics.cuh"

namespace mlsw {

static int grid_for(long work, int threads) {
  long g = (work + threads - 1) / threads;
  if (g > 8192) g = 8192;
  if (g < 1) g = 1;
  return (int)g;
}

// ---------------------------------------------------------------------------
// Row-parallel kernels: blockIdx.x covers the x range of a row in chunks of
// blockDim.x, blockIdx.y runs (grid-stride) over the rows. Index arithmetic
// stays in 32 bits per row; only the final offsets are 64-bit.
// ---------------------------------------------------------------------------
constexpr int kRowThreads = 256;

// About 4096 blocks in all, each looping over many rows: a block per row
// would spend more time being scheduled than storing its one row segment.
static dim3 row_grid(int width, long nrows) {
  const long gx = (width + kRowThreads - 1) / kRowThreads;
  long gy = 4096 / gx;
  if (gy > nrows) gy = nrows;
  if (gy > 65535) gy = 65535;
  if (gy < 1) gy = 1;
  return dim3((unsigned)gx, (unsigned)gy, 1);
}

__device__ __forceinline__ int wrap_any(int v, int n) {
  v %= n;
  return v < 0 ? v + n : v;
}

// Lanes of V consecutive x (V = 4: one 16-byte access).
template <int V>
struct Row;
template <>
struct Row<1> {
  using T = float;
  static __device__ __forceinline__ T load(const float* p) { return *p; }
  static __device__ __forceinline__ void store(float* p, T v) { *p = v; }
  static __device__ __forceinline__ T sub(T a, float b) { return a - b; }
  static __device__ __forceinline__ T add(T a, T b) { return a + b; }
  static __device__ __forceinline__ T splat(float b) { return b; }
  static __device__ __forceinline__ bool ok(T v) { return v > 0.f && isfinite(v); }
};
template <>
struct Row<4> {
  using T = float4;
  static __device__ __forceinline__ T load(const float* p) {
    return *reinterpret_cast<const float4*>(p);
  }
  static __device__ __forceinline__ void store(float* p, T v) {
    *reinterpret_cast<float4*>(p) = v;
  }
  static __device__ __forceinline__ T sub(T a, float b) {
    return make_float4(a.x - b, a.y - b, a.z - b, a.w - b);
  }
  static __device__ __forceinline__ T add(T a, T b) {
    return make_float4(a.x + b.x, a.y + b.y, a.z + b.z, a.w + b.w);
  }
  static __device__ __forceinline__ T splat(float b) { return make_float4(b, b, b, b); }
  static __device__ __forceinline__ bool ok(T v) {
    return Row<1>::ok(v.x) && Row<1>::ok(v.y) && Row<1>::ok(v.z) && Row<1>::ok(v.w);
  }
};

// ---------------------------------------------------------------------------
// f = f_eq(h, U = 0) (Eq. equilibrium_distribution at rest): f_0 = h, else 0.
// One thread owns V cells of a padded row of one layer, reads their heights
// once and writes all Q planes. The x range [-4, nx + 4) covers the ghost
// ring and the two alignment columns on each side, and y runs over
// [-2, ny + 2) when ghosts_y: every ghost takes its periodic image, so no
// separate ghost pass is needed. R rows are in flight per thread, which
// matters when h is page-locked host memory read across the host link.
// ---------------------------------------------------------------------------
template <int Q, int V>
__global__ void __launch_bounds__(kRowThreads)
    init_kernel(int n, Layout L, int ghosts_y, const float* __restrict__ h,
                float* __restrict__ f, KShift sh, int* __restrict__ status) {
  using Rw = Row<V>;
  using T = typename Rw::T;
  constexpr int R = 4;
  const int nx = L.nx, ny = L.ny;
  const int groups = (nx + 8) / V;
  const int yrows = ghosts_y ? ny + 4 : 1;
  const int y0 = ghosts_y ? 2 : 0;
  const long nrows = (long)n * yrows;
  const int gi = blockIdx.x * blockDim.x + threadIdx.x;
  if (gi >= groups) return;
  const int x = gi * V - 4;
  // V = 4 needs nx % 4 == 0, so a group of x maps onto one group of sx
  const int sx = (x >= 0 && x < nx) ? x : wrap_any(x, nx);
  bool bad = false;
  for (long r0 = blockIdx.y; r0 < nrows; r0 += (long)R * gridDim.y) {
    T hv[R];
#pragma unroll
    for (int u = 0; u < R; ++u) {
      const long r = r0 + (long)u * gridDim.y;
      if (r < nrows) {
        const int i = (int)(r / yrows);
        const int y = (int)(r - (long)i * yrows) - y0;
        const int sy = ghosts_y ? ((y >= 0 && y < ny) ? y : wrap_any(y, ny)) : 0;
        hv[u] = Rw::load(h + ((long)i * ny + sy) * nx + sx);
      }
    }
#pragma unroll
    for (int u = 0; u < R; ++u) {
      const long r = r0 + (long)u * gridDim.y;
      if (r < nrows) {
        const int i = (int)(r / yrows);
        const int y = (int)(r - (long)i * yrows) - y0;
        bad |= !Rw::ok(hv[u]);
        float* dst = f + L.at(i * Q, x, y);
        Rw::store(dst, Rw::sub(hv[u], sh.H[i]));  // rest population, shifted by H_i
#pragma unroll
        for (int k = 1; k < Q; ++k) Rw::store(dst + (long)k * L.plane, Rw::splat(0.f));
      }
    }
  }
  if (bad) atomicOr(status, kStatusNonfinite);
}

template <int Q>
static void init_q(const dim3& g, int V, int n, const Layout& L, int gy, const float* h,
                   float* f, const KShift& sh, int* status, cudaStream_t st) {
  if (V == 4)
    init_kernel<Q, 4><<<g, kRowThreads, 0, st>>>(n, L, gy, h, f, sh, status);
  else
    init_kernel<Q, 1><<<g, kRowThreads, 0, st>>>(n, L, gy, h, f, sh, status);
}

cudaError_t launch_init(int Q, int n, const Layout& L, bool ghosts_y, const float* h, float* f,
                        const KShift& sh, int* status, cudaStream_t st) {
  // the written x range [-4, nx + 4) and y range [-2, ny + 2) must lie
  // inside the padding
  if (L.gx != 4 || L.pitch < L.nx + 8 || (ghosts_y && (L.gy != 2 || L.rows < L.ny + 4)))
    return cudaErrorInvalidValue;
  const bool vec = L.nx % 4 == 0 && L.nx >= 4 && (reinterpret_cast<uintptr_t>(h) & 15) == 0 &&
                   (reinterpret_cast<uintptr_t>(f) & 15) == 0 && L.pitch % 4 == 0 &&
                   L.gx == 4 && L.plane % 4 == 0;
  const int V = vec ? 4 : 1;
  const long nrows = (long)n * (ghosts_y ? L.ny + 4 : 1);
  const dim3 g = row_grid((L.nx + 8) / V, nrows);
  if (Q == 9)
    init_q<9>(g, V, n, L, ghosts_y ? 1 : 0, h, f, sh, status, st);
  else if (Q == 3)
    init_q<3>(g, V, n, L, ghosts_y ? 1 : 0, h, f, sh, status, st);
  else
    return cudaErrorInvalidValue;
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// ghost images: rows y in {-2, -1, ny, ny + 1} over x in [-2, nx + 2) and
// columns x in {-2, -1, nx, nx + 1} over y in [0, ny) (x only: the columns
// over y = 0)
// ---------------------------------------------------------------------------
__global__ void fill_ghosts_kernel(int nplanes, Layout L, int ghosts_y, float* __restrict__ f) {
  const int nx = L.nx, ny = L.ny;
  const long rows_part = ghosts_y ? 4L * (nx + 4) : 0;  // four ghost rows
  const long cols_part = 4L * (ghosts_y ? ny : 1);      // four ghost columns
  const long per_plane = rows_part + cols_part;
  const long total = per_plane * nplanes;
  for (long t = blockIdx.x * (long)blockDim.x + threadIdx.x; t < total;
       t += (long)gridDim.x * blockDim.x) {
    const int p = (int)(t / per_plane);
    const long u = t % per_plane;
    int x, y;
    if (u < rows_part) {
      const int g = (int)(u / (nx + 4));
      x = (int)(u % (nx + 4)) - 2;
      y = g == 0 ? -2 : (g == 1 ? -1 : (g == 2 ? ny : ny + 1));
    } else {
      const long v = u - rows_part;
      const int g = (int)(v & 3);
      y = (int)(v >> 2);
      x = g == 0 ? -2 : (g == 1 ? -1 : (g == 2 ? nx : nx + 1));
    }
    const int sx = wrap_any(x, nx), sy = ghosts_y ? wrap_any(y, ny) : 0;
    f[L.at(p, x, y)] = f[L.at(p, sx, sy)];
  }
}

cudaError_t launch_fill_ghosts(int nplanes, const Layout& L, bool ghosts_y, float* f,
                               cudaStream_t st) {
  const long per_plane = (ghosts_y ? 4L * (L.nx + 4) + 4L * L.ny : 4L);
  fill_ghosts_kernel<<<grid_for(per_plane * nplanes, 256), 256, 0, st>>>(nplanes, L,
                                                                         ghosts_y ? 1 : 0, f);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// read-out and representation shifts (real cells only; one row = one layer
// row y of the lattice)
// ---------------------------------------------------------------------------
template <int Q, int V>
__global__ void __launch_bounds__(kRowThreads)
    heights_kernel(int n, Layout L, const float* __restrict__ f, KShift sh,
                   float* __restrict__ h, const int* __restrict__ st_in,
                   int* __restrict__ st_out) {
  using Rw = Row<V>;
  using T = typename Rw::T;
  const int nx = L.nx, ny = L.ny;
  const int x = (blockIdx.x * blockDim.x + threadIdx.x) * V;
  // the status word of the steps before, to its host mirror
  if (st_out && x == 0 && blockIdx.y == 0) *st_out = *st_in;
  if (x >= nx) return;
  for (long r = blockIdx.y; r < (long)n * ny; r += gridDim.y) {
    const int i = (int)(r / ny), y = (int)(r - (long)i * ny);
    const float* src = f + L.at(i * Q, x, y);
    T v[Q];
#pragma unroll
    for (int k = 0; k < Q; ++k) v[k] = Rw::load(src + (long)k * L.plane);
    T s = Rw::splat(sh.H[i]);
    T d = Rw::splat(0.f);
#pragma unroll
    for (int k = 0; k < Q; ++k) d = Rw::add(d, v[k]);
    Rw::store(h + r * nx + x, Rw::add(s, d));
  }
}

template <int Q>
static void heights_q(const dim3& g, int V, int n, const Layout& L, const float* f,
                      const KShift& sh, float* h, const int* st_in, int* st_out,
                      cudaStream_t st) {
  if (V == 4)
    heights_kernel<Q, 4><<<g, kRowThreads, 0, st>>>(n, L, f, sh, h, st_in, st_out);
  else
    heights_kernel<Q, 1><<<g, kRowThreads, 0, st>>>(n, L, f, sh, h, st_in, st_out);
}

cudaError_t launch_heights(int Q, int n, const Layout& L, const float* f, const KShift& sh,
                           float* h, cudaStream_t st, const int* st_in, int* st_out) {
  const bool vec = L.nx % 4 == 0 && (reinterpret_cast<uintptr_t>(h) & 15) == 0 &&
                   (reinterpret_cast<uintptr_t>(f) & 15) == 0 && L.pitch % 4 == 0 &&
                   L.gx % 4 == 0 && L.plane % 4 == 0;
  const int V = vec ? 4 : 1;
  const dim3 g = row_grid(L.nx / V, (long)n * L.ny);
  if (Q == 9)
    heights_q<9>(g, V, n, L, f, sh, h, st_in, st_out, st);
  else if (Q == 3)
    heights_q<3>(g, V, n, L, f, sh, h, st_in, st_out, st);
  else
    return cudaErrorInvalidValue;
  return cudaGetLastError();
}

__global__ void __launch_bounds__(kRowThreads)
    shift_kernel(int Q, int n, Layout L, float* __restrict__ f, KShift sh, float sign) {
  const int nx = L.nx, ny = L.ny;
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  if (x >= nx) return;
  for (long r = blockIdx.y; r < (long)n * ny; r += gridDim.y) {
    const int i = (int)(r / ny), y = (int)(r - (long)i * ny);
    float* p = f + L.at(i * Q, x, y);
    *p = *p + sign * sh.H[i];
  }
}

cudaError_t launch_shift(int Q, int n, const Layout& L, float* f, const KShift& sh, float sign,
                         cudaStream_t st) {
  shift_kernel<<<row_grid(L.nx, (long)n * L.ny), kRowThreads, 0, st>>>(Q, n, L, f, sh, sign);
  return cudaGetLastError();
}

__global__ void __launch_bounds__(kRowThreads)
    rest_planes_kernel(int Q, int n, Layout L, const float* __restrict__ f, KShift sh,
                       float* __restrict__ out) {
  const int nx = L.nx, ny = L.ny;
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  if (x >= nx) return;
  for (long r = blockIdx.y; r < (long)n * ny; r += gridDim.y) {
    const int i = (int)(r / ny), y = (int)(r - (long)i * ny);
    out[r * nx + x] = sh.H[i] + f[L.at(i * Q, x, y)];
  }
}

cudaError_t launch_rest_planes(int Q, int n, const Layout& L, const float* f, const KShift& sh,
                               float* out, cudaStream_t st) {
  rest_planes_kernel<<<row_grid(L.nx, (long)n * L.ny), kRowThreads, 0, st>>>(Q, n, L, f, sh,
                                                                             out);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// diagnostics: per-layer mass, kinetic energy |J|^2 / (2h), min h
// ---------------------------------------------------------------------------
__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  return v;
}
__device__ __forceinline__ double warp_min(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmin(v, __shfl_down_sync(0xffffffffu, v, o));
  return v;
}

constexpr int kDiagThreads = 256;

template <int LAT>
__global__ void __launch_bounds__(kDiagThreads)
    diag_partial_kernel(int n, Layout L, const float* __restrict__ f, KShift sh,
                        double* __restrict__ partials) {
  using Lt = Lattice<LAT>;
  constexpr int Q = Lt::Q;
  __shared__ double red[kDiagThreads / 32][kMaxLayers + 2];
  const long ncell = (long)L.nx * L.ny;
  double mass[kMaxLayers];
  for (int i = 0; i < kMaxLayers; ++i) mass[i] = 0.0;
  double ke = 0.0, hmin = DBL_MAX;
  for (long c = blockIdx.x * (long)blockDim.x + threadIdx.x; c < ncell;
       c += (long)gridDim.x * blockDim.x) {
    const int x = (int)(c % L.nx), y = (int)(c / L.nx);
    for (int i = 0; i < n; ++i) {
      float dh = 0.f, jx = 0.f, jy = 0.f;
#pragma unroll
      for (int k = 0; k < Q; ++k) {
        const float v = f[L.at(i * Q + k, x, y)];
        dh += v;
        jx += (float)Lt::cx(k) * v;
        jy += (float)Lt::cy(k) * v;
      }
      const double h = (double)sh.H[i] + (double)dh;
      mass[i] += h;
      ke += ((double)jx * jx + (double)jy * jy) / (2.0 * h);
      hmin = fmin(hmin, h);
    }
  }
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  for (int i = 0; i < n; ++i) {
    const double s = warp_sum(mass[i]);
    if (lane == 0) red[wid][i] = s;
  }
  {
    const double s = warp_sum(ke);
    const double m = warp_min(hmin);
    if (lane == 0) {
      red[wid][n] = s;
      red[wid][n + 1] = m;
    }
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int q = 0; q < n + 2; ++q) {
      double acc = (q == n + 1) ? DBL_MAX : 0.0;
      for (int w = 0; w < kDiagThreads / 32; ++w)
        acc = (q == n + 1) ? fmin(acc, red[w][q]) : acc + red[w][q];
      partials[(long)blockIdx.x * (n + 2) + q] = acc;
    }
  }
}

__global__ void diag_final_kernel(int n, int nblk, const double* __restrict__ partials,
                                  double* __restrict__ out) {
  const int q = threadIdx.x;
  if (q >= n + 2) return;
  double acc = (q == n + 1) ? DBL_MAX : 0.0;
  for (int b = 0; b < nblk; ++b) {
    const double v = partials[(long)b * (n + 2) + q];
    acc = (q == n + 1) ? fmin(acc, v) : acc + v;
  }
  out[q] = acc;
}

cudaError_t launch_diagnostics(int lattice, int n, const Layout& L, const float* f,
                               const KShift& sh, double* partials, int nblk, double* out,
                               cudaStream_t st) {
  if (lattice == 2)
    diag_partial_kernel<2><<<nblk, kDiagThreads, 0, st>>>(n, L, f, sh, partials);
  else
    diag_partial_kernel<1><<<nblk, kDiagThreads, 0, st>>>(n, L, f, sh, partials);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  diag_final_kernel<<<1, 32, 0, st>>>(n, nblk, partials, out);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// friction of independent cells
// ---------------------------------------------------------------------------
template <int N>
__global__ void friction_eval_kernel(KParams P, long ncell, const float* __restrict__ h,
                                     const float* __restrict__ Jx, const float* __restrict__ Jy,
                                     float* __restrict__ Rx, float* __restrict__ Ry) {
  for (long c = blockIdx.x * (long)blockDim.x + threadIdx.x; c < ncell;
       c += (long)gridDim.x * blockDim.x) {
    float hh[N], jx[N], jy[N], rx[N], ry[N];
#pragma unroll
    for (int i = 0; i < N; ++i) {
      hh[i] = h[(long)i * ncell + c];
      jx[i] = Jx[(long)i * ncell + c];
      jy[i] = Jy ? Jy[(long)i * ncell + c] : 0.f;
    }
    friction<N>(P, hh, jx, jy, rx, ry);
#pragma unroll
    for (int i = 0; i < N; ++i) {
      Rx[(long)i * ncell + c] = rx[i];
      if (Ry) Ry[(long)i * ncell + c] = ry[i];
    }
  }
}

cudaError_t launch_friction_eval(const KParams& P, long ncell, const float* h, const float* Jx,
                                 const float* Jy, float* Rx, float* Ry, cudaStream_t st) {
  const int g = grid_for(ncell, 128);
  switch (P.n) {
    case 1: friction_eval_kernel<1><<<g, 128, 0, st>>>(P, ncell, h, Jx, Jy, Rx, Ry); break;
    case 2: friction_eval_kernel<2><<<g, 128, 0, st>>>(P, ncell, h, Jx, Jy, Rx, Ry); break;
    case 3: friction_eval_kernel<3><<<g, 128, 0, st>>>(P, ncell, h, Jx, Jy, Rx, Ry); break;
    case 4: friction_eval_kernel<4><<<g, 128, 0, st>>>(P, ncell, h, Jx, Jy, Rx, Ry); break;
    case 5: friction_eval_kernel<5><<<g, 128, 0, st>>>(P, ncell, h, Jx, Jy, Rx, Ry); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

}  // namespace mlsw

namespace mlsw {

// ---------------------------------------------------------------------------
// batches: one Fourier mode of every layer of every instance,
//   hhat_i(q) = sum_x h_i(x) exp(-2 pi i (kx x / nx + ky y / ny)),
// one CTA per (instance, layer); the phase is formed from exact integers.
// ---------------------------------------------------------------------------
constexpr int kModeThreads = 256;

__global__ void __launch_bounds__(kModeThreads)
    batch_mode_kernel(const BatchInst* __restrict__ inst, int cur, const int* __restrict__ kx,
                      const int* __restrict__ ky, double* __restrict__ out) {
  const int j = blockIdx.x / kMaxLayers, i = blockIdx.x - j * kMaxLayers;
  const BatchInst& b = inst[j];
  const KParams& P = b.P;
  __shared__ double red[2][kModeThreads / 32];
  if (i >= P.n) {
    if (threadIdx.x == 0) {
      out[2 * blockIdx.x] = 0.0;
      out[2 * blockIdx.x + 1] = 0.0;
    }
    return;
  }
  const Layout& L = P.L;
  const float* __restrict__ f = b.f[cur];
  const int nx = P.nx, ny = P.ny;
  const long ncell = (long)nx * ny;
  const long qx = ((long)kx[j] % nx + nx) % nx, qy = ((long)ky[j] % ny + ny) % ny;
  double re = 0.0, im = 0.0;
  for (long c = threadIdx.x; c < ncell; c += kModeThreads) {
    const int y = (int)(c / nx), x = (int)(c - (long)y * nx);
    const float* src = f + L.at(i * 9, x, y);
    float d = 0.f;
#pragma unroll
    for (int k = 0; k < 9; ++k) d += src[(long)k * L.plane];
    const double h = (double)(P.H[i] + d);
    // phase / (2 pi) = m / (nx ny), m exact
    const long m = ((qx * x) % nx * ny + (qy * y) % ny * nx) % ncell;
    float sn, cs;
    sincospif(2.f * (float)((double)m / (double)ncell), &sn, &cs);
    re += h * (double)cs;
    im -= h * (double)sn;
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    re += __shfl_down_sync(0xffffffffu, re, o);
    im += __shfl_down_sync(0xffffffffu, im, o);
  }
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (lane == 0) {
    red[0][wid] = re;
    red[1][wid] = im;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double a = 0.0, bb = 0.0;
    for (int w = 0; w < kModeThreads / 32; ++w) {
      a += red[0][w];
      bb += red[1][w];
    }
    out[2 * blockIdx.x] = a;
    out[2 * blockIdx.x + 1] = bb;
  }
}

cudaError_t launch_batch_modes(const BatchInst* inst, int count, int cur, const int* kx,
                               const int* ky, double* out, cudaStream_t st) {
  if (count <= 0) return cudaSuccess;
  batch_mode_kernel<<<count * kMaxLayers, kModeThreads, 0, st>>>(inst, cur, kx, ky, out);
  return cudaGetLastError();
}

// heights of one instance of a batch (layout of its buffers)
cudaError_t launch_batch_heights(const BatchInst* inst_host, int cur, float* h, cudaStream_t st) {
  return launch_heights(9, inst_host->P.n, inst_host->P.L, inst_host->f[cur],
                        KShift{{inst_host->P.H[0], inst_host->P.H[1], inst_host->P.H[2],
                                inst_host->P.H[3], inst_host->P.H[4]}},
                        h, st);
}

}  // namespace mlsw

namespace mlsw {

// ---------------------------------------------------------------------------
// free energy, Eq. (free_energy_n_layer) in the long-wave form,
//   F = sum_x [ sum_{i=1..n} gamma_i (1 + |grad z_i|^2 / 2)
//             + sum_{i=0..n-1} sum_{k=1..n-i} S_ik phi_k(z_{i+k} - z_i)
//               (1 + |grad z_i|^2 / 2) ],  z_0 the substrate,
// with the lattice gradient of the step (isotropic stencil), from dense
// heights [n][ny][nx], in FP64. Two passes: per-block partial sums, then
// their sum in a fixed order.
// ---------------------------------------------------------------------------
constexpr int kFreeThreads = 256;

__device__ __forceinline__ double phi_d(const FreeEnergyParams& E, int k, double h) {
  if (E.wet_kind == 1) {
    const double a = exp(-E.kappa * (h - k * E.hstar));
    return 2.0 * a - a * a;
  }
  const double r = k * E.hstar / h;
  return (E.nw * pow(r, (double)E.mw) - E.mw * pow(r, (double)E.nw)) / (double)(E.nw - E.mw);
}

__global__ void __launch_bounds__(kFreeThreads)
    free_energy_partial_kernel(FreeEnergyParams E, const float* __restrict__ h,
                               double* __restrict__ partials) {
  __shared__ double red[kFreeThreads / 32];
  const int n = E.n, nx = E.nx, ny = E.ny;
  const long ncell = (long)nx * ny;
  double acc = 0.0;
  for (long c = blockIdx.x * (long)blockDim.x + threadIdx.x; c < ncell;
       c += (long)gridDim.x * blockDim.x) {
    const int y = (int)(c / nx), x = (int)(c - (long)y * nx);
    const int xe = x + 1 == nx ? 0 : x + 1, xw = x == 0 ? nx - 1 : x - 1;
    const int yn = y + 1 == ny ? 0 : y + 1, ys = y == 0 ? ny - 1 : y - 1;
    double z[kMaxLayers + 1], g2[kMaxLayers + 1];
    // the substrate z_0 at the cell and its neighbours, its squared gradient
    auto z0 = [&](int xx, int yy) {
      if (E.sub_amp == 0.0) return 0.0;
      long m = ((long)E.sub_kx * xx % nx) * ny + ((long)E.sub_ky * yy % ny) * nx;
      m %= ncell;
      if (m < 0) m += ncell;
      return E.sub_amp * cospi(2.0 * (double)m / (double)ncell);
    };
    z[0] = z0(x, y);
    double zE = z0(xe, y), zW = z0(xw, y), zN = 0, zS = 0, zNE = 0, zNW = 0, zSE = 0, zSW = 0;
    if (E.lattice == 2) {
      zN = z0(x, yn);
      zS = z0(x, ys);
      zNE = z0(xe, yn);
      zNW = z0(xw, yn);
      zSE = z0(xe, ys);
      zSW = z0(xw, ys);
      const double gx = (zE - zW) / 3.0 + ((zNE - zNW) + (zSE - zSW)) / 12.0;
      const double gy = (zN - zS) / 3.0 + ((zNE - zSE) + (zNW - zSW)) / 12.0;
      g2[0] = gx * gx + gy * gy;
    } else {
      const double gx = 0.5 * (zE - zW);
      g2[0] = gx * gx;
    }
    for (int i = 1; i <= n; ++i) {
      const float* hi = h + (long)(i - 1) * ncell;
      z[i] = z[i - 1] + (double)hi[(long)y * nx + x];
      zE += hi[(long)y * nx + xe];
      zW += hi[(long)y * nx + xw];
      double gx, gy;
      if (E.lattice == 2) {
        zN += hi[(long)yn * nx + x];
        zS += hi[(long)ys * nx + x];
        zNE += hi[(long)yn * nx + xe];
        zNW += hi[(long)yn * nx + xw];
        zSE += hi[(long)ys * nx + xe];
        zSW += hi[(long)ys * nx + xw];
        // (1/cs^2) sum_k w_k c_k z(x + c_k): 1/3 on the axes, 1/12 on the diagonals
        gx = (zE - zW) / 3.0 + ((zNE - zNW) + (zSE - zSW)) / 12.0;
        gy = (zN - zS) / 3.0 + ((zNE - zSE) + (zNW - zSW)) / 12.0;
      } else {
        gx = 0.5 * (zE - zW);
        gy = 0.0;
      }
      g2[i] = gx * gx + gy * gy;
      acc += E.gamma[i - 1] * (1.0 + 0.5 * g2[i]);
    }
    for (int i = 0; i < n; ++i)
      for (int k = 1; k <= n - i; ++k)
        acc += E.S[i][k - 1] * phi_d(E, k, z[i + k] - z[i]) * (1.0 + 0.5 * g2[i]);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int w = 0; w < kFreeThreads / 32; ++w) s += red[w];
    partials[blockIdx.x] = s;
  }
}

__global__ void free_energy_final_kernel(int nblk, const double* __restrict__ partials,
                                         double* __restrict__ out) {
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    double s = 0.0;
    for (int b = 0; b < nblk; ++b) s += partials[b];
    *out = s;
  }
}

cudaError_t launch_free_energy(const FreeEnergyParams& E, const float* h, double* partials,
                               int nblk, double* out, cudaStream_t st) {
  free_energy_partial_kernel<<<nblk, kFreeThreads, 0, st>>>(E, h, partials);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  free_energy_final_kernel<<<1, 32, 0, st>>>(nblk, partials, out);
  return cudaGetLastError();
}

}  // namespace mlsw

namespace mlsw {

// ---------------------------------------------------------------------------
// Self-test of the bounded mbarrier wait of the step kernels: one CTA waits
// on a barrier that receives its single arrival (arrive != 0) or never does,
// each thread with the given iteration limit; a wait that runs out sets
// kStatusTimeout, as a step kernel's does, and the kernel returns.
// ---------------------------------------------------------------------------
__global__ void wait_selftest_kernel(int arrive, unsigned limit, int* __restrict__ status) {
  __shared__ __align__(8) uint64_t bar;
  if (threadIdx.x == 0) {
    mbar_init(&bar, 1);
    mbar_init_fence();
  }
  __syncthreads();
  if (arrive && threadIdx.x == 0) mbar_arrive_expect_tx(&bar, 0u);  // the one arrival, no bytes
  if (!mbar_wait_bounded(&bar, 0u, limit)) atomicOr(status, kStatusTimeout);
}

cudaError_t launch_wait_selftest(int arrive, unsigned limit, int* status, cudaStream_t st) {
  wait_selftest_kernel<<<1, 128, 0, st>>>(arrive, limit, status);
  return cudaGetLastError();
}

MLSW_DEFINE_BOUNDS_READER(bounds_violations_aux)

}  // namespace mlsw
