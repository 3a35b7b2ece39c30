// aux_kernels.cu -- initialisation, ghost images, height read-out,
// representation shifts, diagnostics reductions and the stand-alone friction
// evaluation. All population arrays use the padded Layout of physics.cuh
// (a dense caller array is the Layout with no ghosts).
#include <cfloat>

#include "kernels.h"
#include "physics.cuh"

namespace mlsw {

static int grid_for(long work, int threads) {
  long g = (work + threads - 1) / threads;
  if (g > 8192) g = 8192;
  if (g < 1) g = 1;
  return (int)g;
}

// ---------------------------------------------------------------------------
// f = f_eq(h, U = 0) (Eq. equilibrium_distribution at rest): f_0 = h, else 0
// ---------------------------------------------------------------------------
__global__ void init_kernel(int Q, int n, Layout L, const float* __restrict__ h,
                            float* __restrict__ f, KShift sh, int* __restrict__ status) {
  const long ncell = (long)L.nx * L.ny;
  const long total = (long)n * Q * ncell;
  bool bad = false;
  for (long t = blockIdx.x * (long)blockDim.x + threadIdx.x; t < total;
       t += (long)gridDim.x * blockDim.x) {
    const long cell = t % ncell;
    const int p = (int)(t / ncell);
    const int k = p % Q, i = p / Q;
    const int x = (int)(cell % L.nx), y = (int)(cell / L.nx);
    float v = 0.f;
    if (k == 0) {
      const float hv = h[(long)i * ncell + cell];
      bad |= !(hv > 0.f) || !isfinite(hv);
      v = hv - sh.H[i];  // stored rest population is shifted by H_i
    }
    f[L.at(p, x, y)] = v;
  }
  if (bad) atomicOr(status, kStatusNonfinite);
}

cudaError_t launch_init(int Q, int n, const Layout& L, const float* h, float* f, const KShift& sh,
                        int* status, cudaStream_t st) {
  const long total = (long)n * Q * L.nx * L.ny;
  init_kernel<<<grid_for(total, 256), 256, 0, st>>>(Q, n, L, h, f, sh, status);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// ghost images: rows y in {-2, -1, ny, ny + 1} over x in [-2, nx + 2) and
// columns x in {-2, -1, nx, nx + 1} over y in [0, ny) (x only: the columns
// over y = 0)
// ---------------------------------------------------------------------------
__device__ __forceinline__ int wrap_any(int v, int n) {
  v %= n;
  return v < 0 ? v + n : v;
}

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
// read-out and representation shifts (real cells only)
// ---------------------------------------------------------------------------
__global__ void heights_kernel(int Q, int n, Layout L, const float* __restrict__ f, KShift sh,
                               float* __restrict__ h) {
  const long ncell = (long)L.nx * L.ny;
  const long total = (long)n * ncell;
  for (long t = blockIdx.x * (long)blockDim.x + threadIdx.x; t < total;
       t += (long)gridDim.x * blockDim.x) {
    const long cell = t % ncell;
    const int i = (int)(t / ncell);
    const int x = (int)(cell % L.nx), y = (int)(cell / L.nx);
    float s = 0.f;
    for (int k = 0; k < Q; ++k) s += f[L.at(i * Q + k, x, y)];
    h[t] = sh.H[i] + s;
  }
}

cudaError_t launch_heights(int Q, int n, const Layout& L, const float* f, const KShift& sh,
                           float* h, cudaStream_t st) {
  heights_kernel<<<grid_for((long)n * L.nx * L.ny, 256), 256, 0, st>>>(Q, n, L, f, sh, h);
  return cudaGetLastError();
}

__global__ void shift_kernel(int Q, int n, Layout L, float* __restrict__ f, KShift sh,
                             float sign) {
  const long ncell = (long)L.nx * L.ny;
  const long total = (long)n * ncell;
  for (long t = blockIdx.x * (long)blockDim.x + threadIdx.x; t < total;
       t += (long)gridDim.x * blockDim.x) {
    const long cell = t % ncell;
    const int i = (int)(t / ncell);
    float* p = f + L.at(i * Q, (int)(cell % L.nx), (int)(cell / L.nx));
    *p = *p + sign * sh.H[i];
  }
}

cudaError_t launch_shift(int Q, int n, const Layout& L, float* f, const KShift& sh, float sign,
                         cudaStream_t st) {
  shift_kernel<<<grid_for((long)n * L.nx * L.ny, 256), 256, 0, st>>>(Q, n, L, f, sh, sign);
  return cudaGetLastError();
}

__global__ void rest_planes_kernel(int Q, int n, Layout L, const float* __restrict__ f, KShift sh,
                                   float* __restrict__ out) {
  const long ncell = (long)L.nx * L.ny;
  const long total = (long)n * ncell;
  for (long t = blockIdx.x * (long)blockDim.x + threadIdx.x; t < total;
       t += (long)gridDim.x * blockDim.x) {
    const long cell = t % ncell;
    const int i = (int)(t / ncell);
    out[t] = sh.H[i] + f[L.at(i * Q, (int)(cell % L.nx), (int)(cell / L.nx))];
  }
}

cudaError_t launch_rest_planes(int Q, int n, const Layout& L, const float* f, const KShift& sh,
                               float* out, cudaStream_t st) {
  rest_planes_kernel<<<grid_for((long)n * L.nx * L.ny, 256), 256, 0, st>>>(Q, n, L, f, sh, out);
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
