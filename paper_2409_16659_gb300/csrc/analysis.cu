// analysis.cu -- analysis of a solver's state on the device:
//   * radially averaged power spectra of the layer heights, the quantity the
//     paper's spinodal-dewetting section follows in time and compares with
//     the growth rates of its linear stability analysis;
//   * azimuthal averages of the interface heights around a drop or lens
//     centre, the profiles its droplet-equilibrium section fits circular
//     arcs to.
//
// Spectra.
// S_i(b) = mean of |H_i(k)|^2 over the integer wavevectors k = (kx, ky),
// kx in (-nx/2, nx/2] and likewise ky, with round(|k|) = b, where H_i is the
// unnormalised 2-D DFT of h_i with its mean removed (the k = 0 term is set
// to zero). Two passes of radix-2 FFTs in shared memory (power-of-two
// sides): rows, which also form the height deviations h_i - H_i from the
// stored populations, then columns, which bin |H|^2 in FP64.
#include <cstdint>

#include "kernels.h"
#include "physics.cuh"

namespace mlsw {

namespace {

__device__ __forceinline__ int bitrev(int v, int bits) {
  return bits == 0 ? 0 : (int)(__brev((unsigned)v) >> (32 - bits));
}

// In-place radix-2 decimation-in-time FFT (forward, e^{-2 pi i j k / len}) of
// `count` contiguous arrays of length len = 2^bits, each loaded in
// bit-reversed order; leaves them in natural order. All threads of the CTA
// take part.
__device__ void fft_inplace(float2* a, int bits, int count) {
  const int len = 1 << bits, half = len >> 1;
  for (int s = 0; s < bits; ++s) {
    const int m = 1 << s;
    for (int t = threadIdx.x; t < count * half; t += blockDim.x) {
      const int arr = t / half, u = t - arr * half;
      const int j = u & (m - 1);
      const int i0 = arr * len + ((u >> s) << (s + 1)) + j, i1 = i0 + m;
      float sn, cs;
      sincospif(-(float)j / (float)m, &sn, &cs);  // j / m is exact (m a power of two)
      const float2 b = a[i1], u0 = a[i0];
      const float2 wb = make_float2(b.x * cs - b.y * sn, b.x * sn + b.y * cs);
      a[i0] = make_float2(u0.x + wb.x, u0.y + wb.y);
      a[i1] = make_float2(u0.x - wb.x, u0.y - wb.y);
    }
    __syncthreads();
  }
}

// One CTA per (row y, layer i): the row of h_i - H_i (the sum of the stored
// populations, whose rest population is shifted by H_i), transformed.
template <int Q>
__global__ void __launch_bounds__(256)
    spectrum_rows_kernel(Layout L, const float* __restrict__ f, int bits_x,
                         float2* __restrict__ work) {
  extern __shared__ float2 row[];
  const int nx = L.nx, ny = L.ny;
  const int y = blockIdx.x, i = blockIdx.y;
  const float* src = f + L.at(i * Q, 0, y);
  for (int x = threadIdx.x; x < nx; x += blockDim.x) {
    float d = 0.f;
#pragma unroll
    for (int k = 0; k < Q; ++k) d += src[(long)k * L.plane + x];
    row[bitrev(x, bits_x)] = make_float2(d, 0.f);
  }
  __syncthreads();
  fft_inplace(row, bits_x, 1);
  float2* dst = work + ((long)i * ny + y) * nx;
  for (int x = threadIdx.x; x < nx; x += blockDim.x) dst[x] = row[x];
}

// One CTA per (cb columns, layer i): the column transforms, then |H|^2 into
// the radial bins (FP64 sums in shared memory, then global atomics). Layer 0
// also counts the wavevectors per bin.
__global__ void __launch_bounds__(256)
    spectrum_cols_kernel(int nx, int ny, int bits_y, int cb, const float2* __restrict__ work,
                         int nbins, double* __restrict__ bins,
                         unsigned long long* __restrict__ counts) {
  extern __shared__ unsigned char sm[];
  float2* col = reinterpret_cast<float2*>(sm);                      // [cb][ny]
  double* sb = reinterpret_cast<double*>(col + (size_t)cb * ny);    // [nbins]
  unsigned* sc = reinterpret_cast<unsigned*>(sb + nbins);           // [nbins]
  const int c0 = blockIdx.x * cb, i = blockIdx.y;
  for (int b = threadIdx.x; b < nbins; b += blockDim.x) {
    sb[b] = 0.0;
    sc[b] = 0u;
  }
  const float2* src = work + (long)i * ny * nx;
  for (int e = threadIdx.x; e < cb * ny; e += blockDim.x) {
    const int y = e / cb, c = e - y * cb;  // neighbouring threads read neighbouring columns
    col[c * ny + bitrev(y, bits_y)] = src[(long)y * nx + c0 + c];
  }
  __syncthreads();
  fft_inplace(col, bits_y, cb);
  for (int e = threadIdx.x; e < cb * ny; e += blockDim.x) {
    const int c = e / ny, yy = e - c * ny;
    const int kxi = c0 + c;
    const int kx = kxi <= nx / 2 ? kxi : kxi - nx, ky = yy <= ny / 2 ? yy : yy - ny;
    const int b = (int)rint(sqrt((double)kx * kx + (double)ky * ky));
    if (b < nbins) {
      const float2 v = col[e];
      const double p = (kx == 0 && ky == 0) ? 0.0 : (double)v.x * v.x + (double)v.y * v.y;
      atomicAdd(sb + b, p);
      atomicAdd(sc + b, 1u);
    }
  }
  __syncthreads();
  for (int b = threadIdx.x; b < nbins; b += blockDim.x) {
    if (sc[b] == 0u) continue;
    atomicAdd(bins + (long)i * nbins + b, sb[b]);
    if (i == 0) atomicAdd(counts + b, (unsigned long long)sc[b]);
  }
}

int log2_exact(int v) {
  if (v < 1 || (v & (v - 1)) != 0) return -1;
  int b = 0;
  while ((1 << b) < v) ++b;
  return b;
}

}  // namespace

bool spectrum_supported(int nx, int ny, int nbins) {
  return log2_exact(nx) >= 0 && log2_exact(ny) >= 0 && nx <= kSpectrumMaxSide &&
         ny <= kSpectrumMaxSide && nbins >= 1 && nbins <= kSpectrumMaxBins;
}

cudaError_t launch_spectrum(int Q, int n, const Layout& L, const float* f, int nbins,
                            float2* work, double* bins, unsigned long long* counts,
                            cudaStream_t st) {
  const int nx = L.nx, ny = L.ny;
  if (!spectrum_supported(nx, ny, nbins) || n < 1) return cudaErrorInvalidValue;
  const int bx = log2_exact(nx), by = log2_exact(ny);
  const size_t row_smem = (size_t)nx * sizeof(float2);
  const int rthreads = nx / 2 < 32 ? 32 : (nx / 2 > 256 ? 256 : nx / 2);
  cudaError_t e;
  if (Q == 9) {
    e = cudaFuncSetAttribute(spectrum_rows_kernel<9>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)row_smem);
    if (e != cudaSuccess) return e;
    spectrum_rows_kernel<9><<<dim3(ny, n), rthreads, row_smem, st>>>(L, f, bx, work);
  } else if (Q == 3) {
    e = cudaFuncSetAttribute(spectrum_rows_kernel<3>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)row_smem);
    if (e != cudaSuccess) return e;
    spectrum_rows_kernel<3><<<dim3(ny, n), rthreads, row_smem, st>>>(L, f, bx, work);
  } else {
    return cudaErrorInvalidValue;
  }
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  // columns per CTA: up to 8, at most 8192 complex values in shared memory
  int cb = 8192 / ny;
  if (cb > 8) cb = 8;
  if (cb < 1) cb = 1;
  if (cb > nx) cb = nx;
  const size_t col_smem = (size_t)cb * ny * sizeof(float2) + (size_t)nbins * (sizeof(double) + 4);
  e = cudaFuncSetAttribute(spectrum_cols_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)col_smem);
  if (e != cudaSuccess) return e;
  spectrum_cols_kernel<<<dim3(nx / cb, n), 256, col_smem, st>>>(nx, ny, by, cb, work, nbins, bins,
                                                                counts);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Azimuthal averages of the interface heights z_0 .. z_n (z_0 the substrate)
// in unit-width rings b = floor(r) around (cx, cy), r the periodic
// (minimum-image) distance; per-cell heights as the read-out gives them
// (h_i = H_i + sum of the stored populations, in FP32), interfaces and sums
// in FP64. One thread per cell, FP64 atomics into sums[m][nbins] and
// counts[nbins].
// ---------------------------------------------------------------------------
template <int Q>
__global__ void __launch_bounds__(256)
    radial_profile_kernel(int n, Layout L, const float* __restrict__ f, KShift sh,
                          ProfileParams A, double* __restrict__ sums,
                          unsigned long long* __restrict__ counts) {
  const int nx = L.nx, ny = L.ny;
  const long cell = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (cell >= (long)nx * ny) return;
  const int y = (int)(cell / nx), x = (int)(cell - (long)y * nx);
  double dx = x - A.cx, dy = y - A.cy;
  dx -= nx * rint(dx / nx);
  dy -= ny * rint(dy / ny);
  const double r = sqrt(dx * dx + dy * dy);
  if (!(r < (double)A.nbins)) return;
  const int b = (int)floor(r);
  double z = 0.0;
  if (A.sub_amp != 0.0) {
    // z_0 = a cos(2 pi (kx x / nx + ky y / ny)), phase reduced in integers
    const long nc = (long)nx * ny;
    long m = (((long)A.sub_kx * x) % nx) * ny + (((long)A.sub_ky * y) % ny) * nx;
    m %= nc;
    if (m < 0) m += nc;
    z = A.sub_amp * cospi(2.0 * (double)m / (double)nc);
  }
  atomicAdd(sums + b, z);
  for (int i = 0; i < n; ++i) {
    const float* src = f + L.at(i * Q, x, y);
    float d = 0.f;
#pragma unroll
    for (int k = 0; k < Q; ++k) d += src[(long)k * L.plane];
    z += (double)(sh.H[i] + d);
    atomicAdd(sums + (long)(i + 1) * A.nbins + b, z);
  }
  atomicAdd(counts + b, 1ull);
}

cudaError_t launch_radial_profile(int Q, int n, const Layout& L, const float* f, const KShift& sh,
                                  const ProfileParams& A, double* sums,
                                  unsigned long long* counts, cudaStream_t st) {
  const long cells = (long)L.nx * L.ny;
  if (A.nbins < 1 || n < 1 || cells < 1) return cudaErrorInvalidValue;
  const unsigned grid = (unsigned)((cells + 255) / 256);
  if (Q == 9)
    radial_profile_kernel<9><<<grid, 256, 0, st>>>(n, L, f, sh, A, sums, counts);
  else if (Q == 3)
    radial_profile_kernel<3><<<grid, 256, 0, st>>>(n, L, f, sh, A, sums, counts);
  else
    return cudaErrorInvalidValue;
  return cudaGetLastError();
}

MLSW_DEFINE_BOUNDS_READER(bounds_violations_analysis)

}  // namespace mlsw
