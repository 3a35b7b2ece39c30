// kernels.h -- internal launch interface between the host library
// (mlswlbm.cu) and the kernel translation units. Not part of the C ABI.
#pragma once

#include <cuda_runtime.h>

#include "physics.cuh"

namespace mlsw {

// Per-layer rest-population shift (see KParams).
struct KShift {
  float H[kMaxLayers];
};

// One fused time step fin -> fout (distinct buffers) for lattice 1 (D1Q3)
// or 2 (D2Q9). status: device int, OR-ed with 1 on h <= 0 / non-finite.
cudaError_t launch_step(int lattice, const float* fin, float* fout, const KParams& P, int* status,
                        cudaStream_t st);

// f = f_eq(h, U = 0): rest population = h (stored as h - H_i), moving
// populations = 0. status is OR-ed with 1 where h <= 0 or h is not finite.
cudaError_t launch_init(int Q, int n, long ncell, const float* h, float* f, const KShift& sh,
                        int* status, cudaStream_t st);

// h[i][cell] = H_i + sum_k g[i][k][cell]
cudaError_t launch_heights(int Q, int n, long ncell, const float* f, const KShift& sh, float* h,
                           cudaStream_t st);

// rest-population planes: f[i][0] += sign * H_i (sign = +1 or -1)
cudaError_t launch_shift(int Q, int n, long ncell, float* f, const KShift& sh, float sign,
                         cudaStream_t st);

// out[i][cell] = H_i + g[i][0][cell], the true rest population
cudaError_t launch_rest_planes(int Q, int n, long ncell, const float* f, const KShift& sh,
                               float* out, cudaStream_t st);

// Two-pass deterministic reduction of per-layer mass, kinetic energy and
// min h. partials: nblk * (n + 2) doubles; out: n + 2 doubles
// (mass[0..n-1], kinetic, hmin).
cudaError_t launch_diagnostics(int lattice, int n, long ncell, const float* f, const KShift& sh,
                               double* partials, int nblk, double* out, cudaStream_t st);

// Friction of independent cells (layout [i][cell]); Jy / Ry may be null.
cudaError_t launch_friction_eval(const KParams& P, long ncell, const float* h, const float* Jx,
                                 const float* Jy, float* Rx, float* Ry, cudaStream_t st);

}  // namespace mlsw
