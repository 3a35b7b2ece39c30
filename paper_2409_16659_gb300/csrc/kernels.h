// kernels.h -- internal launch interface between the host library
// (mlswlbm.cu, noalloc.cu) and the kernel translation units. Not part of
// the C ABI.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>

#include "physics.cuh"

namespace mlsw {

// status word bits (device int OR-ed by the kernels)
constexpr int kStatusNonfinite = 1;  // h <= 0 or a non-finite value
constexpr int kStatusTimeout = 2;    // a bounded mbarrier wait ran out

// Per-layer rest-population shift (see KParams).
struct KShift {
  float H[kMaxLayers];
};

// One fused time step fin -> fout (distinct buffers, layout P.L).
struct StepLaunch {
  int lattice;                  // 1 = D1Q3, 2 = D2Q9
  const float* fin;
  float* fout;
  const CUtensorMap* fin_map;   // D2Q9: 3-D tensor map of fin (box of one tile)
  KParams P;
  int* status;
  int* sched;                   // D2Q9: two zero-initialised tile-scheduler counters
  int num_sms;
  int reverse;                  // D2Q9: 1 = tiles in reverse order (see SingleTiles)
};
cudaError_t launch_step(const StepLaunch& a, cudaStream_t st);

// D1Q3 lattices small enough for one CTA's shared memory run many steps in
// one persistent launch: bytes of shared memory it needs (0: not possible
// for this lattice type), and the launch, which reads a.fin and leaves the
// state after nsteps steps in a.fout (ghost images included).
size_t step_persistent_smem(int n, int lattice, int nx);
cudaError_t launch_step_persistent(const StepLaunch& a, int nsteps, cudaStream_t st);

// ---------------------------------------------------------------------------
// Batches: many independent D2Q9 lattices stepped by one persistent launch
// over one tile table, in which the tiles of instances that share n, kernel
// mode and tile height form a contiguous range (batch_kernels.cu).
// ---------------------------------------------------------------------------
// Tile heights a batch can use: variant 0 = 16 rows with two rows per
// thread (n <= 3 only), variant 1 = 8 rows with one row per thread.
constexpr int kBatchVariants = 2;
__host__ __device__ constexpr int batch_variant(int rows_per_thread) {
  return rows_per_thread == 2 ? 0 : 1;
}
__host__ __device__ constexpr int batch_tile_rows(int variant) { return variant == 0 ? 16 : 8; }

// Device descriptor of one instance (aligned as its tensor maps require).
struct BatchInst {
  CUtensorMap map[kBatchVariants][2];  // [variant][input buffer]: box of one tile + halo
  KParams P;
  float* f[2];  // population buffers
  int ntx;      // tile columns (tiles are 32 cells wide)
};

// Kernel mode of a parameter set: 0 general, 1 tau = 1, 2 fast (tau = 1,
// exponents (3, 2), spreading only between neighbouring interfaces).
int step_mode(const KParams& P);

// Kind of a range of tiles: layer count n (1..5), kernel mode, tile-height
// variant (16-row tiles only for n <= 3).
constexpr int kBatchKinds = 5 * 3 * kBatchVariants;
__host__ __device__ constexpr int batch_kind(int n, int mode, int variant) {
  return ((n - 1) * 3 + mode) * kBatchVariants + variant;
}
bool batch_kind_valid(int n, int mode, int variant);
// dynamic shared memory of the tile loop of one kind
size_t batch_kind_smem(int n, int variant);

// Ends of the ranges of a tile table sorted by kind: the tiles of kind k are
// the entries [end[k - 1], end[k]) (end[-1] = 0), so end is non-decreasing
// and a kind without tiles repeats the previous end.
struct BatchEnds {
  int end[kBatchKinds];
};

// One batch step of every instance in a tile table (device, entries of
// (instance, tile) in ranges), buffers cur -> cur ^ 1: one launch.
struct BatchLaunch {
  const BatchInst* inst;
  const int2* table;
  BatchEnds ends;
  int cur;
  int* status;
  int* sched;  // two zero-initialised counters
  int num_sms;
};
// With an empty table (every end 0) it only configures the kernel
// (shared-memory limit, occupancy) on the current device, so that a later
// launch can be captured.
cudaError_t launch_batch_step(const BatchLaunch& a, cudaStream_t st);

// out[2 (j kMaxLayers + i) + {0, 1}] = real and imaginary part of
// sum_x h_i(x) exp(-2 pi i (kx[j] x / nx + ky[j] y / ny)) for every instance
// j < count and layer i (zero for i >= n_j); kx, ky device arrays.
cudaError_t launch_batch_modes(const BatchInst* inst, int count, int cur, const int* kx,
                               const int* ky, double* out, cudaStream_t st);

// Heights [n][ny][nx] of one instance (its host descriptor) from buffer cur.
cudaError_t launch_batch_heights(const BatchInst* inst_host, int cur, float* h, cudaStream_t st);

// Radially averaged power spectra of the layer heights (analysis.cu): the
// row and column FFT passes into work (n nx ny complex values), bin sums
// bins[n][nbins] and wavevector counts counts[nbins], both zeroed by the
// caller. Power-of-two sides up to kSpectrumMaxSide, 1 <= nbins <=
// kSpectrumMaxBins.
constexpr int kSpectrumMaxSide = 8192;
constexpr int kSpectrumMaxBins = 8192;
bool spectrum_supported(int nx, int ny, int nbins);
cudaError_t launch_spectrum(int Q, int n, const Layout& L, const float* f, int nbins,
                            float2* work, double* bins, unsigned long long* counts,
                            cudaStream_t st);

// Azimuthal averages of the interfaces around (cx, cy) (analysis.cu):
// sums[m][nbins] of z_m and counts[nbins] of cells per unit-width ring,
// both zeroed by the caller; z_0 the substrate of the given parameters.
struct ProfileParams {
  double cx, cy;
  int nbins;
  double sub_amp;
  int sub_kx, sub_ky;
};
cudaError_t launch_radial_profile(int Q, int n, const Layout& L, const float* f, const KShift& sh,
                                  const ProfileParams& A, double* sums,
                                  unsigned long long* counts, cudaStream_t st);

// Tile shape of the step kernels (the padded layout covers whole tiles).
int step_tile_cols(int lattice);
int step_tile_rows(int n, int lattice);

// f = f_eq(h, U = 0) on the real cells and their ghost images (x only
// when ghosts_y is false): rest population h - H_i, moving populations 0;
// h dense [n][ny][nx]. status |= kStatusNonfinite where h <= 0 or h is not
// finite.
cudaError_t launch_init(int Q, int n, const Layout& L, bool ghosts_y, const float* h, float* f,
                        const KShift& sh, int* status, cudaStream_t st);

// Periodic images: every ghost cell within two cells of the real domain
// (x only when ghosts_y is false) copies its real cell, for all nplanes
// planes.
cudaError_t launch_fill_ghosts(int nplanes, const Layout& L, bool ghosts_y, float* f,
                               cudaStream_t st);

// h dense [n][ny][nx] = H_i + sum_k g[i][k]
// With st_out (a device view of page-locked host memory), the first thread
// also copies the status word *st_in there, so that the host reads it after
// the synchronisation it needs anyway.
cudaError_t launch_heights(int Q, int n, const Layout& L, const float* f, const KShift& sh,
                           float* h, cudaStream_t st, const int* st_in = nullptr,
                           int* st_out = nullptr);

// real cells of the rest planes: f[i][0] += sign * H_i
cudaError_t launch_shift(int Q, int n, const Layout& L, float* f, const KShift& sh, float sign,
                         cudaStream_t st);

// out dense [n][ny][nx] = H_i + g[i][0], the true rest population
cudaError_t launch_rest_planes(int Q, int n, const Layout& L, const float* f, const KShift& sh,
                               float* out, cudaStream_t st);

// Two-pass deterministic reduction of per-layer mass, kinetic energy and
// min h over the real cells. partials: nblk * (n + 2) doubles; out: n + 2
// doubles (mass[0..n-1], kinetic, hmin).
cudaError_t launch_diagnostics(int lattice, int n, const Layout& L, const float* f,
                               const KShift& sh, double* partials, int nblk, double* out,
                               cudaStream_t st);

// Free energy of Eq. (free_energy_n_layer) from dense heights [n][ny][nx],
// FP64, with the parameters in double precision. partials: nblk doubles.
struct FreeEnergyParams {
  int n, lattice, nx, ny;
  double gamma[kMaxLayers];
  double S[kMaxLayers][kMaxLayers];
  double hstar;
  int nw, mw;
  double sub_amp;  // substrate z_0 = sub_amp cos(2 pi (kx x / nx + ky y / ny))
  int sub_kx, sub_ky;
  int wet_kind;    // 0 power law (nw, mw), 1 exponential (kappa)
  double kappa;
};
cudaError_t launch_free_energy(const FreeEnergyParams& E, const float* h, double* partials,
                               int nblk, double* out, cudaStream_t st);

// Friction of independent cells (layout [i][cell]); Jy / Ry may be null.
cudaError_t launch_friction_eval(const KParams& P, long ncell, const float* h, const float* Jx,
                                 const float* Jy, float* Rx, float* Ry, cudaStream_t st);

// One CTA waits on an mbarrier with the step kernels' bounded wait (limit
// iterations); the barrier gets its arrival only when arrive != 0. A wait
// that runs out ORs kStatusTimeout into *status.
cudaError_t launch_wait_selftest(int arrive, unsigned limit, int* status, cudaStream_t st);

// Dense layout of a caller-owned population array (no ghosts).
inline Layout dense_layout(int nx, int ny, int nplanes = 0) {
  Layout L;
  L.nx = nx;
  L.ny = ny;
  L.gx = 0;
  L.gy = 0;
  L.pitch = nx;
  L.rows = ny;
  L.plane = (long)nx * ny;
  L.nplanes = nplanes;
  return L;
}

// Bounds-checked build: accesses out of range since the last call, per
// translation unit with device code (0 in release builds; ~0u if the
// counter could not be read).
unsigned bounds_violations_step();
unsigned bounds_violations_aux();
unsigned bounds_violations_analysis();
unsigned bounds_violations_batch();

}  // namespace mlsw
