// batch_kernels.cu -- one D2Q9 step of every instance of a batch in one
// persistent launch.
//
// The tile table lists (instance, tile) pairs sorted by kind (layer count,
// kernel mode, tile height), so the tiles of each kind form one range. A CTA
// starts on tile blockIdx.x and draws later tiles from one counter shared by
// the whole table, so the tiles it takes increase and it passes through the
// ranges in order: it runs the tile loop of each range it has tiles in
// (section LBM, the same loop as the single-lattice step, d2q9_tile.cuh)
// and hands the first tile it drew beyond a range to the next one. No CTA
// waits for another between ranges, so the ranges of a step overlap as the
// tiles of one range do.
// The dynamic shared memory of a launch is the largest of its ranges' tile
// loops, which each fit two CTAs per SM.
#include <algorithm>

#include "d2q9_tile.cuh"

namespace mlsw {

namespace {

// The tiles of kind K, when this CTA's tile t is among them (t < 0: a
// bounded wait ran out, nothing more runs), then those of the next kinds.
// The kinds' tile loops follow one another in straight-line code: inlined
// in a loop over the ranges instead, they spill registers, and compiled as
// separate functions they lose the uniform registers and constant operands
// of a kernel's parameters (both measured slower than kernels of their own).
template <int K>
__device__ __forceinline__ void run_kinds(const BatchInst* __restrict__ inst,
                                          const int2* __restrict__ table, const BatchEnds& E,
                                          int cur, int* __restrict__ status,
                                          int* __restrict__ sched, int& t) {
  constexpr int V = K % kBatchVariants, M = (K / kBatchVariants) % 3;
  constexpr int N = K / (3 * kBatchVariants) + 1;
  if constexpr (V == 1 || N <= 3) {
    if (t >= 0 && t < E.end[K]) {
      const BatchTiles tiles{inst, table, cur, E.end[K], V};
      t = d2q9_tile_loop<N, M, V == 0 ? 2 : 1>(tiles, status, sched, t);
    }
  }
  if constexpr (K + 1 < kBatchKinds) run_kinds<K + 1>(inst, table, E, cur, status, sched, t);
}

}  // namespace

__global__ void __launch_bounds__(256, 2)
    step_d2q9_batch(const BatchInst* __restrict__ inst, const int2* __restrict__ table,
                    const __grid_constant__ BatchEnds E, int cur, int* __restrict__ status,
                    int* __restrict__ sched) {
  int t = blockIdx.x;
  run_kinds<0>(inst, table, E, cur, status, sched, t);
  tile_loop_finish(sched);
}

bool batch_kind_valid(int n, int mode, int variant) {
  return n >= 1 && n <= kMaxLayers && mode >= kGeneral && mode <= kFast && variant >= 0 &&
         variant < kBatchVariants && (variant == 1 || n <= 3);
}

size_t batch_kind_smem(int n, int variant) {
  if (variant == 0) {
    switch (n) {
      case 1: return D2Tile<1, 2>::kSmem;
      case 2: return D2Tile<2, 2>::kSmem;
      default: return D2Tile<3, 2>::kSmem;
    }
  }
  switch (n) {
    case 1: return D2Tile<1, 1>::kSmem;
    case 2: return D2Tile<2, 1>::kSmem;
    case 3: return D2Tile<3, 1>::kSmem;
    case 4: return D2Tile<4, 1>::kSmem;
    default: return D2Tile<5, 1>::kSmem;
  }
}

cudaError_t launch_batch_step(const BatchLaunch& a, cudaStream_t st) {
  // once per device: the kernel's shared-memory limit (the largest tile
  // loop any range can need) and its CTAs per SM at each range kind's
  // shared memory, so that a launch being captured calls no other API
  static unsigned long long configured = 0;
  static int per_sm[64][kMaxLayers][kBatchVariants];
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev >= 64) return cudaErrorInvalidDevice;
  if (!((configured >> dev) & 1ull)) {
    size_t most = 0;
    for (int n = 1; n <= kMaxLayers; ++n)
      for (int v = 0; v < kBatchVariants; ++v)
        if (batch_kind_valid(n, kGeneral, v)) most = std::max(most, batch_kind_smem(n, v));
    e = cudaFuncSetAttribute(step_d2q9_batch, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)most);
    if (e != cudaSuccess) return e;
    for (int n = 1; n <= kMaxLayers; ++n)
      for (int v = 0; v < kBatchVariants; ++v) {
        int nb = 0;
        if (batch_kind_valid(n, kGeneral, v)) {
          e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, step_d2q9_batch, 256,
                                                            batch_kind_smem(n, v));
          if (e != cudaSuccess) return e;
        }
        per_sm[dev][n - 1][v] = nb > 0 ? nb : 1;
      }
    configured |= 1ull << dev;
  }
  // the largest shared memory of the kinds present sets the launch's CTAs
  // per SM
  const BatchEnds& E = a.ends;
  size_t smem = 0;
  int blocks = 1 << 30, prev = 0;
  for (int k = 0; k < kBatchKinds; ++k) {
    if (E.end[k] < prev) return cudaErrorInvalidValue;
    if (E.end[k] == prev) continue;  // no tiles of kind k
    const int v = k % kBatchVariants, m = (k / kBatchVariants) % 3, n = k / (3 * kBatchVariants) + 1;
    if (!batch_kind_valid(n, m, v)) return cudaErrorInvalidValue;
    prev = E.end[k];
    smem = std::max(smem, batch_kind_smem(n, v));
    blocks = std::min(blocks, per_sm[dev][n - 1][v]);
  }
  const int ntiles = prev;
  if (ntiles <= 0) return cudaSuccess;
  const int slots = a.num_sms * blocks;
  const int grid = ntiles < slots ? ntiles : slots;
  step_d2q9_batch<<<grid, 256, smem, st>>>(a.inst, a.table, E, a.cur, a.status, a.sched);
  return cudaGetLastError();
}

MLSW_DEFINE_BOUNDS_READER(bounds_violations_batch)

}  // namespace mlsw
