// noalloc.cu -- mlswlbm_diagnostics_noalloc: the diagnostics reduction with
// its scratch in a static device array, for callers that cannot allocate.
//
// Some callers cannot call cudaMalloc: applications whose device memory is
// already reserved by a pool allocator (a plain cudaMalloc then fails or
// fragments the pool), and latency-critical loops in which cudaMalloc /
// cudaFree would synchronise the whole device. This entry point needs no
// handle and allocates nothing: the per-block partial sums live in
// g_diag_scratch below, which every GPU that loads the library holds until
// the process exits.
#include <cmath>
#include <mutex>

#include "../../include/mlswlbm.h"
#include "kernels.h"
#include "physics.cuh"

namespace {

// Each reduction block sums a fixed run of cells, so the partials needed
// grow with the lattice; the array holds kNoallocBlocks blocks of
// (MLSW_MAX_LAYERS + 2) doubles = 224 KiB.
constexpr long kNoallocCellsPerBlock = 16384;
constexpr int kNoallocBlocks = 4096;
constexpr int kNoallocMaxDevices = 64;

static __device__ __align__(256) double g_diag_scratch[kNoallocBlocks * (MLSW_MAX_LAYERS + 2)];

std::mutex g_setup_mutex[kNoallocMaxDevices];
bool g_ready[kNoallocMaxDevices];  // set only after a successful look-up
double* g_scratch_ptr[kNoallocMaxDevices];

// The host-side name g_diag_scratch is only a stand-in for the device
// array; its device address is looked up per device, with that device
// current, and passed to the kernels. Only a successful look-up is kept: a
// failed one returns the error and is tried again on the next call.
cudaError_t scratch_of_device(int dev, double** out) {
  std::lock_guard<std::mutex> lock(g_setup_mutex[dev]);
  if (!g_ready[dev]) {
    void* ptr = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&ptr, g_diag_scratch);
    if (e != cudaSuccess || !ptr) {
      (void)cudaGetLastError();  // leave no sticky error behind for the caller
      return e != cudaSuccess ? e : cudaErrorInvalidSymbol;
    }
    g_scratch_ptr[dev] = static_cast<double*>(ptr);
    g_ready[dev] = true;
  }
  *out = g_scratch_ptr[dev];
  return cudaSuccess;
}

}  // namespace

extern "C" int mlswlbm_diagnostics_noalloc(const mlsw_params* p, const float* f,
                                           const float* H, double* out, void* stream) {
  if (!p || !f || !out) return MLSW_ERR_ARG;
  if (mlswlbm_check_params(p) != MLSW_OK) return MLSW_ERR_ARG;
  const int n = p->n_layers;
  const long ncell = (long)p->nx * p->ny;
  const long nblk = (ncell + kNoallocCellsPerBlock - 1) / kNoallocCellsPerBlock;
  if (nblk > kNoallocBlocks) return MLSW_ERR_UNSUPPORTED;  // beyond the static scratch
  mlsw::KShift sh;
  for (int i = 0; i < mlsw::kMaxLayers; ++i) {
    sh.H[i] = (H && i < n) ? H[i] : 0.f;
    if (!std::isfinite(sh.H[i])) return MLSW_ERR_ARG;
  }
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return MLSW_ERR_CUDA;
  if (dev < 0 || dev >= kNoallocMaxDevices) return MLSW_ERR_UNSUPPORTED;
  double* scratch = nullptr;
  if (scratch_of_device(dev, &scratch) != cudaSuccess) return MLSW_ERR_CUDA;
  // every block writes its own partials, so nothing needs clearing first
  const cudaError_t e =
      mlsw::launch_diagnostics(p->lattice, n, mlsw::dense_layout(p->nx, p->ny, n * (p->lattice == MLSW_D1Q3 ? 3 : 9)), f, sh,
                               scratch, (int)nblk, out, (cudaStream_t)stream);
  return e == cudaSuccess ? MLSW_OK : MLSW_ERR_CUDA;
}
