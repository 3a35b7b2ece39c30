// mlswlbm.cu -- host side of the C ABI declared in include/mlswlbm.h:
// parameter validation, spreading coefficients, the create-time stability
// check, device buffers and the entry points.
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <algorithm>
#include <new>
#include <vector>

#include "../../include/mlswlbm.h"
#include "host.h"
#include "kernels.h"
#include "physics.cuh"

using mlsw::KParams;

struct mlsw_handle {
  mlsw_params p;
  KParams kp;         // includes the padded layout kp.L
  int Q;
  long ncell;
  size_t flen;        // floats per (padded) population buffer
  float* f[2];
  int cur;            // index of the buffer holding the current state
  float* hbuf;        // n * ncell heights (upload / read-out)
  int* status;        // [0] OR of kernel error bits; [1], [2] tile scheduler
  double* partials;   // diagnostics partials
  double* dout;       // diagnostics result, n + 2 doubles
  int nblk_diag;
  cudaStream_t stream;
  long launches;
  mlsw::KShift sh;    // rest-population shift H_i (also in kp.H)
  int num_sms;
  size_t psmem;       // D1Q3 persistent launch: shared memory bytes (0: not used)
  CUtensorMap map[2]; // D2Q9: tensor map of each buffer, box = one tile + halo
  int* status_host;   // page-locked mirror of status[0], written by the read-out
  int* status_mirror; // its device address
};

namespace mlsw_host {

bool finite_pos(double v) { return std::isfinite(v) && v > 0.0; }

int Qof(int lattice) { return lattice == MLSW_D1Q3 ? 3 : 9; }

// ---------------------------------------------------------------------------
// Explicit-update stability of a uniform flux (derived, not in the paper).
// With tau = 1 the post-collision flux of a uniform state is J + K J, so the
// update is contractive when the spectral radius of I + K is below 1. K is
// built in double by the same shear-stress integration as the device
// friction; rho(I + K) is bounded through ||(I + K)^m||^(1/m), m = 2^12.
// ---------------------------------------------------------------------------
bool friction_matrix(const mlsw_params& p, const double* h, double K[][MLSW_MAX_LAYERS]) {
  const int n = p.n_layers;
  double L[MLSW_MAX_LAYERS][MLSW_MAX_LAYERS];
  for (int j = 0; j < n; ++j) {
    double ub = 0.0;
    for (int i = 0; i < n; ++i) {
      const double s = (j > i) ? -h[j] : 0.0;
      const double g = (i == j) ? 1.0 : 0.0;
      const double mi = 1.0 / p.mu[i], bi = p.beta[i], hi = h[i];
      ub += bi * mi * (s - g * (hi + 0.5 * bi));
      L[i][j] = hi * ub + mi * hi * hi * (0.5 * s - g * hi / 3.0);
      ub += mi * hi * (s - 0.5 * g * hi);
    }
  }
  // X = L^-1 by Gauss-Jordan with partial pivoting
  double A[MLSW_MAX_LAYERS][2 * MLSW_MAX_LAYERS];
  for (int r = 0; r < n; ++r)
    for (int c = 0; c < 2 * n; ++c) A[r][c] = (c < n) ? L[r][c] : (c - n == r ? 1.0 : 0.0);
  for (int c = 0; c < n; ++c) {
    int piv = c;
    for (int r = c + 1; r < n; ++r)
      if (std::fabs(A[r][c]) > std::fabs(A[piv][c])) piv = r;
    if (A[piv][c] == 0.0 || !std::isfinite(A[piv][c])) return false;
    if (piv != c)
      for (int q = 0; q < 2 * n; ++q) std::swap(A[c][q], A[piv][q]);
    const double inv = 1.0 / A[c][c];
    for (int q = 0; q < 2 * n; ++q) A[c][q] *= inv;
    for (int r = 0; r < n; ++r) {
      if (r == c) continue;
      const double l = A[r][c];
      for (int q = 0; q < 2 * n; ++q) A[r][q] -= l * A[c][q];
    }
  }
  for (int r = 0; r < n; ++r)
    for (int c = 0; c < n; ++c) K[r][c] = h[r] * A[r][n + c];
  return true;
}

double spectral_radius_I_plus_K(const mlsw_params& p, const double* h) {
  const int n = p.n_layers;
  double K[MLSW_MAX_LAYERS][MLSW_MAX_LAYERS];
  if (!friction_matrix(p, h, K)) return INFINITY;
  double A[MLSW_MAX_LAYERS][MLSW_MAX_LAYERS], B[MLSW_MAX_LAYERS][MLSW_MAX_LAYERS];
  for (int r = 0; r < n; ++r)
    for (int c = 0; c < n; ++c) A[r][c] = K[r][c] + (r == c ? 1.0 : 0.0);
  double logscale = 0.0;
  const int squarings = 12;
  for (int s = 0; s < squarings; ++s) {
    double mx = 0.0;
    for (int r = 0; r < n; ++r)
      for (int c = 0; c < n; ++c) {
        double acc = 0.0;
        for (int q = 0; q < n; ++q) acc += A[r][q] * A[q][c];
        B[r][c] = acc;
        mx = std::fmax(mx, std::fabs(acc));
      }
    if (!(mx > 0.0)) return 0.0;
    if (!std::isfinite(mx)) return INFINITY;
    logscale = 2.0 * logscale + std::log(mx);
    for (int r = 0; r < n; ++r)
      for (int c = 0; c < n; ++c) A[r][c] = B[r][c] / mx;
  }
  double fro = 0.0;
  for (int r = 0; r < n; ++r)
    for (int c = 0; c < n; ++c) fro += A[r][c] * A[r][c];
  return std::exp((logscale + 0.5 * std::log(fro)) / std::ldexp(1.0, squarings));
}

KParams make_kparams(const mlsw_params& p) {
  KParams k;
  std::memset(&k, 0, sizeof(k));
  k.n = p.n_layers;
  k.nx = p.nx;
  k.ny = p.ny;
  k.omega = (float)(1.0 / p.tau);
  for (int i = 0; i < p.n_layers; ++i) {
    k.gamma[i] = (float)p.gamma[i];
    k.mu_inv[i] = (float)(1.0 / p.mu[i]);
    k.beta[i] = (float)p.beta[i];
    for (int kk = 1; kk <= p.n_layers - i; ++kk) k.S[i][kk - 1] = (float)p.spread[i][kk - 1];
  }
  k.hstar = (float)p.hstar;
  k.nw = p.wet_n;
  k.mw = p.wet_m;
  if (p.wet_kind == 0) {
    k.c_phi = (float)(1.0 / (p.wet_n - p.wet_m));
    k.c_dphi = (float)((double)p.wet_n * p.wet_m / (p.wet_n - p.wet_m));
  }
  k.wet_kind = p.wet_kind;
  k.kappa = (float)p.wet_kappa;
  k.sub_amp = (float)p.sub_amp;
  k.sub_kx = p.sub_kx;
  k.sub_ky = p.sub_ky;
  return k;
}

int check_heights(const mlsw_params& p, const float* h) {
  const long total = (long)p.n_layers * p.nx * p.ny;
  for (long t = 0; t < total; ++t)
    if (!(std::isfinite(h[t]) && h[t] > 0.f)) return MLSW_ERR_ARG;
  return MLSW_OK;
}

#define CU(call)                                     \
  do {                                               \
    if ((call) != cudaSuccess) return MLSW_ERR_CUDA; \
  } while (0)

// ---------------------------------------------------------------------------
// padded layout and tensor maps
// ---------------------------------------------------------------------------
int round_up(int v, int m) { return (v + m - 1) / m * m; }

mlsw::Layout make_layout(const mlsw_params& p) {
  mlsw::Layout L;
  const int tx = mlsw::step_tile_cols(p.lattice);
  const int ty = mlsw::step_tile_rows(p.n_layers, p.lattice);
  L.nx = p.nx;
  L.ny = p.ny;
  L.gx = 4;  // two ghost columns plus two for 16-byte alignment of tile boxes
  L.gy = (p.lattice == MLSW_D2Q9) ? 2 : 0;
  L.pitch = round_up(p.nx, tx) + 8;
  L.rows = (p.lattice == MLSW_D2Q9) ? round_up(p.ny, ty) + 4 : 1;
  L.plane = (long)L.pitch * L.rows;
  L.nplanes = p.n_layers * Qof(p.lattice);
  return L;
}

int wrap_host(int v, int n) {
  v %= n;
  return v < 0 ? v + n : v;
}

void set_ghost_tables(KParams& k, const mlsw_params& p) {
  const int gx[4] = {-2, -1, p.nx, p.nx + 1};
  const int gy[4] = {-2, -1, p.ny, p.ny + 1};
  for (int g = 0; g < 4; ++g) {
    k.gsrcx[g] = wrap_host(gx[g], p.nx);
    k.gsrcy[g] = (p.lattice == MLSW_D2Q9) ? wrap_host(gy[g], p.ny) : -1000;
  }
  k.tiny = (p.nx < 4 || (p.lattice == MLSW_D2Q9 && p.ny < 4)) ? 1 : 0;
}

typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*,
                                  const cuuint64_t*, const cuuint64_t*, const cuuint32_t*,
                                  const cuuint32_t*, CUtensorMapInterleave, CUtensorMapSwizzle,
                                  CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn encode_fn() {
  static EncodeTiledFn fn = nullptr;
  static bool tried = false;
  if (!tried) {
    tried = true;
    void* ptr = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &ptr, 12000, cudaEnableDefault,
                                         &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<EncodeTiledFn>(ptr);
  }
  return fn;
}

// 3-D map (x: pitch, y: rows, z: planes) whose box is one D2Q9 tile with
// its halo: 40 x (TY + 4) x all planes.
bool make_tile_map(CUtensorMap* m, float* base, const mlsw::Layout& L, int nplanes, int box_cols,
                   int box_rows) {
  EncodeTiledFn fn = encode_fn();
  if (!fn) return false;
  cuuint64_t dims[3] = {(cuuint64_t)L.pitch, (cuuint64_t)L.rows, (cuuint64_t)nplanes};
  cuuint64_t strides[2] = {(cuuint64_t)L.pitch * 4, (cuuint64_t)L.plane * 4};
  cuuint32_t box[3] = {(cuuint32_t)box_cols, (cuuint32_t)box_rows, (cuuint32_t)nplanes};
  cuuint32_t es[3] = {1, 1, 1};
  return fn(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, base, dims, strides, box, es,
            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
            CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) ==
         CUDA_SUCCESS;
}

// host <-> device copies of the real cells of every plane
cudaError_t copy_planes(mlsw_handle* h, float* host, const float* dev, bool to_host) {
  const mlsw::Layout& L = h->kp.L;
  const int nplanes = h->p.n_layers * h->Q;
  const size_t row = (size_t)L.nx * sizeof(float);
  for (int pl = 0; pl < nplanes; ++pl) {
    float* hp = host + (size_t)pl * h->ncell;
    const float* dp = dev + L.at(pl, 0, 0);
    cudaError_t e =
        to_host ? cudaMemcpy2DAsync(hp, row, dp, (size_t)L.pitch * sizeof(float), row, L.ny,
                                    cudaMemcpyDeviceToHost, h->stream)
                : cudaMemcpy2DAsync(const_cast<float*>(dp), (size_t)L.pitch * sizeof(float), hp,
                                    row, row, L.ny, cudaMemcpyHostToDevice, h->stream);
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

void set_shift(KParams& kp, mlsw::KShift& sh, int n, const float* H) {
  for (int i = 0; i < mlsw::kMaxLayers; ++i) {
    const float v = (i < n) ? H[i] : 0.f;
    sh.H[i] = v;
    kp.H[i] = v;
  }
  // reference thickness between interfaces l < m, summed in double
  for (int l = 0; l <= mlsw::kMaxLayers; ++l)
    for (int m = 0; m <= mlsw::kMaxLayers; ++m) {
      double acc = 0.0;
      for (int j = l + 1; j <= m; ++j) acc += (double)sh.H[j - 1];
      kp.Hsum[l][m] = (float)acc;
    }
}

void set_shift(mlsw_handle* h, const float* H) { set_shift(h->kp, h->sh, h->p.n_layers, H); }

int prepare_instance(const mlsw_params& p, const float* h_init, KParams& kp, mlsw::KShift& sh) {
  int rc = mlswlbm_check_params(&p);
  if (rc != MLSW_OK) return rc;
  if (!h_init) return MLSW_ERR_ARG;
  rc = check_heights(p, h_init);
  if (rc != MLSW_OK) return rc;
  const int n = p.n_layers;
  const long ncell = (long)p.nx * p.ny;

  double hmin[MLSW_MAX_LAYERS], hmax[MLSW_MAX_LAYERS], hmean[MLSW_MAX_LAYERS],
      hst[MLSW_MAX_LAYERS];
  float shift[MLSW_MAX_LAYERS];
  for (int i = 0; i < n; ++i) {
    double mn = INFINITY, mx = -INFINITY, sum = 0.0;
    for (long c = 0; c < ncell; ++c) {
      const double v = h_init[(long)i * ncell + c];
      mn = std::fmin(mn, v);
      mx = std::fmax(mx, v);
      sum += v;
    }
    hmin[i] = mn;
    hmax[i] = mx;
    hmean[i] = sum / (double)ncell;
    hst[i] = p.hstar;
  }
  // Shift H_i = median of the layer: independent of the order of the cells
  // (a translated field gets the same shift) and close to most cells. The
  // rest population of a cell at h is stored as h - H_i, so cells near H_i
  // keep the small fluxes through them above FP32 rounding: in a nearly
  // flat film the median is its mean level, in a droplet field the
  // precursor that covers most of the layer.
  {
    std::vector<float> buf;
    try {
      buf.resize((size_t)ncell);
    } catch (...) {
      return MLSW_ERR_NOMEM;
    }
    for (int i = 0; i < n; ++i) {
      std::copy(h_init + (long)i * ncell, h_init + (long)(i + 1) * ncell, buf.begin());
      auto mid = buf.begin() + (ncell - 1) / 2;
      std::nth_element(buf.begin(), mid, buf.end());
      shift[i] = *mid;
    }
  }
  if (!(p.flags & MLSW_FLAG_SKIP_STABILITY_CHECK)) {
    const double* states[4] = {hst, hmin, hmean, hmax};
    for (const double* s : states)
      if (!(spectral_radius_I_plus_K(p, s) < 1.0)) return MLSW_ERR_UNSTABLE;
  }
  kp = make_kparams(p);
  kp.L = make_layout(p);
  // the step kernels address a layer's planes with 32-bit offsets
  if ((double)kp.L.plane * Qof(p.lattice) >= 2147483647.0) return MLSW_ERR_UNSUPPORTED;
  set_ghost_tables(kp, p);
  set_shift(kp, sh, n, shift);
  return MLSW_OK;
}

// The address at which kernels on the current device can read or write a
// page-locked host buffer, or nullptr when p is pageable or device memory.
// Kernels then move the heights across the host link themselves, fused
// with the initialisation or the read-out, instead of a separate copy.
const void* mapped_host_ptr(const void* p) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    (void)cudaGetLastError();
    return nullptr;
  }
  return a.type == cudaMemoryTypeHost ? a.devicePointer : nullptr;
}

}  // namespace mlsw_host

using namespace mlsw_host;

extern "C" {

const char* mlswlbm_strerror(int code) {
  switch (code) {
    case MLSW_OK: return "ok";
    case MLSW_ERR_ARG: return "invalid argument";
    case MLSW_ERR_NOMEM: return "out of memory";
    case MLSW_ERR_CUDA: return "CUDA call failed";
    case MLSW_ERR_NONFINITE: return "non-finite value or non-positive layer height";
    case MLSW_ERR_UNSTABLE: return "explicit friction update not contractive";
    case MLSW_ERR_TIMEOUT: return "device wait timed out";
    case MLSW_ERR_UNSUPPORTED: return "unsupported configuration";
    default: return "unknown error";
  }
}

int mlswlbm_spreading_from_tensions(int n, const double* g, mlsw_params* p) {
  if (!g || !p || n < 1 || n > MLSW_MAX_LAYERS) return MLSW_ERR_ARG;
  const int G = n + 2;
  p->n_layers = n;
  for (int i = 0; i < MLSW_MAX_LAYERS; ++i)
    for (int k = 0; k < MLSW_MAX_LAYERS; ++k) p->spread[i][k] = 0.0;
  // Eq. (spreading_parameters)
  for (int i = 0; i < n; ++i)
    for (int k = 1; k <= n - i; ++k) {
      double s;
      if (k == 1)
        s = g[i * G + i + 2] - g[i * G + i + 1] - g[(i + 1) * G + i + 2];
      else
        s = g[i * G + i + k + 1] + g[(i + 1) * G + i + k] - g[i * G + i + k] -
            g[(i + 1) * G + i + k + 1];
      p->spread[i][k - 1] = s;
    }
  for (int i = 1; i <= n; ++i) p->gamma[i - 1] = g[i * G + i + 1];
  return MLSW_OK;
}

int mlswlbm_check_params(const mlsw_params* p) {
  if (!p) return MLSW_ERR_ARG;
  const int n = p->n_layers;
  if (n < 1 || n > MLSW_MAX_LAYERS) return MLSW_ERR_ARG;
  if (p->lattice != MLSW_D1Q3 && p->lattice != MLSW_D2Q9) return MLSW_ERR_ARG;
  if (p->nx < 1 || p->ny < 1) return MLSW_ERR_ARG;
  if (p->lattice == MLSW_D1Q3 && p->ny != 1) return MLSW_ERR_ARG;
  const double cells = (double)p->nx * p->ny * n * Qof(p->lattice);
  if (cells > 4.0e9) return MLSW_ERR_ARG;  // 32-bit tile indexing limit, 16 GB per buffer
  if (!std::isfinite(p->tau) || !(p->tau > 0.5)) return MLSW_ERR_ARG;
  if (!finite_pos(p->hstar)) return MLSW_ERR_ARG;
  if (p->wet_kind != 0 && p->wet_kind != 1) return MLSW_ERR_ARG;
  if (p->wet_kind == 0 && (p->wet_m < 1 || p->wet_n <= p->wet_m || p->wet_n > 64))
    return MLSW_ERR_ARG;
  if (p->wet_kind == 1 && !finite_pos(p->wet_kappa)) return MLSW_ERR_ARG;
  if (!std::isfinite(p->sub_amp)) return MLSW_ERR_ARG;
  if (p->sub_amp != 0.0 && p->lattice == MLSW_D1Q3 && p->sub_ky != 0) return MLSW_ERR_ARG;
  for (int i = 0; i < n; ++i) {
    if (!finite_pos(p->mu[i])) return MLSW_ERR_ARG;
    if (!std::isfinite(p->beta[i]) || p->beta[i] < 0.0) return MLSW_ERR_ARG;
    if (!std::isfinite(p->gamma[i])) return MLSW_ERR_ARG;
    for (int k = 1; k <= n - i; ++k)
      if (!std::isfinite(p->spread[i][k - 1])) return MLSW_ERR_ARG;
  }
  return MLSW_OK;
}

void mlswlbm_destroy(mlsw_handle* h) {
  if (!h) return;
  cudaStreamSynchronize(h->stream);
  cudaFree(h->f[0]);
  cudaFree(h->f[1]);
  cudaFree(h->hbuf);
  cudaFree(h->status);
  cudaFree(h->partials);
  cudaFree(h->dout);
  if (h->status_host) cudaFreeHost(h->status_host);
  delete h;
}

int mlswlbm_create(const mlsw_params* p, const float* h_init, void* stream, mlsw_handle** out) {
  if (!out) return MLSW_ERR_ARG;
  *out = nullptr;
  if (!p) return MLSW_ERR_ARG;
  KParams kp;
  mlsw::KShift sh;
  const int rc0 = prepare_instance(*p, h_init, kp, sh);
  if (rc0 != MLSW_OK) return rc0;
  const int n = p->n_layers;
  const long ncell = (long)p->nx * p->ny;
  int rc = MLSW_OK;

  mlsw_handle* h = new (std::nothrow) mlsw_handle;
  if (!h) return MLSW_ERR_NOMEM;
  std::memset(h, 0, sizeof(*h));
  h->p = *p;
  h->kp = kp;
  h->sh = sh;
  h->Q = Qof(p->lattice);
  h->ncell = ncell;
  h->flen = (size_t)n * h->Q * h->kp.L.plane;
  h->stream = (cudaStream_t)stream;
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
    delete h;
    return MLSW_ERR_CUDA;
  }
  h->num_sms = sms > 0 ? sms : 1;
  h->nblk_diag = 2 * h->num_sms;
  {
    // a buffer that fits in 90 % of the L2 is kept there between steps
    int l2 = 0;
    if (cudaDeviceGetAttribute(&l2, cudaDevAttrL2CacheSize, dev) != cudaSuccess) l2 = 0;
    const double buf = (double)h->flen * sizeof(float);
    h->kp.l2_policy = (l2 > 0 && buf <= 0.9 * l2) ? mlsw::kL2Resident : mlsw::kL2Stream;
  }
  if (!(p->flags & MLSW_FLAG_NO_PERSISTENT)) {
    int optin = 0;
    const size_t need = mlsw::step_persistent_smem(n, p->lattice, p->nx);
    if (need > 0 &&
        cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) == cudaSuccess &&
        need <= (size_t)optin)
      h->psmem = need;
  }
  bool ok = cudaMalloc(&h->f[0], h->flen * sizeof(float)) == cudaSuccess &&
            cudaMalloc(&h->f[1], h->flen * sizeof(float)) == cudaSuccess &&
            cudaMalloc(&h->hbuf, (size_t)n * ncell * sizeof(float)) == cudaSuccess &&
            cudaMalloc(&h->status, 4 * sizeof(int)) == cudaSuccess &&
            cudaMalloc(&h->partials, (size_t)h->nblk_diag * (n + 2) * sizeof(double)) ==
                cudaSuccess &&
            cudaMalloc(&h->dout, (size_t)(n + 2) * sizeof(double)) == cudaSuccess &&
            cudaHostAlloc(&h->status_host, sizeof(int), cudaHostAllocMapped) == cudaSuccess &&
            cudaHostGetDevicePointer(&h->status_mirror, h->status_host, 0) == cudaSuccess;
  if (!ok) {
    cudaGetLastError();
    mlswlbm_destroy(h);
    return MLSW_ERR_NOMEM;
  }
  // zero padding: cells outside the real domain and its ghost ring are read
  // by edge tiles but never feed a real cell
  if (cudaMemsetAsync(h->status, 0, 4 * sizeof(int), h->stream) != cudaSuccess ||
      cudaMemsetAsync(h->f[0], 0, h->flen * sizeof(float), h->stream) != cudaSuccess ||
      cudaMemsetAsync(h->f[1], 0, h->flen * sizeof(float), h->stream) != cudaSuccess) {
    mlswlbm_destroy(h);
    return MLSW_ERR_CUDA;
  }
  if (p->lattice == MLSW_D2Q9) {
    const int bc = mlsw::step_tile_cols(p->lattice) + 8;
    const int br = mlsw::step_tile_rows(n, p->lattice) + 4;
    if (!make_tile_map(&h->map[0], h->f[0], h->kp.L, n * h->Q, bc, br) ||
        !make_tile_map(&h->map[1], h->f[1], h->kp.L, n * h->Q, bc, br)) {
      mlswlbm_destroy(h);
      return MLSW_ERR_CUDA;
    }
  }
  rc = mlswlbm_set_heights(h, h_init);
  if (rc == MLSW_OK && cudaStreamSynchronize(h->stream) != cudaSuccess) rc = MLSW_ERR_CUDA;
  if (rc != MLSW_OK) {
    mlswlbm_destroy(h);
    return rc;
  }
  *out = h;
  return MLSW_OK;
}

int mlswlbm_set_heights(mlsw_handle* h, const float* h_in) {
  if (!h || !h_in) return MLSW_ERR_ARG;
  // page-locked heights are read by the init kernel in place; others are
  // copied to the device first
  const float* src = static_cast<const float*>(mapped_host_ptr(h_in));
  if (!src) {
    const size_t bytes = (size_t)h->p.n_layers * h->ncell * sizeof(float);
    CU(cudaMemcpyAsync(h->hbuf, h_in, bytes, cudaMemcpyHostToDevice, h->stream));
    src = h->hbuf;
  }
  CU(mlsw::launch_init(h->Q, h->p.n_layers, h->kp.L, h->p.lattice == MLSW_D2Q9, src,
                       h->f[h->cur], h->sh, h->status, h->stream));
  h->launches += 1;
  return MLSW_OK;
}

int mlswlbm_set_heights_device(mlsw_handle* h, const float* dev_in) {
  if (!h || !dev_in) return MLSW_ERR_ARG;
  CU(mlsw::launch_init(h->Q, h->p.n_layers, h->kp.L, h->p.lattice == MLSW_D2Q9, dev_in,
                       h->f[h->cur], h->sh, h->status, h->stream));
  h->launches += 1;
  return MLSW_OK;
}

int mlswlbm_step(mlsw_handle* h, long nsteps) {
  if (!h || nsteps < 0) return MLSW_ERR_ARG;
  mlsw::StepLaunch a;
  a.lattice = h->p.lattice;
  a.P = h->kp;
  a.status = h->status;
  a.sched = h->status + 1;
  a.num_sms = h->num_sms;
  a.reverse = 0;
  if (h->psmem) {
    // whole lattice in one CTA: chunks of steps per launch
    constexpr long kChunk = 16384;
    for (long left = nsteps; left > 0;) {
      const int chunk = (int)(left < kChunk ? left : kChunk);
      a.fin = h->f[h->cur];
      a.fout = h->f[h->cur ^ 1];
      CU(mlsw::launch_step_persistent(a, chunk, h->stream));
      h->launches += 1;
      h->cur ^= 1;
      left -= chunk;
    }
    return MLSW_OK;
  }
  for (long s = 0; s < nsteps; ++s) {
    a.fin = h->f[h->cur];
    a.fout = h->f[h->cur ^ 1];
    a.fin_map = &h->map[h->cur];
    // unless a whole buffer stays in the L2, steps from buffer 1 run their
    // tiles in reverse order: every step then begins with the rows its
    // predecessor wrote last, which the L2 still holds (the results do not
    // depend on the order)
    a.reverse = h->kp.l2_policy == mlsw::kL2Stream ? h->cur : 0;
    CU(mlsw::launch_step(a, h->stream));
    h->launches += 1;
    if (h->kp.tiny) {
      // a side below 4 cells: a real cell can have several ghost images,
      // which a separate pass refreshes
      CU(mlsw::launch_fill_ghosts(h->p.n_layers * h->Q, h->kp.L, h->p.lattice == MLSW_D2Q9,
                                  a.fout, h->stream));
      h->launches += 1;
    }
    h->cur ^= 1;
  }
  return MLSW_OK;
}

int mlswlbm_status(mlsw_handle* h) {
  if (!h) return MLSW_ERR_ARG;
  int flag = 0;
  CU(cudaMemcpyAsync(&flag, h->status, sizeof(int), cudaMemcpyDeviceToHost, h->stream));
  CU(cudaStreamSynchronize(h->stream));
  if (flag) {
    CU(cudaMemsetAsync(h->status, 0, sizeof(int), h->stream));
    return (flag & mlsw::kStatusTimeout) ? MLSW_ERR_TIMEOUT : MLSW_ERR_NONFINITE;
  }
  return MLSW_OK;
}

int mlswlbm_get_heights_device(mlsw_handle* h, float* dev_out) {
  if (!h || !dev_out) return MLSW_ERR_ARG;
  CU(mlsw::launch_heights(h->Q, h->p.n_layers, h->kp.L, h->f[h->cur], h->sh, dev_out,
                          h->stream));
  h->launches += 1;
  return MLSW_OK;
}

int mlswlbm_get_heights(mlsw_handle* h, float* out) {
  if (!h || !out) return MLSW_ERR_ARG;
  // page-locked output is written by the read-out kernel in place; the
  // kernel also mirrors the status word to the host, so one
  // synchronisation serves both
  float* mapped = static_cast<float*>(const_cast<void*>(mapped_host_ptr(out)));
  CU(mlsw::launch_heights(h->Q, h->p.n_layers, h->kp.L, h->f[h->cur], h->sh,
                          mapped ? mapped : h->hbuf, h->stream, h->status, h->status_mirror));
  h->launches += 1;
  if (!mapped) {
    const size_t bytes = (size_t)h->p.n_layers * h->ncell * sizeof(float);
    CU(cudaMemcpyAsync(out, h->hbuf, bytes, cudaMemcpyDeviceToHost, h->stream));
  }
  CU(cudaStreamSynchronize(h->stream));
  const int flag = *static_cast<volatile int*>(h->status_host);
  if (!flag) return MLSW_OK;
  return mlswlbm_status(h);  // reports the flag and clears it
}

int mlswlbm_get_state(mlsw_handle* h, float* f_out) {
  if (!h || !f_out) return MLSW_ERR_ARG;
  const int n = h->p.n_layers;
  const size_t plane = (size_t)h->ncell;
  // rest planes H_i + g_0 into the height buffer, all planes raw to the host,
  // then the rest planes over their raw copies
  CU(mlsw::launch_rest_planes(h->Q, n, h->kp.L, h->f[h->cur], h->sh, h->hbuf, h->stream));
  h->launches += 1;
  CU(copy_planes(h, f_out, h->f[h->cur], true));
  for (int i = 0; i < n; ++i)
    CU(cudaMemcpyAsync(f_out + (size_t)i * h->Q * plane, h->hbuf + (size_t)i * plane,
                       plane * sizeof(float), cudaMemcpyDeviceToHost, h->stream));
  CU(cudaStreamSynchronize(h->stream));
  return MLSW_OK;
}

int mlswlbm_set_state(mlsw_handle* h, const float* f_in) {
  if (!h || !f_in) return MLSW_ERR_ARG;
  CU(copy_planes(h, const_cast<float*>(f_in), h->f[h->cur], false));
  CU(mlsw::launch_shift(h->Q, h->p.n_layers, h->kp.L, h->f[h->cur], h->sh, -1.f, h->stream));
  CU(mlsw::launch_fill_ghosts(h->p.n_layers * h->Q, h->kp.L, h->p.lattice == MLSW_D2Q9,
                              h->f[h->cur], h->stream));
  h->launches += 2;
  CU(cudaStreamSynchronize(h->stream));
  return MLSW_OK;
}

int mlswlbm_save_state(mlsw_handle* h, float* H_out, float* g_out) {
  if (!h || !H_out || !g_out) return MLSW_ERR_ARG;
  for (int i = 0; i < h->p.n_layers; ++i) H_out[i] = h->sh.H[i];
  CU(copy_planes(h, g_out, h->f[h->cur], true));
  CU(cudaStreamSynchronize(h->stream));
  return MLSW_OK;
}

int mlswlbm_load_state(mlsw_handle* h, const float* H_in, const float* g_in) {
  if (!h || !H_in || !g_in) return MLSW_ERR_ARG;
  for (int i = 0; i < h->p.n_layers; ++i)
    if (!std::isfinite(H_in[i])) return MLSW_ERR_ARG;
  CU(cudaStreamSynchronize(h->stream));
  set_shift(h, H_in);
  CU(copy_planes(h, const_cast<float*>(g_in), h->f[h->cur], false));
  CU(mlsw::launch_fill_ghosts(h->p.n_layers * h->Q, h->kp.L, h->p.lattice == MLSW_D2Q9,
                              h->f[h->cur], h->stream));
  h->launches += 1;
  CU(cudaStreamSynchronize(h->stream));
  return MLSW_OK;
}

int mlswlbm_get_diagnostics(mlsw_handle* h, double* mass, double* kinetic, double* hmin) {
  if (!h) return MLSW_ERR_ARG;
  const int n = h->p.n_layers;
  CU(mlsw::launch_diagnostics(h->p.lattice, n, h->kp.L, h->f[h->cur], h->sh, h->partials,
                              h->nblk_diag, h->dout, h->stream));
  h->launches += 2;
  double res[MLSW_MAX_LAYERS + 2];
  CU(cudaMemcpyAsync(res, h->dout, (size_t)(n + 2) * sizeof(double), cudaMemcpyDeviceToHost,
                     h->stream));
  CU(cudaStreamSynchronize(h->stream));
  if (mass)
    for (int i = 0; i < n; ++i) mass[i] = res[i];
  if (kinetic) *kinetic = res[n];
  if (hmin) *hmin = res[n + 1];
  return mlswlbm_status(h);
}

int mlswlbm_get_free_energy(mlsw_handle* h, double* F) {
  if (!h || !F) return MLSW_ERR_ARG;
  const mlsw_params& p = h->p;
  mlsw::FreeEnergyParams E;
  std::memset(&E, 0, sizeof(E));
  E.n = p.n_layers;
  E.lattice = p.lattice;
  E.nx = p.nx;
  E.ny = p.ny;
  for (int i = 0; i < p.n_layers; ++i) {
    E.gamma[i] = p.gamma[i];
    for (int k = 1; k <= p.n_layers - i; ++k) E.S[i][k - 1] = p.spread[i][k - 1];
  }
  E.hstar = p.hstar;
  E.nw = p.wet_n;
  E.mw = p.wet_m;
  E.wet_kind = p.wet_kind;
  E.kappa = p.wet_kappa;
  E.sub_amp = p.sub_amp;
  E.sub_kx = p.sub_kx;
  E.sub_ky = p.sub_ky;
  CU(mlsw::launch_heights(h->Q, p.n_layers, h->kp.L, h->f[h->cur], h->sh, h->hbuf, h->stream));
  CU(mlsw::launch_free_energy(E, h->hbuf, h->partials, h->nblk_diag, h->dout, h->stream));
  h->launches += 3;
  CU(cudaMemcpyAsync(F, h->dout, sizeof(double), cudaMemcpyDeviceToHost, h->stream));
  return mlswlbm_status(h);
}

int mlswlbm_get_spectrum(mlsw_handle* h, int nbins, double* out) {
  if (!h || !out || nbins < 1) return MLSW_ERR_ARG;
  const mlsw_params& p = h->p;
  if (!mlsw::spectrum_supported(p.nx, p.ny, nbins)) return MLSW_ERR_UNSUPPORTED;
  const int n = p.n_layers;
  float2* work = nullptr;
  double* bins = nullptr;
  unsigned long long* counts = nullptr;
  cudaStream_t st = h->stream;
  const size_t nwork = (size_t)n * p.nx * p.ny;
  bool ok = cudaMallocAsync(&work, nwork * sizeof(float2), st) == cudaSuccess &&
            cudaMallocAsync(&bins, (size_t)n * nbins * sizeof(double), st) == cudaSuccess &&
            cudaMallocAsync(&counts, (size_t)nbins * sizeof(unsigned long long), st) == cudaSuccess;
  if (!ok) {
    cudaGetLastError();
    if (work) cudaFreeAsync(work, st);
    if (bins) cudaFreeAsync(bins, st);
    if (counts) cudaFreeAsync(counts, st);
    return MLSW_ERR_NOMEM;
  }
  std::vector<double> hb((size_t)n * nbins);
  std::vector<unsigned long long> hc(nbins);
  ok = cudaMemsetAsync(bins, 0, (size_t)n * nbins * sizeof(double), st) == cudaSuccess &&
       cudaMemsetAsync(counts, 0, (size_t)nbins * sizeof(unsigned long long), st) == cudaSuccess &&
       mlsw::launch_spectrum(h->Q, n, h->kp.L, h->f[h->cur], nbins, work, bins, counts, st) ==
           cudaSuccess &&
       cudaMemcpyAsync(hb.data(), bins, hb.size() * sizeof(double), cudaMemcpyDeviceToHost, st) ==
           cudaSuccess &&
       cudaMemcpyAsync(hc.data(), counts, hc.size() * sizeof(unsigned long long),
                       cudaMemcpyDeviceToHost, st) == cudaSuccess;
  cudaFreeAsync(work, st);
  cudaFreeAsync(bins, st);
  cudaFreeAsync(counts, st);
  if (!ok || cudaStreamSynchronize(st) != cudaSuccess) {
    cudaGetLastError();
    return MLSW_ERR_CUDA;
  }
  h->launches += 2;
  for (int i = 0; i < n; ++i)
    for (int b = 0; b < nbins; ++b)
      out[(size_t)i * nbins + b] = hc[b] ? hb[(size_t)i * nbins + b] / (double)hc[b] : 0.0;
  return mlswlbm_status(h);
}

int mlswlbm_get_radial_profile(mlsw_handle* h, double cx, double cy, int nbins, double* out,
                               long long* counts) {
  if (!h || !out || nbins < 1 || !std::isfinite(cx) || !std::isfinite(cy)) return MLSW_ERR_ARG;
  if (h->p.lattice != MLSW_D2Q9) return MLSW_ERR_UNSUPPORTED;
  const int n = h->p.n_layers;
  const size_t nsum = (size_t)(n + 1) * nbins;
  cudaStream_t st = h->stream;
  double* sums = nullptr;
  unsigned long long* cnt = nullptr;
  bool ok = cudaMallocAsync(&sums, nsum * sizeof(double), st) == cudaSuccess &&
            cudaMallocAsync(&cnt, (size_t)nbins * sizeof(unsigned long long), st) == cudaSuccess;
  if (!ok) {
    cudaGetLastError();
    if (sums) cudaFreeAsync(sums, st);
    if (cnt) cudaFreeAsync(cnt, st);
    return MLSW_ERR_NOMEM;
  }
  mlsw::ProfileParams A;
  A.cx = cx;
  A.cy = cy;
  A.nbins = nbins;
  A.sub_amp = h->p.sub_amp;
  A.sub_kx = h->p.sub_kx;
  A.sub_ky = h->p.sub_ky;
  std::vector<double> hs(nsum);
  std::vector<unsigned long long> hc(nbins);
  ok = cudaMemsetAsync(sums, 0, nsum * sizeof(double), st) == cudaSuccess &&
       cudaMemsetAsync(cnt, 0, (size_t)nbins * sizeof(unsigned long long), st) == cudaSuccess &&
       mlsw::launch_radial_profile(h->Q, n, h->kp.L, h->f[h->cur], h->sh, A, sums, cnt, st) ==
           cudaSuccess &&
       cudaMemcpyAsync(hs.data(), sums, nsum * sizeof(double), cudaMemcpyDeviceToHost, st) ==
           cudaSuccess &&
       cudaMemcpyAsync(hc.data(), cnt, (size_t)nbins * sizeof(unsigned long long),
                       cudaMemcpyDeviceToHost, st) == cudaSuccess;
  cudaFreeAsync(sums, st);
  cudaFreeAsync(cnt, st);
  if (!ok || cudaStreamSynchronize(st) != cudaSuccess) {
    cudaGetLastError();
    return MLSW_ERR_CUDA;
  }
  h->launches += 1;
  for (int m = 0; m <= n; ++m)
    for (int b = 0; b < nbins; ++b)
      out[(size_t)m * nbins + b] = hc[b] ? hs[(size_t)m * nbins + b] / (double)hc[b] : 0.0;
  if (counts)
    for (int b = 0; b < nbins; ++b) counts[b] = (long long)hc[b];
  return mlswlbm_status(h);
}

namespace {

// relative volume difference between a radial profile and the circular arc
// of angle theta through its apex prof[0] meeting the level base
double cap_error(const double* prof, const double* area, int nbins, double base, double theta) {
  const double rc = (prof[0] - base) / (1.0 - std::cos(theta));
  double num = 0.0, den = 0.0;
  for (int b = 0; b < nbins; ++b) {
    const double r = b + 0.5;
    const double inside = std::sqrt(std::max(rc * rc - r * r, 0.0));
    const double arc = base + std::max(0.0, inside - rc * std::cos(theta));
    num += area[b] * std::fabs(prof[b] - arc);
    den += area[b] * (prof[b] - base);
  }
  return num / den;
}

}  // namespace

int mlswlbm_fit_cap_angle(const double* prof, const double* area, int nbins, double base,
                          double* theta_deg, double* err) {
  if (!prof || !area || nbins < 2 || !theta_deg || !(prof[0] > base)) return MLSW_ERR_ARG;
  constexpr double kDeg = 3.14159265358979323846 / 180.0;
  // scan 0.5 .. 60 degrees in 0.05-degree steps, then golden section between
  // the neighbours of the best step
  const int nscan = 1190;
  int best = 0;
  double ebest = 0.0;
  for (int j = 0; j < nscan; ++j) {
    const double e = cap_error(prof, area, nbins, base, (0.5 + 0.05 * j) * kDeg);
    if (j == 0 || e < ebest) {
      ebest = e;
      best = j;
    }
  }
  double a = (0.5 + 0.05 * std::max(best - 1, 0)) * kDeg;
  double b = (0.5 + 0.05 * std::min(best + 1, nscan - 1)) * kDeg;
  const double g = (std::sqrt(5.0) - 1.0) / 2.0;
  double c = b - g * (b - a), d = a + g * (b - a);
  for (int it = 0; it < 40; ++it) {
    if (cap_error(prof, area, nbins, base, c) < cap_error(prof, area, nbins, base, d))
      b = d;
    else
      a = c;
    c = b - g * (b - a);
    d = a + g * (b - a);
  }
  const double t = 0.5 * (a + b);
  *theta_deg = t / kDeg;
  if (err) *err = cap_error(prof, area, nbins, base, t);
  return MLSW_OK;
}

int mlswlbm_step_until(mlsw_handle* h, long max_steps, long check_every, double ke_threshold,
                       long* steps_done, double* kinetic) {
  if (!h || max_steps < 0 || check_every < 1) return MLSW_ERR_ARG;
  // a run starts from rest (zero kinetic energy), so the criterion is only
  // tested after steps have been taken
  long done = 0;
  double ke = 0.0;
  int rc = MLSW_OK;
  while (done < max_steps) {
    const long chunk = std::min(check_every, max_steps - done);
    rc = mlswlbm_step(h, chunk);
    if (rc != MLSW_OK) break;
    done += chunk;
    rc = mlswlbm_get_diagnostics(h, nullptr, &ke, nullptr);
    if (rc != MLSW_OK || ke < ke_threshold) break;
  }
  if (steps_done) *steps_done = done;
  if (kinetic) *kinetic = ke;
  return rc;
}

int mlswlbm_selftest_bounded_wait(int arrive, unsigned limit, void* stream) {
  if (limit == 0 || limit > (1u << 22)) return MLSW_ERR_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  int* d = nullptr;
  if (cudaMalloc(&d, sizeof(int)) != cudaSuccess) {
    cudaGetLastError();
    return MLSW_ERR_NOMEM;
  }
  int flag = 0;
  bool ok = cudaMemsetAsync(d, 0, sizeof(int), st) == cudaSuccess &&
            mlsw::launch_wait_selftest(arrive, limit, d, st) == cudaSuccess &&
            cudaMemcpyAsync(&flag, d, sizeof(int), cudaMemcpyDeviceToHost, st) == cudaSuccess &&
            cudaStreamSynchronize(st) == cudaSuccess;
  cudaFree(d);
  if (!ok) return MLSW_ERR_CUDA;
  return (flag & mlsw::kStatusTimeout) ? MLSW_ERR_TIMEOUT : MLSW_OK;
}

int mlswlbm_debug_bounds_violations(unsigned long long* count) {
  if (!count) return MLSW_ERR_ARG;
#ifdef MLSW_DEBUG
  if (cudaDeviceSynchronize() != cudaSuccess) return MLSW_ERR_CUDA;
  const unsigned parts[4] = {mlsw::bounds_violations_step(), mlsw::bounds_violations_aux(),
                             mlsw::bounds_violations_analysis(),
                             mlsw::bounds_violations_batch()};
  unsigned long long total = 0;
  for (unsigned v : parts) {
    if (v == ~0u) return MLSW_ERR_CUDA;
    total += v;
  }
  *count = total;
  return MLSW_OK;
#else
  *count = 0;
  return MLSW_ERR_UNSUPPORTED;
#endif
}

int mlswlbm_set_stream(mlsw_handle* h, void* stream) {
  if (!h) return MLSW_ERR_ARG;
  h->stream = (cudaStream_t)stream;
  return MLSW_OK;
}

long mlswlbm_launch_count(const mlsw_handle* h) { return h ? h->launches : -1; }

int mlswlbm_friction_eval(const mlsw_params* p, long ncell, const float* hh, const float* Jx,
                          const float* Jy, float* Rx, float* Ry, void* stream) {
  if (!p || ncell < 0 || !hh || !Jx || !Rx) return MLSW_ERR_ARG;
  const int n = p->n_layers;
  if (n < 1 || n > MLSW_MAX_LAYERS) return MLSW_ERR_ARG;
  for (int i = 0; i < n; ++i)
    if (!finite_pos(p->mu[i]) || !std::isfinite(p->beta[i]) || p->beta[i] < 0.0)
      return MLSW_ERR_ARG;
  if (ncell == 0) return MLSW_OK;
  KParams k;
  std::memset(&k, 0, sizeof(k));
  k.n = n;
  for (int i = 0; i < n; ++i) {
    k.mu_inv[i] = (float)(1.0 / p->mu[i]);
    k.beta[i] = (float)p->beta[i];
  }
  CU(mlsw::launch_friction_eval(k, ncell, hh, Jx, Jy, Rx, Ry, (cudaStream_t)stream));
  return MLSW_OK;
}

}  // extern "C"
