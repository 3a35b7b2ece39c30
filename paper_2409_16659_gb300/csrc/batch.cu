// batch.cu -- batches of independent D2Q9 lattices (the C ABI's
// mlswlbm_batch_*): one population arena, per-instance device descriptors,
// one tile table in which the instances that share layer count, kernel mode
// and tile height (a group) have a contiguous range, one persistent launch
// per step over the whole table (batch_kernels.cu), captured once in a CUDA
// graph, and a timing autotuner for the tile height of every class of
// alike instances.
#include <algorithm>
#include <cstring>
#include <map>
#include <new>
#include <tuple>
#include <vector>

#include "../../include/mlswlbm.h"
#include "host.h"
#include "kernels.h"
#include "physics.cuh"

using mlsw::BatchInst;
using mlsw::KParams;

namespace {

constexpr int kQ = 9;
constexpr int kMaxGroups = mlsw::kBatchKinds;  // n x mode x variant

struct Group {
  int n, mode, variant;
  int offset, ntiles;  // slice of the tile table
};

}  // namespace

struct mlsw_batch {
  int count;
  std::vector<BatchInst> hinst;  // host copies of the descriptors
  std::vector<int> variant;      // tile-height variant of every instance
  // instances the step advances (mlswlbm_batch_select; all at create) and,
  // for one left out, the buffer index that holds its state
  std::vector<char> selected;
  std::vector<int> home;
  std::vector<Group> groups;
  BatchInst* dinst;
  int2* dtable;  // the tile table, sorted by kind
  float* arena;
  int* dstatus;  // [0] error bits, [1], [2] the step kernel's tile counters
  float* hbuf;   // heights of the largest instance (upload, read-out)
  int* dk;       // 2 count mode numbers
  double* dmode; // 2 kMaxLayers count doubles
  int cur;
  cudaStream_t stream;   // the caller's stream
  cudaStream_t cap;      // private stream the step graph is captured on
  cudaGraphExec_t gexec[2];  // one step from buffer 0, from buffer 1
  long launches;
  int num_sms;
};

namespace {

#define CUB(call)                                    \
  do {                                               \
    if ((call) != cudaSuccess) return MLSW_ERR_CUDA; \
  } while (0)

int tiles_of(const BatchInst& b, int variant) {
  const int ty = mlsw::batch_tile_rows(variant);
  return b.ntx * ((b.P.ny + ty - 1) / ty);
}

// the buffer that holds instance j's state now
int state_buffer(const mlsw_batch* b, int j) { return b->selected[j] ? b->cur : b->home[j]; }

// Moves every left-out instance whose state sits in the other buffer to the
// current one by swapping its two buffers (and their tensor maps) in its
// descriptor, so that every instance's state is in buffer cur.
int align_buffers(mlsw_batch* b) {
  bool changed = false;
  for (int j = 0; j < b->count; ++j) {
    if (b->selected[j] || b->home[j] == b->cur) continue;
    BatchInst& bi = b->hinst[j];
    std::swap(bi.f[0], bi.f[1]);
    for (int v = 0; v < mlsw::kBatchVariants; ++v) std::swap(bi.map[v][0], bi.map[v][1]);
    b->home[j] = b->cur;
    changed = true;
  }
  // pageable source: the copy is staged before the call returns
  if (changed)
    CUB(cudaMemcpyAsync(b->dinst, b->hinst.data(), (size_t)b->count * sizeof(BatchInst),
                        cudaMemcpyHostToDevice, b->stream));
  return MLSW_OK;
}

// (re)initialise every instance from its heights: f = f_eq(h, U = 0)
int init_all(mlsw_batch* b, const float* const* h_init) {
  for (int j = 0; j < b->count; ++j) {
    const KParams& P = b->hinst[j].P;
    const size_t bytes = (size_t)P.n * P.nx * P.ny * sizeof(float);
    mlsw::KShift sh;
    for (int i = 0; i < mlsw::kMaxLayers; ++i) sh.H[i] = P.H[i];
    CUB(cudaMemcpyAsync(b->hbuf, h_init[j], bytes, cudaMemcpyHostToDevice, b->stream));
    CUB(mlsw::launch_init(kQ, P.n, P.L, true, b->hbuf, b->hinst[j].f[0], sh, b->dstatus,
                          b->stream));
    b->launches += 1;
    b->home[j] = 0;
  }
  b->cur = 0;
  return MLSW_OK;
}

// ends of the groups' ranges of the tile table, per kind (the groups come
// in kind order: the map below orders them by (n, mode, variant))
mlsw::BatchEnds ends_of(const mlsw_batch* b) {
  mlsw::BatchEnds E;
  int g = 0, end = 0;
  for (int k = 0; k < mlsw::kBatchKinds; ++k) {
    if (g < (int)b->groups.size()) {
      const Group& G = b->groups[g];
      if (mlsw::batch_kind(G.n, G.mode, G.variant) == k) {
        end = G.offset + G.ntiles;
        ++g;
      }
    }
    E.end[k] = end;
  }
  return E;
}

// the tile table of the groups for the current variant choice, sorted by
// kind
int build_groups(mlsw_batch* b) {
  std::map<std::tuple<int, int, int>, std::vector<int>> members;
  for (int j = 0; j < b->count; ++j) {
    if (!b->selected[j]) continue;
    const KParams& P = b->hinst[j].P;
    members[std::make_tuple(P.n, mlsw::step_mode(P), b->variant[j])].push_back(j);
  }
  std::vector<int2> table;
  b->groups.clear();
  for (auto& kv : members) {
    Group g;
    g.n = std::get<0>(kv.first);
    g.mode = std::get<1>(kv.first);
    g.variant = std::get<2>(kv.first);
    g.offset = (int)table.size();
    for (int j : kv.second) {
      const int nt = tiles_of(b->hinst[j], g.variant);
      for (int t = 0; t < nt; ++t) table.push_back(make_int2(j, t));
    }
    g.ntiles = (int)table.size() - g.offset;
    b->groups.push_back(g);
  }
  if (b->groups.size() > (size_t)kMaxGroups) return MLSW_ERR_UNSUPPORTED;
  // the ranges must cover the table in kind order
  if (ends_of(b).end[mlsw::kBatchKinds - 1] != (int)table.size()) return MLSW_ERR_UNSUPPORTED;
  if (b->dtable) cudaFree(b->dtable);
  b->dtable = nullptr;
  if (cudaMalloc(&b->dtable, std::max<size_t>(1, table.size()) * sizeof(int2)) != cudaSuccess)
    return MLSW_ERR_NOMEM;
  CUB(cudaMemcpy(b->dtable, table.data(), table.size() * sizeof(int2), cudaMemcpyHostToDevice));
  return MLSW_OK;
}

// the step launch over the groups' table, from buffer cur
mlsw::BatchLaunch step_launch(const mlsw_batch* b, int cur) {
  mlsw::BatchLaunch a;
  a.inst = b->dinst;
  a.table = b->dtable;
  a.ends = ends_of(b);
  a.cur = cur;
  a.status = b->dstatus;
  a.sched = b->dstatus + 1;
  a.num_sms = b->num_sms;
  return a;
}

// Captures one step (from buffer cur) as a graph of its one launch.
int capture_step(mlsw_batch* b, int cur, cudaGraphExec_t* exec) {
  // configure the kernel (shared-memory limit) outside capture
  mlsw::BatchLaunch a = step_launch(b, cur);
  mlsw::BatchLaunch none = a;
  for (int k = 0; k < mlsw::kBatchKinds; ++k) none.ends.end[k] = 0;
  CUB(mlsw::launch_batch_step(none, b->cap));
  CUB(cudaStreamBeginCapture(b->cap, cudaStreamCaptureModeThreadLocal));
  const bool ok = mlsw::launch_batch_step(a, b->cap) == cudaSuccess;
  cudaGraph_t graph = nullptr;
  const cudaError_t e = cudaStreamEndCapture(b->cap, &graph);
  if (!ok || e != cudaSuccess || !graph) {
    if (graph) cudaGraphDestroy(graph);
    cudaGetLastError();
    return MLSW_ERR_CUDA;
  }
  const cudaError_t ei = cudaGraphInstantiate(exec, graph, 0);
  cudaGraphDestroy(graph);
  return ei == cudaSuccess ? MLSW_OK : MLSW_ERR_CUDA;
}

// Timing autotuner: for every class of instances with the same n (<= 3),
// mode and size, time a few steps of the class alone with 16-row and with
// 8-row tiles and keep the faster. The steps change the states, which the
// caller resets afterwards.
int autotune(mlsw_batch* b) {
  std::map<std::tuple<int, int, int, int>, std::vector<int>> classes;
  for (int j = 0; j < b->count; ++j) {
    const KParams& P = b->hinst[j].P;
    if (P.n <= 3) classes[std::make_tuple(P.n, mlsw::step_mode(P), P.nx, P.ny)].push_back(j);
  }
  cudaEvent_t e0, e1;
  CUB(cudaEventCreate(&e0));
  if (cudaEventCreate(&e1) != cudaSuccess) {
    cudaEventDestroy(e0);
    return MLSW_ERR_CUDA;
  }
  int rc = MLSW_OK;
  int2* dt = nullptr;
  for (auto& kv : classes) {
    const int n = std::get<0>(kv.first), mode = std::get<1>(kv.first);
    float best = 0.f;
    int best_v = 0;
    for (int v = 0; v < mlsw::kBatchVariants && rc == MLSW_OK; ++v) {
      std::vector<int2> table;
      for (int j : kv.second)
        for (int t = 0; t < tiles_of(b->hinst[j], v); ++t) table.push_back(make_int2(j, t));
      if (dt) cudaFree(dt);
      dt = nullptr;
      if (cudaMalloc(&dt, table.size() * sizeof(int2)) != cudaSuccess ||
          cudaMemcpy(dt, table.data(), table.size() * sizeof(int2), cudaMemcpyHostToDevice) !=
              cudaSuccess) {
        rc = MLSW_ERR_CUDA;
        break;
      }
      mlsw::BatchLaunch a;
      a.inst = b->dinst;
      a.table = dt;
      // one range: kinds before this one end at 0, the others at the end
      const int kind = mlsw::batch_kind(n, mode, v);
      for (int k = 0; k < mlsw::kBatchKinds; ++k) a.ends.end[k] = k < kind ? 0 : (int)table.size();
      a.status = b->dstatus;
      a.sched = b->dstatus + 1;
      a.num_sms = b->num_sms;
      constexpr int kWarm = 2, kTimed = 6;
      float ms = 0.f;
      for (int s = 0; s < kWarm + kTimed && rc == MLSW_OK; ++s) {
        if (s == kWarm && cudaEventRecord(e0, b->stream) != cudaSuccess) rc = MLSW_ERR_CUDA;
        a.cur = s & 1;
        if (mlsw::launch_batch_step(a, b->stream) != cudaSuccess) rc = MLSW_ERR_CUDA;
        b->launches += 1;
      }
      if (rc == MLSW_OK && (cudaEventRecord(e1, b->stream) != cudaSuccess ||
                            cudaEventSynchronize(e1) != cudaSuccess ||
                            cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess))
        rc = MLSW_ERR_CUDA;
      if (rc == MLSW_OK && (v == 0 || ms < best)) {
        best = ms;
        best_v = v;
      }
    }
    if (rc != MLSW_OK) break;
    for (int j : kv.second) b->variant[j] = best_v;
  }
  if (dt) cudaFree(dt);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  return rc;
}

}  // namespace

extern "C" {

void mlswlbm_batch_destroy(mlsw_batch* b) {
  if (!b) return;
  if (b->cap) cudaStreamSynchronize(b->cap);
  cudaStreamSynchronize(b->stream);
  for (int k = 0; k < 2; ++k)
    if (b->gexec[k]) cudaGraphExecDestroy(b->gexec[k]);
  if (b->cap) cudaStreamDestroy(b->cap);
  cudaFree(b->dinst);
  cudaFree(b->dtable);
  cudaFree(b->arena);
  cudaFree(b->dstatus);
  cudaFree(b->hbuf);
  cudaFree(b->dk);
  cudaFree(b->dmode);
  delete b;
}

int mlswlbm_batch_create(int count, const mlsw_params* params, const float* const* h_init,
                         int flags, void* stream, mlsw_batch** out) {
  if (!out) return MLSW_ERR_ARG;
  *out = nullptr;
  if (count < 1 || !params || !h_init) return MLSW_ERR_ARG;
  mlsw_batch* b = new (std::nothrow) mlsw_batch();
  if (!b) return MLSW_ERR_NOMEM;
  b->count = count;
  b->stream = (cudaStream_t)stream;
  int rc = MLSW_OK;
  size_t arena_floats = 0, max_heights = 0;
  std::vector<size_t> off(count);
  try {
    b->hinst.resize(count);
    b->variant.resize(count);
    b->selected.assign(count, 1);
    b->home.assign(count, 0);
  } catch (...) {
    delete b;
    return MLSW_ERR_NOMEM;
  }
  for (int j = 0; j < count && rc == MLSW_OK; ++j) {
    if (params[j].lattice != MLSW_D2Q9) {
      rc = MLSW_ERR_UNSUPPORTED;
      break;
    }
    BatchInst& bi = b->hinst[j];
    std::memset(&bi, 0, sizeof(bi));
    mlsw::KShift sh;
    rc = mlsw_host::prepare_instance(params[j], h_init[j], bi.P, sh);
    if (rc != MLSW_OK) break;
    bi.ntx = (bi.P.nx + 31) / 32;
    const size_t flen = (size_t)bi.P.n * kQ * bi.P.L.plane;
    off[j] = arena_floats;
    arena_floats += 2 * ((flen + 63) / 64 * 64);  // two buffers, 256-byte aligned
    max_heights = std::max(max_heights, (size_t)bi.P.n * bi.P.nx * bi.P.ny);
    b->variant[j] = (flags & MLSW_BATCH_TILE8) || bi.P.n > 3 ? 1 : 0;
  }
  if (rc != MLSW_OK) {
    delete b;
    return rc;
  }
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
    delete b;
    return MLSW_ERR_CUDA;
  }
  b->num_sms = sms > 0 ? sms : 1;
  const int nstat = 3;
  bool ok = cudaMalloc(&b->arena, arena_floats * sizeof(float)) == cudaSuccess &&
            cudaMalloc(&b->dinst, (size_t)count * sizeof(BatchInst)) == cudaSuccess &&
            cudaMalloc(&b->dstatus, nstat * sizeof(int)) == cudaSuccess &&
            cudaMalloc(&b->hbuf, max_heights * sizeof(float)) == cudaSuccess &&
            cudaMalloc(&b->dk, 2 * (size_t)count * sizeof(int)) == cudaSuccess &&
            cudaMalloc(&b->dmode, 2 * (size_t)mlsw::kMaxLayers * count * sizeof(double)) ==
                cudaSuccess;
  if (!ok) {
    cudaGetLastError();
    mlswlbm_batch_destroy(b);
    return MLSW_ERR_NOMEM;
  }
  ok = cudaStreamCreateWithFlags(&b->cap, cudaStreamNonBlocking) == cudaSuccess;
  // zero padding (cells outside the real domains and their ghost rings are
  // read by edge tiles but feed no real cell) and the status words
  ok = ok && cudaMemsetAsync(b->dstatus, 0, nstat * sizeof(int), b->stream) == cudaSuccess &&
       cudaMemsetAsync(b->arena, 0, arena_floats * sizeof(float), b->stream) == cudaSuccess;
  for (int j = 0; j < count && ok; ++j) {
    BatchInst& bi = b->hinst[j];
    const size_t flen = (size_t)bi.P.n * kQ * bi.P.L.plane;
    bi.f[0] = b->arena + off[j];
    bi.f[1] = b->arena + off[j] + (flen + 63) / 64 * 64;
    for (int v = 0; v < mlsw::kBatchVariants && ok; ++v) {
      if (v == 0 && bi.P.n > 3) continue;  // 16-row tiles need n <= 3
      for (int k = 0; k < 2 && ok; ++k)
        ok = mlsw_host::make_tile_map(&bi.map[v][k], bi.f[k], bi.P.L, bi.P.n * kQ, 40,
                                      mlsw::batch_tile_rows(v) + 4);
    }
  }
  ok = ok && cudaMemcpy(b->dinst, b->hinst.data(), (size_t)count * sizeof(BatchInst),
                        cudaMemcpyHostToDevice) == cudaSuccess;
  if (!ok) {
    cudaGetLastError();
    mlswlbm_batch_destroy(b);
    return MLSW_ERR_CUDA;
  }
  rc = init_all(b, h_init);
  if (rc == MLSW_OK && (flags & MLSW_BATCH_AUTOTUNE) && !(flags & MLSW_BATCH_TILE8)) {
    rc = autotune(b);
    if (rc == MLSW_OK) rc = init_all(b, h_init);
  }
  if (rc == MLSW_OK) rc = build_groups(b);
  if (rc == MLSW_OK && cudaStreamSynchronize(b->stream) != cudaSuccess) rc = MLSW_ERR_CUDA;
  if (rc == MLSW_OK) rc = capture_step(b, 0, &b->gexec[0]);
  if (rc == MLSW_OK) rc = capture_step(b, 1, &b->gexec[1]);
  if (rc == MLSW_OK) {
    // a non-finite or non-positive height in h_init was flagged by init
    int flag = 0;
    if (cudaMemcpy(&flag, b->dstatus, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess)
      rc = MLSW_ERR_CUDA;
    else if (flag)
      rc = MLSW_ERR_ARG;
  }
  if (rc != MLSW_OK) {
    mlswlbm_batch_destroy(b);
    return rc;
  }
  *out = b;
  return MLSW_OK;
}

int mlswlbm_batch_step(mlsw_batch* b, long nsteps) {
  if (!b || nsteps < 0) return MLSW_ERR_ARG;
  if (b->groups.empty()) return MLSW_OK;  // no instance selected
  for (long s = 0; s < nsteps; ++s) {
    CUB(cudaGraphLaunch(b->gexec[b->cur], b->stream));
    b->launches += 1;
    b->cur ^= 1;
  }
  return MLSW_OK;
}

int mlswlbm_batch_status(mlsw_batch* b) {
  if (!b) return MLSW_ERR_ARG;
  int flag = 0;
  CUB(cudaMemcpyAsync(&flag, b->dstatus, sizeof(int), cudaMemcpyDeviceToHost, b->stream));
  CUB(cudaStreamSynchronize(b->stream));
  if (flag) {
    CUB(cudaMemsetAsync(b->dstatus, 0, sizeof(int), b->stream));
    return (flag & mlsw::kStatusTimeout) ? MLSW_ERR_TIMEOUT : MLSW_ERR_NONFINITE;
  }
  return MLSW_OK;
}

int mlswlbm_batch_get_heights(mlsw_batch* b, int index, float* out) {
  if (!b || !out || index < 0 || index >= b->count) return MLSW_ERR_ARG;
  const KParams& P = b->hinst[index].P;
  CUB(mlsw::launch_batch_heights(&b->hinst[index], state_buffer(b, index), b->hbuf, b->stream));
  b->launches += 1;
  CUB(cudaMemcpyAsync(out, b->hbuf, (size_t)P.n * P.nx * P.ny * sizeof(float),
                      cudaMemcpyDeviceToHost, b->stream));
  return mlswlbm_batch_status(b);
}

int mlswlbm_batch_get_heights_device(mlsw_batch* b, int index, float* dev_out) {
  if (!b || !dev_out || index < 0 || index >= b->count) return MLSW_ERR_ARG;
  CUB(mlsw::launch_batch_heights(&b->hinst[index], state_buffer(b, index), dev_out, b->stream));
  b->launches += 1;
  return MLSW_OK;
}

int mlswlbm_batch_set_heights_device(mlsw_batch* b, int index, const float* dev_in) {
  if (!b || !dev_in || index < 0 || index >= b->count) return MLSW_ERR_ARG;
  const KParams& P = b->hinst[index].P;
  mlsw::KShift sh;
  for (int i = 0; i < mlsw::kMaxLayers; ++i) sh.H[i] = P.H[i];
  CUB(mlsw::launch_init(kQ, P.n, P.L, true, dev_in, b->hinst[index].f[state_buffer(b, index)],
                        sh, b->dstatus, b->stream));
  b->launches += 1;
  return MLSW_OK;
}

int mlswlbm_batch_get_heights_device_many(mlsw_batch* b, int count, const int* indices,
                                          float* dev_out) {
  if (!b || count < 0 || (count > 0 && (!indices || !dev_out))) return MLSW_ERR_ARG;
  for (int k = 0; k < count; ++k)
    if (indices[k] < 0 || indices[k] >= b->count) return MLSW_ERR_ARG;
  size_t off = 0;
  for (int k = 0; k < count; ++k) {
    const int j = indices[k];
    const KParams& P = b->hinst[j].P;
    CUB(mlsw::launch_batch_heights(&b->hinst[j], state_buffer(b, j), dev_out + off, b->stream));
    b->launches += 1;
    off += (size_t)P.n * P.nx * P.ny;
  }
  return MLSW_OK;
}

int mlswlbm_batch_set_heights_device_many(mlsw_batch* b, int count, const int* indices,
                                          const float* dev_in) {
  if (!b || count < 0 || (count > 0 && (!indices || !dev_in))) return MLSW_ERR_ARG;
  for (int k = 0; k < count; ++k)
    if (indices[k] < 0 || indices[k] >= b->count) return MLSW_ERR_ARG;
  size_t off = 0;
  for (int k = 0; k < count; ++k) {
    const int j = indices[k];
    const KParams& P = b->hinst[j].P;
    mlsw::KShift sh;
    for (int i = 0; i < mlsw::kMaxLayers; ++i) sh.H[i] = P.H[i];
    CUB(mlsw::launch_init(kQ, P.n, P.L, true, dev_in + off, b->hinst[j].f[state_buffer(b, j)],
                          sh, b->dstatus, b->stream));
    b->launches += 1;
    off += (size_t)P.n * P.nx * P.ny;
  }
  return MLSW_OK;
}

int mlswlbm_batch_modes(mlsw_batch* b, const int* kx, const int* ky, double* out) {
  if (!b || !kx || !ky || !out) return MLSW_ERR_ARG;
  const int rc = align_buffers(b);
  if (rc != MLSW_OK) return rc;
  const size_t nk = (size_t)b->count * sizeof(int);
  CUB(cudaMemcpyAsync(b->dk, kx, nk, cudaMemcpyHostToDevice, b->stream));
  CUB(cudaMemcpyAsync(b->dk + b->count, ky, nk, cudaMemcpyHostToDevice, b->stream));
  CUB(mlsw::launch_batch_modes(b->dinst, b->count, b->cur, b->dk, b->dk + b->count, b->dmode,
                               b->stream));
  b->launches += 1;
  CUB(cudaMemcpyAsync(out, b->dmode, 2 * (size_t)mlsw::kMaxLayers * b->count * sizeof(double),
                      cudaMemcpyDeviceToHost, b->stream));
  return mlswlbm_batch_status(b);
}

int mlswlbm_batch_select(mlsw_batch* b, int nsel, const int* indices) {
  if (!b || nsel < 0 || nsel > b->count || (nsel > 0 && !indices)) return MLSW_ERR_ARG;
  std::vector<char> want(b->count, 0);
  for (int k = 0; k < nsel; ++k) {
    const int j = indices[k];
    if (j < 0 || j >= b->count || want[j]) return MLSW_ERR_ARG;
    want[j] = 1;
  }
  // every state into buffer cur first: then leaving out or taking back an
  // instance moves no data
  int rc = align_buffers(b);
  if (rc != MLSW_OK) return rc;
  for (int j = 0; j < b->count; ++j) {
    b->selected[j] = want[j];
    b->home[j] = b->cur;
  }
  // the step graphs read the tile table being replaced
  CUB(cudaStreamSynchronize(b->stream));
  for (int k = 0; k < 2; ++k)
    if (b->gexec[k]) {
      cudaGraphExecDestroy(b->gexec[k]);
      b->gexec[k] = nullptr;
    }
  rc = build_groups(b);
  if (rc == MLSW_OK && !b->groups.empty()) rc = capture_step(b, 0, &b->gexec[0]);
  if (rc == MLSW_OK && !b->groups.empty()) rc = capture_step(b, 1, &b->gexec[1]);
  return rc;
}

int mlswlbm_batch_tile_rows(const mlsw_batch* b, int index) {
  if (!b || index < 0 || index >= b->count) return MLSW_ERR_ARG;
  return mlsw::batch_tile_rows(b->variant[index]);
}

long mlswlbm_batch_launch_count(const mlsw_batch* b) { return b ? b->launches : -1; }

int mlswlbm_batch_groups(const mlsw_batch* b) { return b ? (int)b->groups.size() : -1; }

}  // extern "C"
