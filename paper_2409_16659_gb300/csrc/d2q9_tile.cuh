// d2q9_tile.cuh -- the persistent, TMA-fed tile loop of the fused D2Q9 step
// (section LBM: moments, interfaces and pressures, force, BGK with forcing,
// push-streaming), shared by the single-lattice kernel (step_kernels.cu)
// and the batch kernel (batch_kernels.cu), with the device helpers it uses.
// The phases are described at the top of step_kernels.cu.
#pragma once

#include <type_traits>

#include "kernels.h"
#include "physics.cuh"
#include "tma.cuh"

namespace mlsw {

// ---------------------------------------------------------------------------
// Bounds checks of the debug build (physics.cuh): a shared-memory pointer
// must lie in the CTA's dynamic shared memory, an index in its array, a
// global store in its buffer or plane. Out of range, the access is counted
// and goes to the first element instead. Release builds pass through.
// ---------------------------------------------------------------------------
#ifdef MLSW_DEBUG
extern __shared__ __align__(128) unsigned char dyn_smem_base[];
__device__ __forceinline__ bool dyn_smem_ok(const void* p, int bytes) {
  if (!__isShared(p)) return false;
  uint32_t size;
  asm("mov.u32 %0, %%dynamic_smem_size;" : "=r"(size));
  const uint32_t a = smem_addr(p), lo = smem_addr(dyn_smem_base);
  return a >= lo && a + (uint32_t)bytes <= lo + size;
}
#endif
template <class P>
__device__ __forceinline__ P* chk_smem(P* p) {
#ifdef MLSW_DEBUG
  if (!dyn_smem_ok(p, (int)sizeof(P))) {
    note_bounds_violation();
    return reinterpret_cast<P*>(dyn_smem_base);
  }
#endif
  return p;
}
__device__ __forceinline__ int chk_index(int i, int n) {
#ifdef MLSW_DEBUG
  if (i < 0 || i >= n) {
    note_bounds_violation();
    return 0;
  }
#endif
  return i;
}
// offset of a global store inside its buffer or plane: i in [0, len)
__device__ __forceinline__ long chk_offset(long i, long len) {
#ifdef MLSW_DEBUG
  if (i < 0 || i >= len) {
    note_bounds_violation();
    return 0;
  }
#endif
  return i;
}
// global store target: p inside [base, base + len)
__device__ __forceinline__ float* chk_global(float* base, float* p, long len) {
#ifdef MLSW_DEBUG
  const long i = p - base;
  if (i < 0 || i >= len) {
    note_bounds_violation();
    return base;
  }
#endif
  return p;
}

// ---------------------------------------------------------------------------
// Stores of one post-collision population to its streamed destination
// (dx, dy) (already periodic) and to the ghost cells that image it.
// ---------------------------------------------------------------------------
// Lattices with both sides >= 4 cells: a real column d has at most one
// ghost image (d + n for d < 2, d - n for d >= n - 2), likewise rows, so a
// population near an edge needs at most three extra stores.
constexpr int kNoImage = -(1 << 28);

__device__ __forceinline__ int image_of(int d, int n) {
  return d < 2 ? d + n : (d >= n - 2 ? d - n : kNoImage);
}

__device__ __forceinline__ void store_edge(float* __restrict__ plane_base, const Layout& L,
                                           int dx, int dy, int xi, int yi, float v) {
  // indices into the plane (not derived pointers), so that the stores keep
  // the base pointer's no-alias guarantee
  const long r0 = (long)(dy + L.gy) * L.pitch;
  plane_base[chk_offset(r0 + dx + L.gx, L.plane)] = v;
  if (xi != kNoImage) plane_base[chk_offset(r0 + xi + L.gx, L.plane)] = v;
  if (yi != kNoImage) {
    const long r1 = (long)(yi + L.gy) * L.pitch;
    plane_base[chk_offset(r1 + dx + L.gx, L.plane)] = v;
    if (xi != kNoImage) plane_base[chk_offset(r1 + xi + L.gx, L.plane)] = v;
  }
}

// ---------------------------------------------------------------------------
// The rest population after the collision, g0* = g0 + delta: the stored rest
// population g0 (shifted by H, O(h - H)) plus a small change (the incoming
// moving populations less the outgoing equilibria, times omega when tau !=
// 1). Rounding g0 + delta to FP32 loses up to half an ulp of g0 per cell
// and step, and in a slowly changing film (a dewetted precursor far from H)
// that loss has the same sign step after step. The exact rounding error
// (Fast2Sum, |g0| >= |delta| in the cells where it matters) is passed on
// instead, half to each of two opposite moving populations: their ulp is
// orders of magnitude finer, the momentum they carry is unchanged, and the
// cell's populations sum to the incoming mass to their rounding.
// ---------------------------------------------------------------------------
template <class T>
__device__ __forceinline__ T rest_update(T g0, T delta, T& fa, T& fb) {
  const T out = g0 + delta;
  const T r = delta - (out - g0);  // exact: the part of delta the sum dropped
  fa = fmav(r, 0.5f, fa);
  fb = fmav(r, 0.5f, fb);
  return out;
}

// Equilibrium, BGK with forcing for one layer at one cell; fs[k] receives
// the post-collision populations (rest one stored shifted by H).
// g0: the stored rest population; small: the sum of the stored moving ones
// (h - H = g0 + small); f_old (read only when !TAU1) holds the stored
// pre-collision populations.
template <int LAT, bool TAU1>
__device__ __forceinline__ void collide(const KParams& P, float h, float g0, float small,
                                        float jx, float jy, float Fx, float Fy,
                                        const float* f_old, float (&fs)[Lattice<LAT>::Q]) {
  using Lt = Lattice<LAT>;
  const float inv_h = rcp(h);
  const float ux = jx * inv_h, uy = jy * inv_h;
  const float u2 = ux * ux + uy * uy;
  float sum_eq = 0.f;
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
  // stored shifted by H: g0 + (small - sum_eq), relaxed by omega when
  // tau != 1 (the moving populations then keep 1 - omega of small)
  const float d = small - sum_eq;
  fs[0] = rest_update(g0, TAU1 ? d : P.omega * d, fs[1], fs[2]);
}

// ---------------------------------------------------------------------------
// D2Q9 collision with the opposite directions paired: for c_{k+4} = -c_k the
// equilibria share w_k h (4.5 (c.U)^2 - 1.5 U^2) and differ in the sign of
// 3 w_k h c.U, and the forcing terms 3 w_k c.F are odd, so each pair costs
// one symmetric and one antisymmetric part. Directions: 1 (1,0), 2 (1,1),
// 3 (0,1), 4 (-1,1); 5..8 are their opposites.
// ---------------------------------------------------------------------------
template <bool TAU1, class T>
__device__ __forceinline__ void collide_d2q9(const KParams& P, T h, T g0, T small, T jx, T jy,
                                             T Fx, T Fy, const T* f_old, T (&fs)[9]) {
  const T ih = rcp(h);
  const T ux = jx * ih, uy = jy * ih;
  const T u15 = 1.5f * fmav(ux, ux, uy * uy);
  T sumsym = Num<T>::splat(0.f);
  const T cus[4] = {ux, ux + uy, uy, uy - ux};
  const T cfs[4] = {Fx, Fx + Fy, Fy, Fy - Fx};
  const float ws[4] = {1.f / 9.f, 1.f / 36.f, 1.f / 9.f, 1.f / 36.f};
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const T A = ws[q] * h;
    const T cu = cus[q];
    const T sym = A * fmav(4.5f * cu, cu, -u15);
    sumsym += sym;
    if constexpr (TAU1) {
      const T anti = 3.f * fmav(A, cu, ws[q] * cfs[q]);
      fs[q + 1] = sym + anti;
      fs[q + 5] = sym - anti;
    } else {
      const T aeq = (3.f * A) * cu, afr = (3.f * ws[q]) * cfs[q];
      fs[q + 1] = fmav(P.omega, (sym + aeq) - f_old[q + 1], f_old[q + 1]) + afr;
      fs[q + 5] = fmav(P.omega, (sym - aeq) - f_old[q + 5], f_old[q + 5]) - afr;
    }
  }
  // rest population h - (sum of moving equilibria) = h (1 - w_0 U^2/(2 cs^2)),
  // stored shifted by H: g0 + (small - 2 sumsym), relaxed by omega when
  // tau != 1 (see rest_update)
  const T d = fmav(-2.f, sumsym, small);
  fs[0] = rest_update(g0, TAU1 ? d : P.omega * d, fs[1], fs[5]);
}

// Sum of the eight stored moving populations of one layer at a cell: the
// opposite directions first (their moving parts nearly cancel), then the
// diagonals with the axes. The layer's h - H is the rest population plus
// this sum, added last: adding the small populations to the O(h - H) rest
// population one by one would drop their low bits one direction at a time.
template <class T>
__device__ __forceinline__ T moving_sum(const T (&v)[9]) {
  return ((v[1] + v[5]) + (v[3] + v[7])) + ((v[2] + v[6]) + (v[4] + v[8]));
}

// Loads / stores of one cell (float) or of a pair of cells (f2) at two
// addresses.
template <class T> struct Lanes;
template <> struct Lanes<float> {
  static constexpr int W = 1;
  __device__ static float ld(const float* a, const float*) { return *chk_smem(a); }
  __device__ static void st(float* a, float*, float v) { *chk_smem(a) = v; }
  __device__ static float get(float v, int) { return v; }
  __device__ static float ld2(float a, float) { return a; }
};
template <> struct Lanes<f2> {
  static constexpr int W = 2;
  __device__ static f2 ld(const float* a, const float* b) { return mk2(*chk_smem(a), *chk_smem(b)); }
  __device__ static void st(float* a, float* b, f2 v) {
    *chk_smem(a) = v.v.x;
    *chk_smem(b) = v.v.y;
  }
  __device__ static float get(f2 v, int l) { return l ? v.v.y : v.v.x; }
  __device__ static f2 ld2(float a, float b) { return mk2(a, b); }
};

// ---------------------------------------------------------------------------
// D2Q9, persistent, TMA-fed. Tile 32 x TY, 256 threads (32 x 8), RPT tile
// rows per thread. Shared memory (floats unless noted):
//   stage [9N][TY + 4][40]   TMA box, x from x0 - 4, y from y0 - 2
//   zs    [N][TY + 4][36]    interface-height deviations z_i - sum_{j<=i} H_j
//                            on the two-ring region (their differences give
//                            the layer thicknesses)
//   ps    [N][TY + 2][34]    p_i on the one-ring region
//   js    [2][N][TY][32]     fluxes J_i of the tile cells
//   bar                      mbarrier (8 bytes)
//   next_tile                (int)
//   par   [2] KParams        a batch tile's parameters (two buffers)
// About 113 KB per CTA, so two CTAs share an SM and fill each other's
// barrier waits. With tau = 1 the next tile's copy is issued as soon as the
// moments are formed and lands while this tile is finished.
// ---------------------------------------------------------------------------
template <int N, int RPT_ = (N <= 3 ? 2 : 1)>
struct D2Tile {
  static constexpr int Q = 9, PN = N * Q, TX = 32;
  static constexpr int NT = 256, BY = NT / 32, RPT = RPT_, TY = BY * RPT;
  static constexpr int BW = TX + 8, BH = TY + 4, STAGE = PN * BH * BW;
  static constexpr int RW = TX + 4, RH = TY + 4, PW = TX + 2, PH = TY + 2;
  static constexpr int NHALO = 4 * RW + 4 * TY;
  static constexpr size_t kStageBytes = (size_t)STAGE * 4;
  static constexpr size_t kOffZ = kStageBytes;
  static constexpr size_t kOffP = kOffZ + (size_t)N * RH * RW * 4;
  static constexpr size_t kOffJ = kOffP + (size_t)N * PH * PW * 4;
  static constexpr size_t kOffBar = (kOffJ + (size_t)2 * N * TY * TX * 4 + 15) / 16 * 16;
  // the mbarrier of the stage, then the tile drawn next
  static constexpr size_t kOffNext = kOffBar + 8;
  static constexpr size_t kOffPar = (kOffNext + 4 + 15) / 16 * 16;
  static constexpr size_t kParBytes = (sizeof(KParams) + 15) / 16 * 16;
  static constexpr size_t kSmem = kOffPar + 2 * kParBytes;
  static_assert(kStageBytes % 128 == 0, "stage alignment");
  static_assert(NHALO <= NT, "one halo cell per thread");
  static_assert(RPT * BY == TY, "tile rows");
  // the kernel has no static shared memory: two CTAs and their 1 KB
  // reserved blocks fill the 228 KB of an SM
  static_assert(2 * (kSmem + 1024) <= 233472, "two CTAs per SM");
};

// Kernel modes: the general step for tau != 1 and for tau = 1, and a fast
// step for the case the paper runs (tau = 1, wetting exponents (3, 2),
// spreading coefficients only between neighbouring interfaces).
enum StepMode { kGeneral = 0, kTau1 = 1, kFast = 2 };

// One tile of work: its parameters, the tensor map of its input buffer, its
// output buffer and its position in the tile grid of its lattice.
struct TileRef {
  const KParams* P;
  const CUtensorMap* map;
  float* fout;
  int bx, by;
};

// Tiles of one lattice (the single-solver kernel). Tile t of a step runs
// in row-major order, or in reverse order when rev is set: the solver
// alternates the two, so that each step starts on the rows the previous
// step wrote last, which are still in the L2.
struct SingleTiles {
  const KParams* P;
  const CUtensorMap* map;
  float* fout;
  int ntx, ntiles, rev;
  static constexpr bool kHints = true;  // L2 cache hints (KParams::l2_policy)
  static constexpr bool kChained = false;
  static constexpr bool kStageParams = false;  // parameters in the constant bank
  static constexpr bool kShiftStores = true;  // edge stores: straight store + periodic shifts
  __device__ TileRef operator()(int t) const {
    const int u = rev ? ntiles - 1 - t : t;
    return {P, map, fout, u % ntx, u / ntx};
  }
  __device__ void prefetch() const { tma_prefetch_desc(map); }
};

// Tiles of many lattices (a batch): table[t] = (instance, tile of that
// instance); every instance steps from buffer cur to cur ^ 1. One range of
// the table, of one kind, ends at ntiles.
struct BatchTiles {
  const BatchInst* inst;
  const int2* table;
  int cur, ntiles, variant;  // variant: tensor-map set of this tile height
  static constexpr bool kHints = false;  // plain loads and stores
  static constexpr bool kChained = true;
  static constexpr bool kStageParams = true;  // parameters read from shared memory (d2q9_tile_loop)
  static constexpr bool kShiftStores = false;  // edge stores: wrapped store + explicit images
  __device__ TileRef operator()(int t) const {
    const int2 e = table[t];
    const BatchInst& b = inst[e.x];
    return {&b.P, &b.map[variant][cur], b.f[cur ^ 1], e.y % b.ntx, e.y / b.ntx};
  }
  __device__ void prefetch() const {}
};

// The persistent tile loop of the D2Q9 step, for any source of tiles.
// Runs the tiles t0, then those drawn from the counter sched[0], while they
// are below tiles.ntiles. Returns the first tile drawn beyond that bound
// (not yet copied), or kLoopTimedOut after a bounded wait ran out (the
// status word has the timeout bit). The caller ends the launch with
// tile_loop_finish. A source of tiles with kChained set is one of several
// ranges that a CTA runs one after another (tile indices increase, the
// counter is shared): the loop then releases its mbarrier before it
// returns, so that the next range can lay out the shared memory afresh.
constexpr int kLoopTimedOut = -1;

template <int N, int MODE, int RPT_, class Tiles>
__device__ __forceinline__ int d2q9_tile_loop(const Tiles& tiles, int* __restrict__ status,
                                              int* __restrict__ sched, int t0) {
  constexpr bool TAU1 = MODE != kGeneral, W32 = MODE == kFast, NN = MODE == kFast;
  using Tl = D2Tile<N, RPT_>;
  constexpr int Q = 9, TX = Tl::TX, TY = Tl::TY, BY = Tl::BY, RPT = Tl::RPT;
  constexpr int BW = Tl::BW, BH = Tl::BH, RW = Tl::RW, RH = Tl::RH, PW = Tl::PW, PH = Tl::PH;
  // a thread's two tile rows (iy, iy + BY) are evaluated as one FP32x2 pair
  using T = typename std::conditional<RPT == 2, f2, float>::type;
  using Ln = Lanes<T>;
  constexpr int W = Ln::W;
  static_assert(RPT == W, "one lane per tile row of the thread");
  extern __shared__ __align__(128) unsigned char smem_raw[];
  float* stage = reinterpret_cast<float*>(smem_raw);
  float* zs = reinterpret_cast<float*>(smem_raw + Tl::kOffZ);
  float* ps = reinterpret_cast<float*>(smem_raw + Tl::kOffP);
  float* js = reinterpret_cast<float*>(smem_raw + Tl::kOffJ);
  uint64_t* bar = reinterpret_cast<uint64_t*>(smem_raw + Tl::kOffBar);
  int& next_tile = *reinterpret_cast<int*>(smem_raw + Tl::kOffNext);

  const int tid = threadIdx.x;
  const int ntiles = tiles.ntiles;

  // L2 policies (KParams::l2_policy). For a single lattice the step's
  // output is written evict_last, so that as much of it as the L2 holds is
  // still there when the next step reads it. When a whole buffer fits
  // (kL2Resident), the input is read evict_first: it is dead once read, and
  // the output lines keep the L2. A larger lattice (kL2Stream) reads with
  // the lines' priority unchanged (halo rows are read again by the tile row
  // below) and the solver alternates the tile order, so each step starts on
  // the rows its predecessor wrote last. Batches use plain loads and
  // stores (no hinted instructions at all, which measured faster there):
  // kept output lines would only crowd out the halo rows of other tiles.
  constexpr bool HINTS = Tiles::kHints;
  constexpr bool SHIFT = Tiles::kShiftStores;  // edge-tile store scheme (phase C)
  const int l2pol = HINTS ? tiles(blockIdx.x).P->l2_policy : (int)kL2None;  // grid <= ntiles
  const uint64_t st_pol = l2pol == kL2None ? pol_evict_normal() : pol_evict_last();
  const uint64_t ld_pol = l2pol == kL2Resident ? pol_evict_first()
                          : (l2pol == kL2Stream ? pol_evict_unchanged() : pol_evict_normal());
  auto issue = [&](int t) {
    const TileRef r = tiles(t);
    fence_proxy_async_smem();
#ifdef MLSW_DEBUG
    // the box must start on a 16-byte boundary and lie inside the padded
    // planes; a bad box is not copied (the barrier completes without data)
    const Layout& L = r.P->L;
    if ((r.bx * TX) % 4 != 0 || r.bx * TX + BW > L.pitch || r.by * TY + BH > L.rows ||
        (long)BH * BW * Tl::PN * 4 != (long)Tl::kStageBytes) {
      note_bounds_violation();
      mbar_arrive_expect_tx(bar, 0u);  // the one arrival, no bytes
      return;
    }
#endif
    mbar_arrive_expect_tx(bar, (uint32_t)Tl::kStageBytes);
    // box origin: real (x0 - 4, y0 - 2) = padded (x0, y0) since gx = 4, gy = 2
    if constexpr (HINTS)
      tma_load_3d(stage, r.map, bar, r.bx * TX, r.by * TY, 0, ld_pol);
    else
      tma_load_3d(stage, r.map, bar, r.bx * TX, r.by * TY, 0);
  };
  auto draw_next = [&]() {
    const int nt = (int)gridDim.x + atomicAdd(sched, 1);
    next_tile = nt;
    if (nt < ntiles) issue(nt);
  };
  // two-ring cell of halo index q (the ring around the tile)
  auto halo_cell = [&](int q, int& r, int& c) {
    if (q < 2 * RW) {
      r = q / RW;
      c = q - r * RW;
    } else if (q < 4 * RW) {
      const int u = q - 2 * RW;
      r = RH - 2 + u / RW;
      c = u % RW;
    } else {
      const int u = q - 4 * RW;
      r = 2 + (u >> 2);
      const int c4 = u & 3;
      c = c4 < 2 ? c4 : RW - 4 + c4;
    }
  };

  if (tid == 0) {
    mbar_init(bar, 1);
    mbar_init_fence();
  }
  // Programmatic dependent launch: the next step's grid may be scheduled
  // while this one drains, and this grid's set-up above overlaps the
  // previous step's tail. Every global access (the tile loads, the stores
  // into the previous step's input buffer, the counters) comes after the
  // wait for the previous grid's completion. Both are no-ops in a launch
  // without the programmatic attribute.
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
  asm volatile("griddepcontrol.wait;" ::: "memory");
  __syncthreads();
  if (tid == 0) {
    tiles.prefetch();
    if (t0 < ntiles) issue(t0);
  }

  constexpr bool STAGEP = Tiles::kStageParams;
  // Batch tiles take their parameters from their instance's descriptor in
  // global memory (the single-lattice kernel has them in the constant
  // bank). The pressure and collision phases read them from a copy in
  // shared memory instead, made one tile ahead into the other of two
  // buffers: the first tile's before the loop, the next one's as soon as it
  // is drawn; the barrier before the pressure phase makes it visible. With
  // the loads from global memory the batch ran 2.4 % slower.
  auto stage_params = [&](int tt, int buf) {
    constexpr int NW = (int)(sizeof(KParams) / 4);
    int* dst = reinterpret_cast<int*>(smem_raw + Tl::kOffPar + (size_t)buf * Tl::kParBytes);
    const int* src = reinterpret_cast<const int*>(tiles(tt).P);
    for (int w = tid; w < NW; w += Tl::NT) *chk_smem(dst + w) = src[w];
  };
  static_assert(sizeof(KParams) % 4 == 0, "parameters copied as words");
  if constexpr (STAGEP)
    if (t0 < ntiles) stage_params(t0, 0);
  const int ix = tid % TX, iyb = tid / TX;  // tile cells (ix, iyb + lane * BY)
  bool bad = false;
  uint32_t parity = 0;
  // Tiles: the first one is t0 (blockIdx.x in a launch's first range),
  // later ones come from a global counter (sched[0]), so CTAs that drew
  // cheap tiles take more of them.
  int t = t0;
  for (; t < ntiles; parity ^= 1u) {
    const bool timed_out = !mbar_wait_bounded(bar, parity);
    const TileRef tr = tiles(t);
    const KParams& P = *tr.P;
    const Layout& L = P.L;
    const int nx = P.nx, ny = P.ny;
    const long lplane = (long)Q * L.plane;  // floats per layer
    float* __restrict__ fout = tr.fout;
    const int x0 = tr.bx * TX, y0 = tr.by * TY;
    // a corrugated substrate (never in the fast mode): z starts at z_0
    const bool sub = MODE != kFast && P.sub_amp != 0.f;
    // z_0 at tile-local cell (c, r) of the two-ring region (c, r from -2)
    auto z0_at = [&](int c, int r) { return substrate_at(P, x0 + c, y0 + r); };

    // ---- M. moments: deviations z on the two-ring region, J on the tile ----
    // A tile cell's rest population g0 and the sum of its moving ones stay
    // in registers for the collision (h - H = g0 + small): recovering
    // h - H as z_i - z_{i-1} would round it to the resolution of z_i, and
    // that rounding is not mass-neutral.
    T g0s[N], sms[N];
    {
      const int rA = iyb + 2, rB = iyb + (W - 1) * BY + 2, c = ix + 2;  // two-ring coords
      const float* sA = stage + rA * BW + (c + 2);  // stage column = c + 2
      const float* sB = stage + rB * BW + (c + 2);
      T z = Num<T>::splat(0.f);
      if (sub) z = Ln::ld2(z0_at(ix, rA - 2), z0_at(ix, rB - 2));
#pragma unroll
      for (int i = 0; i < N; ++i) {
        T v[Q];
#pragma unroll
        for (int k = 0; k < Q; ++k) v[k] = Ln::ld(sA + (i * Q + k) * BH * BW, sB + (i * Q + k) * BH * BW);
        g0s[i] = v[0];
        sms[i] = moving_sum(v);
        z += g0s[i] + sms[i];
        Ln::st(zs + (i * RH + rA) * RW + c, zs + (i * RH + rB) * RW + c, z);
        Ln::st(js + ((0 * N + i) * TY + rA - 2) * TX + ix, js + ((0 * N + i) * TY + rB - 2) * TX + ix,
               ((v[1] + v[2]) + v[8]) - ((v[4] + v[5]) + v[6]));
        Ln::st(js + ((1 * N + i) * TY + rA - 2) * TX + ix, js + ((1 * N + i) * TY + rB - 2) * TX + ix,
               ((v[2] + v[3]) + v[4]) - ((v[6] + v[7]) + v[8]));
      }
    }
    // halo cells (sums only), a pair of cells per thread through the same T
    // arithmetic as the tile cells, so every cell's z has the same bits
    // whichever tile computes it (with an odd count the last thread puts
    // one cell in both lanes)
    constexpr int NH = Tl::NHALO, NHP = (W == 2) ? (NH + 1) / 2 : NH;
    if (tid < NHP) {
      int rA, cA, rB, cB;
      halo_cell(tid, rA, cA);
      halo_cell((W == 2 && tid + NHP < NH) ? tid + NHP : tid, rB, cB);
      const float* srcA = stage + rA * BW + (cA + 2);
      const float* srcB = stage + rB * BW + (cB + 2);
      T z = Num<T>::splat(0.f);
      if (sub) z = Ln::ld2(z0_at(cA - 2, rA - 2), z0_at(cB - 2, rB - 2));
#pragma unroll
      for (int i = 0; i < N; ++i) {
        T v[Q];
#pragma unroll
        for (int k = 0; k < Q; ++k)
          v[k] = Ln::ld(srcA + (i * Q + k) * BH * BW, srcB + (i * Q + k) * BH * BW);
        z += v[0] + moving_sum(v);
        Ln::st(zs + (i * RH + rA) * RW + cA, zs + (i * RH + rB) * RW + cB, z);
      }
    }
    if (__syncthreads_or(timed_out)) {
      if (tid == 0) {
        atomicOr(status, kStatusTimeout);
        mbar_wait_bounded(bar, parity);  // let this CTA's copy land before exiting
      }
      return kLoopTimedOut;
    }
    // tau = 1 needs nothing more from the stage: refill it with the next
    // tile, which lands while this tile is finished
    if (TAU1 && tid == 0) draw_next();
    {  // the pressure and collision phases: P is the staged copy in a batch
    const KParams& P = STAGEP ? *reinterpret_cast<const KParams*>(smem_raw + Tl::kOffPar +
                                                                 (size_t)(parity & 1) * Tl::kParBytes)
                              : *tr.P;

    // ---- P. pressures on the one-ring region -------------------------------------
    // Cell q of the region (row-major, width PW). With packed pairs, rounds of
    // NT pairs (q, q + NT) cover whole multiples of 2 NT cells and the rest is
    // done one cell per thread, which keeps the threads evenly loaded.
    {
      auto pressure_cells = [&](auto zero, int qa, int qb) {
        using U = decltype(zero);
        using LU = Lanes<U>;
        const int prA = qa / PW, pcA = qa - prA * PW, prB = qb / PW, pcB = qb - prB * PW;
        U zd[N], gzx[N], gzy[N], lz[N], p[N];
#pragma unroll
        for (int i = 0; i < N; ++i) {
          const float* a = zs + (i * RH + prA + 1) * RW + pcA + 1;
          const float* b = zs + (i * RH + prB + 1) * RW + pcB + 1;
          const U zE = LU::ld(a + 1, b + 1), zW = LU::ld(a - 1, b - 1);
          const U zN = LU::ld(a + RW, b + RW), zS = LU::ld(a - RW, b - RW);
          const U zNE = LU::ld(a + RW + 1, b + RW + 1), zNW = LU::ld(a + RW - 1, b + RW - 1);
          const U zSE = LU::ld(a - RW + 1, b - RW + 1), zSW = LU::ld(a - RW - 1, b - RW - 1);
          zd[i] = LU::ld(a, b);
          // (1/cs^2)(w_1 = 1/9, w_2 = 1/36) -> 1/3 and 1/12
          gzx[i] = fmav(zE - zW, 1.f / 3.f, ((zNE - zNW) + (zSE - zSW)) * (1.f / 12.f));
          gzy[i] = fmav(zN - zS, 1.f / 3.f, ((zNE - zSE) + (zNW - zSW)) * (1.f / 12.f));
          // (2/cs^2) sum_k w_k (z_k - z_0): 2/3 on the edges, 1/6 on the corners
          lz[i] = fmav((zE + zW) + (zN + zS), 2.f / 3.f,
                       fmav((zNE + zNW) + (zSE + zSW), 1.f / 6.f, zd[i] * (-10.f / 3.f)));
        }
        if (sub) {
          // z_0 and 1 + |grad z_0|^2 / 2 (lattice stencil) at the two cells;
          // p-region cell (pr, pc) is tile cell (pc - 1, pr - 1)
          U z0c, sg0;
          {
            float zc[2], sg[2];
            const int ca[2] = {pcA - 1, pcB - 1}, ra[2] = {prA - 1, prB - 1};
#pragma unroll
            for (int l = 0; l < 2; ++l) {
              const float c0 = z0_at(ca[l], ra[l]);
              const float e = z0_at(ca[l] + 1, ra[l]), w = z0_at(ca[l] - 1, ra[l]);
              const float nn = z0_at(ca[l], ra[l] + 1), ss = z0_at(ca[l], ra[l] - 1);
              const float ne = z0_at(ca[l] + 1, ra[l] + 1), nw = z0_at(ca[l] - 1, ra[l] + 1);
              const float se = z0_at(ca[l] + 1, ra[l] - 1), sw = z0_at(ca[l] - 1, ra[l] - 1);
              const float gx = fmaf(e - w, 1.f / 3.f, ((ne - nw) + (se - sw)) * (1.f / 12.f));
              const float gy = fmaf(nn - ss, 1.f / 3.f, ((ne - se) + (nw - sw)) * (1.f / 12.f));
              zc[l] = c0;
              sg[l] = fmaf(0.5f, fmaf(gx, gx, gy * gy), 1.f);
            }
            z0c = LU::ld2(zc[0], zc[1]);
            sg0 = LU::ld2(sg[0], sg[1]);
          }
          layer_pressures_dev<N, W32, U, NN>(P, zd, gzx, gzy, lz, p, z0c, sg0);
        } else {
          layer_pressures_dev<N, W32, U, NN>(P, zd, gzx, gzy, lz, p);
        }
#pragma unroll
        for (int i = 0; i < N; ++i)
          LU::st(ps + (i * PH + prA) * PW + pcA, ps + (i * PH + prB) * PW + pcB, p[i]);
      };
      constexpr int NC = PH * PW;
      constexpr int NPAIRED = (W == 2) ? (NC / (2 * Tl::NT)) * 2 * Tl::NT : 0;
      for (int q = tid; q < NPAIRED / 2; q += Tl::NT) {
        const int base = (q / Tl::NT) * 2 * Tl::NT + q % Tl::NT;
        pressure_cells(Num<T>::splat(0.f), base, base + Tl::NT);
      }
      // the rest in pairs (q, q + RP), through the same T arithmetic, so a
      // cell's pressure has the same bits in every tile (with an odd rest the
      // last pair puts one cell in both lanes)
      constexpr int R = NC - NPAIRED, RP = (W == 2) ? (R + 1) / 2 : R;
      for (int j = tid; j < RP; j += Tl::NT)
        pressure_cells(Num<T>::splat(0.f), NPAIRED + j,
                       (W == 2 && j + RP < R) ? NPAIRED + j + RP : NPAIRED + j);
    }
    __syncthreads();
    // with tau = 1 written by thread 0 before the barrier above
    int tnext = TAU1 ? next_tile : 0;
    if constexpr (STAGEP && TAU1)
      if (tnext < ntiles) stage_params(tnext, (parity ^ 1u) & 1u);

    // ---- C. force, collision, streaming (the thread's rows as one pair) -------
    {
      const int iyA = iyb, iyB = iyb + (W - 1) * BY;
      const int gx = x0 + ix;
      bool valid[W];
#pragma unroll
      for (int l = 0; l < W; ++l) valid[l] = gx < nx && y0 + iyb + l * BY < ny;
      if (valid[0]) {  // lane 0 invalid implies lane 1 invalid
        T hh[N], jx[N], jy[N];
        {
#pragma unroll
          for (int i = 0; i < N; ++i) {
            hh[i] = (g0s[i] + sms[i]) + P.H[i];
            jx[i] = Ln::ld(js + ((0 * N + i) * TY + iyA) * TX + ix, js + ((0 * N + i) * TY + iyB) * TX + ix);
            jy[i] = Ln::ld(js + ((1 * N + i) * TY + iyA) * TX + ix, js + ((1 * N + i) * TY + iyB) * TX + ix);
          }
        }
        T Rx[N], Ry[N];
        friction<N>(P, hh, jx, jy, Rx, Ry);
        // A tile at least three cells from every edge streams without
        // wrap-around or ghost images: all nine destinations are fixed,
        // warp-uniform offsets from one base per cell.
        const bool inner = !P.tiny && x0 >= 3 && x0 + TX + 3 <= nx && y0 >= 3 && y0 + TY + 3 <= ny;
        float* cbase[W];
#pragma unroll
        for (int l = 0; l < W; ++l)
          cbase[l] = fout + (long)(y0 + iyb + l * BY + L.gy) * L.pitch + (gx + L.gx);
        // Edge tiles of lattices with both sides >= 4 cells: a population
        // first goes to the padded cell (x + cx, y + cy) itself, as in an
        // inner tile. That is its destination, or, when it leaves the
        // domain, the ghost cell imaging its wrapped destination. A
        // destination column d in {-1, 0, 1} has its other periodic copy at
        // d + nx, one in {nx - 2, nx - 1, nx} at d - nx (the wrapped real
        // cell or a ghost image), others none; rows likewise. xsh and ysh
        // hold these shifts (0: none) per lane and column / row offset.
        int xsh[W][3], ysh[W][3];
        bool wimg = false;  // some lane of the warp has a shifted copy
        // Lattices with a side below 4 cells: wrapped destinations (koff)
        // only; a separate pass refreshes their ghosts.
        int koff[W][Q];
        if (SHIFT && !inner) {
          bool img = false;
#pragma unroll
          for (int l = 0; l < W; ++l) {
            const int gy = y0 + iyb + l * BY;
#pragma unroll
            for (int c = 0; c < 3; ++c) {
              const int dx = gx + c - 1, dy = gy + c - 1;
              xsh[l][c] = dx < 2 ? nx : (dx >= nx - 2 ? -nx : 0);
              ysh[l][c] = dy < 2 ? ny * L.pitch : (dy >= ny - 2 ? -ny * L.pitch : 0);
              img |= valid[l] && (xsh[l][c] != 0 || ysh[l][c] != 0);
            }
            if (P.tiny) {
              int wx[3], wy[3];
#pragma unroll
              for (int c = 0; c < 3; ++c) {
                int dx = gx + c - 1, dy = gy + c - 1;
                dx += (dx < 0) ? nx : 0;
                dx -= (dx >= nx) ? nx : 0;
                dy += (dy < 0) ? ny : 0;
                dy -= (dy >= ny) ? ny : 0;
                wx[c] = dx;
                wy[c] = dy;
              }
#pragma unroll
              for (int k = 0; k < Q; ++k)
                koff[l][k] = k * (int)L.plane + (wy[Lattice<2>::cy(k) + 1] + L.gy) * L.pitch +
                             wx[Lattice<2>::cx(k) + 1] + L.gx;
            }
          }
          // lanes beyond a ragged edge have left this branch
          wimg = __any_sync(__activemask(), img);
        }
        // the batch kernel's edge stores: wrapped destinations (koff) and
        // their ghost images, written explicitly (store_edge); this form
        // compiles to faster code for the batch's many inlined kinds
        int dxs[W][3], dys[W][3], xis[W][3], yis[W][3];
        bool images[W];
        if constexpr (!SHIFT) {
          // per lane: destinations of the three column / row offsets, images
#pragma unroll
          for (int l = 0; l < W && !inner; ++l) {
            const int gy = y0 + iyb + l * BY;
#pragma unroll
            for (int c = 0; c < 3; ++c) {
              int dx = gx + c - 1, dy = gy + c - 1;
              dx += (dx < 0) ? nx : 0;
              dx -= (dx >= nx) ? nx : 0;
              dy += (dy < 0) ? ny : 0;
              dy -= (dy >= ny) ? ny : 0;
              dxs[l][c] = dx;
              dys[l][c] = dy;
              xis[l][c] = image_of(dx, nx);
              yis[l][c] = image_of(dy, ny);
            }
            // lattices with a side below 4 cells refresh their ghosts in a
            // separate pass; the others write the images here
            images[l] = !P.tiny && ((xis[l][0] != kNoImage) || (xis[l][1] != kNoImage) ||
                                    (xis[l][2] != kNoImage) || (yis[l][0] != kNoImage) ||
                                    (yis[l][1] != kNoImage) || (yis[l][2] != kNoImage));
#pragma unroll
            for (int k = 0; k < Q; ++k)
              koff[l][k] = k * (int)L.plane + (dys[l][Lattice<2>::cy(k) + 1] + L.gy) * L.pitch +
                           dxs[l][Lattice<2>::cx(k) + 1] + L.gx;
          }
        }
#pragma unroll
        for (int i = 0; i < N; ++i) {
          const float* a = ps + (i * PH + iyA + 1) * PW + ix + 1;
          const float* b = ps + (i * PH + iyB + 1) * PW + ix + 1;
          const T pE = Ln::ld(a + 1, b + 1), pW = Ln::ld(a - 1, b - 1);
          const T pN = Ln::ld(a + PW, b + PW), pS = Ln::ld(a - PW, b - PW);
          const T pNE = Ln::ld(a + PW + 1, b + PW + 1), pNW = Ln::ld(a + PW - 1, b + PW - 1);
          const T pSE = Ln::ld(a - PW + 1, b - PW + 1), pSW = Ln::ld(a - PW - 1, b - PW - 1);
          const T gpx = fmav(pE - pW, 1.f / 3.f, ((pNE - pNW) + (pSE - pSW)) * (1.f / 12.f));
          const T gpy = fmav(pN - pS, 1.f / 3.f, ((pNE - pSE) + (pNW - pSW)) * (1.f / 12.f));
          const T h = hh[i];
          const T Fx = fmav(-h, gpx, Rx[i]);
          const T Fy = fmav(-h, gpy, Ry[i]);
#pragma unroll
          for (int l = 0; l < W; ++l)
            if (valid[l])
              bad |= !(Ln::get(h, l) > 0.f) || !isfinite(Ln::get(Fx, l) + Ln::get(Fy, l));
          T fo[Q];
          if constexpr (!TAU1) {
            const float* sA = stage + (iyA + 2) * BW + (ix + 4);
            const float* sB = stage + (iyB + 2) * BW + (ix + 4);
#pragma unroll
            for (int k = 0; k < Q; ++k) fo[k] = Ln::ld(sA + (i * Q + k) * BH * BW, sB + (i * Q + k) * BH * BW);
          }
          T fs[Q];
          collide_d2q9<TAU1>(P, h, g0s[i], sms[i], jx[i], jy[i], Fx, Fy, fo, fs);
          if (inner) {
#pragma unroll
            for (int l = 0; l < W; ++l) {
#pragma unroll
              for (int k = 0; k < Q; ++k) {
                float* dst = chk_global(fout,
                                        &cbase[l][(long)i * lplane + (long)k * L.plane +
                                                  Lattice<2>::cy(k) * L.pitch + Lattice<2>::cx(k)],
                                        L.length());
                if constexpr (HINTS)
                  st_global_hint(dst, Ln::get(fs[k], l), st_pol);
                else
                  *dst = Ln::get(fs[k], l);
              }
            }
            continue;
          }
          if constexpr (!SHIFT) {
            float* obase = fout + (long)i * lplane;
#pragma unroll
            for (int l = 0; l < W; ++l) {
              if (!valid[l]) continue;
              if (!images[l]) {
#pragma unroll
                for (int k = 0; k < Q; ++k)
                  *chk_global(fout, obase + koff[l][k], L.length()) = Ln::get(fs[k], l);
              } else {
#pragma unroll
                for (int k = 0; k < Q; ++k) {
                  const int cxi = Lattice<2>::cx(k) + 1, cyi = Lattice<2>::cy(k) + 1;
                  store_edge(obase + (long)k * L.plane, L, dxs[l][cxi], dys[l][cyi], xis[l][cxi],
                             yis[l][cyi], Ln::get(fs[k], l));
                }
              }
            }
            continue;
          }
          if (P.tiny) {
            float* obase = fout + (long)i * lplane;
#pragma unroll
            for (int l = 0; l < W; ++l) {
              if (!valid[l]) continue;
#pragma unroll
              for (int k = 0; k < Q; ++k)
                *chk_global(fout, obase + koff[l][k], L.length()) = Ln::get(fs[k], l);
            }
            continue;
          }
#pragma unroll
          for (int l = 0; l < W; ++l) {
            if (!valid[l]) continue;
#pragma unroll
            for (int k = 0; k < Q; ++k) {
              const int cx = Lattice<2>::cx(k), cy = Lattice<2>::cy(k);
              const long o = (long)i * lplane + (long)k * L.plane + cy * L.pitch + cx;
              const float v = Ln::get(fs[k], l);
              float* dst = chk_global(fout, &cbase[l][o], L.length());
              if constexpr (HINTS)
                st_global_hint(dst, v, st_pol);
              else
                *dst = v;
              if (wimg) {
                const int xs = xsh[l][cx + 1], ys = ysh[l][cy + 1];
                if (xs) *chk_global(fout, &cbase[l][o + xs], L.length()) = v;
                if (ys) {
                  *chk_global(fout, &cbase[l][o + ys], L.length()) = v;
                  if (xs) *chk_global(fout, &cbase[l][o + xs + ys], L.length()) = v;
                }
              }
            }
          }
        }
      }
    }
    if (!TAU1) {
      __syncthreads();  // every thread has read its pre-collision populations
      if (tid == 0) draw_next();
      __syncthreads();
      tnext = next_tile;
      if constexpr (STAGEP)
        if (tnext < ntiles) stage_params(tnext, (parity ^ 1u) & 1u);
    }
    t = tnext;
    }
  }
  if (bad) atomicOr(status, kStatusNonfinite);
  if constexpr (Tiles::kChained) {
    __syncthreads();  // every thread is done with this range's shared memory
    if (tid == 0) mbar_inval(bar);  // no copy is in flight: t was not issued
  }
  return t;
}

// End of a launch of the tile loop: the last CTA to finish (every CTA has
// drawn its last tile) resets the two counters for the next launch.
__device__ __forceinline__ void tile_loop_finish(int* __restrict__ sched) {
  if (threadIdx.x == 0 && atomicAdd(sched + 1, 1) == (int)gridDim.x - 1) {
    sched[0] = 0;
    sched[1] = 0;
  }
}

}  // namespace mlsw
