// step_kernels.cu -- the fused multilayer shallow-water LBM time step.
//
// One launch = one time step over the whole periodic lattice, in one pass
// over the populations:
//   M. moments: h_i = H_i + sum_k g_ki (rest population stored shifted by
//      H_i, see physics.cuh) on the tile plus a two-cell ring, J_i on the
//      tile -- section LBM;
//   P. on the tile plus one ring: interfaces z_i, their lattice gradient and
//      Laplacian, and the layer pressures p_i (Eqs. Laplace_pressure,
//      disjoining_pressure, p_i = sum_{j>=i} (Lambda_j + Pi_j));
//   C. on the tile: grad p_i, friction (Eq. friction_force), force
//      (Eq. force), equilibrium (Eq. equilibrium_distribution), BGK with
//      forcing (Eq. BGK) and push-streaming into the other buffer, including
//      the periodic ghost images the next step reads.
// Algorithmic traffic is one read and one write of every population.
//
// Discrete derivatives are the isotropic lattice stencils, written as sums
// of differences from the centre so a constant field gives exactly zero:
//   grad phi = (1/c_s^2) sum_k w_k c_k (phi(x + c_k) - phi(x))
//   lap  phi = (2/c_s^2) sum_k w_k (phi(x + c_k) - phi(x)).
//
// D2Q9 runs a persistent kernel, two CTAs per SM, over 32 x TY tiles. The
// tile plus halo of all n*9 population planes (a box of 40 x (TY + 4) x 9n
// floats) arrives in shared memory with one TMA bulk tensor copy completing
// on an mbarrier; each CTA refills its stage with the next tile as soon as
// the moments of the current one are formed, so copies overlap arithmetic.
// D1Q3 (small 1-D lattices) uses a plain tiled kernel.
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
// About 112 KB per CTA, so two CTAs share an SM and fill each other's
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
  static constexpr size_t kSmem = (kOffNext + 4 + 15) / 16 * 16;
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
  __device__ TileRef operator()(int t) const {
    const int u = rev ? ntiles - 1 - t : t;
    return {P, map, fout, u % ntx, u / ntx};
  }
  __device__ void prefetch() const { tma_prefetch_desc(map); }
};

// Tiles of many lattices (a batch): table[t] = (instance, tile of that
// instance); every instance steps from buffer cur to cur ^ 1.
struct BatchTiles {
  const BatchInst* inst;
  const int2* table;
  int cur, ntiles, variant;  // variant: tensor-map set of this tile height
  static constexpr bool kHints = false;  // plain loads and stores
  __device__ TileRef operator()(int t) const {
    const int2 e = table[t];
    const BatchInst& b = inst[e.x];
    return {&b.P, &b.map[variant][cur], b.f[cur ^ 1], e.y % b.ntx, e.y / b.ntx};
  }
  __device__ void prefetch() const {}
};

// The persistent tile loop of the D2Q9 step, for any source of tiles.
template <int N, int MODE, int RPT_, class Tiles>
__device__ __forceinline__ void d2q9_tile_loop(const Tiles& tiles, int* __restrict__ status,
                                               int* __restrict__ sched) {
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
    if ((int)blockIdx.x < ntiles) issue(blockIdx.x);
  }

  const int ix = tid % TX, iyb = tid / TX;  // tile cells (ix, iyb + lane * BY)
  bool bad = false;
  uint32_t parity = 0;
  // Tiles: the first one is blockIdx.x, later ones come from a global
  // counter (sched[0]), so CTAs that drew cheap tiles take more of them.
  // The last CTA to finish resets the counters for the next launch.
  for (int t = blockIdx.x; t < ntiles; parity ^= 1u) {
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
        if (atomicAdd(sched + 1, 1) == (int)gridDim.x - 1) {
          sched[0] = 0;
          sched[1] = 0;
        }
      }
      return;
    }
    // tau = 1 needs nothing more from the stage: refill it with the next
    // tile, which lands while this tile is finished
    if (TAU1 && tid == 0) draw_next();

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
        // per lane: destinations of the three column / row offsets, images
        int koff[W][Q], dxs[W][3], dys[W][3], xis[W][3], yis[W][3];
        bool images[W];
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
        }
      }
    }
    if (!TAU1) {
      __syncthreads();  // every thread has read its pre-collision populations
      if (tid == 0) draw_next();
      __syncthreads();
      tnext = next_tile;
    }
    t = tnext;
  }
  if (bad) atomicOr(status, kStatusNonfinite);
  if (tid == 0 && atomicAdd(sched + 1, 1) == (int)gridDim.x - 1) {
    sched[0] = 0;  // every CTA has drawn its last tile
    sched[1] = 0;
  }
}

template <int N, int MODE>
__global__ void __launch_bounds__(256, 2)
    step_d2q9_tma(const __grid_constant__ CUtensorMap fin_map, float* __restrict__ fout,
                  const __grid_constant__ KParams P, int* __restrict__ status,
                  int* __restrict__ sched, int rev) {
  using Tl = D2Tile<N>;
  const int ntx = (P.nx + Tl::TX - 1) / Tl::TX, nty = (P.ny + Tl::TY - 1) / Tl::TY;
  const SingleTiles tiles{&P, &fin_map, fout, ntx, ntx * nty, rev};
  d2q9_tile_loop<N, MODE, Tl::RPT>(tiles, status, sched);
}

// One step of every instance of a batch group (same n, mode and tile rows):
// one persistent launch over the group's tile table.
template <int N, int MODE, int RPT>
__global__ void __launch_bounds__(256, 2)
    step_d2q9_batch(const BatchInst* __restrict__ inst, const int2* __restrict__ table, int ntiles,
                    int cur, int* __restrict__ status, int* __restrict__ sched) {
  const BatchTiles tiles{inst, table, cur, ntiles, batch_variant(RPT)};
  d2q9_tile_loop<N, MODE, RPT>(tiles, status, sched);
}

// ---------------------------------------------------------------------------
// D1Q3 cell arithmetic shared by the tiled and the persistent kernels, so
// both give the same bits.
// ---------------------------------------------------------------------------
// p_i of one cell from z deviations at x - 1, x, x + 1
// z0w, z0c, z0e: the substrate at x - 1, x, x + 1 (all 0 when flat)
template <int N, bool W32>
__device__ __forceinline__ void d1q3_pressures(const KParams& P, const float (&zw)[N],
                                               const float (&zc)[N], const float (&ze)[N],
                                               float (&p)[N], float z0w = 0.f, float z0c = 0.f,
                                               float z0e = 0.f) {
  float zd[N], gxz[N], gyz[N], lz[N];
#pragma unroll
  for (int i = 0; i < N; ++i) {
    const float e = ze[i] - zc[i], wv = zw[i] - zc[i];
    zd[i] = zc[i];
    gxz[i] = 0.5f * (e - wv);  // (1/cs^2) w_1 = 1/2
    gyz[i] = 0.f;
    lz[i] = e + wv;            // (2/cs^2) w_1 = 1
  }
  if (P.sub_amp != 0.f) {
    const float g0 = 0.5f * (z0e - z0w);
    layer_pressures_dev<N, W32>(P, zd, gxz, gyz, lz, p, z0c, fmaf(0.5f, g0 * g0, 1.f));
  } else {
    layer_pressures_dev<N, W32>(P, zd, gxz, gyz, lz, p);
  }
}

// Force, collision with forcing, for one cell: fs[i][k] receives the
// post-collision populations; f_old is read only when !TAU1. Returns true
// when a height is not positive or a force not finite.
template <int N, bool TAU1>
__device__ __forceinline__ bool d1q3_collide_cell(const KParams& P, const float (&g0)[N],
                                                  const float (&sm)[N],
                                                  const float (&hh)[N], const float (&jx)[N],
                                                  const float (&pw)[N], const float (&pc)[N],
                                                  const float (&pe)[N], const float (&f_old)[N][3],
                                                  float (&fs)[N][3]) {
  float zero[N], Rx[N], Ry[N];
#pragma unroll
  for (int i = 0; i < N; ++i) zero[i] = 0.f;
  friction<N>(P, hh, jx, zero, Rx, Ry);
  bool bad = false;
#pragma unroll
  for (int i = 0; i < N; ++i) {
    const float gpx = 0.5f * ((pe[i] - pc[i]) - (pw[i] - pc[i]));
    const float h = hh[i];
    const float Fx = fmav(-h, gpx, Rx[i]);
    bad |= !(h > 0.f) || !isfinite(Fx) || !isfinite(jx[i]);
    collide<1, TAU1>(P, h, g0[i], sm[i], jx[i], 0.f, Fx, 0.f, f_old[i], fs[i]);
  }
  return bad;
}

// ---------------------------------------------------------------------------
// D1Q3: tile of TX cells, one cell per thread, plain loads (the padded
// layout supplies the periodic images in x).
// ---------------------------------------------------------------------------
template <int N, int TX, bool TAU1, bool W32>
__global__ void __launch_bounds__(TX)
    step_d1q3_kernel(const float* __restrict__ fin, float* __restrict__ fout, const KParams P,
                     int* __restrict__ status) {
  constexpr int Q = 3;
  constexpr int RW = TX + 4, PW = TX + 2;
  __shared__ float zs[N][RW];  // interface-height deviations, see D2Q9
  __shared__ float ps[N][PW];
  const Layout& L = P.L;
  const int nx = P.nx;
  const int x0 = blockIdx.x * TX, tx = threadIdx.x;

  const bool sub = P.sub_amp != 0.f;
  float hh[N], g0[N], sm[N], jx[N];
  {
    float z = sub ? substrate_at(P, x0 + tx, 0) : 0.f;
#pragma unroll
    for (int i = 0; i < N; ++i) {
      const float f0 = __ldg(fin + L.at(i * Q + 0, x0 + tx, 0));
      const float f1 = __ldg(fin + L.at(i * Q + 1, x0 + tx, 0));
      const float f2 = __ldg(fin + L.at(i * Q + 2, x0 + tx, 0));
      const float s = f0 + (f1 + f2);
      g0[i] = f0;
      sm[i] = f1 + f2;
      hh[i] = P.H[i] + s;
      jx[i] = f1 - f2;
      z += s;
      zs[i][tx + 2] = z;
    }
  }
  if (tx < 4) {
    const int rc = tx < 2 ? tx : RW - 4 + tx;  // columns x0 - 2, x0 - 1, x0 + TX, x0 + TX + 1
    const int x = x0 - 2 + rc;
    float z = sub ? substrate_at(P, x, 0) : 0.f;
#pragma unroll
    for (int i = 0; i < N; ++i) {
      const float f0 = __ldg(fin + L.at(i * Q + 0, x, 0));
      const float f1 = __ldg(fin + L.at(i * Q + 1, x, 0));
      const float f2 = __ldg(fin + L.at(i * Q + 2, x, 0));
      z += f0 + (f1 + f2);
      zs[i][chk_index(rc, RW)] = z;
    }
  }
  __syncthreads();
  for (int pc = tx; pc < PW; pc += TX) {
    const int rc = pc + 1;
    float zw[N], zc[N], ze[N], p[N];
#pragma unroll
    for (int i = 0; i < N; ++i) {
      zw[i] = zs[i][chk_index(rc - 1, RW)];
      zc[i] = zs[i][chk_index(rc, RW)];
      ze[i] = zs[i][chk_index(rc + 1, RW)];
    }
    if (sub) {
      const int x = x0 - 1 + pc;
      d1q3_pressures<N, W32>(P, zw, zc, ze, p, substrate_at(P, x - 1, 0), substrate_at(P, x, 0),
                             substrate_at(P, x + 1, 0));
    } else {
      d1q3_pressures<N, W32>(P, zw, zc, ze, p);
    }
#pragma unroll
    for (int i = 0; i < N; ++i) ps[i][chk_index(pc, PW)] = p[i];
  }
  __syncthreads();
  const int gx = x0 + tx;
  if (gx >= nx) return;
  float pw[N], pc[N], pe[N], fo[N][Q], fs[N][Q];
#pragma unroll
  for (int i = 0; i < N; ++i) {
    pw[i] = ps[i][tx];
    pc[i] = ps[i][tx + 1];
    pe[i] = ps[i][tx + 2];
#pragma unroll
    for (int k = 0; k < Q; ++k) fo[i][k] = TAU1 ? 0.f : fin[L.at(i * Q + k, gx, 0)];
  }
  const bool bad = d1q3_collide_cell<N, TAU1>(P, g0, sm, hh, jx, pw, pc, pe, fo, fs);
  int dxs[3], xis[3];
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    int dx = gx + c - 1;
    dx += (dx < 0) ? nx : 0;
    dx -= (dx >= nx) ? nx : 0;
    dxs[c] = dx;
    xis[c] = P.tiny ? kNoImage : image_of(dx, nx);  // tiny lattices refresh ghosts apart
  }
#pragma unroll
  for (int i = 0; i < N; ++i)
#pragma unroll
    for (int k = 0; k < Q; ++k) {
      const int cxi = Lattice<1>::cx(k) + 1;
      store_edge(fout + (long)(i * Q + k) * L.plane, L, dxs[cxi], 0, xis[cxi], kNoImage,
                 fs[i][k]);
    }
  if (bad) atomicOr(status, kStatusNonfinite);
}

// ---------------------------------------------------------------------------
// D1Q3, persistent: one CTA holds the whole lattice in shared memory and
// runs nsteps steps in one launch, with barriers between the phases of a
// step instead of kernel launches. Shared memory (floats): two population
// buffers [3N][nx], z [N][nx], p [N][nx]. The lattice is read from fin and
// the final state written to fout (which may be fin), ghost images
// included. Same cell arithmetic as step_d1q3_kernel.
// ---------------------------------------------------------------------------
constexpr int kD1PT = 256;

template <int N, bool TAU1, bool W32>
__global__ void __launch_bounds__(kD1PT)
    step_d1q3_persistent(const float* fin, float* fout, const KParams P, int nsteps,
                         int* __restrict__ status) {
  constexpr int Q = 3;
  extern __shared__ __align__(16) float sm[];
  const Layout& L = P.L;
  const int nx = P.nx, tid = threadIdx.x;
  float* fa = sm;                     // current populations [i * Q + k][x]
  float* fb = fa + 3 * N * nx;        // next populations
  float* zsm = fb + 3 * N * nx;       // [i][x]
  float* psm = zsm + N * nx;          // [i][x]
  for (int t = tid; t < Q * N * nx; t += kD1PT) {
    const int pl = t / nx, x = t - pl * nx;
    *chk_smem(fa + t) = fin[L.at(pl, x, 0)];
  }
  __syncthreads();
  bool bad = false;
  for (int s = 0; s < nsteps; ++s) {
    // moments -> z
    for (int x = tid; x < nx; x += kD1PT) {
      float z = P.sub_amp != 0.f ? substrate_at(P, x, 0) : 0.f;
#pragma unroll
      for (int i = 0; i < N; ++i) {
        z += *chk_smem(fa + (i * Q + 0) * nx + x) +
             (*chk_smem(fa + (i * Q + 1) * nx + x) + *chk_smem(fa + (i * Q + 2) * nx + x));
        *chk_smem(zsm + i * nx + x) = z;
      }
    }
    __syncthreads();
    // pressures
    for (int x = tid; x < nx; x += kD1PT) {
      const int xw = x == 0 ? nx - 1 : x - 1, xe = x == nx - 1 ? 0 : x + 1;
      float zw[N], zc[N], ze[N], p[N];
#pragma unroll
      for (int i = 0; i < N; ++i) {
        zw[i] = *chk_smem(zsm + i * nx + xw);
        zc[i] = *chk_smem(zsm + i * nx + x);
        ze[i] = *chk_smem(zsm + i * nx + xe);
      }
      if (P.sub_amp != 0.f)
        d1q3_pressures<N, W32>(P, zw, zc, ze, p, substrate_at(P, x - 1, 0),
                               substrate_at(P, x, 0), substrate_at(P, x + 1, 0));
      else
        d1q3_pressures<N, W32>(P, zw, zc, ze, p);
#pragma unroll
      for (int i = 0; i < N; ++i) *chk_smem(psm + i * nx + x) = p[i];
    }
    __syncthreads();
    // force, collision, streaming into fb
    for (int x = tid; x < nx; x += kD1PT) {
      const int xw = x == 0 ? nx - 1 : x - 1, xe = x == nx - 1 ? 0 : x + 1;
      float g0[N], sm[N], hh[N], jx[N], pw[N], pc[N], pe[N], fo[N][Q], fs[N][Q];
#pragma unroll
      for (int i = 0; i < N; ++i) {
        const float f0 = *chk_smem(fa + (i * Q + 0) * nx + x);
        const float f1 = *chk_smem(fa + (i * Q + 1) * nx + x);
        const float f2 = *chk_smem(fa + (i * Q + 2) * nx + x);
        const float sum = f0 + (f1 + f2);
        g0[i] = f0;
        sm[i] = f1 + f2;
        hh[i] = P.H[i] + sum;
        jx[i] = f1 - f2;
        fo[i][0] = f0;
        fo[i][1] = f1;
        fo[i][2] = f2;
        pw[i] = *chk_smem(psm + i * nx + xw);
        pc[i] = *chk_smem(psm + i * nx + x);
        pe[i] = *chk_smem(psm + i * nx + xe);
      }
      bad |= d1q3_collide_cell<N, TAU1>(P, g0, sm, hh, jx, pw, pc, pe, fo, fs);
      const int dst[3] = {x, xe, xw};  // c_k = 0, +1, -1
#pragma unroll
      for (int i = 0; i < N; ++i)
#pragma unroll
        for (int k = 0; k < Q; ++k) *chk_smem(fb + (i * Q + k) * nx + dst[k]) = fs[i][k];
    }
    __syncthreads();
    float* t = fa;
    fa = fb;
    fb = t;
  }
  // final state, real cells and the ghost images x in [-2, nx + 2)
  for (int t = tid; t < Q * N * (nx + 4); t += kD1PT) {
    const int pl = t / (nx + 4), x = t - pl * (nx + 4) - 2;
    int sx = x % nx;
    sx += sx < 0 ? nx : 0;
    fout[L.at(pl, x, 0)] = *chk_smem(fa + pl * nx + sx);
  }
  if (bad) atomicOr(status, kStatusNonfinite);
}

// ---------------------------------------------------------------------------
// dispatch
// ---------------------------------------------------------------------------
constexpr int kD1TX = 128;

template <int N, int MODE>
static cudaError_t launch_d2(const StepLaunch& a, cudaStream_t st) {
  using T = D2Tile<N>;
  auto kern = step_d2q9_tma<N, MODE>;
  // raise the dynamic shared-memory limit and size the persistent grid once
  // per device and instantiation
  static unsigned long long configured = 0;
  static int per_sm[64];
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev >= 64) return cudaErrorInvalidDevice;
  if (!((configured >> dev) & 1ull)) {
    e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)T::kSmem);
    if (e != cudaSuccess) return e;
    int nb = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, kern, T::NT, T::kSmem);
    if (e != cudaSuccess) return e;
    per_sm[dev] = nb > 0 ? nb : 1;
    configured |= 1ull << dev;
  }
  const int ntiles = ((a.P.nx + T::TX - 1) / T::TX) * ((a.P.ny + T::TY - 1) / T::TY);
  const int slots = a.num_sms * per_sm[dev];
  const int grid = ntiles < slots ? ntiles : slots;
  // launched as a programmatic dependent of the previous kernel on the
  // stream (see d2q9_tile_loop)
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(grid);
  cfg.blockDim = dim3(T::NT);
  cfg.dynamicSmemBytes = T::kSmem;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kern, *a.fin_map, a.fout, a.P, a.status, a.sched, a.reverse);
}

int step_mode(const KParams& P) {
  if (P.omega != 1.f) return kGeneral;
  const bool w32 = (P.wet_kind == 0 && P.nw == 3 && P.mw == 2);
  bool nn = true;  // spreading coefficients only between neighbouring interfaces
  for (int l = 0; l < P.n; ++l)
    for (int k = 2; k <= P.n - l; ++k) nn = nn && (P.S[l][k - 1] == 0.f);
  return (w32 && nn && P.sub_amp == 0.f) ? kFast : kTau1;
}

// batch kernels: dynamic shared memory and occupancy, once per device and
// instantiation
template <int N, int MODE, int RPT>
static cudaError_t launch_batch_nmr(const BatchLaunch& a, cudaStream_t st) {
  using T = D2Tile<N, RPT>;
  auto kern = step_d2q9_batch<N, MODE, RPT>;
  static unsigned long long configured = 0;
  static int per_sm[64];
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev >= 64) return cudaErrorInvalidDevice;
  if (!((configured >> dev) & 1ull)) {
    e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)T::kSmem);
    if (e != cudaSuccess) return e;
    int nb = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, kern, T::NT, T::kSmem);
    if (e != cudaSuccess) return e;
    per_sm[dev] = nb > 0 ? nb : 1;
    configured |= 1ull << dev;
  }
  if (a.ntiles <= 0) return cudaSuccess;
  const int slots = a.num_sms * per_sm[dev];
  const int grid = a.ntiles < slots ? a.ntiles : slots;
  kern<<<grid, T::NT, T::kSmem, st>>>(a.inst, a.table, a.ntiles, a.cur, a.status, a.sched);
  return cudaGetLastError();
}

template <int N, int MODE>
static cudaError_t launch_batch_nm(const BatchLaunch& a, cudaStream_t st) {
  if (a.variant == 1) return launch_batch_nmr<N, MODE, 1>(a, st);
  if constexpr (N <= 3) return launch_batch_nmr<N, MODE, 2>(a, st);
  return cudaErrorInvalidValue;  // 16-row tiles do not fit for n >= 4
}

template <int N>
static cudaError_t launch_batch_n(const BatchLaunch& a, cudaStream_t st) {
  switch (a.mode) {
    case kGeneral: return launch_batch_nm<N, kGeneral>(a, st);
    case kTau1: return launch_batch_nm<N, kTau1>(a, st);
    case kFast: return launch_batch_nm<N, kFast>(a, st);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_batch_step(const BatchLaunch& a, cudaStream_t st) {
  switch (a.n) {
    case 1: return launch_batch_n<1>(a, st);
    case 2: return launch_batch_n<2>(a, st);
    case 3: return launch_batch_n<3>(a, st);
    case 4: return launch_batch_n<4>(a, st);
    case 5: return launch_batch_n<5>(a, st);
    default: return cudaErrorInvalidValue;
  }
}

template <int N>
static cudaError_t launch_n(const StepLaunch& a, cudaStream_t st) {
  const bool tau1 = (a.P.omega == 1.f);
  const bool w32 = (a.P.wet_kind == 0 && a.P.nw == 3 && a.P.mw == 2);
  if (a.lattice == 2) {
    switch (step_mode(a.P)) {
      case kGeneral: return launch_d2<N, kGeneral>(a, st);
      case kFast: return launch_d2<N, kFast>(a, st);
      default: return launch_d2<N, kTau1>(a, st);
    }
  }
  dim3 grid((a.P.nx + kD1TX - 1) / kD1TX);
  if (tau1) {
    if (w32)
      step_d1q3_kernel<N, kD1TX, true, true><<<grid, kD1TX, 0, st>>>(a.fin, a.fout, a.P, a.status);
    else
      step_d1q3_kernel<N, kD1TX, true, false><<<grid, kD1TX, 0, st>>>(a.fin, a.fout, a.P, a.status);
  } else {
    step_d1q3_kernel<N, kD1TX, false, false><<<grid, kD1TX, 0, st>>>(a.fin, a.fout, a.P, a.status);
  }
  return cudaGetLastError();
}

size_t step_persistent_smem(int n, int lattice, int nx) {
  if (lattice != 1 || n < 1 || n > kMaxLayers || nx < 1) return 0;
  return (size_t)8 * n * nx * sizeof(float);
}

template <int N, bool TAU1, bool W32>
static cudaError_t launch_d1p(const StepLaunch& a, int nsteps, cudaStream_t st) {
  auto kern = step_d1q3_persistent<N, TAU1, W32>;
  const size_t smem = step_persistent_smem(N, 1, a.P.nx);
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  kern<<<1, kD1PT, smem, st>>>(a.fin, a.fout, a.P, nsteps, a.status);
  return cudaGetLastError();
}

template <int N>
static cudaError_t launch_d1p_n(const StepLaunch& a, int nsteps, cudaStream_t st) {
  const bool tau1 = (a.P.omega == 1.f);
  const bool w32 = (a.P.wet_kind == 0 && a.P.nw == 3 && a.P.mw == 2);
  if (tau1) return w32 ? launch_d1p<N, true, true>(a, nsteps, st) : launch_d1p<N, true, false>(a, nsteps, st);
  return launch_d1p<N, false, false>(a, nsteps, st);
}

cudaError_t launch_step_persistent(const StepLaunch& a, int nsteps, cudaStream_t st) {
  switch (a.P.n) {
    case 1: return launch_d1p_n<1>(a, nsteps, st);
    case 2: return launch_d1p_n<2>(a, nsteps, st);
    case 3: return launch_d1p_n<3>(a, nsteps, st);
    case 4: return launch_d1p_n<4>(a, nsteps, st);
    case 5: return launch_d1p_n<5>(a, nsteps, st);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_step(const StepLaunch& a, cudaStream_t st) {
  switch (a.P.n) {
    case 1: return launch_n<1>(a, st);
    case 2: return launch_n<2>(a, st);
    case 3: return launch_n<3>(a, st);
    case 4: return launch_n<4>(a, st);
    case 5: return launch_n<5>(a, st);
    default: return cudaErrorInvalidValue;
  }
}

int step_tile_cols(int lattice) { return lattice == 2 ? 32 : kD1TX; }

int step_tile_rows(int n, int lattice) {
  if (lattice != 2) return 1;
  switch (n) {
    case 1: return D2Tile<1>::TY;
    case 2: return D2Tile<2>::TY;
    case 3: return D2Tile<3>::TY;
    case 4: return D2Tile<4>::TY;
    default: return D2Tile<5>::TY;
  }
}

MLSW_DEFINE_BOUNDS_READER(bounds_violations_step)

}  // namespace mlsw
