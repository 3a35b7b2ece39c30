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

#include "kernels.h"
#include "physics.cuh"
#include "d2q9_tile.cuh"

namespace mlsw {


template <int N, int MODE>
__global__ void __launch_bounds__(256, 2)
    step_d2q9_tma(const __grid_constant__ CUtensorMap fin_map, float* __restrict__ fout,
                  const __grid_constant__ KParams P, int* __restrict__ status,
                  int* __restrict__ sched, int rev) {
  using Tl = D2Tile<N>;
  const int ntx = (P.nx + Tl::TX - 1) / Tl::TX, nty = (P.ny + Tl::TY - 1) / Tl::TY;
  const SingleTiles tiles{&P, &fin_map, fout, ntx, ntx * nty, rev};
  d2q9_tile_loop<N, MODE, Tl::RPT>(tiles, status, sched, (int)blockIdx.x);
  tile_loop_finish(sched);
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
