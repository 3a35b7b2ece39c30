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
#include "tma.cuh"

namespace mlsw {

// ---------------------------------------------------------------------------
// Stores of one post-collision population to its streamed destination
// (dx, dy) (already periodic) and to every ghost cell that images it.
// xm / ym: bit g set when ghost column / row g (x = -2, -1, nx, nx + 1)
// images the destination column / row.
// ---------------------------------------------------------------------------
__device__ __forceinline__ int ghost_pos(int g, int n) {
  return g == 0 ? -2 : (g == 1 ? -1 : (g == 2 ? n : n + 1));
}

__device__ __forceinline__ unsigned ghost_mask(const int (&src)[4], int d) {
  return (src[0] == d ? 1u : 0u) | (src[1] == d ? 2u : 0u) | (src[2] == d ? 4u : 0u) |
         (src[3] == d ? 8u : 0u);
}

__device__ __forceinline__ void store_images(float* __restrict__ plane_base, const Layout& L,
                                             int dx, int dy, unsigned xm, unsigned ym, float v) {
  plane_base[(long)(dy + L.gy) * L.pitch + dx + L.gx] = v;
  if (xm | ym) {
    for (int gr = -1; gr < 4; ++gr) {
      if (gr >= 0 && !((ym >> gr) & 1u)) continue;
      const int yy = gr < 0 ? dy : ghost_pos(gr, L.ny);
      for (int gc = -1; gc < 4; ++gc) {
        if (gr < 0 && gc < 0) continue;
        if (gc >= 0 && !((xm >> gc) & 1u)) continue;
        const int xx = gc < 0 ? dx : ghost_pos(gc, L.nx);
        plane_base[(long)(yy + L.gy) * L.pitch + xx + L.gx] = v;
      }
    }
  }
}

// Lattices with both sides >= 4 cells: a real column d has at most one
// ghost image (d + n for d < 2, d - n for d >= n - 2), likewise rows, so a
// population near an edge needs at most three extra stores.
constexpr int kNoImage = -(1 << 28);

__device__ __forceinline__ int image_of(int d, int n) {
  return d < 2 ? d + n : (d >= n - 2 ? d - n : kNoImage);
}

__device__ __forceinline__ void store_edge(float* __restrict__ plane_base, const Layout& L,
                                           int dx, int dy, int xi, int yi, float v) {
  const long r0 = (long)(dy + L.gy) * L.pitch;
  plane_base[r0 + dx + L.gx] = v;
  if (xi != kNoImage) plane_base[r0 + xi + L.gx] = v;
  if (yi != kNoImage) {
    const long r1 = (long)(yi + L.gy) * L.pitch;
    plane_base[r1 + dx + L.gx] = v;
    if (xi != kNoImage) plane_base[r1 + xi + L.gx] = v;
  }
}

// Equilibrium, BGK with forcing for one layer at one cell; fs[k] receives
// the post-collision populations (rest one stored shifted by H).
// f_old (read only when !TAU1) holds the stored pre-collision populations.
template <int LAT, bool TAU1>
__device__ __forceinline__ void collide(const KParams& P, float h, float dh, float jx, float jy,
                                        float Fx, float Fy, const float* f_old,
                                        float (&fs)[Lattice<LAT>::Q]) {
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
  // stored shifted by H, i.e. dh - sum_eq
  const float geq0 = dh - sum_eq;
  fs[0] = TAU1 ? geq0 : f_old[0] + P.omega * (geq0 - f_old[0]);
}

// ---------------------------------------------------------------------------
// D2Q9 collision with the opposite directions paired: for c_{k+4} = -c_k the
// equilibria share w_k h (4.5 (c.U)^2 - 1.5 U^2) and differ in the sign of
// 3 w_k h c.U, and the forcing terms 3 w_k c.F are odd, so each pair costs
// one symmetric and one antisymmetric part. Directions: 1 (1,0), 2 (1,1),
// 3 (0,1), 4 (-1,1); 5..8 are their opposites.
// ---------------------------------------------------------------------------
template <bool TAU1>
__device__ __forceinline__ void collide_d2q9(const KParams& P, float h, float dh, float jx,
                                             float jy, float Fx, float Fy, const float* f_old,
                                             float (&fs)[9]) {
  const float ih = rcp(h);
  const float ux = jx * ih, uy = jy * ih;
  const float u15 = 1.5f * (ux * ux + uy * uy);
  float sumsym = 0.f;
  const float cus[4] = {ux, ux + uy, uy, uy - ux};
  const float cfs[4] = {Fx, Fx + Fy, Fy, Fy - Fx};
  const float ws[4] = {1.f / 9.f, 1.f / 36.f, 1.f / 9.f, 1.f / 36.f};
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const float A = ws[q] * h;
    const float cu = cus[q];
    const float sym = A * (4.5f * cu * cu - u15);
    sumsym += sym;
    if (TAU1) {
      const float anti = 3.f * (A * cu + ws[q] * cfs[q]);
      fs[q + 1] = sym + anti;
      fs[q + 5] = sym - anti;
    } else {
      const float aeq = 3.f * A * cu, afr = 3.f * ws[q] * cfs[q];
      fs[q + 1] = f_old[q + 1] + P.omega * ((sym + aeq) - f_old[q + 1]) + afr;
      fs[q + 5] = f_old[q + 5] + P.omega * ((sym - aeq) - f_old[q + 5]) - afr;
    }
  }
  // rest population h - (sum of moving equilibria) = h (1 - w_0 U^2/(2 cs^2)),
  // stored shifted by H
  const float geq0 = dh - 2.f * sumsym;
  fs[0] = TAU1 ? geq0 : f_old[0] + P.omega * (geq0 - f_old[0]);
}

// ---------------------------------------------------------------------------
// D2Q9, persistent, TMA-fed. Tile 32 x TY, NT threads (32 x BY), RPT tile
// rows per thread. Shared memory (floats unless noted):
//   stage [9N][TY + 4][40]   TMA box, x from x0 - 4, y from y0 - 2
//   zs, hs [N][TY + 4][36]   z_i deviation / h_i on the two-ring region
//   ps     [N][TY + 2][34]   p_i on the one-ring region
//   bar                      mbarrier (8 bytes)
// Each CTA needs about 111 KB, so two CTAs share an SM and fill each
// other's barrier waits. With tau = 1 the next tile's copy is issued as soon
// as the moments are formed and lands while this tile finishes.
// ---------------------------------------------------------------------------
template <int N>
struct D2Tile {
  static constexpr int Q = 9, PN = N * Q, TX = 32;
  static constexpr int TY = N <= 3 ? 16 : 8, NT = 256, BY = NT / 32, RPT = TY / BY;
  static constexpr int BW = TX + 8, BH = TY + 4, STAGE = PN * BH * BW;
  static constexpr int RW = TX + 4, RH = TY + 4, PW = TX + 2, PH = TY + 2;
  static constexpr int NHALO = 4 * RW + 4 * TY;
  static constexpr size_t kStageBytes = (size_t)STAGE * 4;
  static constexpr size_t kOffZ = kStageBytes;
  static constexpr size_t kOffH = kOffZ + (size_t)N * RH * RW * 4;
  static constexpr size_t kOffP = kOffH + (size_t)N * RH * RW * 4;
  static constexpr size_t kOffBar = (kOffP + (size_t)N * PH * PW * 4 + 15) / 16 * 16;
  static constexpr size_t kSmem = kOffBar + 16;
  static_assert(kStageBytes % 128 == 0, "stage alignment");
  static_assert(NHALO <= NT, "one halo cell per thread");
  static_assert(RPT * BY == TY, "tile rows");
};

template <int N, bool TAU1, bool W32>
__global__ void __launch_bounds__(256, 2)
    step_d2q9_tma(const __grid_constant__ CUtensorMap fin_map, float* __restrict__ fout,
                  const KParams P, int* __restrict__ status, int* __restrict__ sched) {
  using T = D2Tile<N>;
  constexpr int Q = 9, TX = T::TX, TY = T::TY, BY = T::BY, RPT = T::RPT;
  constexpr int BW = T::BW, BH = T::BH, RW = T::RW, RH = T::RH, PW = T::PW, PH = T::PH;
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  float* stage = reinterpret_cast<float*>(smem_raw);
  float* zs = reinterpret_cast<float*>(smem_raw + T::kOffZ);
  float* hs = reinterpret_cast<float*>(smem_raw + T::kOffH);
  float* ps = reinterpret_cast<float*>(smem_raw + T::kOffP);
  uint64_t* bar = reinterpret_cast<uint64_t*>(smem_raw + T::kOffBar);
  __shared__ int next_tile;

  const int tid = threadIdx.x;
  const Layout& L = P.L;
  const int nx = P.nx, ny = P.ny;
  const int ntx = (nx + TX - 1) / TX, nty = (ny + TY - 1) / TY, ntiles = ntx * nty;

  auto issue = [&](int t) {
    const int bx = t % ntx, by = t / ntx;
    fence_proxy_async_smem();
    mbar_arrive_expect_tx(bar, (uint32_t)T::kStageBytes);
    // box origin: real (x0 - 4, y0 - 2) = padded (x0, y0) since gx = 4, gy = 2
    tma_load_3d(stage, &fin_map, bar, bx * TX, by * TY, 0);
  };

  if (tid == 0) {
    mbar_init(bar, 1);
    mbar_init_fence();
  }
  __syncthreads();
  if (tid == 0) {
    tma_prefetch_desc(&fin_map);
    if ((int)blockIdx.x < ntiles) issue(blockIdx.x);
  }

  const int ix = tid % TX, iyb = tid / TX;  // tile cells (ix, iyb + r * BY)
  const long lplane = (long)Q * L.plane;    // floats per layer
  bool bad = false;
  uint32_t parity = 0;
  // Tiles: the first one is blockIdx.x, later ones come from a global
  // counter (sched[0]), so CTAs that drew cheap tiles take more of them.
  // The last CTA to finish resets the counters for the next launch.
  for (int t = blockIdx.x; t < ntiles; parity ^= 1u) {
    const bool timed_out = !mbar_wait_bounded(bar, parity);
    const int x0 = (t % ntx) * TX, y0 = (t / ntx) * TY;

    // ---- M. moments -------------------------------------------------------
    float hh[RPT][N], dd[RPT][N], jx[RPT][N], jy[RPT][N];
#pragma unroll
    for (int rr = 0; rr < RPT; ++rr) {
      const int r = iyb + rr * BY + 2, c = ix + 2;  // two-ring coordinates
      const float* src = stage + r * BW + (c + 2);  // stage column = c + 2
      float z = 0.f;
#pragma unroll
      for (int i = 0; i < N; ++i) {
        float v[Q];
#pragma unroll
        for (int k = 0; k < Q; ++k) v[k] = src[(i * Q + k) * BH * BW];
        const float sm = ((v[0] + v[1]) + (v[2] + v[3])) + ((v[4] + v[5]) + (v[6] + v[7])) + v[8];
        dd[rr][i] = sm;
        hh[rr][i] = P.H[i] + sm;
        jx[rr][i] = ((v[1] + v[2]) + v[8]) - ((v[4] + v[5]) + v[6]);
        jy[rr][i] = ((v[2] + v[3]) + v[4]) - ((v[6] + v[7]) + v[8]);
        z += sm;
        zs[(i * RH + r) * RW + c] = z;
        hs[(i * RH + r) * RW + c] = hh[rr][i];
      }
    }
    if (tid < T::NHALO) {
      const int q = tid;
      int r, c;
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
      const float* src = stage + r * BW + (c + 2);
      float z = 0.f;
#pragma unroll
      for (int i = 0; i < N; ++i) {
        float v[Q];
#pragma unroll
        for (int k = 0; k < Q; ++k) v[k] = src[(i * Q + k) * BH * BW];
        const float sm = ((v[0] + v[1]) + (v[2] + v[3])) + ((v[4] + v[5]) + (v[6] + v[7])) + v[8];
        z += sm;
        zs[(i * RH + r) * RW + c] = z;
        hs[(i * RH + r) * RW + c] = P.H[i] + sm;
      }
    }
    // !TAU1 keeps the pre-collision populations of its own cells for C
    float fo[TAU1 ? 1 : RPT][TAU1 ? 1 : N][Q];
    if (!TAU1) {
#pragma unroll
      for (int rr = 0; rr < RPT; ++rr) {
        const float* src = stage + (iyb + rr * BY + 2) * BW + (ix + 4);
#pragma unroll
        for (int i = 0; i < N; ++i)
#pragma unroll
          for (int k = 0; k < Q; ++k) fo[TAU1 ? 0 : rr][TAU1 ? 0 : i][k] = src[(i * Q + k) * BH * BW];
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
    // every thread holds what it needs from the stage: refill it with the
    // next tile, which lands while this tile is finished
    if (tid == 0) {
      const int nt = (int)gridDim.x + atomicAdd(sched, 1);
      next_tile = nt;
      if (nt < ntiles) issue(nt);
    }

    // ---- P. pressures on the one-ring region ----------------------------------
    for (int q = tid; q < PH * PW; q += T::NT) {
      const int pr = q / PW, pc = q - pr * PW;
      const int r = pr + 1, c = pc + 1;
      float h[N], gzx[N], gzy[N], lz[N], p[N];
#pragma unroll
      for (int i = 0; i < N; ++i) {
        const float* zc = zs + (i * RH + r) * RW + c;
        const float zE = zc[1], zW = zc[-1], zN = zc[RW], zS = zc[-RW];
        const float zNE = zc[RW + 1], zNW = zc[RW - 1], zSE = zc[-RW + 1], zSW = zc[-RW - 1];
        // (1/cs^2)(w_1 = 1/9, w_2 = 1/36) -> 1/3 and 1/12
        gzx[i] = (zE - zW) * (1.f / 3.f) + ((zNE - zNW) + (zSE - zSW)) * (1.f / 12.f);
        gzy[i] = (zN - zS) * (1.f / 3.f) + ((zNE - zSE) + (zNW - zSW)) * (1.f / 12.f);
        // (2/cs^2) sum_k w_k (z_k - z_0): 2/3 on the edges, 1/6 on the corners
        lz[i] = ((zE + zW) + (zN + zS)) * (2.f / 3.f) + ((zNE + zNW) + (zSE + zSW)) * (1.f / 6.f) -
                zc[0] * (10.f / 3.f);
        h[i] = hs[(i * RH + r) * RW + c];
      }
      layer_pressures<N, W32>(P, h, gzx, gzy, lz, p);
#pragma unroll
      for (int i = 0; i < N; ++i) ps[(i * PH + pr) * PW + pc] = p[i];
    }
    __syncthreads();
    const int tnext = next_tile;  // written by thread 0 before the barrier above

    // ---- C. force, collision, streaming -----------------------------------------
#pragma unroll
    for (int rr = 0; rr < RPT; ++rr) {
      const int iy = iyb + rr * BY;
      const int gx = x0 + ix, gy = y0 + iy;
      if (gx >= nx || gy >= ny) continue;
      float Rx[N], Ry[N];
      friction<N>(P, hh[rr], jx[rr], jy[rr], Rx, Ry);
      // destinations of the three column / row offsets and their images
      int dxs[3], dys[3], xis[3], yis[3];
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        int dx = gx + c - 1, dy = gy + c - 1;
        dx += (dx < 0) ? nx : 0;
        dx -= (dx >= nx) ? nx : 0;
        dy += (dy < 0) ? ny : 0;
        dy -= (dy >= ny) ? ny : 0;
        dxs[c] = dx;
        dys[c] = dy;
        xis[c] = image_of(dx, nx);
        yis[c] = image_of(dy, ny);
      }
      const bool images = P.tiny || (xis[0] != kNoImage) || (xis[1] != kNoImage) ||
                          (xis[2] != kNoImage) || (yis[0] != kNoImage) ||
                          (yis[1] != kNoImage) || (yis[2] != kNoImage);
      int koff[Q];
#pragma unroll
      for (int k = 0; k < Q; ++k)
        koff[k] = k * (int)L.plane + (dys[Lattice<2>::cy(k) + 1] + L.gy) * L.pitch +
                  dxs[Lattice<2>::cx(k) + 1] + L.gx;
#pragma unroll
      for (int i = 0; i < N; ++i) {
        const float* pc = ps + (i * PH + iy + 1) * PW + ix + 1;
        const float gpx = (pc[1] - pc[-1]) * (1.f / 3.f) +
                          ((pc[PW + 1] - pc[PW - 1]) + (pc[-PW + 1] - pc[-PW - 1])) * (1.f / 12.f);
        const float gpy = (pc[PW] - pc[-PW]) * (1.f / 3.f) +
                          ((pc[PW + 1] - pc[-PW + 1]) + (pc[PW - 1] - pc[-PW - 1])) * (1.f / 12.f);
        const float h = hh[rr][i];
        const float Fx = -h * gpx + Rx[i];
        const float Fy = -h * gpy + Ry[i];
        bad |= !(h > 0.f) || !isfinite(Fx + Fy);
        float fs[Q];
        collide_d2q9<TAU1>(P, h, dd[rr][i], jx[rr][i], jy[rr][i], Fx, Fy,
                           fo[TAU1 ? 0 : rr][TAU1 ? 0 : i], fs);
        float* obase = fout + (long)i * lplane;
        if (!images) {
#pragma unroll
          for (int k = 0; k < Q; ++k) obase[koff[k]] = fs[k];
        } else if (!P.tiny) {
#pragma unroll
          for (int k = 0; k < Q; ++k) {
            const int cxi = Lattice<2>::cx(k) + 1, cyi = Lattice<2>::cy(k) + 1;
            store_edge(obase + (long)k * L.plane, L, dxs[cxi], dys[cyi], xis[cxi], yis[cyi],
                       fs[k]);
          }
        } else {
#pragma unroll
          for (int k = 0; k < Q; ++k) {
            const int cxi = Lattice<2>::cx(k) + 1, cyi = Lattice<2>::cy(k) + 1;
            store_images(obase + (long)k * L.plane, L, dxs[cxi], dys[cyi],
                         ghost_mask(P.gsrcx, dxs[cxi]), ghost_mask(P.gsrcy, dys[cyi]), fs[k]);
          }
        }
      }
    }
    t = tnext;
  }
  if (bad) atomicOr(status, kStatusNonfinite);
  if (tid == 0 && atomicAdd(sched + 1, 1) == (int)gridDim.x - 1) {
    sched[0] = 0;  // every CTA has drawn its last tile
    sched[1] = 0;
  }
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
  __shared__ float zs[N][RW];
  __shared__ float hs[N][RW];
  __shared__ float ps[N][PW];
  const Layout& L = P.L;
  const int nx = P.nx;
  const int x0 = blockIdx.x * TX, tx = threadIdx.x;

  float hh[N], dd[N], jx[N];
  {
    float z = 0.f;
#pragma unroll
    for (int i = 0; i < N; ++i) {
      const float f0 = __ldg(fin + L.at(i * Q + 0, x0 + tx, 0));
      const float f1 = __ldg(fin + L.at(i * Q + 1, x0 + tx, 0));
      const float f2 = __ldg(fin + L.at(i * Q + 2, x0 + tx, 0));
      const float s = f0 + (f1 + f2);
      dd[i] = s;
      hh[i] = P.H[i] + s;
      jx[i] = f1 - f2;
      z += s;
      hs[i][tx + 2] = hh[i];
      zs[i][tx + 2] = z;
    }
  }
  if (tx < 4) {
    const int rc = tx < 2 ? tx : RW - 4 + tx;  // columns x0 - 2, x0 - 1, x0 + TX, x0 + TX + 1
    const int x = x0 - 2 + rc;
    float z = 0.f;
#pragma unroll
    for (int i = 0; i < N; ++i) {
      const float s = __ldg(fin + L.at(i * Q + 0, x, 0)) +
                      (__ldg(fin + L.at(i * Q + 1, x, 0)) + __ldg(fin + L.at(i * Q + 2, x, 0)));
      z += s;
      hs[i][rc] = P.H[i] + s;
      zs[i][rc] = z;
    }
  }
  __syncthreads();
  for (int pc = tx; pc < PW; pc += TX) {
    const int rc = pc + 1;
    float h[N], gxz[N], gyz[N], lz[N], p[N];
#pragma unroll
    for (int i = 0; i < N; ++i) {
      const float c = zs[i][rc];
      const float e = zs[i][rc + 1] - c, wv = zs[i][rc - 1] - c;
      gxz[i] = 0.5f * (e - wv);  // (1/cs^2) w_1 = 1/2
      gyz[i] = 0.f;
      lz[i] = e + wv;            // (2/cs^2) w_1 = 1
      h[i] = hs[i][rc];
    }
    layer_pressures<N, W32>(P, h, gxz, gyz, lz, p);
#pragma unroll
    for (int i = 0; i < N; ++i) ps[i][pc] = p[i];
  }
  __syncthreads();
  const int gx = x0 + tx;
  if (gx >= nx) return;
  float zero[N], Rx[N], Ry[N];
#pragma unroll
  for (int i = 0; i < N; ++i) zero[i] = 0.f;
  friction<N>(P, hh, jx, zero, Rx, Ry);
  int dxs[3], xis[3];
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    int dx = gx + c - 1;
    dx += (dx < 0) ? nx : 0;
    dx -= (dx >= nx) ? nx : 0;
    dxs[c] = dx;
    xis[c] = image_of(dx, nx);
  }
  bool bad = false;
#pragma unroll
  for (int i = 0; i < N; ++i) {
    const float c = ps[i][tx + 1];
    const float gpx = 0.5f * ((ps[i][tx + 2] - c) - (ps[i][tx] - c));
    const float h = hh[i];
    const float Fx = -h * gpx + Rx[i];
    bad |= !(h > 0.f) || !isfinite(Fx) || !isfinite(jx[i]);
    float fo[Q];
    if (!TAU1) {
#pragma unroll
      for (int k = 0; k < Q; ++k) fo[k] = fin[L.at(i * Q + k, gx, 0)];
    }
    float fs[Q];
    collide<1, TAU1>(P, h, dd[i], jx[i], 0.f, Fx, 0.f, fo, fs);
#pragma unroll
    for (int k = 0; k < Q; ++k) {
      const int cxi = Lattice<1>::cx(k) + 1;
      float* base = fout + (long)(i * Q + k) * L.plane;
      if (!P.tiny)
        store_edge(base, L, dxs[cxi], 0, xis[cxi], kNoImage, fs[k]);
      else
        store_images(base, L, dxs[cxi], 0, ghost_mask(P.gsrcx, dxs[cxi]), 0u, fs[k]);
    }
  }
  if (bad) atomicOr(status, kStatusNonfinite);
}

// ---------------------------------------------------------------------------
// dispatch
// ---------------------------------------------------------------------------
constexpr int kD1TX = 128;

template <int N, bool TAU1, bool W32>
static cudaError_t launch_d2(const StepLaunch& a, cudaStream_t st) {
  using T = D2Tile<N>;
  auto kern = step_d2q9_tma<N, TAU1, W32>;
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
  kern<<<grid, T::NT, T::kSmem, st>>>(*a.fin_map, a.fout, a.P, a.status, a.sched);
  return cudaGetLastError();
}

template <int N, bool TAU1, bool W32>
static cudaError_t launch_n(const StepLaunch& a, cudaStream_t st) {
  if (a.lattice == 2) return launch_d2<N, TAU1, W32>(a, st);
  dim3 grid((a.P.nx + kD1TX - 1) / kD1TX);
  step_d1q3_kernel<N, kD1TX, TAU1, W32><<<grid, kD1TX, 0, st>>>(a.fin, a.fout, a.P, a.status);
  return cudaGetLastError();
}

template <bool TAU1, bool W32>
static cudaError_t launch_tau(const StepLaunch& a, cudaStream_t st) {
  switch (a.P.n) {
    case 1: return launch_n<1, TAU1, W32>(a, st);
    case 2: return launch_n<2, TAU1, W32>(a, st);
    case 3: return launch_n<3, TAU1, W32>(a, st);
    case 4: return launch_n<4, TAU1, W32>(a, st);
    case 5: return launch_n<5, TAU1, W32>(a, st);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_step(const StepLaunch& a, cudaStream_t st) {
  const bool w32 = (a.P.nw == 3 && a.P.mw == 2);
  const bool tau1 = (a.P.omega == 1.f);
  if (tau1) return w32 ? launch_tau<true, true>(a, st) : launch_tau<true, false>(a, st);
  return w32 ? launch_tau<false, true>(a, st) : launch_tau<false, false>(a, st);
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

}  // namespace mlsw
