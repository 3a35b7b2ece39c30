// unet.cu -- U-Net surrogate of 64 LBM steps on the 5th-generation tensor
// cores (tcgen05), with its training.
//
// The network maps the layer heights h(t) of a periodic lattice to
// h(t + 64 steps). Four levels of 32, 64, 128, 256 channels at full, half,
// quarter and eighth resolution; two 3 x 3 periodic convolutions with ReLU
// per level on the way down (2 x 2 average pooling between levels) and on
// the way up (nearest 2x upsampling, concatenated with the same level's
// features from the way down), then a 3 x 3 convolution to 16 output
// channels, the first n of which are the change of the n layers times
// out_scale. Every sample is normalised by the RMS s of its deviations
// h_i - mean h_i over all its layers: the input planes are
// (h_i - mean h_i) in_scale / s, then the problem's parameters as constant
// planes, then zeros (16 in all), and the change is the output times
// s / out_scale. In the near-linear regime the change over a window scales
// with the deviations, so every window looks alike to the network, and a
// flat film (s = 0) stays exactly flat. The prediction is projected onto
// exact per-layer mass (the change is made mean-free per layer), as the
// LBM conserves it.
//
// Arithmetic: BF16 activations and weights, FP32 accumulation in tensor
// memory. Activations are NHWC with a one-pixel periodic halo ring
// ([B][H+2][W+2][C]) that every kernel writing a tensor keeps current, so
// the tile copies never wrap.
//   * A convolution is an implicit GEMM over 128-pixel tiles: for every tap
//     and every chunk of KC input channels one TMA copy brings the shifted
//     pixels (a box of the activation tensor) and one the weights; one
//     thread issues tcgen05.mma into a TMEM accumulator of 128 x BN; the
//     epilogue (bias, ReLU or a ReLU-gradient mask, BF16, halo images) reads
//     TMEM with tcgen05.ld.
//   * The input gradient is the same kernel with the weights transposed and
//     the taps reversed.
//   * The weight gradient per tap is a GEMM over pixels of two MN-major
//     operands (output gradient and shifted input, channels contiguous),
//     split over CTAs and summed with FP32 atomics.
// Master weights and the Adam moments are FP32.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <new>
#include <random>
#include <vector>

#include "../../include/mlswlbm.h"
#include "tcgen05.cuh"

namespace mlsw {
namespace unet {

typedef __nv_bfloat16 bf16;

constexpr int kCin0 = 16;   // input planes
constexpr int kCout = 16;   // output channels (the first n are used)
constexpr int kLayers = 15;

// Tensors (activations; their gradients use the same index). The four
// levels have 32, 64, 128 and 256 channels.
enum Tensor {
  X0, A0, S0, P1, A1, S1, P2, A2, S2, P3, A3, S3, U2, B2, D2, U1, B1, D1, U0, B0, D0, YG,
  kTensors
};
// channels and level of every tensor (YG: the output gradient, 16 channels)
constexpr int kTC[kTensors] = {16, 32, 32, 32, 64, 64, 64, 128, 128, 128, 256, 256,
                               256, 128, 128, 128, 64, 64, 64, 32, 32, 16};
constexpr int kTL[kTensors] = {0, 0, 0, 1, 1, 1, 2, 2, 2, 3, 3, 3, 2, 2, 2, 1, 1, 1, 0, 0, 0, 0};

struct Layer {
  int in[2];   // input tensors (in[1] = -1: one input); channels concatenated
  int out;     // output tensor (-1: the dense FP32 output)
  int cout;
  bool relu;
};
constexpr Layer kNet[kLayers] = {
    {{X0, -1}, A0, 32, true},  {{A0, -1}, S0, 32, true},  {{P1, -1}, A1, 64, true},
    {{A1, -1}, S1, 64, true},  {{P2, -1}, A2, 128, true}, {{A2, -1}, S2, 128, true},
    {{P3, -1}, A3, 256, true}, {{A3, -1}, S3, 256, true}, {{U2, S2}, B2, 128, true},
    {{B2, -1}, D2, 128, true}, {{U1, S1}, B1, 64, true},  {{B1, -1}, D1, 64, true},
    {{U0, S0}, B0, 32, true},  {{B0, -1}, D0, 32, true},  {{D0, -1}, -1, kCout, false}};

constexpr int layer_cin(int l) {
  return kTC[kNet[l].in[0]] + (kNet[l].in[1] >= 0 ? kTC[kNet[l].in[1]] : 0);
}

// ---------------------------------------------------------------------------
// Implicit-GEMM 3 x 3 convolution on tcgen05.
// ---------------------------------------------------------------------------
struct ConvArgs {
  CUtensorMap in_map[2];  // activations: 4-D [C, W+2, H+2, B], box [KC, BX, BY, 1]
  CUtensorMap w_map;      // weights: 4-D [Cin_tot, rows, 3 dy, 3 dx], box [KC, BN, 3, 1]
  int nin, cin[2], koff[2], cin_tot;
  int H, W;
  int cout;               // output channels
  const float* bias;      // [cout] or null
  int relu;               // ReLU in the epilogue
  int reverse_taps;       // input gradient: tap t reads the pixel at -offset(t)
  // output channels [0, split) go to out[0] (out_c[0] channels), the rest to
  // out[1]; mask[j] (same layout as out[j], or null) multiplies by (mask > 0)
  bf16* out[2];
  int out_c[2], split;
  const bf16* mask[2];
  float* dense;           // FP32 [B][dense_c][H][W] of the first dense_c channels (or null)
  int dense_c;
  int B_tiles;            // 128-pixel tiles of all images of the batch
  int* err;
};

// A convolution tile is 128 output pixels, 16 wide and 8 high. A stage
// holds, for one input, chunk of KC channels and column shift sx in
// {-1, 0, 1}: the 16 x 10 pixels of that shift (rows y0 - 1 .. y0 + 8), a
// K-major operand of 160 rows whose rows 16 (sy + 1) .. + 127 are the
// tile's pixels shifted by (sx, sy), and the BN x KC weights of the three
// taps with that column shift, all by two TMA copies. The three row shifts
// read the pixels at offsets of 16 rows, whole swizzle atoms.
template <int KC, int BN>
struct ConvShape {
  static constexpr int TW = 16, TH = 8;        // the tile of output pixels
  static constexpr int AROWS = TW * (TH + 2);  // rows of a shifted box
  static constexpr int ABYTES = AROWS * KC * 2, BBYTES = BN * KC * 2;
  static constexpr int ASTRIDE = (ABYTES + 1023) / 1024 * 1024;
  static constexpr int BSTRIDE = BBYTES;       // the weight box's dy blocks are contiguous
  static constexpr int STAGE = ASTRIDE + (3 * BBYTES + 1023) / 1024 * 1024;
  static constexpr int ST0 = 204 * 1024 / STAGE;
  // small stages (the 16- and 32-channel layers): six deep, which measured
  // faster than four with more CTAs per SM
  static constexpr int ST = STAGE <= 25 * 1024 ? 6 : (STAGE <= 50 * 1024 ? 4 : (ST0 < 2 ? 2 : ST0));
  static constexpr int ACOLS = BN <= 32 ? 32 : (BN <= 64 ? 64 : 128);
  static constexpr int TCOLS = 2 * ACOLS;          // two accumulators
  static constexpr int CTAS_TMEM = 512 / TCOLS;    // CTAs whose TMEM fits one SM
  static constexpr int kBiasMax = 256;  // output channels whose bias is staged in shared memory
  static constexpr size_t SMEM_NEED = 1024 + (size_t)ST * STAGE + 8 * (2 * ST + 5) + 16 + 4 * kBiasMax;
  // ask for enough shared memory that no more CTAs than CTAS_TMEM share an SM
  static constexpr size_t SMEM_TMEM = 233472 / (CTAS_TMEM + 1) + 1024;
  static constexpr size_t SMEM = SMEM_NEED > SMEM_TMEM ? SMEM_NEED : SMEM_TMEM;
  static_assert(BN <= 128, "output-channel tiles of at most 128");
  static_assert(SMEM_NEED <= 232448, "stages exceed shared memory");
  static_assert(BBYTES % (8 * KC * 2) == 0, "weight blocks are whole swizzle atoms");
};

// 32 bytes to global memory in one 256-bit store (dst 32-byte aligned):
// a lane's 16 BF16 channels fill a whole sector
__device__ __forceinline__ void st_global_v8(void* dst, const uint32_t (&v)[8]) {
  asm volatile("st.global.v8.b32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8};" ::"l"(dst), "r"(v[0]),
               "r"(v[1]), "r"(v[2]), "r"(v[3]), "r"(v[4]), "r"(v[5]), "r"(v[6]), "r"(v[7])
               : "memory");
}

__device__ __forceinline__ uint32_t pack_bf16(float a, float b) {
  __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
  return *reinterpret_cast<uint32_t*>(&h);
}

// Persistent and warp-specialised: warp 0 issues the TMA copies, warp 1
// the MMAs into one of two TMEM accumulators, warps 2..5 drain a finished
// accumulator (epilogue) while the next tile accumulates into the other.
// Work item w of the CTA is tile w / ntn, output-channel tile w % ntn, for
// w = blockIdx.x, + gridDim.x, ...
template <int KC, int BN>
__global__ void __launch_bounds__(192, 1) conv_tc(const __grid_constant__ ConvArgs a, int ntn) {
  using S = ConvShape<KC, BN>;
  extern __shared__ __align__(1024) unsigned char smraw[];
  unsigned char* sm = (unsigned char*)(((uintptr_t)smraw + 1023) & ~(uintptr_t)1023);
  uint64_t* full = (uint64_t*)(sm + S::ST * S::STAGE);
  uint64_t* empty = full + S::ST;
  uint64_t* tfull = empty + S::ST;  // [2] accumulator ready
  uint64_t* tempty = tfull + 2;     // [2] accumulator drained
  uint64_t* drain = tempty + 2;     // every MMA of this CTA has completed
  uint32_t* tslot = (uint32_t*)(drain + 1);
  float* sbias = (float*)(tslot + 4);  // [cout] (16-byte aligned)
  const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
  const int W = a.W, H = a.H;
  const int tpr = W / S::TW, tpi = tpr * (H / S::TH);
  const int nitems = a.B_tiles * ntn;
  const int sgn = a.reverse_taps ? -1 : 1;

  if (threadIdx.x == 0) {
    for (int s = 0; s < S::ST; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    for (int j = 0; j < 2; ++j) {
      mbar_init(&tfull[j], 1);
      mbar_init(&tempty[j], 4);
    }
    mbar_init(drain, 1);
    mbar_init_fence();
  }
  if (warp == 1) tmem_alloc(tslot, S::TCOLS);
  // the bias, read once per CTA (the epilogue adds it from shared memory)
  if (a.bias)
    for (int c = threadIdx.x; c < a.cout; c += blockDim.x) sbias[c] = a.bias[c];
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tslot;
  bool ok = true;
  if (warp == 0) {
    if (lane == 0) {
      int k = 0;  // stage counter over all items
      for (int item = blockIdx.x; item < nitems && ok; item += gridDim.x) {
        const int tile = item / ntn, n0 = (item % ntn) * BN;
        const int b = tile / tpi, r = tile % tpi;
        const int x0 = (r % tpr) * S::TW, y0 = (r / tpr) * S::TH;
        for (int i = 0; i < a.nin && ok; ++i)
          for (int c0 = 0; c0 < a.cin[i] && ok; c0 += KC)
            for (int sx = -1; sx <= 1 && ok; ++sx, ++k) {
              const int s = k % S::ST, it = k / S::ST;
              if (it > 0) ok = mbar_wait_bounded(&empty[s], (it - 1) & 1);
              if (!ok) break;
              unsigned char* st = sm + s * S::STAGE;
              mbar_arrive_expect_tx(&full[s], (uint32_t)(S::ABYTES + 3 * S::BBYTES));
              // halo coordinates: real column x0 + sx is x0 + sx + 1, real
              // row y0 - 1 is y0
              tma_load_4d(st, &a.in_map[i], &full[s], c0, x0 + sx + 1, y0, b);
              // the three taps whose pixels are at column shift sx: tap
              // column sgn sx, rows dy = -1, 0, 1 in that order
              tma_load_4d(st + S::ASTRIDE, &a.w_map, &full[s], a.koff[i] + c0, n0, 0, sgn * sx + 1);
            }
      }
    }
  } else if (warp == 1) {
    if (lane == 0) {
      constexpr uint32_t idesc = idesc_bf16_f32(128, BN);
      int k = 0, local = 0;
      for (int item = blockIdx.x; item < nitems && ok; item += gridDim.x, ++local) {
        const int ab = local & 1, use = local >> 1;
        if (use > 0) ok = mbar_wait_bounded(&tempty[ab], (use - 1) & 1);
        if (!ok) break;
        tc_fence_after();
        const uint32_t acc = tmem + (uint32_t)(ab * S::ACOLS);
        uint32_t accumulate = 0;
        for (int i = 0; i < a.nin && ok; ++i)
          for (int c0 = 0; c0 < a.cin[i] && ok; c0 += KC)
            for (int sx = 0; sx < 3 && ok; ++sx, ++k) {
              const int s = k % S::ST, it = k / S::ST;
              ok = mbar_wait_bounded(&full[s], it & 1);
              if (!ok) break;
              tc_fence_after();
              const unsigned char* st = sm + s * S::STAGE;
#pragma unroll
              for (int sy = 0; sy < 3; ++sy) {
                // pixels at row shift sy - 1 take the weights of tap row
                // sgn (sy - 1), block sgn (sy - 1) + 1 of the weight box
                const int wb = a.reverse_taps ? 2 - sy : sy;
                const unsigned char* pa = st + sy * S::TW * KC * 2;
                const unsigned char* pb = st + S::ASTRIDE + wb * S::BSTRIDE;
#pragma unroll
                for (int kk = 0; kk < KC / 16; ++kk) {
                  tc_mma(acc, sdesc_kmajor<KC * 2>(pa + kk * 32), sdesc_kmajor<KC * 2>(pb + kk * 32),
                         idesc, accumulate);
                  accumulate = 1;
                }
              }
              tc_commit(&empty[s]);
            }
        tc_commit(&tfull[ab]);
      }
      // no MMA may still run when the tensor memory is freed
      tc_commit(drain);
      if (!mbar_wait_bounded(drain, 0)) ok = false;
    }
  } else {
    // epilogue: warp w reads TMEM lanes 32 (w % 4) .. + 31, i.e. pixels
    const int q = warp & 3;
    int local = 0;
    for (int item = blockIdx.x; item < nitems; item += gridDim.x, ++local) {
      const int ab = local & 1, use = local >> 1;
      const bool dok = mbar_wait_bounded(&tfull[ab], use & 1);
      tc_fence_after();
      if (!dok) {
        ok = false;
        break;
      }
      const int tile = item / ntn, n0 = (item % ntn) * BN;
      const int b = tile / tpi, r = tile % tpi;
      const int x0 = (r % tpr) * S::TW, y0 = (r / tpr) * S::TH;
      const int m = q * 32 + lane;
      const int x = x0 + (m & (S::TW - 1)), y = y0 + m / S::TW;
      const int xs[2] = {x + 1, x == 0 ? W + 1 : (x == W - 1 ? 0 : -1)};
      const int ys[2] = {y + 1, y == 0 ? H + 1 : (y == H - 1 ? 0 : -1)};
#pragma unroll 1
      for (int c = 0; c < BN; c += 16) {
        uint32_t rr[16];
        tmem_ld16(tmem + (uint32_t)(ab * S::ACOLS) + ((uint32_t)(q * 32) << 16) + (uint32_t)c, rr);
        const int ch = n0 + c;  // first output channel of this chunk
        if (ch >= a.cout) continue;
        float v[16];
#pragma unroll
        for (int j = 0; j < 16; ++j) {
          float t = __uint_as_float(rr[j]);
          if (a.bias) t += sbias[ch + j];
          if (a.relu) t = fmaxf(t, 0.f);
          v[j] = t;
        }
        if (a.dense) {
#pragma unroll
          for (int j = 0; j < 16; ++j)
            if (ch + j < a.dense_c) a.dense[(((long)b * a.dense_c + ch + j) * H + y) * W + x] = v[j];
          continue;
        }
        const int o = ch < a.split ? 0 : 1;
        const int lc = ch - (o ? a.split : 0);
        const int C = a.out_c[o];
        if (a.mask[o]) {
          const uint4* mp = reinterpret_cast<const uint4*>(
              a.mask[o] + (((long)b * (H + 2) + y + 1) * (W + 2) + x + 1) * C + lc);
          const uint4 m0 = mp[0], m1 = mp[1];
          const uint32_t mw[8] = {m0.x, m0.y, m0.z, m0.w, m1.x, m1.y, m1.z, m1.w};
#pragma unroll
          for (int j = 0; j < 8; ++j) {
            // a BF16 is > 0 when its sign bit is clear and it is not zero
            const uint32_t lo = mw[j] & 0xFFFFu, hi = mw[j] >> 16;
            if (!(lo != 0 && !(lo & 0x8000u))) v[2 * j] = 0.f;
            if (!(hi != 0 && !(hi & 0x8000u))) v[2 * j + 1] = 0.f;
          }
        }
        uint32_t pk[8];
#pragma unroll
        for (int j = 0; j < 8; ++j) pk[j] = pack_bf16(v[2 * j], v[2 * j + 1]);
#pragma unroll
        for (int iy = 0; iy < 2; ++iy)
#pragma unroll
          for (int ix = 0; ix < 2; ++ix) {
            if (ys[iy] < 0 || xs[ix] < 0) continue;
            // 32-byte aligned: every tensor is its own allocation, C and lc
            // are multiples of 16 channels
            st_global_v8(a.out[o] + (((long)b * (H + 2) + ys[iy]) * (W + 2) + xs[ix]) * C + lc, pk);
          }
      }
      // this accumulator may be reused once every epilogue warp has read it
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive_expect_tx(&tempty[ab], 0u);
    }
  }
  if (!ok) atomicOr(a.err, 2);
  tc_fence_before();
  __syncthreads();
  if (warp == 1) tmem_free(tmem, S::TCOLS);
}

// ---------------------------------------------------------------------------
// Weight gradient of one input of a layer on tcgen05:
//   dW[o][t][koff + c] += sum_p dz[p][o] x[p + off(t)][c]
// a GEMM over pixels p (K) of two MN-major operands (channels contiguous):
// the output gradient (M = output channels, tiles of 128) and the input
// (N = input channels, tiles of BN). A CTA takes one column shift dx of the
// taps and a run of 8 x 8-pixel chunks. Per chunk one copy brings the
// output gradient (64 K rows) and one the input's 8 x 10 pixels of the
// chunk's columns shifted by dx (rows y0 - 1 .. y0 + 8, 80 K rows); the
// three taps of the column (dy = -1, 0, 1) read the latter at K offsets of
// 0, 8 and 16 rows (whole swizzle atoms) into three TMEM accumulators.
// Channels beyond a tensor's read as zero; the CTAs' sums are added with
// FP32 atomics.
// ---------------------------------------------------------------------------
struct WgradArgs {
  CUtensorMap dz_map;  // 4-D [Cout, W+2, H+2, B], box [64, 8, 8, 1]
  CUtensorMap x_map;   // 4-D [Cin, W+2, H+2, B], box [64, 8, 10, 1]
  int H, W, B;
  int cout, cin, koff, cin_tot;
  int chunks_per_cta;  // 8 x 8-pixel chunks per CTA
  float* dw;           // [cout][9][cin_tot]
  int* err;
};

template <int BN>
struct WgShape {
  static constexpr int ABOX = 64 * 128;  // 64 K rows x 64 channels of BF16
  static constexpr int BBOX = 80 * 128;  // 80 K rows x 64 channels
  static constexpr int ABYTES = 2 * ABOX, BBYTES = (BN / 64) * BBOX;
  static constexpr int STAGE = ABYTES + BBYTES;
  static constexpr int ST = (190 * 1024 / STAGE) > 6 ? 6 : (190 * 1024 / STAGE);
  static constexpr int TCOLS = 3 * BN <= 256 ? 256 : 512;  // three accumulators of BN columns
  static constexpr size_t SMEM = 1024 + (size_t)ST * STAGE + 256;
  static_assert(3 * BN <= 512, "three accumulators must fit the tensor memory");
};

// dst[0..3] += v[0..3] (FP32 bit patterns), one 16-byte vector reduction in
// the L2; dst 16-byte aligned
__device__ __forceinline__ void red_add_v4(float* dst, const uint32_t* v) {
  asm volatile("red.global.add.v4.f32 [%0], {%1, %2, %3, %4};" ::"l"(dst), "f"(__uint_as_float(v[0])),
               "f"(__uint_as_float(v[1])), "f"(__uint_as_float(v[2])), "f"(__uint_as_float(v[3]))
               : "memory");
}

template <int BN>
__global__ void __launch_bounds__(128) wgrad_tc(const __grid_constant__ WgradArgs a) {
  using S = WgShape<BN>;
  extern __shared__ __align__(1024) unsigned char smraw[];
  unsigned char* sm = (unsigned char*)(((uintptr_t)smraw + 1023) & ~(uintptr_t)1023);
  uint64_t* full = (uint64_t*)(sm + S::ST * S::STAGE);
  uint64_t* empty = full + S::ST;
  uint64_t* done = empty + S::ST;
  uint32_t* tslot = (uint32_t*)(done + 1);
  const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
  const int dx = blockIdx.y % 3 - 1, mt = blockIdx.y / 3, nt = blockIdx.z;
  const int m0 = mt * 128, c0 = nt * BN;
  const int W = a.W, H = a.H;
  const int cpr = W / 8, cpi = cpr * (H / 8);  // chunks per row of chunks, per image
  const long total = (long)a.B * cpi;
  const long k_first = (long)blockIdx.x * a.chunks_per_cta;
  const long k_end = k_first + a.chunks_per_cta < total ? k_first + a.chunks_per_cta : total;
  const int nk = k_end > k_first ? (int)(k_end - k_first) : 0;
  // output-gradient boxes holding real channels (the rest of the A tile
  // feeds accumulator rows that are never read)
  const int na = a.cout > m0 + 64 ? 2 : 1;

  if (threadIdx.x == 0) {
    for (int s = 0; s < S::ST; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    mbar_init(done, 1);
    mbar_init_fence();
  }
  if (warp == 0) tmem_alloc(tslot, S::TCOLS);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tslot;
  bool ok = true;
  if (warp == 0 && lane == 0) {
    for (int kb = 0; kb < nk && ok; ++kb) {
      const int s = kb % S::ST, it = kb / S::ST;
      if (it > 0) ok = mbar_wait_bounded(&empty[s], (it - 1) & 1);
      if (!ok) break;
      const long k = k_first + kb;
      const int b = (int)(k / cpi), q = (int)(k % cpi);
      const int px = (q % cpr) * 8, py = (q / cpr) * 8;
      unsigned char* st = sm + s * S::STAGE;
      mbar_arrive_expect_tx(&full[s], (uint32_t)(na * S::ABOX + S::BBYTES));
      for (int j = 0; j < na; ++j)
        tma_load_4d(st + j * S::ABOX, &a.dz_map, &full[s], m0 + 64 * j, px + 1, py + 1, b);
      // halo coordinates: real column px + dx is px + dx + 1, real row
      // py - 1 is py
      for (int j = 0; j < BN / 64; ++j)
        tma_load_4d(st + S::ABYTES + j * S::BBOX, &a.x_map, &full[s], c0 + 64 * j, px + dx + 1,
                    py, b);
    }
  } else if (warp == 1 && lane == 0) {
    constexpr uint32_t idesc = idesc_bf16_f32(128, BN, true, true);
    for (int kb = 0; kb < nk && ok; ++kb) {
      const int s = kb % S::ST, it = kb / S::ST;
      ok = mbar_wait_bounded(&full[s], it & 1);
      if (!ok) break;
      tc_fence_after();
      unsigned char* st = sm + s * S::STAGE;
#pragma unroll
      for (int j = 0; j < 3; ++j)
#pragma unroll
        for (int kk = 0; kk < 4; ++kk)
          tc_mma(tmem + (uint32_t)(j * BN), sdesc_mnmajor128(st + kk * 16 * 128, S::ABOX),
                 sdesc_mnmajor128(st + S::ABYTES + (j * 8 + kk * 16) * 128, S::BBOX), idesc,
                 (kb | kk) ? 1u : 0u);
      tc_commit(&empty[s]);
    }
    tc_commit(done);
  }
  __syncwarp();
  const bool dok = nk > 0 ? mbar_wait_bounded(done, 0) : true;
  tc_fence_after();
  if (dok && nk > 0) {
    const int o = m0 + warp * 32 + lane;
#pragma unroll 1
    for (int j = 0; j < 3; ++j) {
      const int tap = 3 * j + dx + 1;
#pragma unroll 1
      for (int c = 0; c < BN; c += 16) {
        uint32_t rr[16];
        tmem_ld16(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)(j * BN + c), rr);
        if (o >= a.cout || c0 + c >= a.cin) continue;  // cin is a multiple of 16
        float* dst = a.dw + ((long)o * 9 + tap) * a.cin_tot + a.koff + c0 + c;
#pragma unroll
        for (int i = 0; i < 16; i += 4) red_add_v4(dst + i, rr + i);
      }
    }
  } else if (!dok && threadIdx.x == 0) {
    atomicOr(a.err, 1);
  }
  if (!ok) atomicOr(a.err, 2);
  tc_fence_before();
  __syncthreads();
  if (warp == 0) tmem_free(tmem, S::TCOLS);
}

// ---------------------------------------------------------------------------
// CUDA-core kernels: pooling, upsampling and their gradients with ReLU
// masks, input planes, output, loss, bias gradients, Adam.
// ---------------------------------------------------------------------------
__device__ __forceinline__ long hidx(int b, int y, int x, int H, int W, int C) {
  return (((long)b * (H + 2) + y + 1) * (W + 2) + x + 1) * C;
}

// store one pixel's channel pair (c, c + 1) and its periodic images
__device__ __forceinline__ void st_pair(bf16* t, int b, int y, int x, int H, int W, int C, int c,
                                        float v0, float v1) {
  const __nv_bfloat162 p = __floats2bfloat162_rn(v0, v1);
  const int xs[2] = {x + 1, x == 0 ? W + 1 : (x == W - 1 ? 0 : -1)};
  const int ys[2] = {y + 1, y == 0 ? H + 1 : (y == H - 1 ? 0 : -1)};
  for (int iy = 0; iy < 2; ++iy)
    for (int ix = 0; ix < 2; ++ix)
      if (ys[iy] >= 0 && xs[ix] >= 0)
        *reinterpret_cast<__nv_bfloat162*>(t + (((long)b * (H + 2) + ys[iy]) * (W + 2) + xs[ix]) * C + c) = p;
}

__device__ __forceinline__ float2 ld_pair(const bf16* t, long off) {
  return __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(t + off));
}

// ---------------------------------------------------------------------------
// Pooling, upsampling and their gradients work on 8-channel groups (16
// bytes): a thread takes one group of one output pixel. Tensor sides are
// powers of two (lgW = log2 W), channel counts multiples of 8.
// ---------------------------------------------------------------------------
struct Oct {
  float v[8];
};
__device__ __forceinline__ Oct ld_oct(const bf16* t, long off) {
  const uint4 q = *reinterpret_cast<const uint4*>(t + off);
  const uint32_t w[4] = {q.x, q.y, q.z, q.w};
  Oct o;
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    const float2 f = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(&w[j]));
    o.v[2 * j] = f.x;
    o.v[2 * j + 1] = f.y;
  }
  return o;
}
// one pixel's 8 channels c .. c + 7 and their periodic images
__device__ __forceinline__ void st_oct(bf16* t, int b, int y, int x, int H, int W, int C, int c,
                                       const Oct& o) {
  uint4 q;
  uint32_t* w = reinterpret_cast<uint32_t*>(&q);
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    __nv_bfloat162 h2 = __floats2bfloat162_rn(o.v[2 * j], o.v[2 * j + 1]);
    w[j] = *reinterpret_cast<uint32_t*>(&h2);
  }
  const int xs[2] = {x + 1, x == 0 ? W + 1 : (x == W - 1 ? 0 : -1)};
  const int ys[2] = {y + 1, y == 0 ? H + 1 : (y == H - 1 ? 0 : -1)};
#pragma unroll
  for (int iy = 0; iy < 2; ++iy)
#pragma unroll
    for (int ix = 0; ix < 2; ++ix)
      if (ys[iy] >= 0 && xs[ix] >= 0)
        *reinterpret_cast<uint4*>(t + (((long)b * (H + 2) + ys[iy]) * (W + 2) + xs[ix]) * C + c) = q;
}
// work item i of a (B x H x W pixels) x (C / 8 groups) loop
struct OctIdx {
  int b, y, x, c;
};
__device__ __forceinline__ OctIdx oct_idx(long i, int lgH, int lgW, int lgG) {
  OctIdx r;
  r.c = (int)(i & ((1 << lgG) - 1)) * 8;
  const long p = i >> lgG;
  r.x = (int)(p & ((1 << lgW) - 1));
  r.y = (int)((p >> lgW) & ((1 << lgH) - 1));
  r.b = (int)(p >> (lgW + lgH));
  return r;
}

// dst (H/2 x W/2, lgH, lgW its sides) = 2 x 2 mean of src (H x W)
__global__ void pool_kernel(const bf16* __restrict__ src, bf16* __restrict__ dst, int B, int lgH,
                            int lgW, int lgG) {
  const int H = 1 << lgH, W = 1 << lgW, C = 8 << lgG;
  const long total = (long)B << (lgH + lgW + lgG);
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < total; i += (long)gridDim.x * blockDim.x) {
    const OctIdx k = oct_idx(i, lgH, lgW, lgG);
    Oct s = {};
    for (int q = 0; q < 4; ++q) {
      const Oct v = ld_oct(src, hidx(k.b, 2 * k.y + q / 2, 2 * k.x + q % 2, 2 * H, 2 * W, C) + k.c);
#pragma unroll
      for (int j = 0; j < 8; ++j) s.v[j] += v.v[j];
    }
#pragma unroll
    for (int j = 0; j < 8; ++j) s.v[j] *= 0.25f;
    st_oct(dst, k.b, k.y, k.x, H, W, C, k.c, s);
  }
}

// dst (H x W) = nearest 2x upsampling of src (H/2 x W/2)
__global__ void up_kernel(const bf16* __restrict__ src, bf16* __restrict__ dst, int B, int lgH,
                          int lgW, int lgG) {
  const int H = 1 << lgH, W = 1 << lgW, C = 8 << lgG;
  const long total = (long)B << (lgH + lgW + lgG);
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < total; i += (long)gridDim.x * blockDim.x) {
    const OctIdx k = oct_idx(i, lgH, lgW, lgG);
    st_oct(dst, k.b, k.y, k.x, H, W, C, k.c, ld_oct(src, hidx(k.b, k.y / 2, k.x / 2, H / 2, W / 2, C) + k.c));
  }
}

// dS (H/2 x W/2, the sides given) = (sum of the 2 x 2 fine pixels of dU) * (S > 0)
__global__ void up_grad_mask_kernel(const bf16* __restrict__ dU, const bf16* __restrict__ Sact,
                                    bf16* __restrict__ dS, int B, int lgH, int lgW, int lgG) {
  const int H = 1 << lgH, W = 1 << lgW, C = 8 << lgG;
  const long total = (long)B << (lgH + lgW + lgG);
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < total; i += (long)gridDim.x * blockDim.x) {
    const OctIdx k = oct_idx(i, lgH, lgW, lgG);
    Oct s = {};
    for (int q = 0; q < 4; ++q) {
      const Oct v = ld_oct(dU, hidx(k.b, 2 * k.y + q / 2, 2 * k.x + q % 2, 2 * H, 2 * W, C) + k.c);
#pragma unroll
      for (int j = 0; j < 8; ++j) s.v[j] += v.v[j];
    }
    const Oct m = ld_oct(Sact, hidx(k.b, k.y, k.x, H, W, C) + k.c);
#pragma unroll
    for (int j = 0; j < 8; ++j) s.v[j] = m.v[j] > 0.f ? s.v[j] : 0.f;
    st_oct(dS, k.b, k.y, k.x, H, W, C, k.c, s);
  }
}

// dS (H x W) = (skip + dP(pixel / 2) / 4) * (S > 0)
__global__ void pool_grad_add_mask_kernel(const bf16* __restrict__ dP, const bf16* __restrict__ skip,
                                          const bf16* __restrict__ Sact, bf16* __restrict__ dS, int B,
                                          int lgH, int lgW, int lgG) {
  const int H = 1 << lgH, W = 1 << lgW, C = 8 << lgG;
  const long total = (long)B << (lgH + lgW + lgG);
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < total; i += (long)gridDim.x * blockDim.x) {
    const OctIdx k = oct_idx(i, lgH, lgW, lgG);
    const Oct p = ld_oct(dP, hidx(k.b, k.y / 2, k.x / 2, H / 2, W / 2, C) + k.c);
    const Oct q = ld_oct(skip, hidx(k.b, k.y, k.x, H, W, C) + k.c);
    const Oct m = ld_oct(Sact, hidx(k.b, k.y, k.x, H, W, C) + k.c);
    Oct o;
#pragma unroll
    for (int j = 0; j < 8; ++j) o.v[j] = m.v[j] > 0.f ? q.v[j] + 0.25f * p.v[j] : 0.f;
    st_oct(dS, k.b, k.y, k.x, H, W, C, k.c, o);
  }
}

// ---------------------------------------------------------------------------
// Per-plane sums of a [planes][HW] FP32 array in two levels, deterministic:
// block (chunk, plane) adds kRedChunk elements (FP32 over a thread's 32
// values, FP64 above that), and the last block to finish adds the chunk
// sums of every plane in order.
//   mode 0: out[p] = mean of plane p;
//   mode 1: out[b] = RMS over the n planes of sample b of x - center[plane]
//           (center: the plane means), zero for a flat sample.
// counter: a zeroed word, left zeroed.
// ---------------------------------------------------------------------------
constexpr int kRedChunk = 8192;
__global__ void __launch_bounds__(256) plane_reduce_kernel(const float* __restrict__ x, int planes,
                                                           int HW, int n, int mode,
                                                           const double* __restrict__ center,
                                                           double* __restrict__ partial,
                                                           unsigned* __restrict__ counter,
                                                           double* __restrict__ out) {
  const int nchunk = HW / kRedChunk, pl = blockIdx.y, ch = blockIdx.x;
  const float4* p = reinterpret_cast<const float4*>(x + (long)pl * HW + (long)ch * kRedChunk);
  const float c = mode ? (float)center[pl] : 0.f;
  float s = 0.f;
#pragma unroll
  for (int k = 0; k < kRedChunk / 1024; ++k) {
    const float4 v = p[k * 256 + threadIdx.x];
    if (mode) {
      const float d0 = v.x - c, d1 = v.y - c, d2 = v.z - c, d3 = v.w - c;
      s += (d0 * d0 + d1 * d1) + (d2 * d2 + d3 * d3);
    } else {
      s += (v.x + v.y) + (v.z + v.w);
    }
  }
  double d = s;
  for (int o = 16; o > 0; o >>= 1) d += __shfl_down_sync(0xffffffffu, d, o);
  __shared__ double red[8];
  __shared__ bool last;
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = d;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < 8; ++w) t += red[w];
    partial[(long)pl * nchunk + ch] = t;
    __threadfence();
    last = atomicAdd(counter, 1u) == gridDim.x * gridDim.y - 1;
  }
  __syncthreads();
  if (!last) return;
  __threadfence();
  if (mode == 0) {
    for (int q = threadIdx.x; q < planes; q += blockDim.x) {
      double t = 0.0;
      for (int k = 0; k < nchunk; ++k) t += __ldcg(partial + (long)q * nchunk + k);
      out[q] = t / HW;
    }
  } else {
    for (int b = threadIdx.x; b < planes / n; b += blockDim.x) {
      double t = 0.0;
      for (int q = b * n; q < b * n + n; ++q)
        for (int k = 0; k < nchunk; ++k) t += __ldcg(partial + (long)q * nchunk + k);
      out[b] = sqrt(t / ((double)n * HW));
    }
  }
  if (threadIdx.x == 0) *counter = 0u;
}

// 1 / s of a sample, 0 for a flat one (its planes are then all zero)
__device__ __forceinline__ double inv_or_zero(double s) { return s > 0.0 ? 1.0 / s : 0.0; }

// X0 = (h_i - mean) in_scale / s, parameter planes, zeros (16 channels)
__global__ void input_kernel(const float* __restrict__ h, const double* __restrict__ mean,
                             const double* __restrict__ rms, int B, int n, int H, int W,
                             float in_scale, const float* __restrict__ extra, int n_extra,
                             bf16* __restrict__ x0) {
  const long total = (long)B * H * W;
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < total; i += (long)gridDim.x * blockDim.x) {
    const int x = (int)(i % W);
    const int y = (int)((i / W) % H), b = (int)(i / ((long)W * H));
    float v[kCin0];
    for (int c = 0; c < kCin0; ++c) v[c] = 0.f;
    const double k = in_scale * inv_or_zero(rms[b]);
    for (int c = 0; c < n; ++c)
      v[c] = (float)(((double)h[(((long)b * n + c) * H + y) * W + x] - mean[b * n + c]) * k);
    for (int j = 0; j < n_extra; ++j) v[n + j] = extra[j];
    for (int c = 0; c < kCin0; c += 2) st_pair(x0, b, y, x, H, W, kCin0, c, v[c], v[c + 1]);
  }
}

// out = h + (y - mean y) s / out_scale per (sample, layer); ymean: means of
// y, rms: s of every sample
__global__ void output_kernel(const float* __restrict__ h, const float* __restrict__ y,
                              const double* __restrict__ ymean, const double* __restrict__ rms,
                              long total, int n, int HW, float inv_scale, float* __restrict__ out) {
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < total; i += (long)gridDim.x * blockDim.x)
    out[i] = h[i] + (float)(((double)y[i] - ymean[i / HW]) * rms[i / ((long)n * HW)] * inv_scale);
}

// loss += sum (y - (t - h) out_scale / s)^2 (FP64); dY (NHWC halo, 16
// channels) = 2 (y - (t - h) out_scale / s) / count
__global__ void loss_kernel(const float* __restrict__ y, const float* __restrict__ h,
                            const float* __restrict__ t, const double* __restrict__ rms, int B,
                            int n, int H, int W, float scale, float inv_count,
                            double* __restrict__ loss, bf16* __restrict__ dY) {
  const long total = (long)B * H * W;
  double acc = 0.0;
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < total; i += (long)gridDim.x * blockDim.x) {
    const int x = (int)(i % W);
    const int yy = (int)((i / W) % H), b = (int)(i / ((long)W * H));
    float g[kCout];
    for (int c = 0; c < kCout; ++c) g[c] = 0.f;
    const float ks = (float)(scale * inv_or_zero(rms[b]));
    for (int c = 0; c < n; ++c) {
      const long k = (((long)b * n + c) * H + yy) * W + x;
      const float d = y[k] - (t[k] - h[k]) * ks;
      acc += (double)d * d;
      g[c] = 2.f * d * inv_count;
    }
    for (int c = 0; c < kCout; c += 2) st_pair(dY, b, yy, x, H, W, kCout, c, g[c], g[c + 1]);
  }
  __shared__ double red[256];
  red[threadIdx.x] = acc;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if ((int)threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) atomicAdd(loss, red[0]);
}

// db[c] += sum over the real pixels of dz (NHWC halo, C channels, C = 8 2^lgG
// <= 256). A thread adds one 8-channel group over every (256 / groups)-th
// pixel of the grid-stride loop; the block combines its threads' sums in
// shared memory and adds one atomic per channel.
__global__ void __launch_bounds__(256) bias_grad_kernel(const bf16* __restrict__ dz, int B, int lgH,
                                                        int lgW, int lgG, float* __restrict__ db) {
  const int H = 1 << lgH, W = 1 << lgW, C = 8 << lgG, g = 1 << lgG;
  const int pp = 256 >> lgG;  // pixels per block and iteration
  const int grp = threadIdx.x & (g - 1), sub = threadIdx.x >> lgG;
  const long npix = (long)B << (lgH + lgW);
  float s[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
  for (long q = (long)blockIdx.x * pp + sub; q < npix; q += (long)gridDim.x * pp) {
    const int x = (int)(q & (W - 1)), y = (int)((q >> lgW) & (H - 1)), b = (int)(q >> (lgW + lgH));
    const Oct v = ld_oct(dz, hidx(b, y, x, H, W, C) + grp * 8);
#pragma unroll
    for (int j = 0; j < 8; ++j) s[j] += v.v[j];
  }
  __shared__ float red[256][9];
#pragma unroll
  for (int j = 0; j < 8; ++j) red[threadIdx.x][j] = s[j];
  __syncthreads();
  if ((int)threadIdx.x < C) {
    const int gi = threadIdx.x >> 3, j = threadIdx.x & 7;
    float t = 0.f;
    for (int k = 0; k < pp; ++k) t += red[k * g + gi][j];
    atomicAdd(db + threadIdx.x, t);
  }
}

struct LayerParams {
  long w_off, b_off;  // offsets of the layer's weights and bias in the flat arrays
  int cout, cin, cout_pad, cin_pad;
  bf16* wf;           // forward weights [cout_pad][9][cin]
  bf16* wd;           // input-gradient weights [cin_pad][9][cout], taps as stored
};
struct AdamArgs {
  LayerParams L[kLayers];
  float* p;        // FP32 parameters (flat)
  const float* g;  // their gradients
  float* m;
  float* v;
  long count;
  float lr, b1, b2, eps, c1, c2;  // c1 = 1 / (1 - b1^t), c2 = 1 / (1 - b2^t)
};

// Adam step on the FP32 parameters, then the BF16 copies of every weight:
// forward layout [o][t][c] and the input-gradient layout [c][t][o]
__global__ void adam_kernel(const __grid_constant__ AdamArgs a, int do_step) {
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < a.count; i += (long)gridDim.x * blockDim.x) {
    float w = a.p[i];
    if (do_step) {
      const float g = a.g[i];
      const float m = a.b1 * a.m[i] + (1.f - a.b1) * g;
      const float v = a.b2 * a.v[i] + (1.f - a.b2) * g * g;
      a.m[i] = m;
      a.v[i] = v;
      w -= a.lr * (m * a.c1) / (sqrtf(v * a.c2) + a.eps);
      a.p[i] = w;
    }
    // which layer's weights?
    for (int l = 0; l < kLayers; ++l) {
      const LayerParams& L = a.L[l];
      const long nw = (long)L.cout * 9 * L.cin;
      if (i >= L.w_off && i < L.w_off + nw) {
        const long k = i - L.w_off;
        const int o = (int)(k / (9 * L.cin)), t = (int)((k / L.cin) % 9), c = (int)(k % L.cin);
        const bf16 q = __float2bfloat16_rn(w);
        L.wf[((long)o * 9 + t) * L.cin + c] = q;
        L.wd[((long)c * 9 + t) * L.cout + o] = q;
        break;
      }
    }
  }
}

}  // namespace unet
}  // namespace mlsw

// ===========================================================================
// Host side
// ===========================================================================
namespace {

using namespace mlsw::unet;

typedef CUresult (*EncodeFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                             const cuuint64_t*, const cuuint32_t*, const cuuint32_t*,
                             CUtensorMapInterleave, CUtensorMapSwizzle, CUtensorMapL2promotion,
                             CUtensorMapFloatOOBfill);

EncodeFn encoder() {
  static EncodeFn fn = nullptr;
  static bool tried = false;
  if (!tried) {
    tried = true;
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<EncodeFn>(p);
  }
  return fn;
}

CUtensorMapSwizzle swizzle_of(int inner_bytes) {
  return inner_bytes == 128 ? CU_TENSOR_MAP_SWIZZLE_128B
                            : (inner_bytes == 64 ? CU_TENSOR_MAP_SWIZZLE_64B : CU_TENSOR_MAP_SWIZZLE_32B);
}

// 4-D map of an NHWC tensor with halo: dims [C, W+2, H+2, B], box [bc, bx, by, 1]
bool map_nhwc(CUtensorMap* m, void* base, int C, int W, int H, int B, int bc, int bx, int by) {
  EncodeFn fn = encoder();
  if (!fn) return false;
  cuuint64_t dims[4] = {(cuuint64_t)C, (cuuint64_t)W + 2, (cuuint64_t)H + 2, (cuuint64_t)B};
  cuuint64_t st[3] = {(cuuint64_t)C * 2, (cuuint64_t)C * 2 * (W + 2), (cuuint64_t)C * 2 * (W + 2) * (H + 2)};
  cuuint32_t box[4] = {(cuuint32_t)bc, (cuuint32_t)bx, (cuuint32_t)by, 1};
  cuuint32_t es[4] = {1, 1, 1, 1};
  return fn(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 4, base, dims, st, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
            swizzle_of(bc * 2), CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) ==
         CUDA_SUCCESS;
}

// 2-D map of a weight matrix [rows][K] (K contiguous), box [kc, bn]
// weights [rows][tap][K] (tap = 3 (dy + 1) + (dx + 1)) as a 4-D tensor
// [K, rows, 3 dy, 3 dx]; a box [kc, bn, 3, 1] holds one tap column's three
// taps, each a K-major bn x kc block
bool map_weights(CUtensorMap* m, void* base, int K, int rows, int kc, int bn) {
  EncodeFn fn = encoder();
  if (!fn) return false;
  cuuint64_t dims[4] = {(cuuint64_t)K, (cuuint64_t)rows, 3, 3};
  cuuint64_t st[3] = {(cuuint64_t)K * 2 * 9, (cuuint64_t)K * 2 * 3, (cuuint64_t)K * 2};
  cuuint32_t box[4] = {(cuuint32_t)kc, (cuuint32_t)bn, 3, 1};
  cuuint32_t es[4] = {1, 1, 1, 1};
  return fn(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 4, base, dims, st, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
            swizzle_of(kc * 2), CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) ==
         CUDA_SUCCESS;
}

int kc_fwd(int l) {
  int kc = 64;
  for (int j = 0; j < 2; ++j)
    if (kNet[l].in[j] >= 0) kc = std::min(kc, kTC[kNet[l].in[j]]);
  return kc;
}
int kc_bwd(int l) { return std::min(64, kNet[l].cout); }
int bn_bwd(int l) {
  int bn = kTC[kNet[l].in[0]];
  if (kNet[l].in[1] >= 0) bn = std::min(bn, kTC[kNet[l].in[1]]);
  return std::min(bn, 128);
}
int bn_fwd(int l) { return std::min(kNet[l].cout, 128); }
int bn_wgrad(int cin) { return cin <= 64 ? 64 : 128; }

template <int KC, int BN>
cudaError_t launch_conv_t(const ConvArgs& a, int ntn, int num_sms, cudaStream_t st) {
  using S = ConvShape<KC, BN>;
  static bool attr[64] = {};
  static int per_sm[64] = {};
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev >= 64) return cudaErrorInvalidDevice;
  if (!attr[dev]) {
    e = cudaFuncSetAttribute(conv_tc<KC, BN>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)S::SMEM);
    if (e != cudaSuccess) return e;
    // CTAs per SM by shared memory (228 KB, 1 KB reserved per CTA) and by
    // tensor memory. Registers can hold fewer (the 16-channel input layer:
    // 3 of 6), and the grid is then more than one wave; that measured
    // faster than a grid of only the CTAs resident at once (2.08 against
    // 1.79 ms per batch-32 prediction): CTAs that finish early make room
    // for the rest, which balances the uneven tiles better.
    const int by_smem = 233472 / ((int)S::SMEM + 1024);
    per_sm[dev] = std::max(1, std::min(by_smem, S::CTAS_TMEM));
    attr[dev] = true;
  }
  if (a.bias && a.cout > S::kBiasMax) return cudaErrorInvalidValue;
  const int items = a.B_tiles * ntn;
  const int grid = std::min(items, num_sms * per_sm[dev]);
  conv_tc<KC, BN><<<grid, 192, S::SMEM, st>>>(a, ntn);
  return cudaGetLastError();
}

cudaError_t launch_conv(int kc, int bn, const ConvArgs& a, int ntn, int num_sms, cudaStream_t st) {
#define MLSW_CONV_CASE(K, N) \
  if (kc == K && bn == N) return launch_conv_t<K, N>(a, ntn, num_sms, st);
  MLSW_CONV_CASE(16, 32)
  MLSW_CONV_CASE(32, 16)
  MLSW_CONV_CASE(32, 32)
  MLSW_CONV_CASE(32, 64)
  MLSW_CONV_CASE(64, 32)
  MLSW_CONV_CASE(64, 64)
  MLSW_CONV_CASE(64, 128)
#undef MLSW_CONV_CASE
  return cudaErrorInvalidValue;
}

template <int BN>
cudaError_t launch_wgrad_t(const WgradArgs& a, dim3 grid, cudaStream_t st) {
  using S = WgShape<BN>;
  static bool attr[64] = {};
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 64 && !attr[dev]) {
    e = cudaFuncSetAttribute(wgrad_tc<BN>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)S::SMEM);
    if (e != cudaSuccess) return e;
    attr[dev] = true;
  }
  wgrad_tc<BN><<<grid, 128, S::SMEM, st>>>(a);
  return cudaGetLastError();
}

int grid_for(long work, int threads) {
  long g = (work + threads - 1) / threads;
  return (int)std::max(1L, std::min(g, 4096L));
}

int ilog2(int v) {
  int k = 0;
  while ((1 << (k + 1)) <= v) ++k;
  return k;
}

}  // namespace

struct mlswlbm_unet {
  int n, H, W, Bmax, n_extra, num_sms;
  float in_scale, out_scale;
  cudaStream_t stream;
  int lw[kTensors], lh[kTensors];         // width, height of every tensor's level
  bf16* act[kTensors];
  bf16* grad[kTensors];
  bf16* skipg[3];                         // skip-connection gradients of S0, S1, S2
  float* ydense;                          // [B][n][H][W]
  float* hbuf;                            // predicted heights scratch (train: unused)
  double* means;                          // per (sample, layer) means
  double* rms;                            // per sample RMS deviation
  double* red_part;                       // chunk sums of plane_reduce_kernel
  unsigned* red_count;                    // its completion counter (zero between launches)
  double* dloss;
  float* extra;                           // parameter planes' values
  float *params, *pgrad, *adam_m, *adam_v;
  long nparam;
  long adam_t;
  LayerParams L[kLayers];
  bf16* wbuf;
  CUtensorMap act_map[kTensors];          // as a convolution input (KC of its consumer)
  CUtensorMap grad_map[kTensors];         // as an input-gradient convolution input
  CUtensorMap wg_act[kTensors], wg_grad[kTensors];  // weight-gradient operands
  CUtensorMap wf_map[kLayers], wd_map[kLayers];
  int* err;
};

namespace {

void unet_free(mlswlbm_unet* u) {
  if (!u) return;
  for (int t = 0; t < kTensors; ++t) {
    cudaFree(u->act[t]);
    cudaFree(u->grad[t]);
  }
  for (int j = 0; j < 3; ++j) cudaFree(u->skipg[j]);
  cudaFree(u->ydense);
  cudaFree(u->hbuf);
  cudaFree(u->means);
  cudaFree(u->rms);
  cudaFree(u->red_part);
  cudaFree(u->red_count);
  cudaFree(u->dloss);
  cudaFree(u->extra);
  cudaFree(u->params);
  cudaFree(u->pgrad);
  cudaFree(u->adam_m);
  cudaFree(u->adam_v);
  cudaFree(u->wbuf);
  cudaFree(u->err);
  delete u;
}

size_t tensor_elems(const mlswlbm_unet* u, int t) {
  return (size_t)u->Bmax * (u->lh[t] + 2) * (u->lw[t] + 2) * kTC[t];
}

// the consumer conv of each tensor decides its map's channel chunk
int act_kc(int t) {
  for (int l = 0; l < kLayers; ++l)
    for (int j = 0; j < 2; ++j)
      if (kNet[l].in[j] == t) return kc_fwd(l);
  return 0;
}

cudaError_t conv_forward(mlswlbm_unet* u, int l, int batch) {
  const Layer& N = kNet[l];
  ConvArgs a;
  std::memset(&a, 0, sizeof(a));
  const int t0 = N.in[0];
  a.nin = N.in[1] >= 0 ? 2 : 1;
  for (int j = 0; j < a.nin; ++j) {
    a.in_map[j] = u->act_map[N.in[j]];
    a.cin[j] = kTC[N.in[j]];
    a.koff[j] = j ? kTC[N.in[0]] : 0;
  }
  a.w_map = u->wf_map[l];
  a.cin_tot = layer_cin(l);
  a.H = u->lh[t0];
  a.W = u->lw[t0];
  a.cout = N.cout;
  a.bias = u->params + u->L[l].b_off;
  a.relu = N.relu ? 1 : 0;
  if (N.out >= 0) {
    a.out[0] = u->act[N.out];
    a.out_c[0] = N.cout;
    a.split = N.cout;
  } else {
    a.dense = u->ydense;
    a.dense_c = u->n;
  }
  a.err = u->err;
  a.B_tiles = batch * (a.W / 16) * (a.H / 8);
  return launch_conv(kc_fwd(l), bn_fwd(l), a, N.cout / bn_fwd(l), u->num_sms, u->stream);
}

// input gradient of layer l: from grad of its output to the gradients of its
// inputs (out0, out1), masked by the given activations
cudaError_t conv_input_grad(mlswlbm_unet* u, int l, int batch, bf16* out0, const bf16* mask0,
                            bf16* out1, const bf16* mask1) {
  const Layer& N = kNet[l];
  const int tz = N.out >= 0 ? N.out : YG;
  ConvArgs a;
  std::memset(&a, 0, sizeof(a));
  a.nin = 1;
  a.in_map[0] = u->grad_map[tz];
  a.cin[0] = N.cout;
  a.koff[0] = 0;
  a.w_map = u->wd_map[l];
  a.cin_tot = N.cout;
  a.H = u->lh[N.in[0]];
  a.W = u->lw[N.in[0]];
  a.cout = layer_cin(l);
  a.reverse_taps = 1;
  a.out[0] = out0;
  a.mask[0] = mask0;
  a.out_c[0] = kTC[N.in[0]];
  a.split = kTC[N.in[0]];
  if (N.in[1] >= 0) {
    a.out[1] = out1;
    a.mask[1] = mask1;
    a.out_c[1] = kTC[N.in[1]];
  }
  a.err = u->err;
  a.B_tiles = batch * (a.W / 16) * (a.H / 8);
  const int bn = bn_bwd(l);
  return launch_conv(kc_bwd(l), bn, a, a.cout / bn, u->num_sms, u->stream);
}

cudaError_t weight_grad(mlswlbm_unet* u, int l, int batch) {
  const Layer& N = kNet[l];
  const int tz = N.out >= 0 ? N.out : YG;
  const int H = u->lh[N.in[0]], W = u->lw[N.in[0]];
  for (int j = 0; j < 2; ++j) {
    const int tx = N.in[j];
    if (tx < 0) continue;
    WgradArgs a;
    std::memset(&a, 0, sizeof(a));
    a.dz_map = u->wg_grad[tz];
    a.x_map = u->wg_act[tx];
    a.H = H;
    a.W = W;
    a.B = batch;
    a.cout = N.cout;
    a.cin = kTC[tx];
    a.koff = j ? kTC[N.in[0]] : 0;
    a.cin_tot = layer_cin(l);
    a.dw = u->pgrad + u->L[l].w_off;
    a.err = u->err;
    const int bn = bn_wgrad(a.cin);
    const int mt = (a.cout + 127) / 128, nt = (a.cin + bn - 1) / bn;
    const long chunks = (long)batch * H * W / 64;
    // one CTA per SM over the three column shifts and all tiles (every CTA
    // adds its whole partial dW: fewer, longer CTAs mean fewer reductions)
    const long want = std::max(1L, (long)u->num_sms / (3L * mt * nt));
    const int per = (int)std::max(1L, (chunks + want - 1) / want);
    const dim3 grid((unsigned)((chunks + per - 1) / per), (unsigned)(3 * mt), (unsigned)nt);
    a.chunks_per_cta = per;
    cudaError_t e = bn == 64 ? launch_wgrad_t<64>(a, grid, u->stream)
                             : launch_wgrad_t<128>(a, grid, u->stream);
    if (e != cudaSuccess) return e;
  }
  // the output gradient has the layer's cout channels (YG: kCout)
  const int Cz = kTC[tz];
  const int bgrid = (int)std::max(1L, std::min((long)4 * u->num_sms, (long)batch * H * W * (Cz / 8) / 256));
  bias_grad_kernel<<<bgrid, 256, 0, u->stream>>>(u->grad[tz], batch, ilog2(H), ilog2(W),
                                                 ilog2(Cz / 8), u->pgrad + u->L[l].b_off);
  return cudaGetLastError();
}

// plane means (mode 0) or sample RMS deviations about u->means (mode 1) of
// a [batch][n][H][W] FP32 array
void plane_reduce(mlswlbm_unet* u, const float* x, int batch, int mode, double* out) {
  const int HW = u->H * u->W;
  plane_reduce_kernel<<<dim3(HW / kRedChunk, batch * u->n), 256, 0, u->stream>>>(
      x, batch * u->n, HW, u->n, mode, u->means, u->red_part, u->red_count, out);
}

cudaError_t forward(mlswlbm_unet* u, const float* h, int batch) {
  const int HW = u->H * u->W;
  plane_reduce(u, h, batch, 0, u->means);
  plane_reduce(u, h, batch, 1, u->rms);
  input_kernel<<<grid_for((long)batch * HW, 256), 256, 0, u->stream>>>(
      h, u->means, u->rms, batch, u->n, u->H, u->W, u->in_scale, u->extra, u->n_extra, u->act[X0]);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  for (int l = 0; l < kLayers; ++l) {
    // pooling before the first convolution of a level on the way down,
    // upsampling before the first one on the way up
    struct Pre { int layer, src, dst, up; };
    static const Pre pre[6] = {{2, S0, P1, 0}, {4, S1, P2, 0}, {6, S2, P3, 0},
                               {8, S3, U2, 1}, {10, D2, U1, 1}, {12, D1, U0, 1}};
    for (const Pre& p : pre) {
      if (p.layer != l) continue;
      const int C = kTC[p.dst], Hd = u->lh[p.dst], Wd = u->lw[p.dst];
      const int grid = grid_for((long)batch * Hd * Wd * C / 8, 256);
      if (p.up)
        up_kernel<<<grid, 256, 0, u->stream>>>(u->act[p.src], u->act[p.dst], batch, ilog2(Hd),
                                               ilog2(Wd), ilog2(C / 8));
      else
        pool_kernel<<<grid, 256, 0, u->stream>>>(u->act[p.src], u->act[p.dst], batch, ilog2(Hd),
                                                 ilog2(Wd), ilog2(C / 8));
      e = cudaGetLastError();
      if (e != cudaSuccess) return e;
    }
    e = conv_forward(u, l, batch);
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

cudaError_t backward(mlswlbm_unet* u, int batch) {
  cudaError_t e;
#define MLSW_CK(x)             \
  do {                         \
    e = (x);                   \
    if (e != cudaSuccess) return e; \
  } while (0)
  auto G = [&](int t) { return u->grad[t]; };
  auto Aq = [&](int t) { return (const bf16*)u->act[t]; };
  auto upmask = [&](int dU, int S, int dS) {
    const int C = kTC[S], H = u->lh[dU], W = u->lw[dU];
    up_grad_mask_kernel<<<grid_for((long)batch * (H / 2) * (W / 2) * C / 8, 256), 256, 0, u->stream>>>(
        G(dU), Aq(S), G(dS), batch, ilog2(H / 2), ilog2(W / 2), ilog2(C / 8));
    return cudaGetLastError();
  };
  auto poolmask = [&](int dP, int lev, int S) {
    const int C = kTC[S], H = u->lh[S], W = u->lw[S];
    pool_grad_add_mask_kernel<<<grid_for((long)batch * H * W * C / 8, 256), 256, 0, u->stream>>>(
        G(dP), u->skipg[lev], Aq(S), G(S), batch, ilog2(H), ilog2(W), ilog2(C / 8));
    return cudaGetLastError();
  };
  // layer 14 (out) .. 0, see the table
  MLSW_CK(weight_grad(u, 14, batch));
  MLSW_CK(conv_input_grad(u, 14, batch, G(D0), Aq(D0), nullptr, nullptr));
  MLSW_CK(weight_grad(u, 13, batch));
  MLSW_CK(conv_input_grad(u, 13, batch, G(B0), Aq(B0), nullptr, nullptr));
  MLSW_CK(weight_grad(u, 12, batch));
  MLSW_CK(conv_input_grad(u, 12, batch, G(U0), nullptr, u->skipg[0], nullptr));
  MLSW_CK(upmask(U0, D1, D1));
  MLSW_CK(weight_grad(u, 11, batch));
  MLSW_CK(conv_input_grad(u, 11, batch, G(B1), Aq(B1), nullptr, nullptr));
  MLSW_CK(weight_grad(u, 10, batch));
  MLSW_CK(conv_input_grad(u, 10, batch, G(U1), nullptr, u->skipg[1], nullptr));
  MLSW_CK(upmask(U1, D2, D2));
  MLSW_CK(weight_grad(u, 9, batch));
  MLSW_CK(conv_input_grad(u, 9, batch, G(B2), Aq(B2), nullptr, nullptr));
  MLSW_CK(weight_grad(u, 8, batch));
  MLSW_CK(conv_input_grad(u, 8, batch, G(U2), nullptr, u->skipg[2], nullptr));
  MLSW_CK(upmask(U2, S3, S3));
  MLSW_CK(weight_grad(u, 7, batch));
  MLSW_CK(conv_input_grad(u, 7, batch, G(A3), Aq(A3), nullptr, nullptr));
  MLSW_CK(weight_grad(u, 6, batch));
  MLSW_CK(conv_input_grad(u, 6, batch, G(P3), nullptr, nullptr, nullptr));
  MLSW_CK(poolmask(P3, 2, S2));
  MLSW_CK(weight_grad(u, 5, batch));
  MLSW_CK(conv_input_grad(u, 5, batch, G(A2), Aq(A2), nullptr, nullptr));
  MLSW_CK(weight_grad(u, 4, batch));
  MLSW_CK(conv_input_grad(u, 4, batch, G(P2), nullptr, nullptr, nullptr));
  MLSW_CK(poolmask(P2, 1, S1));
  MLSW_CK(weight_grad(u, 3, batch));
  MLSW_CK(conv_input_grad(u, 3, batch, G(A1), Aq(A1), nullptr, nullptr));
  MLSW_CK(weight_grad(u, 2, batch));
  MLSW_CK(conv_input_grad(u, 2, batch, G(P1), nullptr, nullptr, nullptr));
  MLSW_CK(poolmask(P1, 0, S0));
  MLSW_CK(weight_grad(u, 1, batch));
  MLSW_CK(conv_input_grad(u, 1, batch, G(A0), Aq(A0), nullptr, nullptr));
  MLSW_CK(weight_grad(u, 0, batch));
#undef MLSW_CK
  return cudaSuccess;
}

cudaError_t adam(mlswlbm_unet* u, double lr, int do_step) {
  AdamArgs a;
  std::memset(&a, 0, sizeof(a));
  for (int l = 0; l < kLayers; ++l) a.L[l] = u->L[l];
  a.p = u->params;
  a.g = u->pgrad;
  a.m = u->adam_m;
  a.v = u->adam_v;
  a.count = u->nparam;
  a.lr = (float)lr;
  a.b1 = 0.9f;
  a.b2 = 0.999f;
  a.eps = 1e-8f;
  const double t = (double)(u->adam_t + (do_step ? 1 : 0));
  a.c1 = do_step ? (float)(1.0 / (1.0 - std::pow(0.9, t))) : 1.f;
  a.c2 = do_step ? (float)(1.0 / (1.0 - std::pow(0.999, t))) : 1.f;
  adam_kernel<<<grid_for(u->nparam, 256), 256, 0, u->stream>>>(a, do_step);
  return cudaGetLastError();
}

bool is_pow2(int v) { return v > 0 && (v & (v - 1)) == 0; }

// |x - y|, with a NaN or infinite difference as +inf (a window with a
// non-finite prediction must fail its audit)
__device__ __forceinline__ float abs_diff_or_inf(float x, float y) {
  const float d = fabsf(x - y);
  return d <= 3.402823466e38f ? d : __int_as_float(0x7f800000);
}

// out[j] (zeroed by the caller; the bits of a non-negative float order as
// unsigned integers) = max over item j of |a - b|: a grid-stride loop of
// float4 loads (or scalars when the items are not 16-byte aligned), a
// warp-shuffle and block maximum, one atomic maximum per block and item.
__global__ void __launch_bounds__(256) max_abs_diff_kernel(const float* __restrict__ a,
                                                           const float* __restrict__ b, int count,
                                                           long elems, int vec,
                                                           unsigned* __restrict__ out) {
  __shared__ float wmax[8];
  for (int j = blockIdx.y; j < count; j += gridDim.y) {
    const float* pa = a + (long)j * elems;
    const float* pb = b + (long)j * elems;
    const long stride = (long)gridDim.x * blockDim.x;
    float m = 0.f;
    if (vec) {
      const float4* qa = reinterpret_cast<const float4*>(pa);
      const float4* qb = reinterpret_cast<const float4*>(pb);
      for (long i = (long)blockIdx.x * blockDim.x + threadIdx.x; i < elems / 4; i += stride) {
        const float4 x = __ldg(qa + i), y = __ldg(qb + i);
        m = fmaxf(m, fmaxf(fmaxf(abs_diff_or_inf(x.x, y.x), abs_diff_or_inf(x.y, y.y)),
                           fmaxf(abs_diff_or_inf(x.z, y.z), abs_diff_or_inf(x.w, y.w))));
      }
    } else {
      for (long i = (long)blockIdx.x * blockDim.x + threadIdx.x; i < elems; i += stride)
        m = fmaxf(m, abs_diff_or_inf(__ldg(pa + i), __ldg(pb + i)));
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0) wmax[threadIdx.x >> 5] = m;
    __syncthreads();
    if (threadIdx.x == 0) {
      float t = wmax[0];
      for (int w = 1; w < (int)(blockDim.x >> 5); ++w) t = fmaxf(t, wmax[w]);
      atomicMax(out + j, __float_as_uint(t));
    }
    __syncthreads();  // wmax is reused by the next item
  }
}

}  // namespace

extern "C" {

long mlswlbm_unet_param_count(void) {
  long n = 0;
  for (int l = 0; l < kLayers; ++l) n += (long)kNet[l].cout * 9 * layer_cin(l) + kNet[l].cout;
  return n;
}

int mlswlbm_unet_create(int n_layers, int nx, int ny, int max_batch, int n_extra, const double* extra,
                        unsigned long long seed, double in_scale, double out_scale, void* stream,
                        mlswlbm_unet** out) {
  if (!out) return MLSW_ERR_ARG;
  *out = nullptr;
  if (n_layers < 1 || n_layers > MLSW_MAX_LAYERS || n_extra < 0 || n_layers + n_extra > kCin0 ||
      (n_extra > 0 && !extra) || max_batch < 1 || !(in_scale > 0.0) || !(out_scale > 0.0) ||
      !std::isfinite(in_scale) || !std::isfinite(out_scale))
    return MLSW_ERR_ARG;
  // four levels, the coarsest at least 16 x 16 cells
  if (!is_pow2(nx) || !is_pow2(ny) || nx < 128 || ny < 128 || nx > 4096 || ny > 4096 ||
      (long)max_batch * n_layers > 65535)
    return MLSW_ERR_UNSUPPORTED;
  for (int j = 0; j < n_extra; ++j)
    if (!std::isfinite(extra[j])) return MLSW_ERR_ARG;
  mlswlbm_unet* u = new (std::nothrow) mlswlbm_unet;
  if (!u) return MLSW_ERR_NOMEM;
  std::memset(u, 0, sizeof(*u));
  u->n = n_layers;
  u->H = ny;
  u->W = nx;
  u->Bmax = max_batch;
  u->n_extra = n_extra;
  u->in_scale = (float)in_scale;
  u->out_scale = (float)out_scale;
  u->stream = (cudaStream_t)stream;
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
    delete u;
    return MLSW_ERR_CUDA;
  }
  u->num_sms = std::max(1, sms);
  for (int t = 0; t < kTensors; ++t) {
    u->lw[t] = nx >> kTL[t];
    u->lh[t] = ny >> kTL[t];
  }
  // parameters: every layer's weights [out][9][in], then its bias
  long off = 0;
  size_t wbytes = 0;
  for (int l = 0; l < kLayers; ++l) {
    LayerParams& L = u->L[l];
    L.cout = kNet[l].cout;
    L.cin = layer_cin(l);
    L.cout_pad = L.cout;
    L.cin_pad = L.cin;
    L.w_off = off;
    off += (long)L.cout * 9 * L.cin;
    L.b_off = off;
    off += L.cout;
    wbytes += 2 * (size_t)9 * L.cout * L.cin * sizeof(bf16);
  }
  u->nparam = off;
  bool ok = true;
  for (int t = 0; t < kTensors && ok; ++t) {
    const size_t bytes = tensor_elems(u, t) * sizeof(bf16);
    ok = cudaMalloc(&u->act[t], bytes) == cudaSuccess && cudaMalloc(&u->grad[t], bytes) == cudaSuccess &&
         cudaMemsetAsync(u->act[t], 0, bytes, u->stream) == cudaSuccess &&
         cudaMemsetAsync(u->grad[t], 0, bytes, u->stream) == cudaSuccess;
  }
  const int skipt[3] = {S0, S1, S2};
  for (int j = 0; j < 3 && ok; ++j)
    ok = cudaMalloc(&u->skipg[j], tensor_elems(u, skipt[j]) * sizeof(bf16)) == cudaSuccess;
  const size_t hsz = (size_t)max_batch * n_layers * nx * ny;
  ok = ok && cudaMalloc(&u->ydense, hsz * sizeof(float)) == cudaSuccess &&
       cudaMalloc(&u->hbuf, hsz * sizeof(float)) == cudaSuccess &&
       cudaMalloc(&u->means, (size_t)max_batch * n_layers * sizeof(double)) == cudaSuccess &&
       cudaMalloc(&u->rms, (size_t)max_batch * sizeof(double)) == cudaSuccess &&
       cudaMalloc(&u->red_part, (size_t)max_batch * n_layers * (nx * ny / kRedChunk) *
                                    sizeof(double)) == cudaSuccess &&
       cudaMalloc(&u->red_count, sizeof(unsigned)) == cudaSuccess &&
       cudaMemsetAsync(u->red_count, 0, sizeof(unsigned), u->stream) == cudaSuccess &&
       cudaMalloc(&u->dloss, sizeof(double)) == cudaSuccess &&
       cudaMalloc(&u->extra, (size_t)kCin0 * sizeof(float)) == cudaSuccess &&
       cudaMalloc(&u->params, u->nparam * sizeof(float)) == cudaSuccess &&
       cudaMalloc(&u->pgrad, u->nparam * sizeof(float)) == cudaSuccess &&
       cudaMalloc(&u->adam_m, u->nparam * sizeof(float)) == cudaSuccess &&
       cudaMalloc(&u->adam_v, u->nparam * sizeof(float)) == cudaSuccess &&
       cudaMalloc(&u->wbuf, wbytes) == cudaSuccess && cudaMalloc(&u->err, sizeof(int)) == cudaSuccess;
  if (!ok) {
    cudaGetLastError();
    unet_free(u);
    return MLSW_ERR_NOMEM;
  }
  // BF16 weight copies and their tensor maps
  {
    bf16* w = u->wbuf;
    for (int l = 0; l < kLayers && ok; ++l) {
      LayerParams& L = u->L[l];
      L.wf = w;
      w += (size_t)9 * L.cout * L.cin;
      L.wd = w;
      w += (size_t)9 * L.cout * L.cin;
      ok = map_weights(&u->wf_map[l], L.wf, L.cin, L.cout, kc_fwd(l), bn_fwd(l)) &&
           map_weights(&u->wd_map[l], L.wd, L.cout, L.cin, kc_bwd(l), bn_bwd(l));
    }
  }
  for (int t = 0; t < kTensors && ok; ++t) {
    const int W = u->lw[t], H = u->lh[t], C = kTC[t];
    const int kc = act_kc(t);
    // convolution inputs: boxes of 16 x 10 pixels (a tile and its row halo)
    if (kc) ok = map_nhwc(&u->act_map[t], u->act[t], C, W, H, max_batch, kc, 16, 10);
    // the gradient of a convolution's output feeds its input-gradient
    // convolution with channel chunks of min(64, C)
    ok = ok && map_nhwc(&u->grad_map[t], u->grad[t], C, W, H, max_batch, std::min(64, C), 16, 10) &&
         map_nhwc(&u->wg_act[t], u->act[t], C, W, H, max_batch, 64, 8, 10) &&
         map_nhwc(&u->wg_grad[t], u->grad[t], C, W, H, max_batch, 64, 8, 8);
  }
  if (!ok) {
    unet_free(u);
    return MLSW_ERR_CUDA;
  }
  // He-normal weights (std sqrt(2 / (9 cin))), zero biases, zero Adam moments
  std::vector<float> p(u->nparam, 0.f);
  std::mt19937_64 gen(seed);
  for (int l = 0; l < kLayers; ++l) {
    const LayerParams& L = u->L[l];
    std::normal_distribution<double> nd(0.0, std::sqrt(2.0 / (9.0 * L.cin)));
    for (long k = 0; k < (long)L.cout * 9 * L.cin; ++k) p[L.w_off + k] = (float)nd(gen);
  }
  float ex[kCin0] = {0.f};
  for (int j = 0; j < n_extra; ++j) ex[j] = (float)extra[j];
  ok = cudaMemcpyAsync(u->params, p.data(), u->nparam * sizeof(float), cudaMemcpyHostToDevice, u->stream) ==
           cudaSuccess &&
       cudaMemcpyAsync(u->extra, ex, sizeof(ex), cudaMemcpyHostToDevice, u->stream) == cudaSuccess &&
       cudaMemsetAsync(u->adam_m, 0, u->nparam * sizeof(float), u->stream) == cudaSuccess &&
       cudaMemsetAsync(u->adam_v, 0, u->nparam * sizeof(float), u->stream) == cudaSuccess &&
       cudaMemsetAsync(u->err, 0, sizeof(int), u->stream) == cudaSuccess &&
       adam(u, 0.0, 0) == cudaSuccess && cudaStreamSynchronize(u->stream) == cudaSuccess;
  if (!ok) {
    unet_free(u);
    return MLSW_ERR_CUDA;
  }
  *out = u;
  return MLSW_OK;
}

int mlswlbm_unet_predict(mlswlbm_unet* u, const float* h, float* out, int batch) {
  if (!u || !h || !out || batch < 1 || batch > u->Bmax || out == h) return MLSW_ERR_ARG;
  if (forward(u, h, batch) != cudaSuccess) return MLSW_ERR_CUDA;
  const int HW = u->H * u->W;
  plane_reduce(u, u->ydense, batch, 0, u->means);
  const long total = (long)batch * u->n * HW;
  output_kernel<<<grid_for(total, 256), 256, 0, u->stream>>>(h, u->ydense, u->means, u->rms, total,
                                                              u->n, HW, 1.f / u->out_scale, out);
  return cudaGetLastError() == cudaSuccess ? MLSW_OK : MLSW_ERR_CUDA;
}

int mlswlbm_unet_train_step(mlswlbm_unet* u, const float* h, const float* target, int batch, double lr,
                            double* loss) {
  if (!u || !h || !target || batch < 1 || batch > u->Bmax || !(lr >= 0.0)) return MLSW_ERR_ARG;
  if (forward(u, h, batch) != cudaSuccess) return MLSW_ERR_CUDA;
  const long count = (long)batch * u->n * u->H * u->W;
  if (cudaMemsetAsync(u->dloss, 0, sizeof(double), u->stream) != cudaSuccess ||
      cudaMemsetAsync(u->pgrad, 0, u->nparam * sizeof(float), u->stream) != cudaSuccess)
    return MLSW_ERR_CUDA;
  loss_kernel<<<grid_for((long)batch * u->H * u->W, 256), 256, 0, u->stream>>>(
      u->ydense, h, target, u->rms, batch, u->n, u->H, u->W, u->out_scale, 1.f / (float)count,
      u->dloss, u->grad[YG]);
  if (cudaGetLastError() != cudaSuccess || backward(u, batch) != cudaSuccess) return MLSW_ERR_CUDA;
  if (adam(u, lr, 1) != cudaSuccess) return MLSW_ERR_CUDA;
  u->adam_t += 1;
  if (loss) {
    double s = 0.0;
    if (cudaMemcpyAsync(&s, u->dloss, sizeof(double), cudaMemcpyDeviceToHost, u->stream) != cudaSuccess ||
        cudaStreamSynchronize(u->stream) != cudaSuccess)
      return MLSW_ERR_CUDA;
    *loss = s / (double)count;
  }
  return MLSW_OK;
}

int mlswlbm_unet_status(mlswlbm_unet* u) {
  if (!u) return MLSW_ERR_ARG;
  int e = 0;
  if (cudaMemcpyAsync(&e, u->err, sizeof(int), cudaMemcpyDeviceToHost, u->stream) != cudaSuccess ||
      cudaStreamSynchronize(u->stream) != cudaSuccess)
    return MLSW_ERR_CUDA;
  return e ? MLSW_ERR_TIMEOUT : MLSW_OK;
}

int mlswlbm_unet_set_params(mlswlbm_unet* u, const float* host, long count) {
  if (!u || !host || count != u->nparam) return MLSW_ERR_ARG;
  if (cudaMemcpyAsync(u->params, host, count * sizeof(float), cudaMemcpyHostToDevice, u->stream) != cudaSuccess ||
      cudaMemsetAsync(u->adam_m, 0, count * sizeof(float), u->stream) != cudaSuccess ||
      cudaMemsetAsync(u->adam_v, 0, count * sizeof(float), u->stream) != cudaSuccess ||
      adam(u, 0.0, 0) != cudaSuccess || cudaStreamSynchronize(u->stream) != cudaSuccess)
    return MLSW_ERR_CUDA;
  u->adam_t = 0;
  return MLSW_OK;
}

int mlswlbm_unet_get_params(mlswlbm_unet* u, float* host, long count) {
  if (!u || !host || count != u->nparam) return MLSW_ERR_ARG;
  if (cudaMemcpyAsync(host, u->params, count * sizeof(float), cudaMemcpyDeviceToHost, u->stream) != cudaSuccess ||
      cudaStreamSynchronize(u->stream) != cudaSuccess)
    return MLSW_ERR_CUDA;
  return MLSW_OK;
}

int mlswlbm_unet_debug(mlswlbm_unet* u, int kind, int id, void* out, long bytes) {
  if (!u || !out || bytes < 0) return MLSW_ERR_ARG;
  const void* src = nullptr;
  size_t len = 0;
  if ((kind == 0 || kind == 1) && id >= 0 && id < kTensors) {
    src = kind == 0 ? (const void*)u->act[id] : (const void*)u->grad[id];
    len = tensor_elems(u, id) * sizeof(bf16);
  } else if (kind == 2) {
    src = u->pgrad;
    len = u->nparam * sizeof(float);
  } else if (kind == 3) {
    src = u->ydense;
    len = (size_t)u->Bmax * u->n * u->H * u->W * sizeof(float);
  } else if (kind == 4 && id >= 0 && id < 3) {
    const int skipt[3] = {S0, S1, S2};
    src = u->skipg[id];
    len = tensor_elems(u, skipt[id]) * sizeof(bf16);
  } else {
    return MLSW_ERR_ARG;
  }
  if ((size_t)bytes < len) return MLSW_ERR_ARG;
  if (cudaMemcpyAsync(out, src, len, cudaMemcpyDeviceToHost, u->stream) != cudaSuccess ||
      cudaStreamSynchronize(u->stream) != cudaSuccess)
    return MLSW_ERR_CUDA;
  return MLSW_OK;
}

void mlswlbm_unet_destroy(mlswlbm_unet* u) {
  if (!u) return;
  cudaStreamSynchronize(u->stream);
  unet_free(u);
}

int mlswlbm_max_abs_diff(const float* a, const float* b, int count, long elems, float* out,
                         void* stream) {
  if (!a || !b || !out || count < 1 || elems < 1) return MLSW_ERR_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  if (cudaMemsetAsync(out, 0, (size_t)count * sizeof(float), st) != cudaSuccess)
    return MLSW_ERR_CUDA;
  const bool vec = elems % 4 == 0 && (reinterpret_cast<uintptr_t>(a) % 16) == 0 &&
                   (reinterpret_cast<uintptr_t>(b) % 16) == 0;
  const long work = vec ? elems / 4 : elems;
  const long bx = std::min<long>((work + 256 * 8 - 1) / (256 * 8), 1024);
  const dim3 grid((unsigned)std::max<long>(bx, 1), (unsigned)std::min(count, 65535));
  max_abs_diff_kernel<<<grid, 256, 0, st>>>(a, b, count, elems, vec ? 1 : 0,
                                            reinterpret_cast<unsigned*>(out));
  return cudaGetLastError() == cudaSuccess ? MLSW_OK : MLSW_ERR_CUDA;
}

}  // extern "C"
