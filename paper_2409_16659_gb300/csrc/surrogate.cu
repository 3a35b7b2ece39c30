// surrogate.cu -- a small convolutional surrogate of 64 LBM steps.
//
// The network maps the layer heights h(t) of a periodic lattice to the
// change h(t + 64 steps) - h(t): three K x K convolutions (K = 5, periodic
// padding) with 16 -> 32 -> 32 -> 16 channels and ReLU between them. The
// input channels are the n layer heights minus their means, times in_scale,
// and zero channels up to 16; the first n output channels are the change
// times out_scale. The prediction is projected back onto exact per-layer
// mass (the change is made mean-free per layer), as the LBM conserves it.
//
// Arithmetic: activations and weights in BF16, products accumulated in FP32
// on the tensor cores (warp-level mma.sync m16n8k16). Activations are NHWC
// (channels innermost). A convolution is an implicit GEMM
//   out[p][o] = sum_{d, i} in[p + off(d)][i] * W[d][i][o]
// over pixels p; its gradient with respect to the input is the same form
// with the offsets reversed and W transposed (so the forward kernel serves
// both), and its weight gradient is a GEMM over pixels, split over CTAs and
// summed with FP32 atomics. Master weights and the Adam moments are FP32.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>
#include <new>
#include <cstring>
#include <random>
#include <vector>

#include "mlswlbm.h"

namespace {

constexpr int KS = 5, KR = KS / 2, KD = KS * KS;
constexpr int C0 = 16, C1 = 32, C2 = 32, C3 = 16;
constexpr int NCONV = 3;
constexpr int CIN[NCONV] = {C0, C1, C2};
constexpr int COUT[NCONV] = {C1, C2, C3};

__device__ __forceinline__ void mma_bf16(float (&c)[4], uint32_t a0, uint32_t a1, uint32_t a2,
                                         uint32_t a3, uint32_t b0, uint32_t b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, "
      "{%8,%9}, {%0,%1,%2,%3};"
      : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
      : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
}

__device__ __forceinline__ uint32_t ld32(const __nv_bfloat16* p) {
  return *reinterpret_cast<const uint32_t*>(p);
}
__device__ __forceinline__ uint32_t pack2(__nv_bfloat16 lo, __nv_bfloat16 hi) {
  return (uint32_t)__bfloat16_as_ushort(lo) | ((uint32_t)__bfloat16_as_ushort(hi) << 16);
}

// periodic neighbour of pixel (b, y, x) at offset d (dy, dx in -KR..KR)
__device__ __forceinline__ long nb_pixel(int b, int y, int x, int d, int H, int W) {
  int yy = y + d / KS - KR, xx = x + d % KS - KR;
  yy += (yy < 0) ? H : 0;
  yy -= (yy >= H) ? H : 0;
  xx += (xx < 0) ? W : 0;
  xx -= (xx >= W) ? W : 0;
  return ((long)b * H + yy) * W + xx;
}

// ---------------------------------------------------------------------------
// Convolution as implicit GEMM. One warp: 16 consecutive pixels of a row
// (W a multiple of 16) times all COUT channels. Weights wt[d][o][i] (BF16,
// i innermost). Epilogue: + bias, then ReLU (RELU), or times (mask > 0)
// (MASK: the backward of a ReLU whose output is `mask`), stored BF16, or
// FP32 (OUTF).
// ---------------------------------------------------------------------------
template <int CI, int CO, bool RELU, bool MASK, bool OUTF>
__global__ void __launch_bounds__(128)
    conv_kernel(const __nv_bfloat16* __restrict__ in, const __nv_bfloat16* __restrict__ wt,
                const float* __restrict__ bias, const __nv_bfloat16* __restrict__ mask,
                void* __restrict__ out, int B, int H, int W) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const long seg = (long)blockIdx.x * 4 + warp;  // 16-pixel row segment
  const long nseg = (long)B * H * (W / 16);
  if (seg >= nseg) return;
  const int x0 = (int)(seg % (W / 16)) * 16;
  const long row = seg / (W / 16);
  const int y = (int)(row % H), b = (int)(row / H);
  const int g = lane >> 2, t = lane & 3;
  float acc[CO / 8][4];
#pragma unroll
  for (int n = 0; n < CO / 8; ++n) acc[n][0] = acc[n][1] = acc[n][2] = acc[n][3] = 0.f;
  for (int d = 0; d < KD; ++d) {
    const __nv_bfloat16* r0 = in + nb_pixel(b, y, x0 + g, d, H, W) * CI;
    const __nv_bfloat16* r1 = in + nb_pixel(b, y, x0 + g + 8, d, H, W) * CI;
#pragma unroll
    for (int c0 = 0; c0 < CI; c0 += 16) {
      const uint32_t a0 = ld32(r0 + c0 + 2 * t), a1 = ld32(r1 + c0 + 2 * t);
      const uint32_t a2 = ld32(r0 + c0 + 2 * t + 8), a3 = ld32(r1 + c0 + 2 * t + 8);
#pragma unroll
      for (int n = 0; n < CO / 8; ++n) {
        const __nv_bfloat16* wp = wt + ((long)d * CO + n * 8 + g) * CI + c0 + 2 * t;
        mma_bf16(acc[n], a0, a1, a2, a3, ld32(wp), ld32(wp + 8));
      }
    }
  }
  const long p0 = ((long)b * H + y) * W + x0 + g, p1 = p0 + 8;
#pragma unroll
  for (int n = 0; n < CO / 8; ++n) {
    const int o = n * 8 + 2 * t;
    float v[4] = {acc[n][0], acc[n][1], acc[n][2], acc[n][3]};
    if (bias) {
      v[0] += bias[o];
      v[1] += bias[o + 1];
      v[2] += bias[o];
      v[3] += bias[o + 1];
    }
    if (RELU) {
#pragma unroll
      for (int j = 0; j < 4; ++j) v[j] = fmaxf(v[j], 0.f);
    }
    if (MASK) {
      const __nv_bfloat16* m0 = mask + p0 * CO + o;
      const __nv_bfloat16* m1 = mask + p1 * CO + o;
      v[0] = __bfloat162float(m0[0]) > 0.f ? v[0] : 0.f;
      v[1] = __bfloat162float(m0[1]) > 0.f ? v[1] : 0.f;
      v[2] = __bfloat162float(m1[0]) > 0.f ? v[2] : 0.f;
      v[3] = __bfloat162float(m1[1]) > 0.f ? v[3] : 0.f;
    }
    if (OUTF) {
      float* of = static_cast<float*>(out);
      *reinterpret_cast<float2*>(of + p0 * CO + o) = make_float2(v[0], v[1]);
      *reinterpret_cast<float2*>(of + p1 * CO + o) = make_float2(v[2], v[3]);
    } else {
      __nv_bfloat16* ob = static_cast<__nv_bfloat16*>(out);
      *reinterpret_cast<__nv_bfloat162*>(ob + p0 * CO + o) = __floats2bfloat162_rn(v[0], v[1]);
      *reinterpret_cast<__nv_bfloat162*>(ob + p1 * CO + o) = __floats2bfloat162_rn(v[2], v[3]);
    }
  }
}

// ---------------------------------------------------------------------------
// Weight gradient dW[d][i][o] += sum_p in[p + off(d)][i] * dout[p][o] over
// one chunk of pixels (blockIdx.x) for one offset d (blockIdx.y); one warp
// per 16 x 8 tile of (i, o). The bias gradient db[o] = sum_p dout[p][o] is
// bias_grad_kernel.
// ---------------------------------------------------------------------------
constexpr int kChunk = 1024;  // pixels per CTA

template <int CI, int CO>
__global__ void wgrad_kernel(const __nv_bfloat16* __restrict__ in,
                             const __nv_bfloat16* __restrict__ dout, float* __restrict__ dw,
                             int B, int H, int W) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  constexpr int TN = CO / 8;
  const int ti = warp / TN, tn = warp % TN;  // tile (16 i) x (8 o)
  const int d = blockIdx.y;
  const long npix = (long)B * H * W;
  const long pbeg = (long)blockIdx.x * kChunk;
  const int g = lane >> 2, t = lane & 3;
  const int i0 = ti * 16 + g, o0 = tn * 8 + g;
  float acc[4] = {0.f, 0.f, 0.f, 0.f};
  for (long k = pbeg; k < pbeg + kChunk && k < npix; k += 16) {
    // pixels of this k-step for columns 2t, 2t+1 and 2t+8, 2t+9
    long pk[4];
    long nbk[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const long p = k + 2 * t + (j & 1) + (j >> 1) * 8;
      pk[j] = p < npix ? p : -1;
      if (pk[j] >= 0) {
        const int x = (int)(p % W);
        const long r = p / W;
        nbk[j] = nb_pixel((int)(r / H), (int)(r % H), x, d, H, W);
      } else {
        nbk[j] = -1;
      }
    }
    auto inv = [&](int j, int i) {
      return nbk[j] >= 0 ? in[nbk[j] * CI + i] : __float2bfloat16(0.f);
    };
    auto dov = [&](int j, int o) {
      return pk[j] >= 0 ? dout[pk[j] * CO + o] : __float2bfloat16(0.f);
    };
    const uint32_t a0 = pack2(inv(0, i0), inv(1, i0));
    const uint32_t a1 = pack2(inv(0, i0 + 8), inv(1, i0 + 8));
    const uint32_t a2 = pack2(inv(2, i0), inv(3, i0));
    const uint32_t a3 = pack2(inv(2, i0 + 8), inv(3, i0 + 8));
    const uint32_t b0 = pack2(dov(0, o0), dov(1, o0));
    const uint32_t b1 = pack2(dov(2, o0), dov(3, o0));
    mma_bf16(acc, a0, a1, a2, a3, b0, b1);
  }
  const int oc = tn * 8 + 2 * t;
  float* base = dw + (long)d * CI * CO;
  atomicAdd(base + (long)i0 * CO + oc, acc[0]);
  atomicAdd(base + (long)i0 * CO + oc + 1, acc[1]);
  atomicAdd(base + (long)(i0 + 8) * CO + oc, acc[2]);
  atomicAdd(base + (long)(i0 + 8) * CO + oc + 1, acc[3]);
}

template <int CO>
__global__ void bias_grad_kernel(const __nv_bfloat16* __restrict__ dout, float* __restrict__ db,
                                 long npix) {
  __shared__ float s[CO];
  for (int o = threadIdx.x; o < CO; o += blockDim.x) s[o] = 0.f;
  __syncthreads();
  for (long e = (long)blockIdx.x * blockDim.x + threadIdx.x; e < npix * CO;
       e += (long)gridDim.x * blockDim.x)
    atomicAdd(s + (int)(e % CO), __bfloat162float(dout[e]));
  __syncthreads();
  for (int o = threadIdx.x; o < CO; o += blockDim.x) atomicAdd(db + o, s[o]);
}

// ---------------------------------------------------------------------------
// input, output, loss
// ---------------------------------------------------------------------------
// per (sample, layer) sums of h (FP64), for the input means
__global__ void layer_sum_kernel(const float* __restrict__ h, long cells, double* __restrict__ sums) {
  const long base = (long)blockIdx.y * cells;
  double acc = 0.0;
  for (long c = (long)blockIdx.x * blockDim.x + threadIdx.x; c < cells;
       c += (long)gridDim.x * blockDim.x)
    acc += h[base + c];
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0) atomicAdd(sums + blockIdx.y, acc);
}

// x0[b][y][x][c] = (h[b][c][y][x] - mean[b][c]) * s for c < n, 0 above
__global__ void input_kernel(const float* __restrict__ h, const double* __restrict__ sums, int n,
                             long cells, float s, __nv_bfloat16* __restrict__ x0, long npix) {
  const long e = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= npix * C0) return;
  const int c = (int)(e % C0);
  const long p = e / C0;
  const long b = p / cells, cell = p - b * cells;
  float v = 0.f;
  if (c < n) {
    const float mean = (float)(sums[b * n + c] / (double)cells);
    v = (h[(b * n + c) * cells + cell] - mean) * s;
  }
  x0[e] = __float2bfloat16(v);
}

// out[b][c][cell] = h + (y / s) - (mean over the layer of y / s), c < n:
// the change projected onto exact per-layer mass. ysum: per (b, c) sums of y.
__global__ void output_kernel(const float* __restrict__ h, const float* __restrict__ y,
                              const double* __restrict__ ysum, int n, long cells, float inv_s,
                              float* __restrict__ out, long total) {
  const long e = (long)blockIdx.x * blockDim.x + threadIdx.x;  // over b, c, cell
  if (e >= total) return;
  const long cell = e % cells, bc = e / cells;
  const int c = (int)(bc % n);
  const long b = bc / n;
  const float mean = (float)(ysum[bc] / (double)cells);
  out[e] = h[e] + (y[(b * cells + cell) * C3 + c] - mean) * inv_s;
}

// per (b, c < n) sums of the network output y [pixel][C3]
__global__ void out_sum_kernel(const float* __restrict__ y, int n, long cells,
                               double* __restrict__ sums) {
  const int bc = blockIdx.y, b = bc / n, c = bc % n;
  double acc = 0.0;
  for (long cell = (long)blockIdx.x * blockDim.x + threadIdx.x; cell < cells;
       cell += (long)gridDim.x * blockDim.x)
    acc += y[((long)b * cells + cell) * C3 + c];
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0) atomicAdd(sums + bc, acc);
}

// loss = mean over (b, c < n, cell) of (y - (target - h) s)^2, and its
// gradient dy (BF16, zero for c >= n)
__global__ void loss_kernel(const float* __restrict__ y, const float* __restrict__ h,
                            const float* __restrict__ target, int n, long cells, float s,
                            float inv_count, __nv_bfloat16* __restrict__ dy,
                            double* __restrict__ loss, long npix) {
  double acc = 0.0;
  for (long e = (long)blockIdx.x * blockDim.x + threadIdx.x; e < npix * C3;
       e += (long)gridDim.x * blockDim.x) {
    const int c = (int)(e % C3);
    const long p = e / C3;
    float gval = 0.f;
    if (c < n) {
      const long b = p / cells, cell = p - b * cells;
      const long hi = (b * n + c) * cells + cell;
      const float r = y[e] - (target[hi] - h[hi]) * s;
      acc += (double)r * r;
      gval = 2.f * r * inv_count;
    }
    dy[e] = __float2bfloat16(gval);
  }
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0) atomicAdd(loss, acc * inv_count);
}

// Adam on FP32 master parameters; then the BF16 copies: wf[d][o][i] for the
// forward pass and wb[KD - 1 - d][i][o] for the input gradient
__global__ void adam_kernel(float* __restrict__ w, const float* __restrict__ gr,
                            float* __restrict__ m, float* __restrict__ v, long count, float lr,
                            float b1, float b2, float c1, float c2, float eps) {
  const long e = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= count) return;
  const float g = gr[e];
  const float mm = b1 * m[e] + (1.f - b1) * g, vv = b2 * v[e] + (1.f - b2) * g * g;
  m[e] = mm;
  v[e] = vv;
  w[e] -= lr * (mm * c1) / (sqrtf(vv * c2) + eps);
}

__global__ void weight_copies_kernel(const float* __restrict__ w, int ci, int co,
                                     __nv_bfloat16* __restrict__ wf,
                                     __nv_bfloat16* __restrict__ wb) {
  const long e = (long)blockIdx.x * blockDim.x + threadIdx.x;  // over d, i, o of w
  if (e >= (long)KD * ci * co) return;
  const int o = (int)(e % co), i = (int)((e / co) % ci), d = (int)(e / ((long)ci * co));
  const __nv_bfloat16 v = __float2bfloat16(w[e]);
  wf[((long)d * co + o) * ci + i] = v;
  wb[((long)(KD - 1 - d) * ci + i) * co + o] = v;
}

unsigned blocks(long n, int t) { return (unsigned)((n + t - 1) / t); }

}  // namespace

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
struct mlswlbm_surrogate {
  int n, nx, ny, max_batch;
  float in_scale, out_scale;
  cudaStream_t st;
  long woff[NCONV + 1];  // offsets of each layer's weights in the parameter vector
  long boff[NCONV];      // offsets of each layer's biases
  long nparam;
  float* param;          // FP32 master parameters (weights w[d][i][o], then biases)
  float* grad;
  float* adam_m;
  float* adam_v;
  __nv_bfloat16* wf[NCONV];
  __nv_bfloat16* wb[NCONV];
  __nv_bfloat16* act[NCONV];  // x0, a1, a2 (inputs of the three convolutions)
  __nv_bfloat16* dact[NCONV]; // gradients with respect to them (dact[0] unused)
  float* y;                   // network output, [pixel][C3] FP32
  __nv_bfloat16* dy;          // its gradient (BF16)
  double* sums;               // input layer sums, output sums, loss
  long step;
};

namespace {

#define SU(call)                                     \
  do {                                               \
    if ((call) != cudaSuccess) return MLSW_ERR_CUDA; \
  } while (0)

cudaError_t refresh_copies(mlswlbm_surrogate* s) {
  for (int l = 0; l < NCONV; ++l) {
    const long cnt = (long)KD * CIN[l] * COUT[l];
    weight_copies_kernel<<<blocks(cnt, 256), 256, 0, s->st>>>(s->param + s->woff[l], CIN[l],
                                                                COUT[l], s->wf[l], s->wb[l]);
  }
  return cudaGetLastError();
}

cudaError_t forward(mlswlbm_surrogate* s, const float* h, int B) {
  const long cells = (long)s->nx * s->ny, npix = B * cells;
  const int n = s->n;
  double* insum = s->sums;
  cudaError_t e = cudaMemsetAsync(insum, 0, sizeof(double) * B * n, s->st);
  if (e != cudaSuccess) return e;
  layer_sum_kernel<<<dim3(64, B * n), 256, 0, s->st>>>(h, cells, insum);
  input_kernel<<<blocks(npix * C0, 256), 256, 0, s->st>>>(h, insum, n, cells, s->in_scale,
                                                          s->act[0], npix);
  const unsigned g = blocks(npix / 16, 4);
  conv_kernel<C0, C1, true, false, false><<<g, 128, 0, s->st>>>(
      s->act[0], s->wf[0], s->param + s->boff[0], nullptr, s->act[1], B, s->ny, s->nx);
  conv_kernel<C1, C2, true, false, false><<<g, 128, 0, s->st>>>(
      s->act[1], s->wf[1], s->param + s->boff[1], nullptr, s->act[2], B, s->ny, s->nx);
  conv_kernel<C2, C3, false, false, true><<<g, 128, 0, s->st>>>(
      s->act[2], s->wf[2], s->param + s->boff[2], nullptr, s->y, B, s->ny, s->nx);
  return cudaGetLastError();
}

}  // namespace

extern "C" {

long mlswlbm_surrogate_param_count(void) {
  long c = 0;
  for (int l = 0; l < NCONV; ++l) c += (long)KD * CIN[l] * COUT[l] + COUT[l];
  return c;
}

int mlswlbm_surrogate_create(int n_layers, int nx, int ny, int max_batch, unsigned long long seed,
                             double in_scale, double out_scale, void* stream,
                             mlswlbm_surrogate** out) {
  if (!out) return MLSW_ERR_ARG;
  *out = nullptr;
  if (n_layers < 1 || n_layers > MLSW_MAX_LAYERS || nx < 16 || nx % 16 != 0 || ny < 1 ||
      max_batch < 1 || !(in_scale > 0.0) || !(out_scale > 0.0) || !std::isfinite(in_scale) ||
      !std::isfinite(out_scale))
    return MLSW_ERR_ARG;
  mlswlbm_surrogate* s = new (std::nothrow) mlswlbm_surrogate;
  if (!s) return MLSW_ERR_NOMEM;
  std::memset(s, 0, sizeof(*s));
  s->n = n_layers;
  s->nx = nx;
  s->ny = ny;
  s->max_batch = max_batch;
  s->in_scale = (float)in_scale;
  s->out_scale = (float)out_scale;
  s->st = (cudaStream_t)stream;
  long off = 0;
  for (int l = 0; l < NCONV; ++l) {
    s->woff[l] = off;
    off += (long)KD * CIN[l] * COUT[l];
  }
  for (int l = 0; l < NCONV; ++l) {
    s->boff[l] = off;
    off += COUT[l];
  }
  s->nparam = off;
  const long npix = (long)max_batch * nx * ny;
  bool ok = cudaMalloc(&s->param, off * sizeof(float)) == cudaSuccess &&
            cudaMalloc(&s->grad, off * sizeof(float)) == cudaSuccess &&
            cudaMalloc(&s->adam_m, off * sizeof(float)) == cudaSuccess &&
            cudaMalloc(&s->adam_v, off * sizeof(float)) == cudaSuccess &&
            cudaMalloc(&s->y, npix * C3 * sizeof(float)) == cudaSuccess &&
            cudaMalloc(&s->dy, npix * C3 * sizeof(__nv_bfloat16)) == cudaSuccess &&
            cudaMalloc(&s->sums, (2 * (size_t)max_batch * n_layers + 1) * sizeof(double)) ==
                cudaSuccess;
  for (int l = 0; l < NCONV && ok; ++l) {
    ok = cudaMalloc(&s->wf[l], (size_t)KD * CIN[l] * COUT[l] * 2) == cudaSuccess &&
         cudaMalloc(&s->wb[l], (size_t)KD * CIN[l] * COUT[l] * 2) == cudaSuccess &&
         cudaMalloc(&s->act[l], (size_t)npix * CIN[l] * 2) == cudaSuccess &&
         cudaMalloc(&s->dact[l], (size_t)npix * CIN[l] * 2) == cudaSuccess;
  }
  if (!ok) {
    cudaGetLastError();
    mlswlbm_surrogate_destroy(s);
    return MLSW_ERR_NOMEM;
  }
  // He-normal weights from a seeded generator, zero biases
  std::vector<float> w(off, 0.f);
  std::mt19937_64 rng(seed);
  for (int l = 0; l < NCONV; ++l) {
    std::normal_distribution<float> nd(0.f, std::sqrt(2.f / (float)(KD * CIN[l])));
    for (long e = 0; e < (long)KD * CIN[l] * COUT[l]; ++e) w[s->woff[l] + e] = nd(rng);
  }
  const int rc = mlswlbm_surrogate_set_params(s, w.data(), off);
  if (rc != MLSW_OK) {
    mlswlbm_surrogate_destroy(s);
    return rc;
  }
  *out = s;
  return MLSW_OK;
}

int mlswlbm_surrogate_set_params(mlswlbm_surrogate* s, const float* host, long count) {
  if (!s || !host || count != s->nparam) return MLSW_ERR_ARG;
  SU(cudaMemcpyAsync(s->param, host, count * sizeof(float), cudaMemcpyHostToDevice, s->st));
  SU(cudaMemsetAsync(s->adam_m, 0, count * sizeof(float), s->st));
  SU(cudaMemsetAsync(s->adam_v, 0, count * sizeof(float), s->st));
  s->step = 0;
  SU(refresh_copies(s));
  SU(cudaStreamSynchronize(s->st));
  return MLSW_OK;
}

int mlswlbm_surrogate_get_params(mlswlbm_surrogate* s, float* host, long count) {
  if (!s || !host || count != s->nparam) return MLSW_ERR_ARG;
  SU(cudaMemcpyAsync(host, s->param, count * sizeof(float), cudaMemcpyDeviceToHost, s->st));
  SU(cudaStreamSynchronize(s->st));
  return MLSW_OK;
}

int mlswlbm_surrogate_predict(mlswlbm_surrogate* s, const float* h, float* out, int batch) {
  if (!s || !h || !out || batch < 1 || batch > s->max_batch) return MLSW_ERR_ARG;
  const long cells = (long)s->nx * s->ny, total = (long)batch * s->n * cells;
  SU(forward(s, h, batch));
  double* ysum = s->sums + (size_t)s->max_batch * s->n;
  SU(cudaMemsetAsync(ysum, 0, sizeof(double) * batch * s->n, s->st));
  out_sum_kernel<<<dim3(64, batch * s->n), 256, 0, s->st>>>(s->y, s->n, cells, ysum);
  output_kernel<<<blocks(total, 256), 256, 0, s->st>>>(h, s->y, ysum, s->n, cells,
                                                        1.f / s->out_scale, out, total);
  SU(cudaGetLastError());
  return MLSW_OK;
}

int mlswlbm_surrogate_train_step(mlswlbm_surrogate* s, const float* h, const float* target,
                                 int batch, double lr, double* loss) {
  if (!s || !h || !target || batch < 1 || batch > s->max_batch || !(lr > 0.0)) return MLSW_ERR_ARG;
  const long cells = (long)s->nx * s->ny, npix = batch * cells;
  const int H = s->ny, W = s->nx;
  SU(forward(s, h, batch));
  double* dloss = s->sums + 2 * (size_t)s->max_batch * s->n;
  SU(cudaMemsetAsync(dloss, 0, sizeof(double), s->st));
  SU(cudaMemsetAsync(s->grad, 0, s->nparam * sizeof(float), s->st));
  loss_kernel<<<256, 256, 0, s->st>>>(s->y, h, target, s->n, cells, s->out_scale,
                                      1.f / (float)(npix * s->n), s->dy, dloss, npix);
  const unsigned g = blocks(npix / 16, 4);
  const dim3 gw(blocks(npix, kChunk), KD);
  // layer 2 (32 -> 16): weight and bias gradients, then the gradient of a2
  wgrad_kernel<C2, C3><<<gw, 32 * (C2 / 16) * (C3 / 8), 0, s->st>>>(s->act[2], s->dy,
                                                                     s->grad + s->woff[2], batch, H, W);
  bias_grad_kernel<C3><<<128, 256, 0, s->st>>>(s->dy, s->grad + s->boff[2], npix);
  conv_kernel<C3, C2, false, true, false><<<g, 128, 0, s->st>>>(s->dy, s->wb[2], nullptr,
                                                                 s->act[2], s->dact[2], batch, H, W);
  // layer 1 (32 -> 32)
  wgrad_kernel<C1, C2><<<gw, 32 * (C1 / 16) * (C2 / 8), 0, s->st>>>(s->act[1], s->dact[2],
                                                                     s->grad + s->woff[1], batch, H, W);
  bias_grad_kernel<C2><<<128, 256, 0, s->st>>>(s->dact[2], s->grad + s->boff[1], npix);
  conv_kernel<C2, C1, false, true, false><<<g, 128, 0, s->st>>>(s->dact[2], s->wb[1], nullptr,
                                                                 s->act[1], s->dact[1], batch, H, W);
  // layer 0 (16 -> 32): no input gradient needed
  wgrad_kernel<C0, C1><<<gw, 32 * (C0 / 16) * (C1 / 8), 0, s->st>>>(s->act[0], s->dact[1],
                                                                     s->grad + s->woff[0], batch, H, W);
  bias_grad_kernel<C1><<<128, 256, 0, s->st>>>(s->dact[1], s->grad + s->boff[0], npix);
  // Adam (beta 0.9, 0.999), then the BF16 copies
  s->step += 1;
  const float b1 = 0.9f, b2 = 0.999f;
  const float c1 = 1.f / (1.f - std::pow(b1, (float)s->step));
  const float c2 = 1.f / (1.f - std::pow(b2, (float)s->step));
  adam_kernel<<<blocks(s->nparam, 256), 256, 0, s->st>>>(s->param, s->grad, s->adam_m, s->adam_v,
                                                          s->nparam, (float)lr, b1, b2, c1, c2, 1e-8f);
  SU(cudaGetLastError());
  SU(refresh_copies(s));
  if (loss) {
    SU(cudaMemcpyAsync(loss, dloss, sizeof(double), cudaMemcpyDeviceToHost, s->st));
    SU(cudaStreamSynchronize(s->st));
  }
  return MLSW_OK;
}

int mlswlbm_surrogate_debug(mlswlbm_surrogate* s, int what, void* out, long bytes) {
  // copies internal buffers for the tests: 0 = y (FP32 [pixel][16]),
  // 1 = gradient of the parameters (FP32), 2 = x0 (BF16 [pixel][16]),
  // 3 = a1, 4 = a2 (BF16 [pixel][32]), 5 = dy (BF16), 6 = d a2, 7 = d a1
  if (!s || !out || bytes < 0) return MLSW_ERR_ARG;
  const void* src = nullptr;
  switch (what) {
    case 0: src = s->y; break;
    case 1: src = s->grad; break;
    case 2: src = s->act[0]; break;
    case 3: src = s->act[1]; break;
    case 4: src = s->act[2]; break;
    case 5: src = s->dy; break;
    case 6: src = s->dact[2]; break;
    case 7: src = s->dact[1]; break;
    default: return MLSW_ERR_ARG;
  }
  SU(cudaMemcpyAsync(out, src, bytes, cudaMemcpyDeviceToHost, s->st));
  SU(cudaStreamSynchronize(s->st));
  return MLSW_OK;
}

void mlswlbm_surrogate_destroy(mlswlbm_surrogate* s) {
  if (!s) return;
  if (s->st) cudaStreamSynchronize(s->st);
  cudaFree(s->param);
  cudaFree(s->grad);
  cudaFree(s->adam_m);
  cudaFree(s->adam_v);
  cudaFree(s->y);
  cudaFree(s->dy);
  cudaFree(s->sums);
  for (int l = 0; l < NCONV; ++l) {
    cudaFree(s->wf[l]);
    cudaFree(s->wb[l]);
    cudaFree(s->act[l]);
    cudaFree(s->dact[l]);
  }
  delete s;
}

}  // extern "C"
