// Per-coordinate warm-start network: 5 -> 64 -> 64 -> 1, ReLU after both
// hidden layers, inputs standardised as (x - shift) / scale; the child's
// starting point is beta^P_j + f(x_j) (the parent warm start of Sec. 5.3 plus a
// learned correction).  Weights live in one FP32 vector (layout in
// include/warmstart.h); with bf16 != 0 every kernel evaluates the network
// with the trainable entries rounded to BF16, accumulating in FP32.
//
// forward: BF16 weights: the 64 x 64 layer on the tensor cores (mma.sync
//          m16n8k16, BF16 operands, FP32 accumulation), 16 rows per warp:
//          each lane computes layer 1 for the A-fragment entries it holds and
//          splits them into three BF16 planes (exactly the FP32 value), so the
//          products are exact and only the FP32 sums round; layer 2's bias,
//          ReLU and the output layer follow on the accumulator fragments.
//          FP32 weights (the reference build of the network): one thread per
//          row on the CUDA cores, layer 2 fused with the output layer.
// grad:    tiles of 128 rows per CTA; per row the forward and the backward
//          sweep run in registers and leave h1, h2, dL/da2, dL/da1 in shared
//          memory; the CTA then folds the tile into its weight-gradient
//          accumulators (registers), and writes one partial per CTA.  A second
//          kernel sums the partials in CTA order, so the gradient is
//          bit-reproducible for a given row count.
// adam:    one thread per trainable entry (Kingma and Ba, 2015).
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>

#include "warmstart.h"

namespace {

constexpr int NIN = 5, NH = 64;
constexpr int O_W1 = 0, O_B1 = NH * NIN, O_W2 = O_B1 + NH, O_B2 = O_W2 + NH * NH, O_W3 = O_B2 + NH,
              O_B3 = O_W3 + NH, O_SHIFT = O_B3 + 1, O_SCALE = O_SHIFT + NIN;
static_assert(O_SHIFT == RELAX_MLP_NTRAIN, "layout");
static_assert(O_SCALE + NIN == RELAX_MLP_NPARAM, "layout");

constexpr int FWD_THREADS = 128;
constexpr int TILE = 128;       // rows per tile of the gradient kernel (= its threads)
constexpr int HS = NH + 1;      // padded row stride of the shared activation tiles

__device__ __forceinline__ float wround(float w, int bf16) {
  return bf16 ? __bfloat162float(__float2bfloat16_rn(w)) : w;
}

// the network's parameters in shared memory, FP32 (BF16-rounded when asked)
struct SW {
  float W1[NH * NIN], b1[NH], W2[NH * NH], b2[NH], w3[NH], b3, shift[NIN], iscale[NIN];
};

__device__ void load_weights(SW& s, const float* theta, int bf16) {
  for (int i = threadIdx.x; i < NH * NIN; i += blockDim.x) s.W1[i] = wround(theta[O_W1 + i], bf16);
  for (int i = threadIdx.x; i < NH * NH; i += blockDim.x) s.W2[i] = wround(theta[O_W2 + i], bf16);
  for (int i = threadIdx.x; i < NH; i += blockDim.x) {
    s.b1[i] = wround(theta[O_B1 + i], bf16);
    s.b2[i] = wround(theta[O_B2 + i], bf16);
    s.w3[i] = wround(theta[O_W3 + i], bf16);
  }
  if (threadIdx.x < NIN) {
    s.shift[threadIdx.x] = theta[O_SHIFT + threadIdx.x];
    s.iscale[threadIdx.x] = 1.0f / theta[O_SCALE + threadIdx.x];
  }
  if (threadIdx.x == 0) s.b3 = wround(theta[O_B3], bf16);
}

// layer 1 of one row: h1 = relu(W1 xs + b1)
__device__ __forceinline__ void layer1(const SW& s, const float* xs, float* h1) {
#pragma unroll
  for (int h = 0; h < NH; ++h) {
    float a = s.b1[h];
#pragma unroll
    for (int i = 0; i < NIN; ++i) a = fmaf(s.W1[h * NIN + i], xs[i], a);
    h1[h] = a > 0.f ? a : 0.f;
  }
}

__device__ __forceinline__ float dot64(const float* w, const float* h) {
  float a0 = 0.f, a1 = 0.f, a2 = 0.f, a3 = 0.f;
#pragma unroll
  for (int k = 0; k < NH; k += 4) {
    a0 = fmaf(w[k], h[k], a0);
    a1 = fmaf(w[k + 1], h[k + 1], a1);
    a2 = fmaf(w[k + 2], h[k + 2], a2);
    a3 = fmaf(w[k + 3], h[k + 3], a3);
  }
  return (a0 + a1) + (a2 + a3);
}

// ---- tensor-core forward (BF16 weights)
__device__ __forceinline__ uint32_t pack_bf16(__nv_bfloat16 lo, __nv_bfloat16 hi) {
  return (uint32_t)__bfloat16_as_ushort(lo) | ((uint32_t)__bfloat16_as_ushort(hi) << 16);
}
// x = p0 + p1 + p2 exactly (8 + 8 + 8 significand bits of an FP32 value)
__device__ __forceinline__ void split3_f32(float x, __nv_bfloat16 (&q)[3]) {
  q[0] = __float2bfloat16_rn(x);
  const float r1 = x - __bfloat162float(q[0]);
  q[1] = __float2bfloat16_rn(r1);
  q[2] = __float2bfloat16_rn(r1 - __bfloat162float(q[1]));
}
__device__ __forceinline__ void mma_bf16_16816(float (&d)[4], const uint32_t (&a)[4], uint32_t b0, uint32_t b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0, %1, %2, %3}, {%4, %5, %6, %7}, {%8, %9}, "
      "{%0, %1, %2, %3};"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

constexpr int MMA_WARPS = 4;
constexpr int W2LD = NH + 8;   // padded row of W2 in shared memory: the 8 row groups hit distinct banks

__global__ void __launch_bounds__(32 * MMA_WARPS) mlp_forward_mma_kernel(const float* theta, const float* feat,
                                                                        const float* base, int64_t rows, float* out) {
  __shared__ SW s;
  __shared__ __align__(16) __nv_bfloat16 W2b[NH * W2LD];   // W2 [o][h], exact in BF16
  load_weights(s, theta, 1);
  for (int i = threadIdx.x; i < NH * NH; i += blockDim.x) W2b[(i / NH) * W2LD + i % NH] = __float2bfloat16_rn(s.W2[i]);
  __syncthreads();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int g = lane >> 2, t4 = lane & 3;   // fragment row group, column pair
  const int64_t ntiles = (rows + 15) / 16;
  for (int64_t tile = (int64_t)blockIdx.x * MMA_WARPS + warp; tile < ntiles; tile += (int64_t)gridDim.x * MMA_WARPS) {
    const int64_t r0 = tile * 16 + g, r1 = r0 + 8;
    float x0[NIN], x1[NIN];
#pragma unroll
    for (int i = 0; i < NIN; ++i) {
      x0[i] = r0 < rows ? (feat[r0 * NIN + i] - s.shift[i]) * s.iscale[i] : 0.f;
      x1[i] = r1 < rows ? (feat[r1 * NIN + i] - s.shift[i]) * s.iscale[i] : 0.f;
    }
    // A fragments of layer 2's input h1 (rows r0, r1 x 64 hidden units), three planes
    uint32_t A[3][4][4];
#pragma unroll
    for (int kc = 0; kc < 4; ++kc) {
#pragma unroll
      for (int hh = 0; hh < 2; ++hh) {            // columns 2 t4 (+1) and 2 t4 + 8 (+1)
        __nv_bfloat16 q00[3], q01[3], q10[3], q11[3];
        const int h = kc * 16 + 2 * t4 + 8 * hh;
        float a00 = s.b1[h], a01 = s.b1[h + 1], a10 = s.b1[h], a11 = s.b1[h + 1];
#pragma unroll
        for (int i = 0; i < NIN; ++i) {
          a00 = fmaf(s.W1[h * NIN + i], x0[i], a00);
          a01 = fmaf(s.W1[(h + 1) * NIN + i], x0[i], a01);
          a10 = fmaf(s.W1[h * NIN + i], x1[i], a10);
          a11 = fmaf(s.W1[(h + 1) * NIN + i], x1[i], a11);
        }
        split3_f32(a00 > 0.f ? a00 : 0.f, q00);
        split3_f32(a01 > 0.f ? a01 : 0.f, q01);
        split3_f32(a10 > 0.f ? a10 : 0.f, q10);
        split3_f32(a11 > 0.f ? a11 : 0.f, q11);
#pragma unroll
        for (int pl = 0; pl < 3; ++pl) {
          A[pl][kc][2 * hh] = pack_bf16(q00[pl], q01[pl]);       // row g
          A[pl][kc][2 * hh + 1] = pack_bf16(q10[pl], q11[pl]);   // row g + 8
        }
      }
    }
    float y0 = 0.f, y1 = 0.f;
#pragma unroll
    for (int nt = 0; nt < NH / 8; ++nt) {
      float d[4] = {0.f, 0.f, 0.f, 0.f};
      const __nv_bfloat16* wrow = W2b + (nt * 8 + g) * W2LD;   // output unit nt*8+g, k contiguous
#pragma unroll
      for (int kc = 0; kc < 4; ++kc) {
        const uint32_t b0 = *reinterpret_cast<const uint32_t*>(wrow + kc * 16 + 2 * t4);
        const uint32_t b1 = *reinterpret_cast<const uint32_t*>(wrow + kc * 16 + 2 * t4 + 8);
#pragma unroll
        for (int pl = 2; pl >= 0; --pl) mma_bf16_16816(d, A[pl][kc], b0, b1);   // small planes first
      }
      // d: (row g, cols o, o+1), (row g + 8, cols o, o+1), o = nt*8 + 2 t4
      const int o = nt * 8 + 2 * t4;
      const float h00 = d[0] + s.b2[o], h01 = d[1] + s.b2[o + 1];
      const float h10 = d[2] + s.b2[o], h11 = d[3] + s.b2[o + 1];
      if (h00 > 0.f) y0 = fmaf(s.w3[o], h00, y0);
      if (h01 > 0.f) y0 = fmaf(s.w3[o + 1], h01, y0);
      if (h10 > 0.f) y1 = fmaf(s.w3[o], h10, y1);
      if (h11 > 0.f) y1 = fmaf(s.w3[o + 1], h11, y1);
    }
    // the four lanes of a row group hold disjoint output units: sum them
    y0 += __shfl_xor_sync(0xffffffffu, y0, 1);
    y0 += __shfl_xor_sync(0xffffffffu, y0, 2);
    y1 += __shfl_xor_sync(0xffffffffu, y1, 1);
    y1 += __shfl_xor_sync(0xffffffffu, y1, 2);
    if (t4 == 0) {
      if (r0 < rows) {
        const float y = s.b3 + y0;
        out[r0] = base ? (feat[r0 * NIN + 2] < -0.5f ? 0.f : base[r0] + y) : y;
      }
      if (r1 < rows) {
        const float y = s.b3 + y1;
        out[r1] = base ? (feat[r1 * NIN + 2] < -0.5f ? 0.f : base[r1] + y) : y;
      }
    }
  }
}

__global__ void __launch_bounds__(FWD_THREADS) mlp_forward_kernel(const float* theta, int bf16, const float* feat,
                                                                 const float* base, int64_t rows, float* out) {
  __shared__ SW s;
  load_weights(s, theta, bf16);
  __syncthreads();
  // one row per thread (no row loop: the compiler would hoist the weights out
  // of it into registers)
  const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (r < rows) {
    float xs[NIN], h1[NH];
#pragma unroll
    for (int i = 0; i < NIN; ++i) xs[i] = (feat[r * NIN + i] - s.shift[i]) * s.iscale[i];
    layer1(s, xs, h1);
    float y = s.b3;
#pragma unroll 1
    for (int o = 0; o < NH; ++o) {
      const float a = s.b2[o] + dot64(&s.W2[o * NH], h1);
      if (a > 0.f) y = fmaf(s.w3[o], a, y);
    }
    // a start: zero on the child's J0 (fix feature -1), base + f elsewhere
    out[r] = base ? (feat[r * NIN + 2] < -0.5f ? 0.f : base[r] + y) : y;
  }
}

// per-CTA partial gradient: part[blockIdx.x][0 .. NTRAIN) and the partial sum
// of squared residuals at part[blockIdx.x][NTRAIN]
__global__ void __launch_bounds__(TILE) mlp_grad_kernel(const float* theta, int bf16, const float* feat,
                                                       const float* base, const float* target, int64_t rows,
                                                       float* part) {
  extern __shared__ __align__(16) float dyn[];
  __shared__ SW s;
  float* H1 = dyn;                 // [TILE][HS] h1
  float* H2 = H1 + TILE * HS;      // [TILE][HS] h2
  float* DA2 = H2 + TILE * HS;     // [TILE][HS] dL/da2
  float* DA1 = DA2 + TILE * HS;    // [TILE][HS] dL/da1
  float* XS = DA1 + TILE * HS;     // [TILE][NIN] standardised inputs
  float* D = XS + TILE * NIN;      // [TILE] dL/dout
  load_weights(s, theta, bf16);
  __syncthreads();
  const int t = threadIdx.x;
  const float inv_n = 1.0f / (float)rows;
  // accumulators: W2 entries (o = t / 64 + 2 k, h = t % 64), 32 per thread;
  // W1 entries t, t + 128, t + 256 (< 320); b2 / w3 (t < 64) or b1 (t >= 64)
  float gW2[32], gW1[3] = {0.f, 0.f, 0.f}, gA = 0.f, gB = 0.f, gb3 = 0.f;
  double sq = 0.0;
#pragma unroll
  for (int k = 0; k < 32; ++k) gW2[k] = 0.f;
  const int64_t ntiles = (rows + TILE - 1) / TILE;
  for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    const int64_t r = tile * TILE + t;
    const bool live = r < rows;
    // ---- forward of this thread's row
    float xs[NIN], h1[NH];
#pragma unroll
    for (int i = 0; i < NIN; ++i) {
      xs[i] = live ? (feat[r * NIN + i] - s.shift[i]) * s.iscale[i] : 0.f;
      XS[t * NIN + i] = xs[i];
    }
    layer1(s, xs, h1);
#pragma unroll
    for (int h = 0; h < NH; ++h) H1[t * HS + h] = h1[h];
    float y = s.b3;
    for (int o = 0; o < NH; ++o) {
      const float a = s.b2[o] + dot64(&s.W2[o * NH], h1);
      const float h2 = a > 0.f ? a : 0.f;
      H2[t * HS + o] = h2;
      y = fmaf(s.w3[o], h2, y);
    }
    float d_out = 0.f;
    if (live) {
      const float res = base[r] + y - target[r];
      sq += (double)res * (double)res;
      d_out = 2.0f * res * inv_n;
    }
    D[t] = d_out;
    // ---- backward of the row: dL/da2, then dL/dh1 = W2' dL/da2, dL/da1
    float dh1[NH];
#pragma unroll
    for (int h = 0; h < NH; ++h) dh1[h] = 0.f;
    for (int o = 0; o < NH; ++o) {
      const float da2 = H2[t * HS + o] > 0.f ? d_out * s.w3[o] : 0.f;
      DA2[t * HS + o] = da2;
#pragma unroll
      for (int h = 0; h < NH; ++h) dh1[h] = fmaf(s.W2[o * NH + h], da2, dh1[h]);
    }
#pragma unroll
    for (int h = 0; h < NH; ++h) DA1[t * HS + h] = h1[h] > 0.f ? dh1[h] : 0.f;
    __syncthreads();
    // ---- fold the tile into the weight gradients (fixed row order)
    {
      const int h = t & (NH - 1), o0 = t >> 6;
      for (int rr = 0; rr < TILE; ++rr) {
        const float hv = H1[rr * HS + h];
#pragma unroll
        for (int k = 0; k < 32; ++k) gW2[k] = fmaf(DA2[rr * HS + o0 + 2 * k], hv, gW2[k]);
      }
#pragma unroll
      for (int k = 0; k < 3; ++k) {
        const int e = t + TILE * k;
        if (e < NH * NIN) {
          const int hh = e / NIN, i = e % NIN;
          float acc = 0.f;
          for (int rr = 0; rr < TILE; ++rr) acc = fmaf(DA1[rr * HS + hh], XS[rr * NIN + i], acc);
          gW1[k] += acc;
        }
      }
      if (t < NH) {
        float a = 0.f, b = 0.f;
        for (int rr = 0; rr < TILE; ++rr) {
          a += DA2[rr * HS + t];
          b = fmaf(D[rr], H2[rr * HS + t], b);
        }
        gA += a;      // b2[t]
        gB += b;      // w3[t]
      } else {
        float a = 0.f;
        for (int rr = 0; rr < TILE; ++rr) a += DA1[rr * HS + (t - NH)];
        gA += a;      // b1[t - 64]
      }
      if (t == 0) {
        float a = 0.f;
        for (int rr = 0; rr < TILE; ++rr) a += D[rr];
        gb3 += a;
      }
    }
    __syncthreads();
  }
  float* P = part + (size_t)blockIdx.x * (RELAX_MLP_NTRAIN + 1);
  {
    const int h = t & (NH - 1), o0 = t >> 6;
#pragma unroll
    for (int k = 0; k < 32; ++k) P[O_W2 + (o0 + 2 * k) * NH + h] = gW2[k];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      const int e = t + TILE * k;
      if (e < NH * NIN) P[O_W1 + e] = gW1[k];
    }
    if (t < NH) {
      P[O_B2 + t] = gA;
      P[O_W3 + t] = gB;
    } else {
      P[O_B1 + (t - NH)] = gA;
    }
    if (t == 0) P[O_B3] = gb3;
  }
  // the CTA's sum of squared residuals, reduced in thread order
  __shared__ double sqs[TILE];
  sqs[t] = sq;
  __syncthreads();
  if (t == 0) {
    double a = 0.0;
    for (int i = 0; i < TILE; ++i) a += sqs[i];
    P[RELAX_MLP_NTRAIN] = (float)(a / (double)rows);
  }
}

// grad[i] = sum over CTAs (in order) of part[c][i]; loss = sum of the partial means
__global__ void mlp_reduce_kernel(const float* part, int nparts, float* grad, float* loss) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i <= RELAX_MLP_NTRAIN; i += gridDim.x * blockDim.x) {
    float a = 0.f;
    for (int c = 0; c < nparts; ++c) a += part[(size_t)c * (RELAX_MLP_NTRAIN + 1) + i];
    if (i < RELAX_MLP_NTRAIN) grad[i] = a;
    else if (loss) *loss = a;
  }
  for (int i = RELAX_MLP_NTRAIN + blockIdx.x * blockDim.x + threadIdx.x; i < RELAX_MLP_NPARAM;
       i += gridDim.x * blockDim.x)
    grad[i] = 0.f;   // shift and scale are not trained
}

// b1, b2 and their complements come separately: 1 - b in FP32 from an FP32 b
// near 1 would carry b's rounding error magnified (0.999f: 1.3e-5 relative)
__global__ void mlp_adam_kernel(float* theta, const float* grad, float* m, float* v, float lr, float b1, float omb1,
                                float b2, float omb2, float eps, float c1, float c2) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= RELAX_MLP_NTRAIN) return;
  const float g = grad[i];
  const float mi = b1 * m[i] + omb1 * g;
  const float vi = b2 * v[i] + omb2 * g * g;
  m[i] = mi;
  v[i] = vi;
  theta[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
}

int sm_count() {
  int dev = 0, n = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
  return n > 0 ? n : 1;
}

constexpr size_t grad_smem() { return (size_t)(4 * TILE * HS + TILE * NIN + TILE) * sizeof(float); }

relax_status cuda_status(cudaError_t e) {
  if (e == cudaSuccess) return RELAX_OK;
  return e == cudaErrorMemoryAllocation ? RELAX_ENOMEM : RELAX_ECUDA;
}

}  // namespace

extern "C" {

relax_status relax_mlp_forward(const float* theta, int32_t bf16, const float* feat, const float* base, int64_t rows,
                               float* out, void* stream) {
  if (!theta || !feat || !out || rows < 0) return RELAX_EINVAL;
  if (rows == 0) return RELAX_OK;
  if (bf16) {   // BF16 weights: the tensor-core forward, grid-stride over 16-row tiles
    const int64_t tiles = (rows + 15) / 16;
    const int64_t want = (tiles + MMA_WARPS - 1) / MMA_WARPS;
    const unsigned grid = (unsigned)(want < 8 * sm_count() ? want : 8 * sm_count());
    mlp_forward_mma_kernel<<<grid, 32 * MMA_WARPS, 0, (cudaStream_t)stream>>>(theta, feat, base, rows, out);
    return cuda_status(cudaGetLastError());
  }
  const int64_t grid = (rows + FWD_THREADS - 1) / FWD_THREADS;
  if (grid > INT32_MAX) return RELAX_ENOTSUP;
  mlp_forward_kernel<<<(unsigned)grid, FWD_THREADS, 0, (cudaStream_t)stream>>>(theta, 0, feat, base, rows, out);
  return cuda_status(cudaGetLastError());
}

relax_status relax_mlp_grad(const float* theta, int32_t bf16, const float* feat, const float* base,
                            const float* target, int64_t rows, float* grad, float* loss, void* stream) {
  if (!theta || !feat || !base || !target || !grad || rows <= 0) return RELAX_EINVAL;
  cudaStream_t st = (cudaStream_t)stream;
  // per device (the current one): cheap, so set on every call
  cudaError_t e = cudaFuncSetAttribute(mlp_grad_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)grad_smem());
  if (e != cudaSuccess) return cuda_status(e);
  const int64_t ntiles = (rows + TILE - 1) / TILE;
  const int nparts = (int)(ntiles < sm_count() ? ntiles : sm_count());
  float* part = nullptr;
  e = cudaMallocAsync((void**)&part, (size_t)nparts * (RELAX_MLP_NTRAIN + 1) * sizeof(float), st);
  if (e != cudaSuccess) return cuda_status(e);
  mlp_grad_kernel<<<nparts, TILE, grad_smem(), st>>>(theta, bf16 ? 1 : 0, feat, base, target, rows, part);
  e = cudaGetLastError();
  if (e == cudaSuccess) {
    mlp_reduce_kernel<<<(RELAX_MLP_NPARAM + 255) / 256, 256, 0, st>>>(part, nparts, grad, loss);
    e = cudaGetLastError();
  }
  cudaFreeAsync(part, st);
  return cuda_status(e);
}

relax_status relax_mlp_adam(float* theta, const float* grad, float* m, float* v, int32_t t, double lr, double beta1,
                            double beta2, double eps, void* stream) {
  if (!theta || !grad || !m || !v || t < 1 || !(lr >= 0.0) || !(beta1 >= 0.0 && beta1 < 1.0) ||
      !(beta2 >= 0.0 && beta2 < 1.0) || !(eps >= 0.0))
    return RELAX_EINVAL;
  const double c1 = 1.0 - std::pow(beta1, (double)t), c2 = 1.0 - std::pow(beta2, (double)t);
  mlp_adam_kernel<<<(RELAX_MLP_NTRAIN + 255) / 256, 256, 0, (cudaStream_t)stream>>>(
      theta, grad, m, v, (float)lr, (float)beta1, (float)(1.0 - beta1), (float)beta2, (float)(1.0 - beta2), (float)eps,
      (float)c1, (float)c2);
  return cuda_status(cudaGetLastError());
}

}  // extern "C"
