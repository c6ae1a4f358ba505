// Tensor-core products of the batched node solves (see bgemm.cuh): the
// persistent split-K kernel on tcgen05 / TMEM / TMA, its planner, the BF16
// plane split of X, and the fused reductions around the two products.
#include <algorithm>
#include <cstdint>
#include <cstdio>

#include "bgemm.cuh"
#include "umma.cuh"
#include "xpass.cuh"

namespace relax {

namespace {

// One piece of a CTA's range: K blocks [kb0, kb1) of tile t, written to
// partial slot `slot` of the tile.
struct BGSeg {
  int t, kb0, kb1, slot;
};
__device__ __forceinline__ BGSeg bg_seg(const BGArgs& a, int64_t i, int64_t iend, int64_t T) {
  BGSeg g;
  g.t = (int)(i / a.nkb);
  const int64_t t0 = (int64_t)g.t * a.nkb;
  g.kb0 = (int)(i - t0);
  g.kb1 = (int)(min(iend, t0 + a.nkb) - t0);
  g.slot = (int)blockIdx.x - (int)bg_owner(t0, T, (int)gridDim.x);
  return g;
}

__host__ __device__ inline uint32_t bg_stage_bytes(int BN) {
  const uint32_t raw = (uint32_t)BG_PLANES * (BG_BM + BN) * BG_SW;
  return (raw + 1023u) / 1024u * 1024u;
}

// Persistent: CTA c takes its contiguous range of (tile, K block) iterations
// (bgemm.cuh), one piece per tile it meets.  The K blocks of a piece are
// taken BG_DRAIN at a time (a period): the MMAs of a period accumulate in one
// of BG_NBUF TMEM buffer pairs (main product, corrections), which the
// epilogue then adds into the piece's FP32 sums in registers while the MMAs
// fill the next pair.
//   warp 0 lane 0: TMA producer (A and B planes of one K block per stage)
//   warp 1:        TMEM allocation; lane 0 issues the MMAs and commits
//   warps 2..9:    epilogue; warp w reads TMEM lanes 32 (w mod 4) .. +31 and
//                  columns 64 ((w - 2) / 4) .. +63 of the tile
// Every wait is bounded; on expiry the kernel records ST_TIMEOUT, stops
// issuing, lets its copies and MMAs finish (bounded) and frees its TMEM.
__global__ void __launch_bounds__(BG_THREADS, 1) bgemm_kernel(const __grid_constant__ BGArgs a) {
  extern __shared__ __align__(1024) unsigned char bg_raw[];
  __shared__ __align__(8) uint64_t full[BG_MAXS], empty[BG_MAXS], tfull[BG_NBUF], tempty[BG_NBUF], drain;
  __shared__ uint32_t tmem_sh;
  __shared__ volatile int tmo;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  unsigned char* smem = bg_raw + ((1024u - (smem_u32(bg_raw) & 1023u)) & 1023u);
  const uint32_t a_plane = (uint32_t)BG_BM * BG_SW;   // one plane of an A tile
  const uint32_t b_plane = (uint32_t)a.BN * BG_SW;
  const uint32_t a_bytes = BG_PLANES * a_plane;
  const uint32_t b_bytes = BG_PLANES * b_plane;
  const uint32_t sstride = bg_stage_bytes(a.BN);
  const int S = a.stages;
  if (threadIdx.x == 0) {
    tmo = 0;
    for (int s = 0; s < S; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    for (int b = 0; b < BG_NBUF; ++b) {
      mbar_init(&tfull[b], 1);
      mbar_init(&tempty[b], 8);
    }
    mbar_init(&drain, 1);
    fence_mbar_init_cluster();
  }
  if (warp == 1) {
    tmem_alloc(&tmem_sh, 2 * BG_NBUF * BG_MAXN);
    tmem_relinquish();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = tmem_sh;
  const int64_t T = (int64_t)a.MT * a.NT * a.nkb;
  const int64_t ibeg = (int64_t)blockIdx.x * T / gridDim.x, iend = (int64_t)(blockIdx.x + 1) * T / gridDim.x;

  if (warp == 0) {
    if (lane == 0) {
      // ------------------------------------------------------ TMA producer
      int it = 0;
      for (int64_t i = ibeg; i < iend && !tmo;) {
        const BGSeg g = bg_seg(a, i, iend, T);
        i += g.kb1 - g.kb0;
        const int nt = g.t % a.NT, mt = g.t / a.NT;
        for (int kb = g.kb0; kb < g.kb1; ++kb) {
          const int s = it % S;
          if (it >= S && !mbar_wait<false>(&empty[s], ((it / S) - 1) & 1, a.limit_ns, a.status)) {
            tmo = 1;
            break;
          }
          if (tmo) break;
          unsigned char* dst = smem + (size_t)s * sstride;
          mbar_arrive_expect_tx(&full[s], a_bytes + b_bytes);
          tma_load_3d(dst, &a.tmA, kb * BG_BK, mt * BG_BM, 0, &full[s]);
          tma_load_3d(dst + a_bytes, &a.tmB, kb * BG_BK, nt * a.BN, 0, &full[s]);
          ++it;
        }
      }
      // the copies in flight land before the CTA may exit
      for (int k = max(0, it - S); k < it; ++k) mbar_wait<false>(&full[k % S], (k / S) & 1, a.limit_ns, a.status);
    }
  } else if (warp == 1) {
    if (lane == 0) {
      // ----------------------------------------------------------- MMA issue
      const uint32_t idesc = umma_idesc_bf16(BG_BM, a.BN);
      const uint32_t sbase = smem_u32(smem);
      int it = 0, gp = 0;   // K blocks and drain periods issued by this CTA
      for (int64_t i = ibeg; i < iend && !tmo;) {
        const BGSeg g = bg_seg(a, i, iend, T);
        i += g.kb1 - g.kb0;
        const int kb1 = g.kb1;
        for (int pb = g.kb0; pb < kb1 && !tmo; pb += BG_DRAIN, ++gp) {
          const int b = gp % BG_NBUF;
          if (gp >= BG_NBUF && !mbar_wait<false>(&tempty[b], ((gp / BG_NBUF) - 1) & 1, a.limit_ns, a.status)) {
            tmo = 1;
            break;
          }
          tc_fence_after();
          const uint32_t d = tmem + (uint32_t)(2 * b * BG_MAXN);   // main; corrections at + BG_MAXN
          const uint32_t e = d + BG_MAXN;
          uint32_t acc = 0;
          const int pe = min(kb1, pb + BG_DRAIN);
          for (int kb = pb; kb < pe; ++kb, ++it) {
            const int s = it % S;
            if (!mbar_wait<false>(&full[s], (it / S) & 1, a.limit_ns, a.status)) {
              tmo = 1;
              break;
            }
            tc_fence_after();
            const uint32_t sa = sbase + (uint32_t)s * sstride, sb = sa + a_bytes;
#pragma unroll
            for (int ks = 0; ks < BG_SW / 32; ++ks) {     // 16 BF16 = 32 bytes of K per MMA
              // (plane of A, plane of B) of the six products kept, of
              // significance 2^0, 2^-8 (twice), 2^-16 (three times; the
              // dropped ones are below 2^-23 relative), grouped by the plane
              // of A so that each A plane is read from shared memory once:
              // the main product in its own accumulator, the rest in the second
              const uint32_t oa = sa + ks * 32, ob = sb + ks * 32;
              const uint64_t a0 = sdesc_kmajor<BG_SW>(oa), a1 = sdesc_kmajor<BG_SW>(oa + a_plane),
                             a2 = sdesc_kmajor<BG_SW>(oa + 2 * a_plane);
              const uint64_t b0 = sdesc_kmajor<BG_SW>(ob), b1 = sdesc_kmajor<BG_SW>(ob + b_plane),
                             b2 = sdesc_kmajor<BG_SW>(ob + 2 * b_plane);
              umma_bf16_col<1>(d, a0, b0, idesc, acc & 1u);
              umma_bf16_col<2>(e, a0, b1, idesc, acc >> 1);
              umma_bf16_col<3>(e, a0, b2, idesc, 1u);
              umma_bf16_col<1>(e, a1, b0, idesc, 1u);
              umma_bf16_col<3>(e, a1, b1, idesc, 1u);
              umma_bf16_col<0>(e, a2, b0, idesc, 1u);
              acc = 3u;
            }
            umma_commit(&empty[s]);   // the stage is free once these MMAs have read it
          }
          if (tmo) break;
          umma_commit(&tfull[b]);     // the period's sum is complete
        }
      }
      // no MMA may be in flight when the TMEM is freed
      umma_commit(&drain);
      mbar_wait<false>(&drain, 0, a.limit_ns, a.status);
    }
    __syncwarp();
  } else {
    // ------------------------------------------------------------- epilogue
    const int q = warp & 3;                  // TMEM lane quarter of this warp
    const int c0 = ((warp - 2) >> 2) * 64;   // this warp's 64 columns of the tile
    int gp = 0;
    for (int64_t i = ibeg; i < iend && !tmo;) {
      const BGSeg g = bg_seg(a, i, iend, T);
      i += g.kb1 - g.kb0;
      const int nt = g.t % a.NT, mt = g.t / a.NT;
      const int kb0 = g.kb0, kb1 = g.kb1;
      const int ncols = min(a.BN, a.N - nt * a.BN);
      const int mine = min(64, ncols - c0);   // columns of this warp (<= 0: none)
      const uint32_t lane_base = tmem + ((uint32_t)(q * 32) << 16);
      float hi[64];
#pragma unroll
      for (int j = 0; j < 64; ++j) hi[j] = 0.f;
      bool ok = true;
      for (int pb = kb0; pb < kb1; pb += BG_DRAIN, ++gp) {
        const int b = gp % BG_NBUF;
        ok = __all_sync(0xffffffffu, mbar_wait<false>(&tfull[b], (gp / BG_NBUF) & 1, a.limit_ns, a.status));
        if (!ok) break;
        tc_fence_after();
        const uint32_t col = (uint32_t)(2 * b * BG_MAXN + c0);
#pragma unroll
        for (int h = 0; h < 4; ++h) {
          if (h * 16 < mine) {   // uniform across the warp
            uint32_t r[16], e[16];
            tmem_ld16(lane_base + col + h * 16, r);              // main product
            tmem_ld16(lane_base + col + BG_MAXN + h * 16, e);    // corrections
            tmem_ld_wait();
#pragma unroll
            for (int j = 0; j < 16; ++j)
              hi[h * 16 + j] += __uint_as_float(r[j]) + __uint_as_float(e[j]);
          }
        }
        tc_fence_before();
        __syncwarp();
        if (lane == 0) mbar_arrive(&tempty[b]);
      }
      if (!ok) {
        tmo = 1;
        break;
      }
      const int row = mt * BG_BM + q * 32 + lane;
      if (row < a.M) {
        double* dst = a.P + ((size_t)g.slot * a.N + (size_t)nt * a.BN + c0) * a.M + row;
#pragma unroll
        for (int j = 0; j < 64; ++j)
          if (j < mine) __stcg(dst + (size_t)j * a.M, (double)hi[j]);
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (warp == 1) tmem_dealloc(tmem, 2 * BG_NBUF * BG_MAXN);
}

// ------------------------------------------------------------ plane splits
__device__ __forceinline__ void split3(float x, __nv_bfloat16& b1, __nv_bfloat16& b2, __nv_bfloat16& b3) {
  b1 = __float2bfloat16_rn(x);
  const float r1 = x - __bfloat162float(b1);   // exact: the rounding error of a coarser format
  b2 = __float2bfloat16_rn(r1);
  const float r2 = r1 - __bfloat162float(b2);
  b3 = __float2bfloat16_rn(r2);                // r2 has at most 8 significant bits: exact
}
__device__ __forceinline__ void split3(double x, __nv_bfloat16& b1, __nv_bfloat16& b2, __nv_bfloat16& b3) {
  b1 = __double2bfloat16(x);
  const double r1 = x - (double)__bfloat162float(b1);
  b2 = __double2bfloat16(r1);
  const double r2 = r1 - (double)__bfloat162float(b2);
  b3 = __double2bfloat16(r2);
}

__global__ void split_x_kernel(const float* X, int64_t n, int64_t p, int64_t ldx, __nv_bfloat16* P, int64_t ld) {
  const int64_t plane = n * ld;
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < plane; t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = t / ld, j = t - i * ld;
    const float x = j < p ? X[i * ldx + j] : 0.0f;
    __nv_bfloat16 b1, b2, b3;
    split3(x, b1, b2, b3);
    P[t] = b1;
    P[plane + t] = b2;
    P[2 * plane + t] = b3;
  }
}

// transposed: planes [3][p][ld] with K = n along a row; 32 x 32 tiles through
// shared memory (coalesced reads of X's rows and writes of the planes' rows)
__global__ void split_xt_kernel(const float* X, int64_t n, int64_t p, int64_t ldx, __nv_bfloat16* P, int64_t ld) {
  __shared__ float tile[32][33];
  const int64_t plane = p * ld;
  const int64_t i0 = (int64_t)blockIdx.x * 32, j0 = (int64_t)blockIdx.y * 32;
  for (int r = threadIdx.y; r < 32; r += blockDim.y) {
    const int64_t i = i0 + r, j = j0 + threadIdx.x;
    tile[r][threadIdx.x] = (i < n && j < p) ? X[i * ldx + j] : 0.0f;
  }
  __syncthreads();
  for (int r = threadIdx.y; r < 32; r += blockDim.y) {
    const int64_t j = j0 + r, i = i0 + threadIdx.x;
    if (j < p && i < ld) {
      __nv_bfloat16 b1, b2, b3;
      split3(tile[threadIdx.x][r], b1, b2, b3);
      const int64_t t = j * ld + i;
      P[t] = b1;
      P[plane + t] = b2;
      P[2 * plane + t] = b3;
    }
  }
}

// ------------------------------------------------- batched-solve kernels
__global__ void pack_kernel(const BatchIo io) {
  const int s = blockIdx.y;
  if (s >= io.m) return;
  const double* b = io.st ? static_cast<const double*>(io.st[io.active[s]].ps.beta) : io.bsrc + (int64_t)s * io.p;
  const int64_t plane = (int64_t)io.nb * io.ldp;
  __nv_bfloat16* row = io.Bp + (int64_t)s * io.ldp;
  for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < io.p; j += (int64_t)gridDim.x * blockDim.x) {
    __nv_bfloat16 b1, b2, b3;
    split3(b[j], b1, b2, b3);
    row[j] = b1;
    row[plane + j] = b2;
    row[2 * plane + j] = b3;
  }
}

__global__ void reduce_link_kernel(const BatchIo io) {
  const int s = blockIdx.y;
  if (s >= io.m) return;
  double* zout = io.zdst + (int64_t)s * io.n;
  const double* zprev = nullptr;
  double mom = 0.0;
  if (io.st) {
    const IterState& S = io.st[io.active[s]];
    if (S.done) return;
    zout = static_cast<double*>(S.ps.zout);
    zprev = static_cast<const double*>(S.ps.zprev);
    mom = S.ps.mom;
  }
  const int64_t plane = (int64_t)io.NB * io.nb * io.ldn;
  const int64_t chunk = (int64_t)io.m * io.n;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < io.n; i += (int64_t)gridDim.x * blockDim.x) {
    const double* src = io.P1 + (int64_t)s * io.n + i;
    const int ns = bg_slots(io.s1, (int)(i / BG_BM) * io.s1.NT + s / io.s1.BN);
    double z = 0.0;
    for (int kc = 0; kc < ns; ++kc) z += __ldcg(src + kc * chunk);   // fixed order
    zout[i] = z;
    const double yd = io.y ? io.y[i] : 0.0;
    double r0, r1 = 0.0;
    if (io.loss < 0) {
      r0 = z;
    } else if (io.loss == 0) {
      r0 = 2.0 * (z - yd);
    } else {
      r0 = -yd / (1.0 + exp(yd * z));
      const double zy = (1.0 + mom) * z - mom * zprev[i];
      r1 = -yd / (1.0 + exp(yd * zy));
    }
    __nv_bfloat16 b1, b2, b3;
    split3(r0, b1, b2, b3);
    __nv_bfloat16* row = io.Rp + (int64_t)s * io.ldn + i;
    row[0] = b1;
    row[plane] = b2;
    row[2 * plane] = b3;
    if (io.NB > 1) {
      split3(r1, b1, b2, b3);
      row = io.Rp + (int64_t)(io.m + s) * io.ldn + i;
      row[0] = b1;
      row[plane] = b2;
      row[2 * plane] = b3;
    }
  }
}

__global__ void reduce_grad_kernel(const BatchIo io) {
  const int s = blockIdx.y;
  if (s >= io.m) return;
  if (io.st && io.st[io.active[s]].done) return;
  const int64_t chunk = (int64_t)io.NB * io.m * io.p;
  for (int q = 0; q < io.NB; ++q) {
    const double* src = io.P2 + ((int64_t)q * io.m + s) * io.p;
    double* dst = io.part + ((int64_t)s * io.NB + q) * io.p;
    const int nt = (q * io.m + s) / io.s2.BN;
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < io.p; j += (int64_t)gridDim.x * blockDim.x) {
      const int ns = bg_slots(io.s2, (int)(j / BG_BM) * io.s2.NT + nt);
      double g = 0.0;
      for (int kc = 0; kc < ns; ++kc) g += __ldcg(src + kc * chunk + j);
      dst[j] = g;
    }
  }
}

typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
EncodeTiledFn encode_fn() {
  static EncodeTiledFn fn = nullptr;
  if (!fn) {
    void* ptr = nullptr;
    cudaDriverEntryPointQueryResult q{};
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &ptr, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<EncodeTiledFn>(ptr);
  }
  return fn;
}

inline unsigned grid1(int64_t work, int block) {
  return (unsigned)std::max<int64_t>(1, std::min<int64_t>((work + block - 1) / block, 1024));
}

}  // namespace

cudaError_t bgemm_plan(BGPlan& pl, int M, int N, int K) {
  pl = BGPlan{};
  if (M < 1 || N < 1 || K < 1) return cudaErrorInvalidValue;
  int dev = 0, nsm = 0, optin = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  pl.M = M;
  pl.N = N;
  pl.K = K;
  pl.NT = (N + BG_MAXN - 1) / BG_MAXN;
  pl.BN = ((N + pl.NT - 1) / pl.NT + 15) / 16 * 16;   // balanced N-tiles, a multiple of 16
  pl.MT = (M + BG_BM - 1) / BG_BM;
  pl.nkb = (K + BG_BK - 1) / BG_BK;
  const int tiles = pl.MT * pl.NT;
  const int64_t T = (int64_t)tiles * pl.nkb;
  // one range per SM; fewer when a tile would be cut into more than BG_MAXKC pieces
  int G = (int)std::min<int64_t>({(int64_t)std::max(nsm, 1), T, (int64_t)(BG_MAXKC - 1) * tiles});
  for (;; --G) {
    pl.grid = G;
    const BGSplit sp = pl.split();
    int kc = 1;
    for (int t = 0; t < tiles; ++t) kc = std::max(kc, bg_slots(sp, t));
    pl.KC = kc;
    if (kc <= BG_MAXKC || G == 1) break;
  }
  const uint32_t sb = bg_stage_bytes(pl.BN);
  const int fixed = 1024 + 512;   // alignment slack, static shared memory
  pl.stages = std::min(BG_MAXS, (optin - fixed) / (int)sb);
  if (pl.stages < 2) return cudaErrorNotSupported;
  pl.smem = (size_t)pl.stages * sb + 1024;
  cudaFuncAttributes fa{};
  cudaError_t e = cudaFuncGetAttributes(&fa, reinterpret_cast<const void*>(&bgemm_kernel));
  if (e != cudaSuccess) return e;
  if (fa.maxDynamicSharedSizeBytes < (int)pl.smem) {
    e = cudaFuncSetAttribute(reinterpret_cast<const void*>(&bgemm_kernel),
                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)pl.smem);
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

cudaError_t bgemm_encode(CUtensorMap* tm, const void* planes, int64_t K, int64_t rows, int64_t ld, int64_t plane_rows,
                         int box_rows) {
  if ((reinterpret_cast<uintptr_t>(planes) & 15u) != 0 || ld % 8 != 0 || ld < K || rows > plane_rows || box_rows < 1 ||
      box_rows > 256)
    return cudaErrorInvalidValue;
  EncodeTiledFn enc = encode_fn();
  if (!enc) return cudaErrorNotSupported;
  const cuuint64_t dims[3] = {(cuuint64_t)K, (cuuint64_t)rows, (cuuint64_t)BG_PLANES};
  const cuuint64_t strides[2] = {(cuuint64_t)ld * 2, (cuuint64_t)plane_rows * ld * 2};
  const cuuint32_t box[3] = {(cuuint32_t)BG_BK, (cuuint32_t)box_rows, (cuuint32_t)BG_PLANES};
  const cuuint32_t estr[3] = {1, 1, 1};
  const CUresult r = enc(tm, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, const_cast<void*>(planes), dims, strides, box, estr,
                         CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_64B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                         CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

cudaError_t bgemm_launch(const BGPlan& pl, const BGArgs& a, cudaStream_t st) {
  if (a.BN != pl.BN || a.stages != pl.stages || a.NT != pl.NT || a.MT != pl.MT || a.nkb != pl.nkb ||
      pl.KC > BG_MAXKC || pl.grid < 1)
    return cudaErrorInvalidValue;
  bgemm_kernel<<<pl.grid, BG_THREADS, pl.smem, st>>>(a);
  return cudaGetLastError();
}

cudaError_t bgemm_split_x(const float* X, int64_t n, int64_t p, int64_t ldx, bool transpose, __nv_bfloat16* planes,
                          int64_t ld, cudaStream_t st) {
  if (!transpose) {
    if (ld < p) return cudaErrorInvalidValue;
    split_x_kernel<<<4096, 256, 0, st>>>(X, n, p, ldx, planes, ld);
  } else {
    if (ld < n) return cudaErrorInvalidValue;
    // blocks over (i, j) tiles; every plane row j < p gets ld columns (zeros past n)
    dim3 grid((unsigned)((ld + 31) / 32), (unsigned)((p + 31) / 32));
    split_xt_kernel<<<grid, dim3(32, 8), 0, st>>>(X, n, p, ldx, planes, ld);
  }
  return cudaGetLastError();
}

cudaError_t batch_pack(const BatchIo& io, cudaStream_t st) {
  dim3 grid(grid1(io.p, 256) > 64 ? 64 : grid1(io.p, 256), (unsigned)io.m);
  pack_kernel<<<grid, 256, 0, st>>>(io);
  return cudaGetLastError();
}

cudaError_t batch_reduce_link(const BatchIo& io, cudaStream_t st) {
  dim3 grid(grid1(io.n, 256) > 64 ? 64 : grid1(io.n, 256), (unsigned)io.m);
  reduce_link_kernel<<<grid, 256, 0, st>>>(io);
  return cudaGetLastError();
}

cudaError_t batch_reduce_grad(const BatchIo& io, cudaStream_t st) {
  dim3 grid(grid1(io.p, 256) > 64 ? 64 : grid1(io.p, 256), (unsigned)io.m);
  reduce_grad_kernel<<<grid, 256, 0, st>>>(io);
  return cudaGetLastError();
}

}  // namespace relax
