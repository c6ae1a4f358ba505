// Fused pass over X by L2 row blocking: z = X beta, r = link(z), g = X' r,
// with X read from HBM once per pass.
//
// This is the matrix-vector work that dominates the method (Sec. 5.2.3); the
// induced dual point zeta = -grad F(X beta) (Sec. 3.3) comes out of it as -r.
//
// Schedule (persistent grid, one CTA per SM, co-resident):
//  * X is cut into row blocks of B rows (a block is a few tens of MB, so the
//    last few blocks stay resident in the 126 MB L2).
//  * Phase A warps (12 per CTA) stream X from HBM: a work item is one row x
//    one column chunk; the warp forms the chunk's partial dot product with
//    beta (held in shared memory) as a compensated FP32 pair and stores it.
//    The warp that completes a row's last chunk (per-row counter) sums the
//    row's partials in chunk order, applies the link (r = grad F(z), or the
//    certification terms) and counts the row in done[block].
//  * Phase B warps (4 per CTA) own a fixed column strip of the CTA.  For each
//    block whose rows are all done they accumulate X' r over the strip,
//    re-reading the block from L2.  Each CTA writes its own columns of X' r:
//    no cross-CTA reduction.
//  * Phase A may run at most `lag` blocks ahead of the slowest CTA's phase B
//    (bdone counters), which bounds the L2 footprint.
// Every wait is bounded (the kernel records ST_TIMEOUT and carries on without
// waiting); counters are zeroed before each launch.
#pragma once
#include <cuda_bf16.h>
#include <cuda_fp8.h>

#include "xpass.cuh"

namespace relax {

constexpr int XB_WA = 12;                       // phase A warps per CTA
constexpr int XB_WB = 4;                        // phase B warps per CTA
constexpr int XB_THREADS = (XB_WA + XB_WB) * 32;
// Phase A keeps XB_U vectors in flight per lane and phase B covers XB_TV
// vectors of the strip per lane; both scale with the vector width so that a
// lane holds the same number of elements (32 / 16) for every storage type.
template <int VEC> struct XBShape {
  static constexpr int U = VEC >= 16 ? 2 : (VEC >= 8 ? 4 : 8);
  static constexpr int TV = VEC >= 16 ? 1 : (VEC >= 8 ? 2 : 4);
};

struct XBArgs {
  const void* X;
  int64_t ldx, n, p;
  int64_t cw;            // columns per phase-A chunk (multiple of the vector width)
  int nchunk;            // chunks per row
  int B;                 // rows per block
  int nblk;              // blocks
  int lag;               // phase A lead over phase B, in blocks
  int64_t sw;            // columns per CTA strip (multiple of the vector width)
  int beta_smem;         // 1: beta staged in shared memory
  int link;
  const double* y;
  const float* colscale;
  PassState* ps;
  double* part;          // [n][nchunk][NF] row-chunk partials (FP32 pair bits or FP64)
  double* r;             // [NB][n] link values of the rows
  double* g;             // [NB][p] X' r
  double* lterm;         // [n][2] per-row {F, -F*(-zeta)} (certification links) or NULL
  unsigned* done;        // [nblk] rows of the block finished   } one zeroed
  unsigned* bdone;       // [nblk] CTAs that finished the block  } contiguous
  unsigned* rowcnt;      // [n] chunks of the row finished       } allocation
  int* status;
  uint64_t limit_ns;
};

__device__ __forceinline__ unsigned ld_acquire_u32(const unsigned* p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

// bounded wait until *ctr >= target; false (and ST_TIMEOUT) after limit_ns
__device__ __forceinline__ bool wait_count(const unsigned* ctr, unsigned target, uint64_t limit_ns, int* status) {
  if (ld_acquire_u32(ctr) >= target) return true;
  const uint64_t t0 = globaltimer_ns();
  for (uint32_t it = 1;; ++it) {
    if (ld_acquire_u32(ctr) >= target) return true;
    if ((it & 15u) == 0u) {
      if (globaltimer_ns() - t0 > limit_ns) {
        atomicCAS(status, ST_OK, ST_TIMEOUT);
        return false;
      }
      __nanosleep(32);
    }
  }
}

// VEC consecutive TA values from shared memory in 16-byte pieces
template <typename TA, int VEC>
__device__ __forceinline__ void load_smem_vec(const TA* p, TA* o) {
  constexpr int PER = 16 / sizeof(TA);
#pragma unroll
  for (int k = 0; k < (VEC * (int)sizeof(TA) + 15) / 16; ++k) {
    if constexpr (sizeof(TA) == 4) {
      const float4 v = *reinterpret_cast<const float4*>(p + k * PER);
      if (k * PER + 0 < VEC) o[k * PER + 0] = v.x;
      if (k * PER + 1 < VEC) o[k * PER + 1] = v.y;
      if (k * PER + 2 < VEC) o[k * PER + 2] = v.z;
      if (k * PER + 3 < VEC) o[k * PER + 3] = v.w;
    } else {
      const double2 v = *reinterpret_cast<const double2*>(p + k * PER);
      if (k * PER + 0 < VEC) o[k * PER + 0] = v.x;
      if (k * PER + 1 < VEC) o[k * PER + 1] = v.y;
    }
  }
}

template <typename TX, typename TA, int NF, int NB>
__global__ void __launch_bounds__(XB_THREADS, 1) xblock_kernel(const XBArgs a) {
  constexpr int VEC = XTraits<TX>::VEC;
  constexpr int XB_U = XBShape<VEC>::U;
  constexpr bool kF32 = sizeof(TA) == 4;
  extern __shared__ __align__(16) unsigned char smem[];
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  __shared__ volatile int tmo;   // a bounded wait expired: no more waiting, same control flow
  __shared__ int skip;
  if (tid == 0) { tmo = 0; skip = a.ps->done; }
  __syncthreads();
  if (skip) return;   // uniform (same flag everywhere)

  const PassState* ps = a.ps;
  const int64_t p = a.p, n = a.n;
  const TX* X = static_cast<const TX*>(a.X);
  // shared: [beta (NF x pst TA) if staged] | r of the block [NB][B] | strip combine [XB_WB][NB][sw]
  // pst = p rounded up to 16 elements: every staged vector starts 16-byte aligned
  const int64_t pst = (p + 15) / 16 * 16;
  TA* bsm = reinterpret_cast<TA*>(smem);
  const size_t bbytes = a.beta_smem ? (size_t)NF * pst * sizeof(TA) + 64 : 0;
  TA* rsm = reinterpret_cast<TA*>(smem + bbytes);
  double* csm = reinterpret_cast<double*>(smem + bbytes + ((size_t)NB * a.B * sizeof(TA) + 15) / 16 * 16);

  if (a.beta_smem) {
    // beta (times the column scales of a quantized X), zero-padded
    const int64_t pp = (int64_t)(bbytes / sizeof(TA));
    for (int64_t j = tid; j < pp; j += XB_THREADS) {
      const int64_t jj = j % pst, f = j / pst;
      double v = 0.0;
      if (f < NF && jj < p) {
        const double sc = a.colscale ? (double)a.colscale[jj] : 1.0;
        v = static_cast<const double*>(f == 0 ? ps->beta : ps->beta2)[jj] * sc;
      }
      bsm[j] = (TA)v;
    }
  }
  __syncthreads();

  if (warp < XB_WA) {
    // -------------------------------------------------------------- phase A
    const int nwA = gridDim.x * XB_WA;
    const int gw = blockIdx.x * XB_WA + warp;
    const unsigned items_per_blk = (unsigned)(a.B * a.nchunk);
    const int64_t total = (int64_t)a.nblk * items_per_blk;
    const double* bg0 = static_cast<const double*>(ps->beta);
    const double* bg1 = static_cast<const double*>(ps->beta2);
    const double* zprev = static_cast<const double*>(ps->zprev);
    double* zout = static_cast<double*>(ps->zout);
    const double mom = ps->mom;
    for (int64_t item = gw; item < total; item += nwA) {
      const int b = (int)(item / items_per_blk);
      const int within = (int)(item - (int64_t)b * items_per_blk);
      const int64_t row = (int64_t)b * a.B + within / a.nchunk;
      const int chunk = within % a.nchunk;
      if (b >= a.lag && !tmo) {
        bool ok = true;
        if (lane == 0) ok = wait_count(&a.bdone[b - a.lag], gridDim.x, a.limit_ns, a.status);
        if (!__shfl_sync(0xffffffffu, ok ? 1 : 0, 0)) tmo = 1;
      }
      if (row >= n) {   // past the last row: count it once
        if (chunk == 0 && lane == 0) atomicAdd(&a.done[b], 1u);
        continue;
      }
      const int64_t c0 = (int64_t)chunk * a.cw;
      const int64_t c1 = (c0 + a.cw < p) ? c0 + a.cw : p;
      const int nv = (int)((c1 - c0 + VEC - 1) / VEC);
      const TX* xr = X + row * a.ldx + c0;
      TA acc[NF];
      TA accl[NF];
#pragma unroll
      for (int f = 0; f < NF; ++f) { acc[f] = (TA)0; accl[f] = (TA)0; }
      for (int v0 = 0; v0 < nv; v0 += 32 * XB_U) {
        TA xs[XB_U][VEC];
#pragma unroll
        for (int u = 0; u < XB_U; ++u) {
          const int v = v0 + lane + 32 * u;
          if (v < nv) XTraits<TX>::load_global(xr + (int64_t)v * VEC, xs[u]);
        }
        TA part_s[NF];
#pragma unroll
        for (int f = 0; f < NF; ++f) part_s[f] = (TA)0;
#pragma unroll
        for (int u = 0; u < XB_U; ++u) {
          const int v = v0 + lane + 32 * u;
          if (v < nv) {
            const int64_t col = c0 + (int64_t)v * VEC;
            TA bv[NF][VEC];
            if (a.beta_smem) {
#pragma unroll
              for (int f = 0; f < NF; ++f) load_smem_vec<TA, VEC>(bsm + (int64_t)f * pst + col, bv[f]);
            } else {
#pragma unroll
              for (int l = 0; l < VEC; ++l) {
                const double sc = (a.colscale && col + l < p) ? (double)a.colscale[col + l] : 1.0;
#pragma unroll
                for (int f = 0; f < NF; ++f)
                  bv[f][l] = (col + l < p) ? (TA)((f == 0 ? bg0 : bg1)[col + l] * sc) : (TA)0;
              }
            }
            if (col + VEC > p) {   // past column p: padding may hold anything
#pragma unroll
              for (int l = 0; l < VEC; ++l)
                if (col + l >= p) {
                  xs[u][l] = (TA)0;
#pragma unroll
                  for (int f = 0; f < NF; ++f) bv[f][l] = (TA)0;
                }
            }
#pragma unroll
            for (int l = 0; l < VEC; ++l)
#pragma unroll
              for (int f = 0; f < NF; ++f) part_s[f] += xs[u][l] * bv[f][l];
          }
        }
#pragma unroll
        for (int f = 0; f < NF; ++f) {
          if constexpr (kF32) two_sum_acc(acc[f], accl[f], part_s[f]);
          else acc[f] += part_s[f];
        }
      }
      double* dst = a.part + ((size_t)row * a.nchunk + chunk) * NF;
#pragma unroll
      for (int f = 0; f < NF; ++f) {
        if constexpr (kF32) {
          float hi = acc[f], lo = accl[f];
          warp_sum_pair(hi, lo);
          if (lane == 0) dst[f] = pack_pair(hi, lo);
        } else {
          const double s = warp_sum((double)acc[f]);
          if (lane == 0) dst[f] = s;
        }
      }
      if (lane == 0) {
        __threadfence();
        const unsigned prev = atomicAdd(&a.rowcnt[row], 1u);
        if (prev + 1 == (unsigned)a.nchunk) {
          // last chunk of the row: z in chunk order, then the link
          __threadfence();
          const double* pr = a.part + (size_t)row * a.nchunk * NF;
          double z[NF];
#pragma unroll
          for (int f = 0; f < NF; ++f) {
            if constexpr (kF32) {
              float hi = 0.f, lo = 0.f;
              for (int c = 0; c < a.nchunk; ++c) add_pair(hi, lo, __ldcg(pr + (size_t)c * NF + f));
              z[f] = (double)hi + (double)lo;
            } else {
              double s = 0.0;
              for (int c = 0; c < a.nchunk; ++c) s += __ldcg(pr + (size_t)c * NF + f);
              z[f] = s;
            }
          }
          const double yd = a.y[row];
          double w[NB];
#pragma unroll
          for (int q = 0; q < NB; ++q) w[q] = 0.0;
          double lf = 0.0, ld = 0.0;
          switch (a.link) {
            case LINK_LS:
              w[0] = 2.0 * (z[0] - yd);
              break;
            case LINK_LOGISTIC:
              w[0] = -yd / (1.0 + exp(yd * z[0]));
              if (NB > 1) {
                const double zy = (1.0 + mom) * z[0] - mom * zprev[row];
                w[NB - 1] = -yd / (1.0 + exp(yd * zy));
              }
              break;
            case LINK_IDENT:
              w[0] = z[0];
              break;
            case LINK_CERT_LS:
            case LINK_CERTZ_LS: {
              const double zd = a.link == LINK_CERT_LS ? z[NF - 1] : zprev[row];
              const double d0 = z[0] - yd, d1 = zd - yd, zeta = -2.0 * d1;
              w[0] = 2.0 * d1;
              lf = d0 * d0;
              ld = zeta * yd - 0.25 * zeta * zeta;
              break;
            }
            case LINK_CERT_LOGI:
            case LINK_CERTZ_LOGI: {
              const double zd = a.link == LINK_CERT_LOGI ? z[NF - 1] : zprev[row];
              w[0] = -yd / (1.0 + exp(yd * zd));
              lf = softplus_neg(yd * z[0]);
              ld = entropy_of(yd * zd);
              break;
            }
            default: break;
          }
#pragma unroll
          for (int q = 0; q < NB; ++q) a.r[(size_t)q * n + row] = w[q];
          if (zout) zout[row] = z[0];
          if (a.lterm) { a.lterm[2 * row] = lf; a.lterm[2 * row + 1] = ld; }
          __threadfence();
          atomicAdd(&a.done[b], 1u);
        }
      }
      __syncwarp();
    }
    return;
  }

  // ---------------------------------------------------------------- phase B
  const int wb = warp - XB_WA;                 // 0 .. XB_WB-1
  const int tb = tid - XB_WA * 32;             // 0 .. XB_WB*32-1
  const int64_t s0 = (int64_t)blockIdx.x * a.sw;
  const int64_t s1 = (s0 + a.sw < p) ? s0 + a.sw : p;
  const int nvs = s1 > s0 ? (int)((s1 - s0 + VEC - 1) / VEC) : 0;   // vectors of the strip
  constexpr int TV = XBShape<VEC>::TV;          // strip vectors per lane (<= 32*TV*VEC columns)
  TA acc[NB][TV][VEC];
  float ahi[kF32 ? NB : 1][TV][VEC], alo[kF32 ? NB : 1][TV][VEC];
#pragma unroll
  for (int q = 0; q < NB; ++q)
#pragma unroll
    for (int t = 0; t < TV; ++t)
#pragma unroll
      for (int l = 0; l < VEC; ++l) {
        acc[q][t][l] = (TA)0;
        if constexpr (kF32) { ahi[q][t][l] = 0.f; alo[q][t][l] = 0.f; }
      }
  for (int b = 0; b < a.nblk; ++b) {
    if (!tmo) {
      bool ok = true;
      if (tb == 0) ok = wait_count(&a.done[b], (unsigned)a.B, a.limit_ns, a.status);
      if (!ok) tmo = 1;
    }
    named_sync(2, XB_WB * 32);
    const int64_t r0 = (int64_t)b * a.B;
    const int rows = (int)((n - r0) < a.B ? (n - r0) : a.B);
    for (int i = tb; i < rows; i += XB_WB * 32)
#pragma unroll
      for (int q = 0; q < NB; ++q) rsm[q * a.B + i] = (TA)__ldcg(a.r + (size_t)q * n + r0 + i);
    named_sync(2, XB_WB * 32);
    // X' r over the strip: warp wb takes rows wb, wb + XB_WB, ... of the block
    for (int i = wb; i < rows; i += XB_WB) {
      const TX* xr = X + (r0 + i) * a.ldx + s0;
      TA wi[NB];
#pragma unroll
      for (int q = 0; q < NB; ++q) wi[q] = rsm[q * a.B + i];
#pragma unroll
      for (int t = 0; t < TV; ++t) {
        const int v = lane + 32 * t;
        if (v < nvs) {
          TA x[VEC];
          XTraits<TX>::load_global_last(xr + (int64_t)v * VEC, x);
#pragma unroll
          for (int l = 0; l < VEC; ++l)
#pragma unroll
            for (int q = 0; q < NB; ++q) acc[q][t][l] += wi[q] * x[l];
        }
      }
    }
    if constexpr (kF32) {   // fold FP32 block sums into the compensated pair
#pragma unroll
      for (int q = 0; q < NB; ++q)
#pragma unroll
        for (int t = 0; t < TV; ++t)
#pragma unroll
          for (int l = 0; l < VEC; ++l) {
            two_sum_acc(ahi[q][t][l], alo[q][t][l], (float)acc[q][t][l]);
            acc[q][t][l] = (TA)0;
          }
    }
    named_sync(2, XB_WB * 32);
    if (tb == 0) {
      __threadfence();
      atomicAdd(&a.bdone[b], 1u);
    }
  }
  // combine the XB_WB warps' strip sums in a fixed order and write X' r
#pragma unroll
  for (int q = 0; q < NB; ++q)
#pragma unroll
    for (int t = 0; t < TV; ++t)
#pragma unroll
      for (int l = 0; l < VEC; ++l) {
        const int e = (lane + 32 * t) * VEC + l;
        if (e < a.sw) {
          const double v = kF32 ? (double)ahi[q][t][l] + (double)alo[q][t][l] : (double)acc[q][t][l];
          csm[((size_t)wb * NB + q) * a.sw + e] = v;
        }
      }
  named_sync(2, XB_WB * 32);
  for (int64_t e = tb; e < (s1 - s0); e += XB_WB * 32) {
    const double sc = a.colscale ? (double)a.colscale[s0 + e] : 1.0;
#pragma unroll
    for (int q = 0; q < NB; ++q) {
      double s = 0.0;
      for (int w = 0; w < XB_WB; ++w) s += csm[((size_t)w * NB + q) * a.sw + e];
      a.g[(size_t)q * p + s0 + e] = s * sc;
    }
  }
}

}  // namespace relax
