// Fused pass over X, strip-stationary: z = X beta, r = link(z), g = X' r, with
// X read from HBM once per pass.
//
// This is the matrix-vector work that dominates the method (Sec. 5.2.3); the
// induced dual point zeta = -grad F(X beta) (Sec. 3.3) comes out of it as -r.
//
// Decomposition.  The grid is Gc x Gr CTAs, one per SM, co-resident.  CTA
// (cc, cr) owns the column strip cc (a few KB of every row) and the row blocks
// b = cr, cr + Gr, ... (B rows each).  Its strip of beta lives in registers and
// its strip of X' r is accumulated in registers, so no CTA ever needs the whole
// of beta or of g.
//
// Per CTA, warp-specialized:
//  * lane 0 of warp 0 streams the CTA's strip tiles of its blocks from HBM into
//    ring A (RA = mA * SA stages; a tile is nbox 2-D tensor boxes of B rows x
//    `inner` columns, loaded by TMA, which zero-fills columns >= p and rows
//    >= n); lane 0 of warp 1 loads the same tiles again, from L2, into ring B
//    (RB = mB * SB stages);
//  * SA "dot" warps (warp a owns stages a, a + SA, ... of ring A; block k
//    goes to stage k mod RA): per row the strip's partial
//    dot product with beta, added to the row's z in 64-bit fixed point
//    (integer additions commute, so z does not depend on the arrival order of
//    the Gc strips), then the block is counted in cnt[b];
//  * SB "axpy" warps (warp e owns stages e, e + SB, ... of ring B): once cnt[b] = Gc each
//    reads z of the block's rows, applies the link and accumulates X' r over
//    its strip; CTA (k mod Gc) of the row group records z and the loss terms
//    of the group's k-th block; at the end the axpy warps' strip sums are
//    combined in a fixed order into g[cr][q][strip].
// Fixed point: z = Z * 2^-S with S chosen per pass from a bound of every
// partial and of their sum, max_i ||x_i||_1 * max_j |beta_j| < 2^(61-S); the
// grid agrees on max_j |beta_j| through one atomic max and a counter, which the
// dot warps wait for only before their first addition (the HBM stream starts
// at once).
// Each stage has exactly one consumer warp, which therefore never waits on a
// barrier phase more than one ahead of the last one it saw (the reason the
// ring depths are multiples of the warp counts).  A stage is held from its
// TMA issue until its warp has read the block, so the stages per ring, not
// the warps, set the bytes in flight: narrow element types, whose blocks are
// small, take several stages per warp.  Phase A may lead
// phase B by at most `lag` blocks of the CTA (L2 footprint).  Every wait is
// bounded: on expiry the kernel records ST_TIMEOUT, stops issuing and waiting,
// lets the copies in flight land and returns.
#pragma once
#include <climits>

#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_fp8.h>

#include "xpass.cuh"

namespace relax {

constexpr int XS_MAXS = 4;        // warps per phase at most
constexpr int XS_MAXR = 12;       // stages per ring at most
constexpr int XS_MAXB = 16;       // rows per block at most (one butterfly group)
constexpr int XS_MAXT = 256;      // 2 + SA + SB warps: at most two per scheduler
// 16-byte vectors of the strip per lane: a lane holds the same number of
// accumulators (24 FP32 or 12 FP64 columns, 24/32 for 16/8-bit X) for every type
template <int VEC> struct XSShape {
  static constexpr int TV = VEC == 2 ? 6 : VEC == 4 ? 6 : VEC == 8 ? 3 : 2;
};

struct XSArgs {
  CUtensorMap tm;        // X as a 2-D tensor (p columns x n rows), box `inner` x B
  int64_t n, p;
  int Gc, Gr;            // column strips x row groups; grid = Gc * Gr
  int64_t sw;            // strip columns = nbox * inner
  int inner, nbox;       // box columns (multiple of the vector width, <= 256); boxes per strip
  int boxb;              // bytes per box in shared memory (B * inner * size, padded to 128)
  int B, nblk;           // rows per block, blocks
  int SA, SB, lag;       // dot / axpy warps; lead of phase A over phase B (blocks)
  int RA, RB;            // ring stages (multiples of SA / SB)
  int link;
  const double* y;
  const float* colscale;
  PassState* ps;
  unsigned long long* zfix;   // [NF][n] z in fixed point (two's complement)   } zeroed
  unsigned long long* zmax;   // [NF] max_j |beta_j| (bits of a nonnegative double) } before
  unsigned* zcnt;             // CTAs that have added to zmax                   } the launch
  double rowl1;               // max_i ||x_i||_1 of the stored X (NaN when X holds a NaN)
  double* g;             // [Gr][NB][p] X' r per row group
  double* lterm;         // [n][2] per-row {F, -F*(-zeta)} (certification links) or NULL
  double* lterm2;        // [n][2] the same at the second dual point (LINK_CERT2_*) or NULL
  unsigned* cnt;         // [nblk] CTAs done with the block's dots (zeroed before the launch)
  int* status;
  uint64_t limit_ns;
};

__device__ __forceinline__ unsigned ld_acquire_u32(const unsigned* p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_release_u32(unsigned* p, unsigned v) {
  asm volatile("st.release.gpu.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
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
      __nanosleep(20);
    }
  }
}

// bounded wait until a shared-memory counter reaches target
__device__ __forceinline__ bool wait_smem(const volatile unsigned* ctr, unsigned target, uint64_t limit_ns,
                                          int* status) {
  if (*ctr >= target) return true;
  const uint64_t t0 = globaltimer_ns();
  for (uint32_t it = 1;; ++it) {
    if (*ctr >= target) return true;
    if ((it & 15u) == 0u && globaltimer_ns() - t0 > limit_ns) {
      atomicCAS(status, ST_OK, ST_TIMEOUT);
      return false;
    }
  }
}

// 2-D tensor box (x = column, y = row) -> shared memory, completion on `bar`
__device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* map, int x, int y, uint64_t* bar,
                                            uint64_t policy) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes.L2::cache_hint"
      " [%0], [%1, {%2, %3}], [%4], %5;" ::"r"(smem_u32(dst)),
      "l"(map), "r"(x), "r"(y), "r"(smem_u32(bar)), "l"(policy)
      : "memory");
}

__device__ __forceinline__ uint64_t policy_evict_last() {
  uint64_t p;
  asm volatile("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(p));
  return p;
}
__device__ __forceinline__ uint64_t policy_evict_normal() {
  uint64_t p;
  asm volatile("createpolicy.fractional.L2::evict_normal.b64 %0, 1.0;" : "=l"(p));
  return p;
}

// Scale exponent of the fixed-point z for the bound `bz` of every partial and
// of their sum: |value| * 2^S < 2^61.  INT_MIN marks a bound that is not
// finite (NaN or Inf in X or beta): z is then NaN.
__device__ __forceinline__ int fixed_scale(double bz) {
  if (!(bz < INFINITY)) return INT_MIN;
  if (bz == 0.0) return 0;
  int e = 0;
  frexp(bz, &e);   // bz < 2^e
  return max(-1000, min(1000, 61 - e));
}

// (h, l) += (rh, rl) for compensated FP32 pairs
__device__ __forceinline__ void pair_add(float& h, float& l, float rh, float rl) {
  float e = 0.f;
  float s = h;
  two_sum_acc(s, e, rh);
  h = s;
  l = l + rl + e;
}

// Steps of a transposed butterfly over N = 2^m rows, at lane strides o0,
// o0/2, ...: each step sends half of the remaining rows to the partner lane
// and keeps the other half (the upper half on lanes with the stride's bit
// set); afterwards h[0], l[0] hold the sum over those m lane bits of the row
// whose index bits, high to low, are the lane's bits o0, o0/2, ...
template <int N>
__device__ __forceinline__ void bfly_steps(float (&h)[N], float (&l)[N], int lane, int o0) {
#pragma unroll
  for (int half = N / 2, o = o0; half >= 1; half >>= 1, o >>= 1) {
    const bool up = (lane & o) != 0;
#pragma unroll
    for (int i = 0; i < half; ++i) {
      const float sh = up ? h[i] : h[i + half], sl = up ? l[i] : l[i + half];
      const float kh = up ? h[i + half] : h[i], kl = up ? l[i + half] : l[i];
      const float rh = __shfl_xor_sync(0xffffffffu, sh, o), rl = __shfl_xor_sync(0xffffffffu, sl, o);
      h[i] = kh;
      l[i] = kl;
      pair_add(h[i], l[i], rh, rl);
    }
  }
}

// Transposed butterfly over 16 rows: on entry lane L holds its partial of
// every row in h[0..15] (l = low parts); on exit h[0], l[0] of lane L hold the
// warp total of row (L >> 1) & 15.  Each step sends half of the remaining rows
// to the partner lane and keeps the other half: 8+4+2+1+1 shuffles of pairs
// instead of 16 x 5.
__device__ __forceinline__ void butterfly16(float (&h)[16], float (&l)[16], int lane) {
#pragma unroll
  for (int half = 8, o = 16; half >= 1; half >>= 1, o >>= 1) {
    const bool up = (lane & o) != 0;
#pragma unroll
    for (int i = 0; i < half; ++i) {
      const float sh = up ? h[i] : h[i + half], sl = up ? l[i] : l[i + half];
      const float kh = up ? h[i + half] : h[i], kl = up ? l[i + half] : l[i];
      const float rh = __shfl_xor_sync(0xffffffffu, sh, o), rl = __shfl_xor_sync(0xffffffffu, sl, o);
      h[i] = kh;
      l[i] = kl;
      pair_add(h[i], l[i], rh, rl);
    }
  }
  const float rh = __shfl_xor_sync(0xffffffffu, h[0], 1), rl = __shfl_xor_sync(0xffffffffu, l[0], 1);
  pair_add(h[0], l[0], rh, rl);
}
__device__ __forceinline__ void butterfly16(double (&h)[16], int lane) {
#pragma unroll
  for (int half = 8, o = 16; half >= 1; half >>= 1, o >>= 1) {
    const bool up = (lane & o) != 0;
#pragma unroll
    for (int i = 0; i < half; ++i) {
      const double sh = up ? h[i] : h[i + half];
      const double kh = up ? h[i + half] : h[i];
      h[i] = kh + __shfl_xor_sync(0xffffffffu, sh, o);
    }
  }
  h[0] += __shfl_xor_sync(0xffffffffu, h[0], 1);
}

// Link of one row: w[q] = the gradient weights of the row (r = grad F at z, and
// at the momentum point for the logistic loop), lf = F term at z[0],
// ld = -F*(-zeta) term of the dual point (certification links).  zp is the
// row's entry of ps.zprev (z of the previous iterate, or the given dual point).
// LOWP (the loop's FP32-accumulating passes): the logistic link in FP32
// (FP64 exp on this GPU costs about as much as streaming the row block);
// the float-float and FP64 passes keep it in FP64.
template <int NF, int NB, bool LOWP = false>
__device__ __forceinline__ void link_of(int link, const double* z, double yd, double zp, double mom, double* w,
                                        double& lf, double& ld, double& ld2) {
  ld2 = 0.0;
#pragma unroll
  for (int q = 0; q < NB; ++q) w[q] = 0.0;
  lf = 0.0;
  ld = 0.0;
  switch (link) {
    case LINK_LS:
      w[0] = 2.0 * (z[0] - yd);
      break;
    case LINK_LOGISTIC:
      if constexpr (LOWP) {
        const float yf = (float)yd;
        w[0] = (double)(-yf / (1.0f + expf(yf * (float)z[0])));
        if (NB > 1) {
          const double zy = (1.0 + mom) * z[0] - mom * zp;
          w[NB - 1] = (double)(-yf / (1.0f + expf(yf * (float)zy)));
        }
      } else {
        w[0] = -yd / (1.0 + exp(yd * z[0]));
        if (NB > 1) {
          const double zy = (1.0 + mom) * z[0] - mom * zp;
          w[NB - 1] = -yd / (1.0 + exp(yd * zy));
        }
      }
      break;
    case LINK_IDENT:
      w[0] = z[0];
      break;
    case LINK_CERT_LS:
    case LINK_CERTZ_LS: {
      const double zd = link == LINK_CERT_LS ? z[NF - 1] : zp;
      const double d0 = z[0] - yd, d1 = zd - yd, zeta = -2.0 * d1;
      w[0] = 2.0 * d1;
      lf = d0 * d0;
      ld = zeta * yd - 0.25 * zeta * zeta;
      break;
    }
    case LINK_CERT_LOGI:
    case LINK_CERTZ_LOGI: {
      const double zd = link == LINK_CERT_LOGI ? z[NF - 1] : zp;
      w[0] = -yd / (1.0 + exp(yd * zd));
      lf = softplus_neg(yd * z[0]);
      ld = entropy_of(yd * zd);
      break;
    }
    case LINK_CERT2_LS: {
      const double d0 = z[0] - yd, d1 = zp - yd;
      w[0] = 2.0 * d1;
      if (NB > 1) w[NB - 1] = 2.0 * d0;
      const double zeta1 = -2.0 * d1, zeta0 = -2.0 * d0;
      lf = d0 * d0;
      ld = zeta1 * yd - 0.25 * zeta1 * zeta1;
      ld2 = zeta0 * yd - 0.25 * zeta0 * zeta0;
      break;
    }
    case LINK_CERT2_LOGI: {
      w[0] = -yd / (1.0 + exp(yd * zp));
      if (NB > 1) w[NB - 1] = -yd / (1.0 + exp(yd * z[0]));
      lf = softplus_neg(yd * z[0]);
      ld = entropy_of(yd * zp);
      ld2 = entropy_of(yd * z[0]);
      break;
    }
    default: break;
  }
}

// FF (FP32 X, TA = float): float-float arithmetic for the certificate and
// the power iteration: each product x beta (and x r) is formed exactly as
// the FMA pair (x bh, fma(x, bh, -x bh)) plus x bl, beta = bh + bl, and
// summed with TwoSum (about 48 significant bits).  This GPU issues FP64 at
// about 1/70 of the FP32 rate, which made the FP64-accumulating pass
// compute-bound; the float-float one streams X like the loop's pass.
template <typename TX, typename TA, int NF, int NB, bool FF = false>
__global__ void __launch_bounds__(XS_MAXT, 1) xstrip_kernel(const __grid_constant__ XSArgs a) {
  constexpr int VEC = XTraits<TX>::VEC;
  constexpr int TV = XSShape<VEC>::TV;
  constexpr bool kF32 = sizeof(TA) == 4;
  // FP32 sums on packed pairs (f32x2): measured faster wherever the pass does
  // more than one FMA per 4 bytes of X (two right-hand sides, BF16 / FP8
  // elements); the one-right-hand-side FP32 pass ran 10% slower on pairs
  constexpr bool kPair = kF32 && !FF && !(sizeof(TX) == 4 && NB == 1);
  // FP8 (16 elements per vector): the dot warps' rows in a rolled loop of
  // four-row groups (measured faster there, slower for FP32 and BF16)
  constexpr bool kGroup = kPair && sizeof(TX) == 1;
  static_assert(!FF || (sizeof(TX) == 4 && kF32), "float-float: FP32 X and FP32 pairs");
  extern __shared__ __align__(128) unsigned char smem_raw[];
  __shared__ __align__(8) uint64_t fullA[XS_MAXR], emptyA[XS_MAXR], fullB[XS_MAXR], emptyB[XS_MAXR];
  __shared__ volatile int tmo;        // a bounded wait expired: stop issuing and waiting
  __shared__ volatile unsigned bcnt;  // blocks finished by phase B in this CTA
  __shared__ int skip;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  if (tid == 0) {
    tmo = 0;
    bcnt = 0;
    skip = a.ps->done;
    for (int s = 0; s < a.RA; ++s) { mbar_init(&fullA[s], 1); mbar_init(&emptyA[s], 1); }
    for (int s = 0; s < a.RB; ++s) { mbar_init(&fullB[s], 1); mbar_init(&emptyB[s], 1); }
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  if (skip) return;   // uniform (same flag everywhere)

  // tensor boxes land on 128-byte aligned addresses (128 bytes of slack are allocated)
  unsigned char* smem = smem_raw + ((128u - (smem_u32(smem_raw) & 127u)) & 127u);
  const int cc = blockIdx.x % a.Gc, cr = blockIdx.x / a.Gc;
  const int64_t n = a.n, p = a.p;
  const int64_t s0 = (int64_t)cc * a.sw;
  const int64_t s1 = (s0 + a.sw < p) ? s0 + a.sw : p;
  const int nvs = (int)((s1 - s0 + VEC - 1) / VEC);          // vectors of the strip
  const uint32_t tilebytes = (uint32_t)a.nbox * a.B * a.inner * (uint32_t)sizeof(TX);   // tx bytes per tile
  const int rowpitch = a.inner * (int)sizeof(TX);   // bytes per row inside a box
  // byte offsets of this lane's vectors in row 0 of a tile (box, then vector in
  // the box row); lanes past the strip read its last vector (their beta is zero
  // and their sums are never written)
  uint32_t voff[TV];
  {
    const int vpb = a.inner / VEC;
#pragma unroll
    for (int t = 0; t < TV; ++t) {
      const int v = min(lane + 32 * t, max(nvs - 1, 0));
      voff[t] = (uint32_t)((v / vpb) * a.boxb + (v % vpb) * 16);
    }
  }
  const int kloc = (cr < a.nblk) ? (a.nblk - cr + a.Gr - 1) / a.Gr : 0;   // blocks of this CTA
  const size_t stage = (size_t)a.nbox * a.boxb;
  unsigned char* ringA = smem;
  unsigned char* ringB = smem + (size_t)a.RA * stage;
  {
    // the fixed-shape row loops read every row of a tile; keep never-loaded
    // stage memory finite
    float4* z4 = reinterpret_cast<float4*>(smem);
    const size_t nz = (size_t)(a.RA + a.RB) * stage / 16;
    for (size_t i = tid; i < nz; i += blockDim.x) z4[i] = make_float4(0.f, 0.f, 0.f, 0.f);
    __syncthreads();
  }
  // phase-B accumulators (used by the axpy warps only)
  TA acc[NB][TV][VEC];
  float ahi[kF32 && !FF ? NB : 1][TV][VEC], alo[kF32 && !FF ? NB : 1][TV][VEC];
  float accl[FF ? NB : 1][TV][VEC];   // FF: low parts of acc
  const bool axpy = warp >= 2 + a.SA && warp < 2 + a.SA + a.SB;

  if (warp == 0) {
    // ------------------------------------------------ producer A: HBM -> ring A
    if (lane == 0) {
      const uint64_t pol = policy_evict_normal();
      int issued = 0;
      for (int k = 0; k < kloc; ++k) {
        const int s = k % a.RA;
        if (tmo) break;
        if (k >= a.RA && !mbar_wait<false>(&emptyA[s], ((k / a.RA) - 1) & 1, a.limit_ns, a.status)) { tmo = 1; break; }
        if (k > a.lag && !wait_smem(&bcnt, (unsigned)(k - a.lag), a.limit_ns, a.status)) { tmo = 1; break; }
        const int y0 = (cr + k * a.Gr) * a.B;
        mbar_arrive_expect_tx(&fullA[s], tilebytes);
        for (int i = 0; i < a.nbox; ++i)
          tma_load_2d(ringA + s * stage + (size_t)i * a.boxb, &a.tm, (int)s0 + i * a.inner, y0, &fullA[s], pol);
        issued = k + 1;
      }
      // let every copy in flight land before the CTA may exit
      for (int k = (issued > a.RA ? issued - a.RA : 0); k < issued; ++k)
        mbar_wait<false>(&fullA[k % a.RA], (k / a.RA) & 1, a.limit_ns, a.status);
    }
  } else if (warp == 1) {
    // ---------------------------------- producer B: L2 -> ring B (its own warp,
    // so that its waits and copies never serialise with producer A's)
    if (lane == 0) {
      const uint64_t pol = policy_evict_first();
      int issued = 0;
      for (int k = 0; k < kloc; ++k) {
        const int s = k % a.RB;
        if (tmo) break;
        if (k >= a.RB && !mbar_wait<false>(&emptyB[s], ((k / a.RB) - 1) & 1, a.limit_ns, a.status)) { tmo = 1; break; }
        const int y0 = (cr + k * a.Gr) * a.B;
        mbar_arrive_expect_tx(&fullB[s], tilebytes);
        for (int i = 0; i < a.nbox; ++i)
          tma_load_2d(ringB + s * stage + (size_t)i * a.boxb, &a.tm, (int)s0 + i * a.inner, y0, &fullB[s], pol);
        issued = k + 1;
      }
      for (int k = (issued > a.RB ? issued - a.RB : 0); k < issued; ++k)
        mbar_wait<false>(&fullB[k % a.RB], (k / a.RB) & 1, a.limit_ns, a.status);
    }
  } else if (warp < 2 + a.SA) {
    // ------------------------------------------------ phase A: strip dot products
    const int st = warp - 2;
    TA bv[NF][TV][VEC];
    float bl[FF ? NF : 1][TV][VEC];   // FF: low parts of beta
#pragma unroll
    for (int t = 0; t < TV; ++t) {
      const int v = lane + 32 * t;
#pragma unroll
      for (int l = 0; l < VEC; ++l) {
        const int64_t col = s0 + (int64_t)v * VEC + l;
        const bool in = v < nvs && col < p;
        const double sc = (in && a.colscale) ? (double)a.colscale[col] : 1.0;
#pragma unroll
        for (int f = 0; f < NF; ++f) {
          const double bd = in ? static_cast<const double*>(f == 0 ? a.ps->beta : a.ps->beta2)[col] * sc : 0.0;
          bv[f][t][l] = (TA)bd;
          if constexpr (FF) bl[f][t][l] = (float)(bd - (double)bv[f][t][l]);
        }
      }
    }
    if (st == 0) {
      // this CTA's max |beta_j| (NaN dominates: its bits compare above +Inf)
#pragma unroll
      for (int f = 0; f < NF; ++f) {
        unsigned long long mb = 0ull;
#pragma unroll
        for (int t = 0; t < TV; ++t)
#pragma unroll
          for (int l = 0; l < VEC; ++l) {
            double bb = (double)bv[f][t][l];
            if constexpr (FF) bb += (double)bl[f][t][l];
            const unsigned long long bits = (unsigned long long)__double_as_longlong(fabs(bb));
            mb = bits > mb ? bits : mb;
          }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
          const unsigned long long other = __shfl_xor_sync(0xffffffffu, mb, o);
          mb = other > mb ? other : mb;
        }
        if (lane == 0) atomicMax(&a.zmax[f], mb);
      }
      __threadfence();
      __syncwarp();
      if (lane == 0) atomicAdd(a.zcnt, 1u);
    }
    int zs[NF];          // fixed-point exponents, known after the first block's dots
    double zf[NF];       // 2^zs
    bool have_scale = false;
    for (int k = st; k < kloc; k += a.SA) {
      if (tmo) break;
      const int sa = k % a.RA;   // one of this warp's stages
      if (!__all_sync(0xffffffffu, mbar_wait<false>(&fullA[sa], (k / a.RA) & 1, a.limit_ns, a.status))) {
        tmo = 1;
        break;
      }
      const int b = cr + k * a.Gr;
      const int64_t r0 = (int64_t)b * a.B;
      const int rows = (int)((n - r0) < a.B ? (n - r0) : a.B);
      const unsigned char* tile = ringA + sa * stage;
      // per-lane partials of the block's rows (plain FP32 over the lane's
      // columns), then one transposed butterfly per forward vector
      TA ph[NF][XS_MAXB];
      float phl[FF ? NF : 1][XS_MAXB];   // FF: low parts
      float vh[NF][4], vl[NF][4];        // kGroup: the four row groups after two butterfly steps
      if constexpr (FF) {
        // float-float: one row at a time (the fully unrolled block of
        // float-float sums outgrew the instruction cache); the row partials
        // go to a per-lane array for the butterfly
#pragma unroll 1
        for (int jj = 0; jj < XS_MAXB; ++jj) {
          float hh[NF], ll[NF];
#pragma unroll
          for (int f = 0; f < NF; ++f) { hh[f] = 0.f; ll[f] = 0.f; }
          const int jr = jj < a.B ? jj : a.B - 1;   // rows >= rows: zero-filled or repeated, discarded
          const unsigned char* rowp = tile + (size_t)jr * rowpitch;
#pragma unroll
          for (int t = 0; t < TV; ++t) {
            TA x[VEC];
            XTraits<TX>::load(reinterpret_cast<const TX*>(rowp + voff[t]), x);
#pragma unroll
            for (int f = 0; f < NF; ++f)
#pragma unroll
              for (int l = 0; l < VEC; ++l) {
                const float pr = x[l] * bv[f][t][l];
                const float lo = fmaf(x[l], bl[f][t][l], fmaf(x[l], bv[f][t][l], -pr));   // exact error + x bl
                const float sacc = hh[f] + pr;
                const float bp = sacc - hh[f];
                ll[f] += ((hh[f] - (sacc - bp)) + (pr - bp)) + lo;
                hh[f] = sacc;
              }
          }
#pragma unroll
          for (int f = 0; f < NF; ++f) { ph[f][jj] = hh[f]; phl[f][jj] = ll[f]; }
        }
      } else if constexpr (kGroup) {
        // FP32 sums, rows in four groups of four (a rolled loop, for the
        // schedulers' instruction caches): group g holds rows g, g+4, g+8,
        // g+12, whose partials take the butterfly's first two steps (lane
        // strides 16, 8) in the group and the last ones (4, 2, 1) after the
        // loop -- the additions of the 16-row butterfly, in its order
#pragma unroll 1
        for (int g = 0; g < 4; ++g) {
          float gh[NF][4], gl[NF][4];
#pragma unroll
          for (int i = 0; i < 4; ++i) {
            const int jj = g + 4 * i;
            const int jr = jj < a.B ? jj : a.B - 1;   // rows >= rows: zero-filled or repeated, discarded
            const unsigned char* rowp = tile + (size_t)jr * rowpitch;
            if constexpr (kPair) {
              // even and odd columns in the two halves of a packed pair
              float2 p2[NF];
#pragma unroll
              for (int f = 0; f < NF; ++f) p2[f] = make_float2(0.f, 0.f);
#pragma unroll
              for (int t = 0; t < TV; ++t) {
                TA x[VEC];
                XTraits<TX>::load(reinterpret_cast<const TX*>(rowp + voff[t]), x);
#pragma unroll
                for (int f = 0; f < NF; ++f)
#pragma unroll
                  for (int l = 0; l < VEC; l += 2)
                    p2[f] = fma2(make_float2(x[l], x[l + 1]), make_float2(bv[f][t][l], bv[f][t][l + 1]), p2[f]);
              }
#pragma unroll
              for (int f = 0; f < NF; ++f) gh[f][i] = p2[f].x + p2[f].y;
            } else {
#pragma unroll
              for (int f = 0; f < NF; ++f) gh[f][i] = 0.f;
#pragma unroll
              for (int t = 0; t < TV; ++t) {
                TA x[VEC];
                XTraits<TX>::load(reinterpret_cast<const TX*>(rowp + voff[t]), x);
#pragma unroll
                for (int f = 0; f < NF; ++f)
#pragma unroll
                  for (int l = 0; l < VEC; ++l) gh[f][i] += x[l] * bv[f][t][l];
              }
            }
#pragma unroll
            for (int f = 0; f < NF; ++f) gl[f][i] = 0.f;
          }
#pragma unroll
          for (int f = 0; f < NF; ++f) {
            bfly_steps<4>(gh[f], gl[f], lane, 16);
#pragma unroll
            for (int gg = 0; gg < 4; ++gg)   // registers, not an indexed array
              if (gg == g) { vh[f][gg] = gh[f][0]; vl[f][gg] = gl[f][0]; }
          }
        }
      } else {
#pragma unroll
      for (int jj = 0; jj < XS_MAXB; ++jj) {
#pragma unroll
        for (int f = 0; f < NF; ++f) ph[f][jj] = (TA)0;
        const int jr = jj < a.B ? jj : a.B - 1;   // rows >= rows: zero-filled or repeated, discarded
        const unsigned char* rowp = tile + (size_t)jr * rowpitch;
        if constexpr (kPair) {
          // FP32: even and odd columns in the two halves of a packed pair
          float2 p2[NF];
#pragma unroll
          for (int f = 0; f < NF; ++f) p2[f] = make_float2(0.f, 0.f);
#pragma unroll
          for (int t = 0; t < TV; ++t) {
            TA x[VEC];
            XTraits<TX>::load(reinterpret_cast<const TX*>(rowp + voff[t]), x);
#pragma unroll
            for (int f = 0; f < NF; ++f)
#pragma unroll
              for (int l = 0; l < VEC; l += 2)
                p2[f] = fma2(make_float2(x[l], x[l + 1]), make_float2(bv[f][t][l], bv[f][t][l + 1]), p2[f]);
          }
#pragma unroll
          for (int f = 0; f < NF; ++f) ph[f][jj] = p2[f].x + p2[f].y;
        } else {
#pragma unroll
          for (int t = 0; t < TV; ++t) {
            TA x[VEC];
            XTraits<TX>::load(reinterpret_cast<const TX*>(rowp + voff[t]), x);
#pragma unroll
            for (int f = 0; f < NF; ++f)
#pragma unroll
              for (int l = 0; l < VEC; ++l) ph[f][jj] += x[l] * bv[f][t][l];
          }
        }
      }
      }
      // every read of the stage is done (the partials are in registers):
      // hand it back to the producer before the butterfly
      __syncwarp();
      if (lane == 0) mbar_arrive(&emptyA[sa]);
      // lane 2j: the strip partial of row j, as (hi, lo)
      TA mh[NF], ml[NF];
#pragma unroll
      for (int f = 0; f < NF; ++f) {
        if constexpr (FF) {
          butterfly16(ph[f], phl[f], lane);
          mh[f] = ph[f][0];
          ml[f] = phl[f][0];
        } else if constexpr (kGroup) {
          bfly_steps<4>(vh[f], vl[f], lane, 4);
          const float rh = __shfl_xor_sync(0xffffffffu, vh[f][0], 1), rl = __shfl_xor_sync(0xffffffffu, vl[f][0], 1);
          pair_add(vh[f][0], vl[f][0], rh, rl);
          mh[f] = vh[f][0];
          ml[f] = vl[f][0];
        } else if constexpr (kF32) {
          float pl[XS_MAXB];
#pragma unroll
          for (int jj = 0; jj < XS_MAXB; ++jj) pl[jj] = 0.f;
          butterfly16(ph[f], pl, lane);
          mh[f] = ph[f][0];
          ml[f] = pl[0];
        } else {
          butterfly16(ph[f], lane);
          mh[f] = ph[f][0];
          ml[f] = (TA)0;
        }
      }
      if (!have_scale) {
        // every CTA's max |beta_j| is in: the common scale of this pass
        if (!__all_sync(0xffffffffu, wait_count(a.zcnt, gridDim.x, a.limit_ns, a.status))) {
          tmo = 1;
          break;
        }
#pragma unroll
        for (int f = 0; f < NF; ++f) {
          zs[f] = fixed_scale(a.rowl1 * __longlong_as_double((long long)__ldcg(&a.zmax[f])));
          zf[f] = zs[f] == INT_MIN ? 0.0 : ldexp(1.0, zs[f]);
        }
        have_scale = true;
      }
      if ((lane & 1) == 0 && (lane >> 1) < rows) {
#pragma unroll
        for (int f = 0; f < NF; ++f) {
          if (zs[f] == INT_MIN) continue;
          const long long q = __double2ll_rn((double)mh[f] * zf[f]) + __double2ll_rn((double)ml[f] * zf[f]);
          atomicAdd(&a.zfix[(size_t)f * n + r0 + (lane >> 1)], (unsigned long long)q);
        }
      }
      // the block is counted with release semantics: after the warp barrier the
      // lanes' fixed-point additions above are ordered before the increment
      // that phase B's acquire-loads observe (cheaper than a full fence)
      __syncwarp();
      if (lane == 0) asm volatile("red.release.gpu.global.add.u32 [%0], 1;" ::"l"(&a.cnt[b]) : "memory");
    }
  } else if (axpy) {
    // ------------------------------------------------ phase B: X' r over the strip
    const int st = warp - 2 - a.SA;
#pragma unroll
    for (int q = 0; q < NB; ++q)
#pragma unroll
      for (int t = 0; t < TV; ++t)
#pragma unroll
        for (int l = 0; l < VEC; ++l) {
          acc[q][t][l] = (TA)0;
          if constexpr (FF) accl[q][t][l] = 0.f;
          else if constexpr (kF32) { ahi[q][t][l] = 0.f; alo[q][t][l] = 0.f; }
        }
    const bool need_zp = a.link == LINK_CERTZ_LS || a.link == LINK_CERTZ_LOGI || a.link == LINK_CERT2_LS ||
                         a.link == LINK_CERT2_LOGI || (a.link == LINK_LOGISTIC && NB > 1);
    const double* zprev = static_cast<const double*>(a.ps->zprev);
    double* zout = static_cast<double*>(a.ps->zout);
    const double mom = a.ps->mom;
    const int jl = lane & 15, hb = lane >> 4;   // the block row this lane evaluates (hb: duplicate)
    double zinv[NF];
    bool have_scale = false;
    for (int k = st; k < kloc; k += a.SB) {
      if (tmo) break;
      const int b = cr + k * a.Gr;
      const int64_t r0 = (int64_t)b * a.B;
      const int rows = (int)((n - r0) < a.B ? (n - r0) : a.B);
      const int64_t rowj = r0 + (jl < rows ? jl : rows - 1);
      const double yd = a.y[rowj];
      const double zp = need_zp ? zprev[rowj] : 0.0;
      if (!__all_sync(0xffffffffu, wait_count(&a.cnt[b], (unsigned)a.Gc, a.limit_ns, a.status))) {
        tmo = 1;
        break;
      }
      if (!have_scale) {   // final once any block is complete
#pragma unroll
        for (int f = 0; f < NF; ++f) {
          const int zs = fixed_scale(a.rowl1 * __longlong_as_double((long long)__ldcg(&a.zmax[f])));
          zinv[f] = zs == INT_MIN ? __longlong_as_double(0x7ff8000000000000ll) : ldexp(1.0, -zs);
        }
        have_scale = true;
      }
      double z[NF];
#pragma unroll
      for (int f = 0; f < NF; ++f) z[f] = (double)(long long)__ldcg(&a.zfix[(size_t)f * n + rowj]) * zinv[f];
      double rv[NB], lf, ld, ld2;
      link_of<NF, NB, kF32 && !FF>(a.link, z, yd, zp, mom, rv, lf, ld, ld2);
      if (jl >= rows) {
#pragma unroll
        for (int q = 0; q < NB; ++q) rv[q] = 0.0;   // rows past the end carry weight 0
      }
      // the row's weights in the accumulation type, formed once by the lane
      // that owns the row (FF: as a float pair)
      TA rvh[NB];
      float rvl[FF ? NB : 1];
#pragma unroll
      for (int q = 0; q < NB; ++q) {
        rvh[q] = (TA)rv[q];
        if constexpr (FF) rvl[q] = (float)(rv[q] - (double)rvh[q]);
      }
      if (cc == k % a.Gc && hb == 0 && jl < rows) {   // this CTA records the block
        if (zout) zout[r0 + jl] = z[0];
        if (a.lterm) { a.lterm[2 * (r0 + jl)] = lf; a.lterm[2 * (r0 + jl) + 1] = ld; }
        if (a.lterm2) { a.lterm2[2 * (r0 + jl)] = lf; a.lterm2[2 * (r0 + jl) + 1] = ld2; }
      }
      const int sb = k % a.RB;   // one of this warp's stages
      if (!__all_sync(0xffffffffu, mbar_wait<false>(&fullB[sb], (k / a.RB) & 1, a.limit_ns, a.status))) {
        tmo = 1;
        break;
      }
      const unsigned char* tile = ringB + sb * stage;
      // rows four at a time (the accumulators are indexed by column only): a
      // fully unrolled block of rows ran slower, its loop and the dot warps'
      // sharing the schedulers' instruction caches
#pragma unroll(FF ? 1 : 4)
      for (int j = 0; j < XS_MAXB; ++j) {
        const int jr = j < a.B ? j : a.B - 1;   // rows >= rows carry weight 0
        TA w[NB];
        float wl[FF ? NB : 1];   // FF: low parts of the row's weights
#pragma unroll
        for (int q = 0; q < NB; ++q) {
          w[q] = __shfl_sync(0xffffffffu, rvh[q], j);
          if constexpr (FF) wl[q] = __shfl_sync(0xffffffffu, rvl[q], j);
        }
        const unsigned char* rowp = tile + (size_t)jr * rowpitch;
#pragma unroll
        for (int t = 0; t < TV; ++t) {
          TA x[VEC];
          XTraits<TX>::load(reinterpret_cast<const TX*>(rowp + voff[t]), x);
          if constexpr (kPair) {
            // two columns per packed FP32 FMA (the same roundings as two scalar FMAs)
#pragma unroll
            for (int l = 0; l < VEC; l += 2)
#pragma unroll
              for (int q = 0; q < NB; ++q) {
                const float2 r2 = fma2(make_float2(w[q], w[q]), make_float2(x[l], x[l + 1]),
                                       make_float2(acc[q][t][l], acc[q][t][l + 1]));
                acc[q][t][l] = r2.x;
                acc[q][t][l + 1] = r2.y;
              }
          } else {
#pragma unroll
            for (int l = 0; l < VEC; ++l)
#pragma unroll
              for (int q = 0; q < NB; ++q) {
                if constexpr (FF) {
                  const float pr = w[q] * x[l];
                  const float lo = fmaf(wl[q], x[l], fmaf(w[q], x[l], -pr));
                  const float sacc = acc[q][t][l] + pr;
                  const float bp = sacc - acc[q][t][l];
                  accl[q][t][l] += ((acc[q][t][l] - (sacc - bp)) + (pr - bp)) + lo;
                  acc[q][t][l] = sacc;
                } else {
                  acc[q][t][l] += w[q] * x[l];
                }
              }
          }
        }
      }
      __syncwarp();
      if (lane == 0) {
        mbar_arrive(&emptyB[sb]);
        atomicAdd((unsigned*)&bcnt, 1u);
      }
      if constexpr (kF32 && !FF) {   // fold the block's FP32 sums into the compensated pair
#pragma unroll
        for (int q = 0; q < NB; ++q)
#pragma unroll
          for (int t = 0; t < TV; ++t)
#pragma unroll
            for (int l = 0; l < VEC; l += 2) {
              if constexpr (kPair) {
                float2 h2 = make_float2(ahi[q][t][l], ahi[q][t][l + 1]);
                float2 l2 = make_float2(alo[q][t][l], alo[q][t][l + 1]);
                two_sum_acc2(h2, l2, make_float2((float)acc[q][t][l], (float)acc[q][t][l + 1]));
                ahi[q][t][l] = h2.x;
                ahi[q][t][l + 1] = h2.y;
                alo[q][t][l] = l2.x;
                alo[q][t][l + 1] = l2.y;
              } else {
                two_sum_acc(ahi[q][t][l], alo[q][t][l], (float)acc[q][t][l]);
                two_sum_acc(ahi[q][t][l + 1], alo[q][t][l + 1], (float)acc[q][t][l + 1]);
              }
              acc[q][t][l] = (TA)0;
              acc[q][t][l + 1] = (TA)0;
            }
      }
    }
  }
  __syncthreads();   // every copy has landed: the rings are free
  const int wcols = nvs * VEC;
  double* comb = reinterpret_cast<double*>(smem);   // [SB][NB][wcols] strip sums of the axpy warps
  if (axpy) {
    const int st = warp - 2 - a.SA;
#pragma unroll
    for (int q = 0; q < NB; ++q)
#pragma unroll
      for (int t = 0; t < TV; ++t)
#pragma unroll
        for (int l = 0; l < VEC; ++l) {
          const int e = (lane + 32 * t) * VEC + l;
          if (e < wcols) {
            double v;
            if constexpr (FF) v = (double)acc[q][t][l] + (double)accl[q][t][l];
            else v = kF32 ? (double)ahi[q][t][l] + (double)alo[q][t][l] : (double)acc[q][t][l];
            comb[((size_t)st * NB + q) * wcols + e] = v;
          }
        }
  }
  __syncthreads();
  // fixed-order sum of the SB warps' strip sums -> g[cr][q][s0 + e]
  const int64_t ncol = s1 - s0;
  for (int64_t e = tid; e < ncol; e += blockDim.x) {
    const double sc = a.colscale ? (double)a.colscale[s0 + e] : 1.0;
#pragma unroll
    for (int q = 0; q < NB; ++q) {
      double sum = 0.0;
      for (int w = 0; w < a.SB; ++w) sum += comb[((size_t)w * NB + q) * wcols + e];
      a.g[((size_t)cr * NB + q) * p + s0 + e] = sum * sc;
    }
  }
}

}  // namespace relax
