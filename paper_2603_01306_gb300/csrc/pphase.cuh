// p-phase: everything an iteration does on p-vectors, in one cooperative launch.
//
//   P0  G^t = sum of the per-cluster X'r partials; a = -G^t/(2 lambda2) (the
//       argument of g* in Psi, since X'zeta = -G^t); |beta^t| statistics.
//   S1  TopSum_{kbar} H_M(|a_Jf|) of Lemma 4.2 through its variational form
//       TopSum_k(h) = min_t k t + sum_j (h_j - t)_+ at t = the kbar-th largest h,
//       found by a radix select over key bits (32 candidates per round, one per
//       lane).  The certification and the standalone g* use the exact keys of
//       the values; the loop selects on FP32-rounded keys, which makes the sum an
//       upper bound within FP32 rounding (Psi stays a valid bound).
//   S2  g_N(beta^t) (Thm 4.4 / Algorithm 1): the water level w of Algorithm 1
//       is the root of sum_j min(|beta_j|, w) = kbar w; a multisection over the
//       bits of w brackets it, an exact FP64 closed-form step finishes it:
//       w = S_below / (kbar - N_above), g = (sum_J1 b^2 + sum_{|b|>w} b^2 + w S_below)/2.
//   D   Phi, Psi, gap; best bounds; gap-based restart (Sec. 3.4); stop test.
//   P1  v = y^t - s grad F at y^t (FISTA, Beck 2017 Sec. 10.7).
//   S3  prox of rho g_N (Algorithm 2 + Eq. prox:gN).  The pooled block of
//       Algorithm 2 is described by one threshold c >= 0: with
//       w(c) = min(c/rho, M) and z_j(c) = min((|v_j| - c)_+ / w(c), 1), c is the
//       root of sum_Jf z_j(c) = kbar (c = 0 when the budget is slack), and
//          beta_j = sign(v_j) max(0, min(|v_j| - c, |v_j|/(1+rho), M))   on Jf,
//       clip(v_j/(1+rho), +-M) on J1, 0 on J0.  Coordinates with z_j = 1 are the
//       positions before the pooled block; those with 0 < z_j < 1 form the block.
//       The root is bracketed by a multisection over the bits of c and finished
//       by an exact FP64 closed form on the breakpoint-free piece:
//          c = rho S_mid / (kbar - N_top + rho N_mid)           (c <= rho M)
//          c = (S_mid - M (kbar - N_top)) / N_mid              (c >  rho M)
//   P2  beta^{t+1}.
//
// Multisection rounds evaluate FP32-rounded values; every decision that fixes
// an output (classification against a threshold, closed forms, sums) is FP64.
// Grid-wide steps use a bounded barrier (the grid is co-resident: cooperative
// launch sized by occupancy).  Round counters are exact integer atomics (the
// z-sums in 32.32 fixed point), so every block takes identical decisions; FP64
// sums go through per-block partials summed in a fixed order (deterministic).
#pragma once
#include <cmath>
#include <cstring>
#include <type_traits>

#include "common.cuh"
#include "xpass.cuh"

namespace relax {

constexpr int PQ = 32;          // candidates per multisection round (one per lane)
constexpr int PBLOCK = 256;
constexpr int PNW = PBLOCK / 32;
constexpr int PEPT = 4;         // max elements per thread
constexpr int PEPT_CLUSTER = 8; // the same for the cluster-per-problem batched launch
constexpr int NFIELD = 8;       // round accumulator fields
constexpr int ACC_STRIDE = NFIELD * PQ;
constexpr int NBP = 10;         // doubles per block partial
constexpr int MAX_POLISH = 8;

enum PMode : int { PM_ITER = 0, PM_EVAL = 1, PM_PROX = 2, PM_GVAL = 3, PM_GSTAR = 4 };

// accumulator fields
enum : int { F_S1 = 0, F_S2Z = 1, F_S2C = 2, F_S3Z = 3, F_S3CM = 4, F_S3CT = 5, F_S3NZ = 6 };

struct IterState {
  PassState ps;                 // the pass's view; ps.beta == beta_cur
  void* beta_prev;
  void* beta_cur;
  void* G_prev;
  void* G_cur;
  void* z_prev;
  void* z_cur;
  void* beta_best;              // argmin Phi so far
  void* beta_dbest;             // beta whose induced zeta gave max Psi
  void* z_dbest;                // z^t = X beta^t of that iterate (its dual point zeta = -grad F(z))
  double tau;                   // FISTA t_k
  double gap_ref;               // gap at the start of the current restart epoch
  double phi_best, psi_best;
  double phi_t, psi_t, g_t, c_last;
  double tol;                   // stop when (Phi_best - Psi_best) <= tol * max(1, |Phi_best|)
  int iter, restarts, have_ref, done, kbar, pbar, n_nz, n_top;
  double t1_last, w2_last;      // S1's t* and S2's water level of the last iteration (0: none)
  double stall_gap;             // best gap when it last fell by 10%
  int stall_iter;               // iteration of that fall
  int stalled;                  // 1: the loop stopped on the stall rule
  int cut_rule;                 // dynamic termination of Sec. 5.3: 1 Phi <= cutoff, 2 Psi >= cutoff
  int cutoff_on;                // dynamic termination against `cutoff` (0: off)
  double cutoff;                // the incumbent's objective f(X b) + lambda2 ||b||^2
  // step rule (backtracking, Beck Sec. 10.4.2): the current L, the rho of the
  // prox that produced beta^t, and what the sufficient-decrease test of the
  // pending trial point needs: <grad F(y), x - y>, ||x - y||^2 and X y (F(y)
  // is summed from it with the next iteration's loss terms), with y and its
  // gradient kept for a retry
  double Lk, rho_last, dgy, dxy2;
  void* y_keep;
  void* gy_keep;
  void* zy_keep;                // n: X y of the pending test
  int bt_pending;               // 1: beta^t is a trial point whose test is pending
  int backtracks;               // retries so far (each doubles L)
  unsigned long long bar_base;  // grid-barrier counter value at the start of a launch
};

// Scalars of a launch that follow from lambda2, M, the step and eta: taken
// once on the host (FP64 on this GPU is slow enough that a chain of scalar
// divisions in one thread shows in every iteration).
struct PConst {
  double inv2l;      // 1 / (2 lambda2)
  double Mtol;       // M (1 + 1e-6): dom g with a relative tolerance
  double inv1r;      // 1 / (1 + rho)
  double kTc;        // (1 + rho) / rho: T(c) = c kTc for c <= rho M
  double rhoM;       // rho M
  float M, inv2l_f, s_f, M1r_f, rr_f, inv_rho_f;   // FP32 forms (M (1 + rho), rho / (1 + rho))
  uint32_t krho;     // FP32 key of rhoM rounded up
};
__host__ __device__ inline PConst pconst_make(double lambda2, double M, double step, double rho) {
  PConst k;
  k.inv2l = 1.0 / (2.0 * lambda2);
  k.Mtol = M * (1.0 + 1e-6);
  k.inv1r = 1.0 / (1.0 + rho);
  k.kTc = (1.0 + rho) / rho;
  k.rhoM = rho * M;
  k.M = (float)M;
  k.inv2l_f = (float)k.inv2l;
  k.s_f = (float)step;
  k.M1r_f = (float)(M * (1.0 + rho));
  k.rr_f = (float)(rho / (1.0 + rho));
  k.inv_rho_f = (float)(1.0 / rho);
#ifdef __CUDA_ARCH__
  const float ru = __double2float_ru(k.rhoM);
#else
  float ru = (float)k.rhoM;
  if ((double)ru < k.rhoM) ru = std::nextafter(ru, INFINITY);
#endif
  uint32_t bits;
  memcpy(&bits, &ru, 4);
  k.krho = bits;
  return k;
}

struct PArgs {
  PConst kc;                    // pconst_make(lambda2, M, step, rho) of this launch
  int mode;
  int loss;
  int64_t p;
  int k;                        // cardinality
  double lambda2, M, step, rho, eta, tol;
  int max_iters;
  int stall_min;                // stall rule's least window (0: off)
  int method;                   // 0 FISTA, 1 PGD (the convergence study of Sec. 5.2)
  int restart_rule;             // 0 duality gap (Sec. 3.4), 1 function value, 2 none
  int backtrack;                // 0 fixed step 1/L, 1 backtracking from L/64
  const int8_t* fix;            // NULL = root
  const void* part;             // [ncl][NB][p] doubles
  int ncl, NB;
  const double* lossp;          // [n][2] per-row loss terms (certification); NULL: from z and y
  const double* y;              // n: response (loss terms from z^t in the loop)
  int64_t n;
  IterState* st;
  const void* vin;              // PROX: v; GVAL: beta; GSTAR: alpha; EVAL: beta_primal
  void* vout;                   // PROX output
  int* counts;                  // PROX: {n_top, n_nz}
  double* out;                  // EVAL: {Phi, Psi}; GVAL: g; GSTAR: g*
  int fast_s1;                  // select the kbar-th largest |a| on FP32 keys (loop)
  unsigned long long* acc;      // [3][ACC_STRIDE], zero between launches
  double* bpart;                // [2][gridDim][NBP]
  unsigned long long* bar;      // grid barrier counter
  unsigned long long bar_base;  // used when st == NULL
  int* status;
  uint64_t limit_ns;
  // Segmented launch (batched node solves, PM_ITER): seg_blocks > 0 splits
  // the grid into segments of seg_blocks CTAs; segment s works on node
  // seg_node[s] with its own state st[node], accumulators acc + node * 3 *
  // ACC_STRIDE, block partials bpart + node * 2 * seg_blocks * NBP, barrier
  // counter bar[node], fixings fix + node * fix_stride, and the gradients of
  // its column, part + s * part_stride.  seg_blocks = 0: one problem, the
  // whole grid.
  int seg_blocks;
  const int* seg_node;
  int64_t fix_stride, part_stride;
  // cluster = 1 (segmented launches only): every segment is one thread-block
  // cluster of seg_blocks CTAs, whose hardware barrier replaces the counter
  // barrier; segments are independent, so the grid needs no co-residency
  int cluster;
};

template <typename T> __device__ __forceinline__ T huber_d(T a, T M) {
  a = a < (T)0 ? -a : a;
  return a <= M ? (T)0.5 * a * a : M * a - (T)0.5 * M * M;
}

template <typename KT>
__device__ __forceinline__ KT cand(KT lo, KT hi, int q) {
  // lo + 1 + floor((hi - lo - 1) (q+1) / (PQ+1)), strictly inside (lo, hi) when hi - lo >= 2
  const KT d = hi - lo - 1;
  const KT qq = (KT)(q + 1);
  return lo + 1 + (d / (KT)(PQ + 1)) * qq + ((d % (KT)(PQ + 1)) * qq) / (KT)(PQ + 1);
}

// First-round candidates around the previous iteration's threshold key kc:
// lane q sits at kc - 2^(15-q) (q < 16), kc (q = 16), kc + 2^(q-17) (q > 16),
// offsets in units of 2^shift keys, clamped into (lo, hi).  The thresholds move
// little from one iteration to the next, so after this round the bracket is
// about as wide as the move; the rounds that follow split it uniformly.  Any
// candidates inside (lo, hi) keep the bracket's invariant, so the result is
// the same as from uniform rounds.
template <typename KT>
__device__ __forceinline__ KT warm_cand(KT kc, KT lo, KT hi, int q, int shift) {
  long long off = q < 16 ? -(1ll << (15 - q)) : (q == 16 ? 0ll : (1ll << (q - 17)));
  long long x = (long long)kc + off * (1ll << shift);
  if (x <= (long long)lo) x = (long long)lo + 1;
  if (x >= (long long)hi) x = (long long)hi - 1;
  return (KT)x;
}

// Float-float sums (Knuth's TwoSum; about 48 significant bits from FP32
// instructions).  This GPU issues FP64 arithmetic, comparisons and
// conversions at about 1.6 lanes per clock per SM against about 112 for FP32
// (measured), so the loop's per-coordinate work on FP32 data (the FAST
// instantiation) is FP32 with float-float sums.
struct ffs {
  float hi, lo;
};
// s += x
__device__ __forceinline__ void ff_acc(ffs& s, float x) {
  const float t = s.hi + x;
  const float bp = t - s.hi;
  s.lo += (s.hi - (t - bp)) + (x - bp);
  s.hi = t;
}
// s += x for an FP64 x (split into two floats first)
__device__ __forceinline__ void ff_acc(ffs& s, double x) {
  const float h = (float)x;
  ff_acc(s, h);
  s.lo += (float)(x - (double)h);
}
// a + b, renormalised; symmetric in a and b (every lane of a butterfly gets
// the same bits)
__device__ __forceinline__ ffs ff_add(ffs a, ffs b) {
  const float t = a.hi + b.hi;
  const float bp = t - a.hi;
  const float e = (a.hi - (t - bp)) + (b.hi - bp);
  const float lo = e + (a.lo + b.lo);
  const float h = t + lo;
  return ffs{h, lo - (h - t)};
}
__device__ __forceinline__ ffs ff_of(double x) {
  const float h = (float)x;
  return ffs{h, (float)(x - (double)h)};
}
__device__ __forceinline__ bool is_zero_bits(double x) { return (__double_as_longlong(x) << 1) == 0; }

// The logistic loss terms of one row in FP32 (the FAST loop), t = y z:
// log(1 + exp(-t)), and the entropy -(u log u + v log v) of u = 1/(1 + e^t),
// v = 1 - u, written with e = exp(-|t|) <= 1 and L = log1p(e) so that
// neither term loses its small part when the sigmoid saturates.
__device__ __forceinline__ void logistic_terms_f(float t, float& f, float& h) {
  const float s = fabsf(t);
  const float e = expf(-s);
  const float L = log1pf(e);
  f = fmaxf(-t, 0.f) + L;
  const float big = 1.f / (1.f + e), small = e * big;   // the two probabilities
  // t >= 0: u = small (pays s + L), v = big (pays L); t < 0 the other way
  h = small * (s + L) + big * L;
}

// One multisection decision, taken by every warp on its own: lane q holds
// candidate x (non-decreasing in q) and `ge`, whether its field reaches the
// target, which holds on a prefix of the lanes (the fields do not increase
// with the candidate).  The bracket's new lower end is the largest candidate
// with ge, its upper end the smallest without; qlo / qhi are their lanes (-1 /
// 32: none).
template <typename KT>
__device__ __forceinline__ void bracket_step(KT x, bool ge, KT& lo, KT& hi, int& qlo, int& qhi) {
  const unsigned b = __ballot_sync(0xffffffffu, ge);
  qlo = b ? 31 - __clz(b) : -1;
  qhi = ~b ? __ffs(~b) - 1 : 32;
  const KT xlo = __shfl_sync(0xffffffffu, x, qlo >= 0 ? qlo : 0);
  const KT xhi = __shfl_sync(0xffffffffu, x, qhi < 32 ? qhi : 0);
  if (qlo >= 0 && xlo > lo) lo = xlo; else qlo = -1;
  if (qhi < 32 && xhi < hi) hi = xhi; else qhi = 32;
}

__device__ __forceinline__ unsigned long long fixp(float z) {
  return __float2ull_rz(z * 4294967296.0f);
}
__device__ __forceinline__ unsigned long long fixp(double z) {
  return __double2ull_rz(z * 4294967296.0);
}

// The hardware barrier of a thread-block cluster, every thread of every CTA
// of the cluster taking part; release / acquire at cluster scope orders the
// CTAs' global-memory traffic around it, as the counter barrier does for a
// cooperative grid.
__device__ __forceinline__ void cluster_barrier() {
  asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}

// TV: element type of the p-vectors (double in the loop and certification;
// float or double for the standalone entry points).  EPT: elements per thread
// (at most), so one CTA covers PBLOCK * EPT coordinates.  BT: the backtracking
// step rule is compiled in (its test and retry cost registers that the
// fixed-step loop does not pay).  CL: the cluster-per-problem launch, whose
// sums go through distributed shared memory.  FAST (the loop on FP32 data,
// PM_ITER only): the per-coordinate arithmetic in FP32 with float-float
// sums; FP64 only where beta^t or beta^{t-1} is nonzero (the iterate's FP64
// accumulation), for the prox outputs that are nonzero, and per row of the
// loss.  Every threshold decision stays exact for the values it classifies.
template <typename TV, int EPT = PEPT, bool BT = false, bool CL = false, bool FAST = false>
__global__ void __launch_bounds__(PBLOCK) pphase_kernel(const PArgs a_in) {
  static_assert(!FAST || (sizeof(TV) == 8 && !BT), "FAST: FP64 iterates, fixed step");
  // S1 keys: FP32 or FP64 bit patterns of |a|
  using KG = typename std::conditional<FAST, uint32_t, unsigned long long>::type;
  using KV = uint32_t;             // FP32 keys of the S2 / S3 thresholds
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  // this CTA's problem: the whole grid, or its segment of a batched launch
  const int nbk = a_in.seg_blocks > 0 ? a_in.seg_blocks : (int)gridDim.x;
  const int seg = (int)blockIdx.x / nbk;
  const int lbk = (int)blockIdx.x - seg * nbk;
  PArgs a = a_in;
  if (a_in.seg_blocks > 0) {
    const int node = a_in.seg_node ? a_in.seg_node[seg] : seg;
    a.st = a_in.st + node;
    a.acc = a_in.acc + (size_t)node * 3 * ACC_STRIDE;
    a.bpart = a_in.bpart + (size_t)node * 2 * nbk * NBP;
    a.bar = a_in.bar + node;
    if (a_in.fix) a.fix = a_in.fix + (size_t)node * a_in.fix_stride;
    a.part = static_cast<const double*>(a_in.part) + (size_t)seg * a_in.part_stride;
  }
  const int nthr = nbk * PBLOCK;
  const int gt = lbk * PBLOCK + tid;
  const int mode = a.mode;
  IterState* st = a.st;

  __shared__ unsigned long long red_u[PNW][NFIELD * PQ];
  __shared__ unsigned long long sh_acc[NFIELD * PQ];
  __shared__ double red_d[PNW][NBP];
  __shared__ double sh_tot[NBP];
  __shared__ int sh_done;
  // cluster launches: this CTA's partial of each grid-wide sum, read by the
  // cluster's CTAs from distributed shared memory (two buffers, alternating:
  // a buffer is rewritten only after the next barrier, which every CTA
  // reaches after its reads of the previous use)
  __shared__ unsigned long long cl_u[2][NFIELD * PQ];
  __shared__ double cl_d[2][NBP];
  __shared__ float2 red_f[PNW][NBP];
  __shared__ float2 cl_f[2][NBP];

  if (tid == 0) sh_done = (st != nullptr) ? st->done : 0;
  __syncthreads();
  if (sh_done) return;   // uniform: every block reads the same flag
  // the host plans FAST for the loop and the certificate's evaluation only
  if (FAST && !((a_in.mode == PM_ITER && st != nullptr) || (a_in.mode == PM_EVAL && st == nullptr))) {
    if (blockIdx.x == 0 && tid == 0) atomicCAS(a_in.status, ST_OK, ST_INTERNAL);
    return;
  }
  // the node's state, read once into shared memory: the scalar stages below
  // (taken by thread 0) would otherwise wait on one global load after another
  __shared__ IterState sst;
  if (st) {
    const unsigned long long* sw = reinterpret_cast<const unsigned long long*>(st);
    unsigned long long* dw = reinterpret_cast<unsigned long long*>(&sst);
    for (int i = tid; i < (int)(sizeof(IterState) / 8); i += PBLOCK) dw[i] = sw[i];
  }
  __syncthreads();
  const IterState* sr = st ? &sst : nullptr;   // reads; the epilogue writes st

  const unsigned long long bar0 = st ? sr->bar_base : a.bar_base;
  int nbar = 0;
  bool alive = true;
  auto barrier = [&]() {
    ++nbar;
    if (CL) {
      cluster_barrier();
      return;
    }
    if (alive && !grid_barrier(a.bar, bar0 + (unsigned long long)nbar * nbk, a.limit_ns, a.status))
      alive = false;
  };
  int nstep = 0;
  // grid-wide deterministic FP64 sum of NV values: block partials summed by
  // lane (block b on lane b mod 32) and a warp butterfly, the same order for
  // the global-memory partials of a cooperative grid and the distributed
  // shared memory of a cluster
  auto gsum = [&](double* v, int nv) {
    const int buf = nstep & 1;
    double* bp = CL ? nullptr : a.bpart + (size_t)buf * nbk * NBP;
    ++nstep;
    for (int i = 0; i < nv; ++i) {
      double s = warp_sum(v[i]);
      if (lane == 0) red_d[warp][i] = s;
    }
    __syncthreads();
    if (tid < nv) {
      double s = 0.0;
      for (int w = 0; w < PNW; ++w) s += red_d[w][tid];
      if (CL) cl_d[buf][tid] = s;
      else bp[(size_t)lbk * NBP + tid] = s;
    }
    barrier();
    for (int c = warp; c < nv; c += PNW) {
      double s = 0.0;
      if (CL) {
        if (lane < nbk) s = ld_cluster_f64(mapa(&cl_d[buf][c], (uint32_t)lane));
      } else {
        for (int b = lane; b < nbk; b += 32) s += __ldcg(bp + (size_t)b * NBP + c);
      }
      s = warp_sum(s);
      if (lane == 0) sh_tot[c] = s;
    }
    __syncthreads();
    for (int i = 0; i < nv; ++i) v[i] = sh_tot[i];
    __syncthreads();
  };
  // the same over float-float partials (FAST): a warp butterfly, the warps in
  // order, the blocks' partials (two floats each) by lane and a butterfly;
  // the totals in FP64
  auto gsum_ff = [&](ffs* v, int nv, double* out) {
    const int buf = nstep & 1;
    float2* bp = CL ? nullptr : reinterpret_cast<float2*>(a.bpart + (size_t)buf * nbk * NBP);
    ++nstep;
    for (int i = 0; i < nv; ++i) {
      ffs s = v[i];
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        const ffs t{__shfl_xor_sync(0xffffffffu, s.hi, o), __shfl_xor_sync(0xffffffffu, s.lo, o)};
        s = ff_add(s, t);
      }
      if (lane == 0) red_f[warp][i] = make_float2(s.hi, s.lo);
    }
    __syncthreads();
    if (tid < nv) {
      ffs s{red_f[0][tid].x, red_f[0][tid].y};
      for (int w = 1; w < PNW; ++w) s = ff_add(s, ffs{red_f[w][tid].x, red_f[w][tid].y});
      if (CL) cl_f[buf][tid] = make_float2(s.hi, s.lo);
      else bp[(size_t)lbk * NBP + tid] = make_float2(s.hi, s.lo);
    }
    barrier();
    for (int c = warp; c < nv; c += PNW) {
      ffs s{0.f, 0.f};
      if (CL) {
        if (lane < nbk) {
          const uint32_t ra = mapa(&cl_f[buf][c], (uint32_t)lane);
          float hi, lo;
          asm volatile("ld.shared::cluster.v2.f32 {%0, %1}, [%2];" : "=f"(hi), "=f"(lo) : "r"(ra) : "memory");
          s = ffs{hi, lo};
        }
      } else {
        for (int b = lane; b < nbk; b += 32) {
          const float2 q = __ldcg(bp + (size_t)b * NBP + c);
          s = ff_add(s, ffs{q.x, q.y});
        }
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        const ffs t{__shfl_xor_sync(0xffffffffu, s.hi, o), __shfl_xor_sync(0xffffffffu, s.lo, o)};
        s = ff_add(s, t);
      }
      if (lane == 0) sh_tot[c] = (double)s.hi + (double)s.lo;
    }
    __syncthreads();
    for (int i = 0; i < nv; ++i) out[i] = sh_tot[i];
    __syncthreads();
  };
  int nround = 0;
  // publish per-lane round fields (lane = candidate) and fetch the grid totals
  auto round_reduce = [&](unsigned long long (&f)[NFIELD], int nf) {
    const int buf = nround & 1;
    unsigned long long* accb = a.acc + (size_t)(nround % 3) * ACC_STRIDE;
    unsigned long long* accz = a.acc + (size_t)((nround + 1) % 3) * ACC_STRIDE;
    ++nround;
    for (int i = 0; i < nf; ++i) red_u[warp][i * PQ + lane] = f[i];
    __syncthreads();
    for (int t = tid; t < nf * PQ; t += PBLOCK) {
      unsigned long long s = 0;
      for (int w = 0; w < PNW; ++w) s += red_u[w][t];
      if (CL) cl_u[buf][t] = s;
      else if (s) atomicAdd(accb + t, s);
    }
    if (!CL && lbk == 0)
      for (int t = tid; t < ACC_STRIDE; t += PBLOCK) accz[t] = 0ull;
    barrier();
    if (CL) {
      for (int t = tid; t < nf * PQ; t += PBLOCK) {
        const uint32_t loc = smem_u32(&cl_u[buf][t]);
        unsigned long long s = 0;
#pragma unroll 4
        for (int r = 0; r < nbk; ++r) {
          uint32_t ra;
          asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(ra) : "r"(loc), "r"(r));
          s += ld_cluster_u64(ra);
        }
        sh_acc[t] = s;
      }
    } else {
      for (int t = tid; t < nf * PQ; t += PBLOCK) sh_acc[t] = __ldcg(accb + t);
    }
    __syncthreads();
  };

  const int64_t p = a.p;
  const double M = a.M;
  const double lam2 = a.lambda2;
  // the step of this iteration's prox: 1/L, or 1/L_k under backtracking
  // (doubled below when the pending trial point fails its test)
  double step = a.step;
  double rho = a.rho;
  if (BT && mode == PM_ITER && a.backtrack) {
    step = 1.0 / sr->Lk;
    rho = 2.0 * lam2 * step;
  }
  const TV Mv = (TV)M;

  // ---------------------------------------------------------------- P0
  const TV* bcur = nullptr;
  const TV* bprev = nullptr;
  const double* Gprev = nullptr;
  double* Gcur = nullptr;
  if (mode == PM_ITER) {
    bcur = static_cast<const TV*>(sr->beta_cur);
    bprev = static_cast<const TV*>(sr->beta_prev);
    Gprev = static_cast<const double*>(sr->G_prev);
    Gcur = static_cast<double*>(sr->G_cur);
  } else if (mode == PM_EVAL || mode == PM_GVAL) {
    bcur = static_cast<const TV*>(a.vin);
  }
  const double* part = static_cast<const double*>(a.part);
  // S1 keys: FP64 patterns when the values are FP64 and exactness is asked for
  const bool key64 = !FAST && !a.fast_s1 && (mode == PM_EVAL || sizeof(TV) == 8);
  // FAST: the FP32 forms of the scalars
  const double inv2l = a.kc.inv2l;
  const double Mtol = a.kc.Mtol;
  const float M32 = a.kc.M;
  const float inv2l32 = a.kc.inv2l_f;
  // the step's constants (the backtracking variant changes the step in flight)
  PConst kr = a.kc;
  if (BT && mode == PM_ITER && a.backtrack) kr = pconst_make(lam2, M, step, rho);

  int8_t fx[EPT];
  KG ka[EPT];        // S1 keys: |a| on Jf, 0 elsewhere
  TV bm[EPT];        // S2: |beta| on Jf, 0 elsewhere
  float bmf[EPT];    // the same, rounded to FP32 for the multisection rounds
  TV bt[EPT];        // beta^t
  double gg[EPT];    // G^t
  double gy[EPT];    // logistic: X' grad F at the tentative y^t
  // sums: 0 sum_J1 H(a), 1 sum_J1 b^2, 2 sum_Jf |b|, 3 sum_Jf b^2, 4 nnz_Jf(b),
  //       5 domain violations, 6 non-finite, 7 sum_Jf H(a), 8 F(z), 9 -F*(-zeta)
  double s0[NBP] = {0, 0, 0, 0, 0, 0, 0, 0, 0, 0};
  double fy_sum = 0.0;   // backtracking: F at the kept momentum point
  ffs lf8{0.f, 0.f}, lf9{0.f, 0.f};   // FAST, logistic: the loss terms in float-float
  if (a.lossp) {
    // per-row loss terms written by the certification pass
    for (int64_t i = gt; i < a.n; i += nthr) {
      s0[8] += a.lossp[2 * i];
      s0[9] += a.lossp[2 * i + 1];
    }
  } else if (mode == PM_ITER) {
    // loss terms of Eq. 6-7 at z^t = X beta^t, zeta = -grad F(z^t), in FP64;
    // with a backtracking test pending, also F at the kept momentum point
    const double* zt = static_cast<const double*>(sr->z_cur);
    const double* zy = (BT && a.backtrack && sr->bt_pending) ? static_cast<const double*>(sr->zy_keep) : nullptr;
    for (int64_t i = gt; i < a.n; i += nthr) {
      const double yi = a.y[i], zi = zt[i];
      if (FAST && a.loss != 0) {
        float f, hh;
        logistic_terms_f((float)(yi * zi), f, hh);
        ff_acc(lf8, f);
        ff_acc(lf9, hh);
        continue;
      }
      if (a.loss == 0) {
        const double d = zi - yi, zeta = -2.0 * d;
        s0[8] += d * d;
        s0[9] += zeta * yi - 0.25 * zeta * zeta;
        if (zy) {
          const double dy = zy[i] - yi;
          fy_sum += dy * dy;
        }
      } else {
        s0[8] += softplus_neg(yi * zi);
        s0[9] += entropy_of(yi * zi);
        if (zy) fy_sum += softplus_neg(yi * zy[i]);
      }
    }
  }
  const bool need_a = (mode == PM_ITER || mode == PM_EVAL || mode == PM_GSTAR);
  const bool need_b = (mode == PM_ITER || mode == PM_EVAL || mode == PM_GVAL);
  float gf[EPT];     // FAST: G^t in FP32
  float gyf[EPT];    // FAST: the logistic second gradient in FP32
  ffs sf[NBP];       // FAST: the sums s0 as float-float
  if constexpr (FAST) {
    // The bulk of the coordinates (beta^t_j = 0, not fixed) costs FP32 work
    // only; the terms of Phi and Psi that are not zero there (fixed-in
    // coordinates, nonzero beta^t_j, and the whole free set when the
    // cardinality budget is slack) are FP64, as are their sums (float-float).
    int c_nnz = 0, c_dom = 0, c_bad = 0;
#pragma unroll
    for (int i = 0; i < NBP; ++i) sf[i] = ffs{0.f, 0.f};
#pragma unroll
    for (int e = 0; e < EPT; ++e) {
      const int64_t j = (int64_t)gt + (int64_t)e * nthr;
      fx[e] = 0; ka[e] = 0; bmf[e] = 0.f; bt[e] = (TV)0; gf[e] = 0.f; gyf[e] = 0.f;
      if (j >= p) { fx[e] = -2; continue; }
      const int8_t f = a.fix ? a.fix[j] : (int8_t)0;
      fx[e] = f;
      double G = 0.0, Gy = 0.0;   // partials summed in FP64, fixed order
      for (int c = 0; c < a.ncl; ++c) {
        G += part[((int64_t)c * a.NB) * p + j];
        if (a.NB > 1) Gy += part[((int64_t)c * a.NB + 1) * p + j];
      }
      if (mode == PM_ITER) Gcur[j] = G;
      gf[e] = (float)G;
      if (a.NB > 1) gyf[e] = (float)Gy;
      const float aa = fabsf(gf[e]) * inv2l32;   // |a_j| in FP32 (keys), a = -G / (2 lambda2)
      if (!isfinite(aa)) ++c_bad;
      if (f > 0) ff_acc(sf[0], huber_d<double>(fabs(G) * inv2l, M));
      if (f == 0) ka[e] = key_of(aa);   // a slack budget's sum over the free set: in the finishing
      const TV b = bcur[j];
      bt[e] = b;
      if (!is_zero_bits((double)b)) {          // most coordinates of beta^t are zero
        const double bd = (double)b;
        const double ab = fabs(bd);
        if (!isfinite(bd)) ++c_bad;
        if (f > 0) { ff_acc(sf[1], bd * bd); if (ab > Mtol) ++c_dom; }
        else if (f < 0) ++c_dom;
        else {
          bmf[e] = (float)ab;
          ff_acc(sf[2], ab);
          ff_acc(sf[3], ab * ab);
          ++c_nnz;
          if (ab > Mtol) ++c_dom;
        }
      }
    }
    sf[4] = ffs{(float)c_nnz, 0.f};
    sf[5] = ffs{(float)c_dom, 0.f};
    sf[6] = ffs{(float)c_bad, 0.f};
    const bool own_loss = a.loss != 0 && !a.lossp && mode == PM_ITER;   // the float-float loss loop ran
    sf[8] = own_loss ? lf8 : ff_of(s0[8]);
    sf[9] = own_loss ? lf9 : ff_of(s0[9]);
  } else {
#pragma unroll
  for (int e = 0; e < EPT; ++e) {
    const int64_t j = (int64_t)gt + (int64_t)e * nthr;
    fx[e] = 0; ka[e] = 0; bm[e] = (TV)0; bmf[e] = 0.f; bt[e] = (TV)0; gg[e] = 0.0; gy[e] = 0.0;
    if (j >= p) { fx[e] = -2; continue; }
    const int8_t f = a.fix ? a.fix[j] : (int8_t)0;
    fx[e] = f;
    if (need_a) {
      double av;
      if (mode == PM_GSTAR) {
        av = (double)static_cast<const TV*>(a.vin)[j];
      } else {
        double G = 0.0, Gy = 0.0;   // cluster partials summed in FP64, fixed order
        for (int c = 0; c < a.ncl; ++c) {
          G += part[((int64_t)c * a.NB) * p + j];
          if (a.NB > 1) Gy += part[((int64_t)c * a.NB + 1) * p + j];
        }
        gg[e] = G;
        gy[e] = Gy;
        if (mode == PM_ITER) Gcur[j] = G;
        av = -G / (2.0 * lam2);
      }
      if (!isfinite(av)) s0[6] += 1.0;
      const double aa = fabs(av);
      if (f > 0) s0[0] += huber_d<double>(aa, M);
      if (f == 0) {
        ka[e] = key64 ? (KG)key_of(aa) : (KG)key_of((float)aa);
        s0[7] += huber_d<double>(aa, M);
      }
    }
    if (need_b) {
      const TV b = bcur[j];
      bt[e] = b;
      if (!isfinite((double)b)) s0[6] += 1.0;
      const TV ab = b < (TV)0 ? -b : b;
      if (f > 0) { s0[1] += (double)b * (double)b; if ((double)ab > M * (1.0 + 1e-6)) s0[5] += 1.0; }
      else if (f < 0) { if (b != (TV)0) s0[5] += 1.0; }
      else {
        bm[e] = ab;
        bmf[e] = (float)ab;
        s0[2] += (double)ab;
        s0[3] += (double)ab * (double)ab;
        if (ab > (TV)0) s0[4] += 1.0;
        if ((double)ab > M * (1.0 + 1e-6)) s0[5] += 1.0;
      }
    }
  }
  }
  const int kbar = st ? sr->kbar : 0;   // filled below for the standalone modes
  int kb = kbar, pb = st ? sr->pbar : 0;
  double tot[NBP];
  for (int i = 0; i < NBP; ++i) tot[i] = s0[i];
  // standalone modes need |J1| and |Jf|; reuse the sum for counts
  double cnt2[2] = {0, 0};
  if (!st) {
    for (int e = 0; e < EPT; ++e) {
      if (fx[e] > 0) cnt2[0] += 1.0;
      if (fx[e] == 0) cnt2[1] += 1.0;
    }
  }
  if constexpr (FAST) gsum_ff(sf, NBP, tot);
  else gsum(tot, NBP);
  if (!st) {
    gsum(cnt2, 2);
    kb = a.k - (int)cnt2[0];
    pb = (int)cnt2[1];
  }
  (void)kbar;
  const double Ftot = tot[8];
  const double Dtot = tot[9];
  const bool nonfinite = tot[6] > 0.0;
  // Backtracking (Beck Sec. 10.4.2): beta^t = prox at y^{t-1} with step 1/L_k
  // is accepted when F(X beta^t) <= F(y) + <grad F(y), beta^t - y> +
  // L_k/2 ||beta^t - y||^2 (with an FP64 rounding slack of 1e-12 |F(y)|);
  // otherwise L_k doubles and the prox is taken again from the kept y and
  // its gradient, and this iteration evaluates nothing else.
  bool retry = false;
  if (BT && mode == PM_ITER && a.backtrack && sr->bt_pending) {
    gsum(&fy_sum, 1);   // uniform: every block reads the same pending flag
    const double Fy = fy_sum;
    const double rhs = Fy + sr->dgy + 0.5 * sr->Lk * sr->dxy2 + 1e-12 * fmax(1.0, fabs(Fy));
    retry = Ftot > rhs;
    if (retry) {
      step = 0.5 / sr->Lk;
      rho = 2.0 * lam2 * step;
      kr = pconst_make(lam2, M, step, rho);
    }
  }

  // ------------------------------------------------------ S1 / S2 setup
  // The scalar decisions of each stage are taken by thread 0 and read by the
  // others from shared memory: FP64 on this GPU is slow enough that 256
  // copies of the same scalar arithmetic cost as much as the coordinates.
  struct ScA {
    double topsum, gval, w_closed;
    unsigned long long c2lo, kc1;
    unsigned kc2;
    int s1, s2, w_known, g_inf, warm1, warm2, slack;
  };
  __shared__ ScA sca;
  if (tid == 0) {
    ScA r{};
    if (need_a) {
      if (kb <= 0) r.topsum = 0.0;
      else if (pb <= kb) { r.topsum = tot[7]; r.slack = FAST; }   // FAST: summed in the finishing
      else r.s1 = 1;
    }
    // In the loop beta^t (t >= 1) is the prox output of the last iteration,
    // whose threshold c fixes its water level: stationarity of the prox in
    // beta_j and the water filling in z_j give |beta_j| = |v_j| - rho w on the
    // fractional coordinates, i.e. w = c / rho (M at most), the w of the
    // prox's own z_j(c).  g then needs one classification at w instead of
    // S2's rounds.
    const double c_prev = (mode == PM_ITER) ? sr->c_last : 0.0;
    r.w_known = mode == PM_ITER && sr->iter >= 1 && c_prev > 0.0 && isfinite(c_prev);
    r.w_closed = r.w_known ? fmin(c_prev / sr->rho_last, M) : 0.0;
    if (need_b) {
      const bool check_dom = (mode != PM_ITER) || (sr->iter == 0);
      if (check_dom && (tot[5] > 0.0 || (kb > 0 && tot[2] > M * (double)kb * (1.0 + 1e-6)) ||
                        (kb <= 0 && tot[2] > 0.0)))
        r.g_inf = 1;
      if (r.g_inf) r.gval = INFINITY;
      else if (kb <= 0) r.gval = 0.5 * tot[1];
      else if (tot[4] <= (double)kb) r.gval = 0.5 * (tot[1] + tot[3]);
      else if (!r.w_known) { r.s2 = 1; r.c2lo = (unsigned long long)tot[4]; }
    }
    // warm first rounds from the last iteration's t* and water level (loop only)
    const double t1p = (mode == PM_ITER) ? sr->t1_last : 0.0;
    const double w2p = (mode == PM_ITER) ? sr->w2_last : 0.0;
    r.warm1 = r.s1 && t1p > 0.0 && isfinite(t1p);
    r.warm2 = r.s2 && w2p > 0.0 && isfinite(w2p);
    r.kc1 = r.warm1 ? (key64 ? (unsigned long long)key_of(t1p) : (unsigned long long)key_of((float)t1p)) : 0ull;
    r.kc2 = r.warm2 ? key_of((float)w2p) : 0u;
    sca = r;
  }
  __syncthreads();
  bool s1 = sca.s1 != 0, s2 = sca.s2 != 0;
  double topsum = sca.topsum, gval = sca.gval;
  KG lo1 = 0, hi1 = key64 ? (KG)(KeyOf<double>::kInf + 1) : (KG)(KeyOf<float>::kInf + 1);
  KV lo2 = 0, hi2 = (KV)KeyOf<float>::kInf;
  unsigned long long c2lo = sca.c2lo, c2hi = 0;   // #{|b| > lo2}, #{|b| > hi2}
  const bool w_known = sca.w_known != 0;
  const double w_closed = sca.w_closed;
  const bool g_inf = sca.g_inf != 0;

  // ------------------------------------------------------- S1 / S2 rounds
  bool warm1 = sca.warm1 != 0;
  bool warm2 = sca.warm2 != 0;
  const KG kc1 = (KG)sca.kc1;
  const KV kc2 = (KV)sca.kc2;
  const int sh1 = key64 ? 29 : 0;   // FP64 keys: 29 more mantissa bits per FP32 step
  if (retry) { s1 = false; s2 = false; warm1 = false; warm2 = false; }
  auto cand1 = [&](int q) { return warm1 ? warm_cand<KG>(kc1, lo1, hi1, q, sh1) : cand<KG>(lo1, hi1, q); };
  auto cand2 = [&](int q) { return warm2 ? warm_cand<KV>(kc2, lo2, hi2, q, 0) : cand<KV>(lo2, hi2, q); };
  while (s1 || s2) {
    unsigned long long fld[NFIELD] = {0, 0, 0, 0, 0, 0, 0, 0};
    const KG x1 = s1 ? cand1(lane) : (KG)0;
    const KV x2 = s2 ? cand2(lane) : (KV)0;
    const float w2 = from_key(x2, 0.f);
    const float inv2 = s2 ? 1.0f / w2 : 0.f;
    if (s1) {
      // a key below the round's smallest candidate (candidates do not decrease
      // with the lane) counts for no lane: only the keys at or above it are
      // broadcast, which in a warm round are few
      const KG x1min = cand1(0);
#pragma unroll
      for (int e = 0; e < EPT; ++e) {
        unsigned act = __ballot_sync(0xffffffffu, ka[e] >= x1min);
        while (act) {
          const int src = __ffs(act) - 1;
          act &= act - 1u;
          const KG kv = __shfl_sync(0xffffffffu, ka[e], src);
          fld[F_S1] += (kv >= x1) ? 1ull : 0ull;
        }
      }
    }
    if (s2) {
      for (int src = 0; src < 32; ++src) {
#pragma unroll
        for (int e = 0; e < EPT; ++e) {
          const float b = __shfl_sync(0xffffffffu, bmf[e], src);
          if (b > 0.f) {
            const float z = b * inv2;
            fld[F_S2Z] += fixp(z < 1.f ? z : 1.f);
            fld[F_S2C] += (b > w2) ? 1ull : 0ull;
          }
        }
      }
    }
    round_reduce(fld, 3);
    if (s1) {
      // largest candidate with count >= kb -> new lo; smallest with count < kb
      // -> new hi.  A candidate x whose count is exactly kb ends the search:
      // for any t with exactly kb keys at or above it, kb H(t) +
      // sum (H(|a_j|) - H(t))_+ is the sum of the kb largest H(|a_j|)
      // (TopSum's variational form), so t* = x serves as well as the
      // kb-th largest key itself.
      const unsigned long long cnt = sh_acc[F_S1 * PQ + lane];
      int qlo, qhi;
      bracket_step<KG>(x1, cnt >= (unsigned long long)kb, lo1, hi1, qlo, qhi);
      const unsigned beq = __ballot_sync(0xffffffffu, cnt == (unsigned long long)kb);
      warm1 = false;
      if (beq) {
        lo1 = __shfl_sync(0xffffffffu, x1, 31 - __clz(beq));
        s1 = false;
      }
      if (hi1 - lo1 <= 1) s1 = false;
    }
    if (s2) {
      const unsigned long long thr = (unsigned long long)kb << 32;
      const unsigned long long cq = sh_acc[F_S2C * PQ + lane];
      int qlo, qhi;
      bracket_step<KV>(x2, sh_acc[F_S2Z * PQ + lane] >= thr, lo2, hi2, qlo, qhi);
      if (qlo >= 0) c2lo = __shfl_sync(0xffffffffu, cq, qlo);
      if (qhi < 32) c2hi = __shfl_sync(0xffffffffu, cq, qhi);
      warm2 = false;
      if (c2lo == c2hi || hi2 - lo2 <= 1) s2 = false;
    }
  }

  // ---------------------------------------------- exact S1 / S2 finishing
  // S1: t* = the kbar-th largest |a| (key lo1); TopSum = kbar H(t*) + sum (H(|a|) - H(t*))_+
  // S2: w on the bracket's piece, polished until the classification is stable.
  const bool fin1 = need_a && kb > 0 && pb > kb && !retry;
  const bool fins = FAST && sca.slack && !retry;   // the whole free set, in FP64 (it has at most kbar coordinates)
  // FP64 G_j: the loop's stored G^t, or the partials again (evaluation)
  auto G64 = [&](int64_t j) {
    if (mode == PM_ITER) return Gcur[j];
    double G = 0.0;
    for (int c = 0; c < a.ncl; ++c) G += part[((int64_t)c * a.NB) * p + j];
    return G;
  };
  // thread 0: the scalars of the finishing (the others read them below)
  __shared__ double shw[5];   // htstar, wcur, topsum, gval, wlast
  __shared__ int shw_pol2;
  double tstar = 0.0, wlo = 0.0, whi = 0.0, nprev = -1.0;   // thread 0's
  int npol = 0;
  if (tid == 0) {
    tstar = fin1 ? (key64 ? from_key((unsigned long long)lo1, 0.0) : (double)from_key((uint32_t)lo1, 0.f)) : 0.0;
    const bool p2 = need_b && !g_inf && kb > 0 && tot[4] > (double)kb && !retry;
    shw[0] = huber_d<double>(tstar, M);
    shw[1] = p2 ? (w_known ? w_closed : (double)from_key(hi2, 0.f)) : 0.0;
    shw[2] = topsum;
    shw[3] = gval;
    shw[4] = 0.0;
    shw_pol2 = p2;
    wlo = (double)from_key(lo2, 0.f);
    whi = (double)from_key(hi2, 0.f);
  }
  __syncthreads();
  const double htstar = shw[0];
  double wcur = shw[1];
  bool pol2 = shw_pol2 != 0;
  bool first = true;
  while (first || pol2) {
    double v[NBP] = {0, 0, 0, 0, 0, 0, 0, 0, 0, 0};
    if constexpr (FAST) {
      // only the coordinates at or above t* (FP32 keys: the others have
      // |a_j| < t*) and the nonzero |beta_j| contribute: FP64 for those
      ffs vf[5] = {{0.f, 0.f}, {0.f, 0.f}, {0.f, 0.f}, {0.f, 0.f}, {0.f, 0.f}};
      int nab = 0;
      if (first && fin1) {
        for (int e = 0; e < EPT; ++e) {
          // keys are FP32 |a| (within two ulps of the FP64 value): a margin
          // keeps every coordinate whose FP64 |a| exceeds t*
          if (fx[e] != 0 || ka[e] + 4u < (KG)lo1) continue;
          const int64_t j = (int64_t)gt + (int64_t)e * nthr;
          const double hv = huber_d<double>(fabs(G64(j)) * inv2l, M) - htstar;
          if (hv > 0.0) ff_acc(vf[0], hv);
        }
      }
      if (first && fins) {
        for (int e = 0; e < EPT; ++e) {
          if (fx[e] != 0) continue;
          const int64_t j = (int64_t)gt + (int64_t)e * nthr;
          ff_acc(vf[0], huber_d<double>(fabs(G64(j)) * inv2l, M));
        }
      }
      if (pol2) {
        for (int e = 0; e < EPT; ++e) {
          if (!(bmf[e] > 0.f)) continue;
          const double m = fabs((double)bt[e]);
          if (m > wcur) {
            ++nab;
            ff_acc(vf[3], m);
            ff_acc(vf[4], m * m);
          }
        }
      }
      vf[2] = ffs{(float)nab, 0.f};
      gsum_ff(vf, 5, v);
    } else {
    if (first && fin1) {
      const TV* av_src = mode == PM_GSTAR ? static_cast<const TV*>(a.vin) : nullptr;
      for (int e = 0; e < EPT; ++e) {
        if (fx[e] != 0) continue;
        const int64_t j = (int64_t)gt + (int64_t)e * nthr;
        const double aa = av_src ? fabs((double)av_src[j]) : fabs(gg[e]) / (2.0 * lam2);
        const double hv = huber_d<double>(aa, M) - htstar;
        if (hv > 0.0) v[0] += hv;
      }
    }
    if (pol2) {
      for (int e = 0; e < EPT; ++e) {
        if ((double)bm[e] > wcur) {
          v[2] += 1.0;
          v[3] += (double)bm[e];
          v[4] += (double)bm[e] * (double)bm[e];
        }
      }
    }
    gsum(v, 5);
    }
    if (tid == 0) {
      if (first && fin1) shw[2] = (double)kb * htstar + v[0];
      if (first && fins) shw[2] = v[0];
      if (pol2) {
        // classification at wcur: N_above, S_above, Q_above
        const double Nab = v[2], Sab = v[3], Qab = v[4];
        const double Sbel = tot[2] - Sab;
        if ((double)kb - Nab <= 0.5) {   // budget filled by coordinates above: no water level
          shw[3] = 0.5 * (tot[1] + tot[3]);
          shw_pol2 = 0;
        } else {
          const double wn = Sbel / ((double)kb - Nab);
          // the closed-form level classifies exactly: one pass (a coordinate
          // with |beta_j| = w adds w |beta_j| = beta_j^2 on either side)
          const bool stable = w_known || (Nab == nprev) || (wn > wlo && wn <= whi && c2lo == c2hi && npol == 0);
          if (stable || npol >= MAX_POLISH) {
            shw[3] = 0.5 * (tot[1] + Qab + wn * Sbel);
            shw[4] = wn;
            shw_pol2 = 0;
          } else {
            nprev = Nab;
            shw[1] = wn;
            ++npol;
          }
        }
      }
    }
    first = false;
    __syncthreads();
    pol2 = shw_pol2 != 0;
    wcur = shw[1];
  }
  topsum = shw[2];
  gval = shw[3];
  const double wlast = shw[4];   // the water level found (0: none)

  // ---------------------------------------------------------------- D
  // thread 0 evaluates Phi, Psi and the loop's decisions; the others read
  // what they need (stop, the best-iterate flags, the momentum)
  double phi = 0.0, psi = 0.0;
  bool stop = false, restart = false, imp_p = false, imp_d = false;
  double mu = 0.0, tau_new = 1.0, gap_ref = 0.0, phi_best = 0.0, psi_best = 0.0;
  int have_ref = 0, restarts = 0, stall_iter = 0, stalled = 0, cut_rule = 0;
  double stall_gap = 0.0;
  const int t = st ? sr->iter : 0;
  __shared__ double shd_mu;
  __shared__ int shd_flags;
  if (tid == 0) {
  if (mode == PM_ITER || mode == PM_EVAL) {
    phi = Ftot + 2.0 * lam2 * gval;
    psi = Dtot - 2.0 * lam2 * (tot[0] + topsum);
  }
  if (mode == PM_EVAL) {
    if (lbk == 0 && tid == 0) {
      a.out[0] = phi;
      a.out[1] = psi;
      if (nonfinite) atomicCAS(a.status, ST_OK, ST_NUMERIC);
    }
  } else if (mode == PM_GVAL) {
    if (lbk == 0 && tid == 0) a.out[0] = gval;
  } else if (mode == PM_GSTAR) {
    if (lbk == 0 && tid == 0) a.out[0] = tot[0] + topsum;
  }

  if (mode == PM_ITER && !retry) {
    const double tau = sr->tau;
    gap_ref = sr->gap_ref;
    have_ref = sr->have_ref;
    phi_best = sr->phi_best;
    psi_best = sr->psi_best;
    restarts = sr->restarts;
    if (nonfinite) stop = true;
    if (phi < phi_best) { phi_best = phi; imp_p = true; }
    if (psi > psi_best) { psi_best = psi; imp_d = true; }
    const double gap = phi - psi;
    if (a.method == 0 && a.restart_rule == 0) {         // duality-gap restart (Sec. 3.4)
      if (!have_ref) {
        if (isfinite(gap)) { gap_ref = gap; have_ref = 1; }
      } else if (t >= 1 && gap <= gap_ref / a.eta) {
        restart = true;
        gap_ref = gap;
        ++restarts;
      }
    } else if (a.method == 0 && a.restart_rule == 1) {  // function value (O'Donoghue and Candes)
      if (t > 1 && phi > sr->phi_t) {
        restart = true;
        ++restarts;
      }
    }
    if (a.method == 1) { mu = 0.0; tau_new = 1.0; }      // PGD: the prox step from beta^t itself
    else if (t == 0) { mu = 0.0; tau_new = tau; }
    else if (restart) { mu = 0.0; tau_new = 1.0; }
    else {
      const double tn = 0.5 * (1.0 + sqrt(1.0 + 4.0 * tau * tau));
      mu = (tau - 1.0) / tn;
      tau_new = tn;
    }
    if (isfinite(phi_best) && phi_best - psi_best <= sr->tol * fmax(1.0, fabs(phi_best))) stop = true;
    if (t >= a.max_iters) stop = true;
    // Stall rule: with the gap restarts of Sec. 3.4 the best gap keeps falling
    // (geometrically while the restarts fire, at least as 1/t^2 between them);
    // one that has not fallen by 10% over the last quarter of the run, and over
    // at least stall_min iterations, sits on the floor of the loop's
    // arithmetic, and further iterations cannot lower it.
    stall_gap = sr->stall_gap;
    stall_iter = sr->stall_iter;
    const double gbest = phi_best - psi_best;
    if (!(gbest >= 0.9 * stall_gap)) {
      stall_gap = gbest;
      stall_iter = t;
    } else if (a.stall_min > 0 && t - stall_iter >= max(a.stall_min, t / 4)) {
      stop = true;
      stalled = 1;
    }
    // Dynamic termination (Sec. 5.3): once Phi falls to the incumbent's
    // objective the node will not be pruned, so branch now; once Psi reaches
    // it the node is pruned.  Pruning wins when both hold.
    if (sr->cutoff_on) {
      if (isfinite(phi_best) && phi_best <= sr->cutoff) { stop = true; cut_rule = 1; }
      if (psi_best >= sr->cutoff) { stop = true; cut_rule = 2; }
    }
  }

    shd_mu = mu;
    shd_flags = (stop ? 1 : 0) | (imp_p ? 2 : 0) | (imp_d ? 4 : 0);
  }
  __syncthreads();
  mu = shd_mu;
  stop = (shd_flags & 1) != 0;
  imp_p = (shd_flags & 2) != 0;
  imp_d = (shd_flags & 4) != 0;

  // best iterates (also on the stopping iteration); for the best dual value the
  // loop's own dual point (z^t) is kept, so that the FP64 certificate
  // evaluates Psi at exactly that point
  if (mode == PM_ITER && (imp_p || imp_d)) {
    TV* bbest = static_cast<TV*>(sr->beta_best);
    TV* bdbest = static_cast<TV*>(sr->beta_dbest);
#pragma unroll
    for (int e = 0; e < EPT; ++e) {
      const int64_t j = (int64_t)gt + (int64_t)e * nthr;
      if (j >= p) continue;
      if (imp_p) bbest[j] = bt[e];
      if (imp_d) bdbest[j] = bt[e];
    }
    if (imp_d) {
      const double* zt = static_cast<const double*>(sr->z_cur);
      double* zb = static_cast<double*>(sr->z_dbest);
      for (int64_t i = gt; i < a.n; i += nthr) zb[i] = zt[i];
    }
  }

  // ---------------------------------------------------------------- P1
  const bool do_prox = (mode == PM_PROX) || (mode == PM_ITER && !stop);
  const bool keep = BT && mode == PM_ITER && a.backtrack;
  if (do_prox && keep && !retry) {
    // X y^t = (1 + mu) z^t - mu z^{t-1}, for the test of the next trial point
    const double* zc = static_cast<const double*>(sr->z_cur);
    const double* zp = static_cast<const double*>(sr->z_prev);
    double* zk = static_cast<double*>(sr->zy_keep);
    for (int64_t i = gt; i < a.n; i += nthr) zk[i] = (1.0 + mu) * zc[i] - mu * zp[i];
  }
  TV vv[EPT];
  TV mm[EPT];      // |v| on Jf
  float mmf[EPT];  // |v| rounded to FP32 (rounds)
  float ti[EPT];   // T^{-1}(|v|) in FP32: where coordinate j reaches z_j = 1
  double nzv = 0.0;
  double nbad = 0.0;   // standalone prox: non-finite inputs (the output is then all NaN)
  // FAST: bit e of `wide` set when v_j is FP64 (vv[e]: beta^t_j or
  // beta^{t-1}_j nonzero, or j fixed in the support); otherwise v_j is the
  // FP32 value -s gy_j with |v_j| = mmf[e] and its sign in bit e of `negm`
  unsigned wide = 0, negm = 0;
  if (do_prox && FAST) {
    // v_j = y_j - s gy_j: FP64 where beta^t_j or beta^{t-1}_j is nonzero (or
    // j is fixed in), FP32 elsewhere, where y_j = 0
    __shared__ float shv[2];   // mu, 1 + mu in FP32
    __shared__ int shv_mu0;
    if (tid == 0) {
      shv[0] = (float)mu;
      shv[1] = (float)(1.0 + mu);
      shv_mu0 = mu == 0.0;
    }
    __syncthreads();
    const float mu32 = shv[0], opm32 = shv[1], s32 = kr.s_f, M1r32 = kr.M1r_f, rr32 = kr.rr_f;
    const bool mu0 = shv_mu0 != 0;
    int c_nz = 0;
#pragma unroll
    for (int e = 0; e < EPT; ++e) {
      const int64_t j = (int64_t)gt + (int64_t)e * nthr;
      vv[e] = (TV)0; mmf[e] = 0.f; ti[e] = 0.f;
      if (j >= p) continue;
      const double b = (double)bt[e];
      const double bp = (double)bprev[j];
      float v32;
      if (fx[e] > 0 || !is_zero_bits(b) || !is_zero_bits(bp)) {
        double gyv;
        if (a.loss == 0) {
          gyv = mu0 ? Gcur[j] : (1.0 + mu) * Gcur[j] - mu * Gprev[j];
        } else if (mu0) {
          gyv = Gcur[j];
        } else {
          gyv = 0.0;
          for (int c = 0; c < a.ncl; ++c) gyv += part[((int64_t)c * a.NB + 1) * p + j];
        }
        const double v = (b + mu * (b - bp)) - step * gyv;   // the iterate's FP64 accumulation
        vv[e] = v;
        v32 = (float)v;
        wide |= 1u << e;
      } else {
        float gyv;
        if (a.loss == 0) gyv = mu0 ? gf[e] : opm32 * gf[e] - mu32 * (float)Gprev[j];
        else gyv = mu0 ? gf[e] : gyf[e];
        v32 = -(s32 * gyv);
      }
      if (v32 < 0.f) negm |= 1u << e;
      if (fx[e] == 0) {
        const float m = fabsf(v32);
        mmf[e] = m;
        ti[e] = m <= M1r32 ? m * rr32 : m - M32;
        if (m > 0.f) ++c_nz;
      }
    }
    nzv = (double)c_nz;
  } else if (do_prox) {
    const TV* vin = static_cast<const TV*>(a.vin);
    const TV muv = (TV)mu;
    const TV sv = (TV)step;
    TV* ykeep = keep ? static_cast<TV*>(sr->y_keep) : nullptr;
    TV* gkeep = keep ? static_cast<TV*>(sr->gy_keep) : nullptr;
#pragma unroll
    for (int e = 0; e < EPT; ++e) {
      const int64_t j = (int64_t)gt + (int64_t)e * nthr;
      vv[e] = (TV)0; mm[e] = (TV)0; mmf[e] = 0.f; ti[e] = 0.f;
      if (j >= p) continue;
      TV v;
      if (mode == PM_ITER) {
        TV y;
        double gyv;
        if (retry) {
          y = ykeep[j];
          gyv = (double)gkeep[j];
        } else {
          const TV b = bt[e];
          const TV bp = bprev[j];
          y = b + muv * (b - bp);
          if (a.loss == 0) gyv = (1.0 + mu) * gg[e] - mu * Gprev[j];
          else gyv = (mu == 0.0) ? gg[e] : gy[e];
          if (keep) {
            ykeep[j] = y;
            gkeep[j] = (TV)gyv;
          }
        }
        v = y - sv * (TV)gyv;
      } else {
        v = vin[j];
        if (!isfinite((double)v)) nbad += 1.0;
      }
      vv[e] = v;
      if (fx[e] == 0) {
        const TV m = v < (TV)0 ? -v : v;
        mm[e] = m;
        mmf[e] = (float)m;
        const double md = (double)m;
        ti[e] = (float)((md <= M * (1.0 + rho)) ? md * (rho / (1.0 + rho)) : md - M);
        if (m > (TV)0) nzv += 1.0;
      }
    }
  }

  // ---------------------------------------------------------------- S3
  double c = 0.0;
  int n_top = 0, n_nz = 0;
  if (do_prox) {
    {
      double nv[2] = {nzv, nbad};
      if constexpr (FAST) {
        ffs t[2] = {{(float)nzv, 0.f}, {0.f, 0.f}};
        gsum_ff(t, 2, nv);
      } else {
        gsum(nv, 2);
      }
      nzv = nv[0];
      nbad = nv[1];
    }
    // thread 0: the scalars of the threshold search
    struct ScS3 {
      double c, rhoM;
      unsigned long long nz;
      float inv_rho32;
      KV kc3, krho;
      int s3, warm3, fin;
    };
    __shared__ ScS3 sc3;
    if (tid == 0) {
      ScS3 r{};
      if (kb <= 0) r.c = INFINITY;
      else if (nzv <= (double)kb || nbad > 0.0) r.c = 0.0;   // no threshold search on a non-finite input
      else r.s3 = 1;
      r.rhoM = kr.rhoM;
      // for an FP32 x: rhoM > x iff x < rhoM rounded up, rhoM <= x iff x >= it
      r.krho = kr.krho;
      const double c3p = (mode == PM_ITER) ? sr->c_last : 0.0;
      r.warm3 = r.s3 && c3p > 0.0 && isfinite(c3p);
      r.kc3 = r.warm3 ? key_of((float)c3p) : (KV)0;
      r.inv_rho32 = kr.inv_rho_f;
      r.nz = (unsigned long long)nzv;
      r.fin = kb > 0 && nzv > (double)kb && nbad == 0.0;
      sc3 = r;
    }
    __syncthreads();
    c = sc3.c;
    const float inv_rho32 = sc3.inv_rho32;
    bool s3 = sc3.s3 != 0;
    KV lo3 = 0, hi3 = (KV)KeyOf<float>::kInf;
    // #{m > lo}, #{m > hi}, the same for T^-1
    unsigned long long cmlo = sc3.nz, cmhi = 0, ctlo = sc3.nz, cthi = 0;
    const KV krho = sc3.krho;
    bool warm3 = sc3.warm3 != 0;
    const KV kc3 = sc3.kc3;
    auto cand3 = [&](int q) { return warm3 ? warm_cand<KV>(kc3, lo3, hi3, q, 0) : cand<KV>(lo3, hi3, q); };
    while (s3) {
      unsigned long long fld[NFIELD] = {0, 0, 0, 0, 0, 0, 0, 0};
      const KV x3 = cand3(lane);
      const float cq = from_key(x3, 0.f);
      const float wq = fminf(cq * inv_rho32, M32);   // bracketing only: FP32
      const float invw = 1.0f / wq;
      // |v_j| at or below the round's smallest candidate adds nothing for any
      // lane (and T^-1(|v_j|) <= |v_j| neither): only the coordinates above
      // it are broadcast, which after the first round are about the top kbar
      // and the bracket's
      const float cmin = from_key(cand3(0), 0.f);
#pragma unroll
      for (int e = 0; e < EPT; ++e) {
        unsigned act = __ballot_sync(0xffffffffu, mmf[e] > cmin);
        while (act) {
          const int src = __ffs(act) - 1;
          act &= act - 1u;
          const float m = __shfl_sync(0xffffffffu, mmf[e], src);
          const float tv = __shfl_sync(0xffffffffu, ti[e], src);
          if (m > cq) {
            const float z = (m - cq) * invw;
            fld[F_S3Z] += fixp(z < 1.f ? z : 1.f);
            fld[F_S3CM] += 1ull;
          }
          fld[F_S3CT] += (tv > cq) ? 1ull : 0ull;
        }
      }
      // fields 3..5 live at indices F_S3Z.. ; reduce fields 0..5 (0..2 unused here)
      round_reduce(fld, 6);
      {
        const unsigned long long thr = (unsigned long long)kb << 32;
        const unsigned long long cm = sh_acc[F_S3CM * PQ + lane], ct = sh_acc[F_S3CT * PQ + lane];
        int qlo, qhi;
        bracket_step<KV>(x3, sh_acc[F_S3Z * PQ + lane] >= thr, lo3, hi3, qlo, qhi);
        if (qlo >= 0) { cmlo = __shfl_sync(0xffffffffu, cm, qlo); ctlo = __shfl_sync(0xffffffffu, ct, qlo); }
        if (qhi < 32) { cmhi = __shfl_sync(0xffffffffu, cm, qhi); cthi = __shfl_sync(0xffffffffu, ct, qhi); }
      }
      warm3 = false;
      const bool regime_inside = lo3 < krho && hi3 >= krho;   // rhoM in (c_lo, c_hi]
      if ((cmlo == cmhi && ctlo == cthi && !regime_inside) || hi3 - lo3 <= 1) s3 = false;
    }
    if (sc3.fin) {
      // exact finishing on the bracket's piece, polished until stable; thread
      // 0 takes the closed forms, every thread classifies its coordinates
      __shared__ double shp[3];   // ccur, Tc, the root found
      __shared__ float shpf[2];   // Tc rounded up, ccur rounded down
      __shared__ int shp_done;
      const double rhoM = sc3.rhoM;
      double clo = 0.0, chi = 0.0, ntop_prev = -1.0, nmid_prev = -1.0;   // thread 0's
      auto set_c = [&](double cc) {   // thread 0
        const double Tc = (cc <= rhoM) ? cc * kr.kTc : cc + M;
        shp[0] = cc;
        shp[1] = Tc;
        shpf[0] = __double2float_ru(Tc);
        shpf[1] = __double2float_rd(cc);
      };
      if (tid == 0) {
        clo = (double)from_key(lo3, 0.f);
        chi = (double)from_key(hi3, 0.f);
        set_c(chi);
        shp_done = 0;
      }
      __syncthreads();
      for (int it = 0; it <= MAX_POLISH; ++it) {
        const double ccur = shp[0], Tc = shp[1];
        double v[NBP] = {0, 0, 0, 0, 0, 0, 0, 0, 0, 0};
        if constexpr (FAST) {
          // an FP32 m satisfies m >= Tc iff m >= Tc rounded up, m > ccur iff
          // m > ccur rounded down: exact classification in FP32
          const float tcu = shpf[0], ccd = shpf[1];
          int ntop = 0, nmid = 0;
          ffs sm{0.f, 0.f};
          for (int e = 0; e < EPT; ++e) {
            if (fx[e] != 0) continue;
            if (wide >> e & 1u) {
              const double m = fabs((double)vv[e]);
              if (m >= Tc) ++ntop;
              else if (m > ccur) { ++nmid; ff_acc(sm, m); }
            } else {
              const float m = mmf[e];
              if (m >= tcu) ++ntop;
              else if (m > ccd) { ++nmid; ff_acc(sm, m); }
            }
          }
          ffs t[3] = {{(float)ntop, 0.f}, {(float)nmid, 0.f}, sm};
          gsum_ff(t, 3, v);
        } else {
        for (int e = 0; e < EPT; ++e) {
          if (fx[e] != 0) continue;
          const double m = (double)mm[e];
          if (m >= Tc) v[0] += 1.0;
          else if (m > ccur) { v[1] += 1.0; v[2] += m; }
        }
        gsum(v, 3);
        }
        if (tid == 0) {
          const double Ntop = v[0], Nmid = v[1], Smid = v[2];
          double cn;
          if (Nmid == 0.0) cn = ccur;   // flat piece: any c on it is a root when Ntop == kbar
          else if (ccur <= rhoM) cn = rho * Smid / ((double)kb - Ntop + rho * Nmid);
          else cn = (Smid - M * ((double)kb - Ntop)) / Nmid;
          const bool inside = (it == 0) && cn > clo && cn <= chi && cmlo == cmhi && ctlo == cthi &&
                              !(rhoM > clo && rhoM <= chi);
          const bool stable = (Ntop == ntop_prev && Nmid == nmid_prev);
          if (inside || stable || it == MAX_POLISH || !(cn > 0.0) || !isfinite(cn)) {
            shp[2] = (isfinite(cn) && cn > 0.0) ? cn : ccur;
            shp_done = 1;
          } else {
            ntop_prev = Ntop;
            nmid_prev = Nmid;
            set_c(cn);
          }
        }
        __syncthreads();
        if (shp_done) break;
      }
      c = shp[2];
    }
  }

  // ---------------------------------------------------------------- P2
  double tst_out[2] = {0.0, 0.0};
  if (do_prox) {
    // the next iterate goes to the buffer that becomes beta_cur after the
    // rotation; a retried trial point replaces the rejected one in place
    TV* out = mode == PM_ITER ? static_cast<TV*>(retry ? sr->beta_cur : sr->beta_prev) : static_cast<TV*>(a.vout);
    double tst[2] = {0.0, 0.0};   // backtracking: <grad F(y), x - y>, ||x - y||^2
    __shared__ double shq[2];     // T_c, 1 / (1 + rho)
    __shared__ float shq_c;       // c rounded down
    if (tid == 0) {
      shq[0] = (c <= kr.rhoM) ? c * kr.kTc : c + M;
      shq[1] = kr.inv1r;
      shq_c = __double2float_rd(c);
    }
    __syncthreads();
    const double T_c = shq[0];
    double cnt[2] = {0, 0};
    if constexpr (FAST) {
      // FP64 only for the outputs that are nonzero (about the support)
      const double inv1r = shq[1];
      const float ccd = shq_c;   // an FP32 m exceeds c iff it exceeds ccd
#pragma unroll
      for (int e = 0; e < EPT; ++e) {
        const int64_t j = (int64_t)gt + (int64_t)e * nthr;
        if (j >= p) continue;
        double b = 0.0;
        if (fx[e] > 0) {
          b = fmin(fmax((double)vv[e] * inv1r, -M), M);   // fixed in: v_j is FP64
        } else if (fx[e] == 0) {
          const bool w = (wide >> e) & 1u;
          double m = 0.0;
          bool nz;
          if (w) {
            m = fabs((double)vv[e]);
            nz = m > c;
          } else {
            nz = mmf[e] > ccd;
            if (nz) m = (double)mmf[e];
          }
          if (nz) {
            const double r = fmax(0.0, fmin(fmin(m - c, m * inv1r), M));
            b = ((negm >> e) & 1u) ? -r : r;
          }
        }
        out[j] = (TV)b;
      }
    } else {
    // Standalone prox: a non-finite input, or a bounded wait of this block
    // that expired (its threshold then rests on incomplete sums), gives NaN
    // outputs instead of silently wrong ones; the counts get a sentinel below.
    const bool poison = mode == PM_PROX && (nbad > 0.0 || !alive);
#pragma unroll
    for (int e = 0; e < EPT; ++e) {
      const int64_t j = (int64_t)gt + (int64_t)e * nthr;
      if (j >= p) continue;
      const double v = (double)vv[e];
      double b;
      if (poison) b = __longlong_as_double(0x7ff8000000000000ll);
      else if (fx[e] < 0) b = 0.0;
      else if (fx[e] > 0) b = fmin(fmax(v / (1.0 + rho), -M), M);
      else {
        const double m = fabs(v);
        const double r = fmax(0.0, fmin(fmin(m - c, m / (1.0 + rho)), M));
        b = v < 0.0 ? -r : r;
        if (r > 0.0) {
          cnt[1] += 1.0;
          if (m >= T_c) cnt[0] += 1.0;
        }
      }
      out[j] = (TV)b;
      if (keep) {   // y^t and its gradient as P1 kept them (this thread's own writes)
        const double d = b - (double)static_cast<const TV*>(sr->y_keep)[j];
        tst[0] += (double)static_cast<const TV*>(sr->gy_keep)[j] * d;
        tst[1] += d * d;
      }
    }
    if (keep) {
      gsum(tst, 2);
      tst_out[0] = tst[0];
      tst_out[1] = tst[1];
    }
    if (mode == PM_PROX && a.counts) {
      gsum(cnt, 2);
      if (lbk == 0 && tid == 0) {
        // any block's expired wait has recorded its status by now (a block that
        // gives up stops arriving, so every later barrier expires too)
        const bool failed = poison || !alive || *(volatile int*)a.status != ST_OK;
        a.counts[0] = failed ? -1 : (int)cnt[0];
        a.counts[1] = failed ? -1 : (int)cnt[1];
      }
    }
    if (mode == PM_PROX && nbad > 0.0 && lbk == 0 && tid == 0) atomicCAS(a.status, ST_OK, ST_NUMERIC);
    }
  }

  // ------------------------------------------------------------- epilogue
  // Everyone must be done with the round accumulators before CTA 0 clears
  // them: in the loop of a cooperative grid the last round is followed by a
  // finishing sum, whose barrier already ensures that; a cluster also waits
  // until no CTA reads another's shared memory, and the standalone modes and
  // the backtracking variant keep the barrier.
  if (CL || BT || mode != PM_ITER) barrier();
  if (lbk == 0) {
    if (!CL)
      for (int i = tid; i < 3 * ACC_STRIDE; i += PBLOCK) a.acc[i] = 0ull;
    if (tid == 0 && mode == PM_ITER && retry) {
      // a rejected trial point: the same iteration again, with L doubled
      st->Lk *= 2.0;
      st->rho_last = rho;
      st->dgy = tst_out[0];
      st->dxy2 = tst_out[1];
      st->bt_pending = 1;
      st->backtracks += 1;
      st->c_last = c;
      st->bar_base = bar0 + (unsigned long long)nbar * nbk;
    } else if (tid == 0) {
      if (mode == PM_ITER) {
        if (nonfinite) atomicCAS(a.status, ST_OK, ST_NUMERIC);
        st->rho_last = rho;
        if (a.backtrack && !stop) {
          st->dgy = tst_out[0];
          st->dxy2 = tst_out[1];
          st->bt_pending = 1;
        }
        st->phi_t = phi;
        st->psi_t = psi;
        st->g_t = gval;
        st->phi_best = phi_best;
        st->psi_best = psi_best;
        st->gap_ref = gap_ref;
        st->have_ref = have_ref;
        st->restarts = restarts;
        st->c_last = c;
        st->t1_last = fin1 ? tstar : 0.0;
        st->w2_last = wlast;
        st->stall_gap = stall_gap;
        st->stall_iter = stall_iter;
        st->stalled = stalled;
        st->cut_rule = cut_rule;
        if (stop) {
          st->done = 1;
          st->ps.done = 1;
        } else {
          // rotate: beta_prev <- beta^t, beta_cur <- beta^{t+1} (written into the old prev)
          void* b_old_prev = st->beta_prev;
          st->beta_prev = st->beta_cur;
          st->beta_cur = b_old_prev;
          void* g_old_prev = st->G_prev;
          st->G_prev = st->G_cur;
          st->G_cur = g_old_prev;
          void* z_old_prev = st->z_prev;
          st->z_prev = st->z_cur;
          st->z_cur = z_old_prev;
          st->tau = tau_new;
          st->iter = t + 1;
          st->ps.beta = st->beta_cur;
          st->ps.zout = st->z_cur;
          st->ps.zprev = st->z_prev;
          // tentative momentum for the pass at beta^{t+1} (the no-restart value)
          const double tn = 0.5 * (1.0 + sqrt(1.0 + 4.0 * tau_new * tau_new));
          st->ps.mom = a.method == 1 ? 0.0 : (tau_new - 1.0) / tn;
        }
        st->bar_base = bar0 + (unsigned long long)nbar * nbk;
      }
    }
  }
  (void)n_top; (void)n_nz;
}

}  // namespace relax
