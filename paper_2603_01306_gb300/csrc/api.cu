// C ABI of the library (include/relax.h): handle lifecycle, the solve loop,
// FP64 certification and the standalone regularizer entry points.
#include <cuda_bf16.h>
#include <cuda_fp8.h>

#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <cstdio>
#include <cstring>
#include <new>
#include <vector>

#include "bgemm.cuh"
#include "launch.cuh"
#include "relax.h"
#include "warmstart.h"

using namespace relax;

namespace {

thread_local char g_detail[256] = "";

void set_detail(const char* what, cudaError_t e, int line) {
  snprintf(g_detail, sizeof(g_detail), "%s failed: %s (api.cu:%d)", what, cudaGetErrorString(e), line);
  (void)cudaGetLastError();   // a non-sticky error must not surface again in a later call
}

#define CU(call)                                                \
  do {                                                          \
    cudaError_t e_ = (call);                                    \
    if (e_ != cudaSuccess) {                                    \
      set_detail(#call, e_, __LINE__);                          \
      return map_cuda(e_);                                      \
    }                                                           \
  } while (0)

relax_status map_cuda(cudaError_t e) {
  if (e == cudaErrorMemoryAllocation) return RELAX_ENOMEM;
  if (e == cudaErrorNotSupported) return RELAX_ENOTSUP;
  return RELAX_ECUDA;
}

relax_status map_dev_status(int s) {
  switch (s) {
    case ST_OK: return RELAX_OK;
    case ST_TIMEOUT: return RELAX_ETIMEOUT;
    case ST_NUMERIC: return RELAX_ENUMERIC;
    default: return RELAX_ECUDA;
  }
}

// ------------------------------------------------------------ small kernels
__global__ void count_fix_kernel(const int8_t* fix, int64_t p, int* out) {
  int j1 = 0, jf = 0, bad = 0;
  for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < p; j += (int64_t)gridDim.x * blockDim.x) {
    const int8_t f = fix[j];
    j1 += f == 1;
    jf += f == 0;
    bad += (f < -1 || f > 1);
  }
  j1 = warp_sum(j1); jf = warp_sum(jf); bad = warp_sum(bad);
  if ((threadIdx.x & 31) == 0) {
    if (j1) atomicAdd(out + 0, j1);
    if (jf) atomicAdd(out + 1, jf);
    if (bad) atomicAdd(out + 2, bad);
  }
}

// the same for the rows of a [rows][p] fixing matrix: row blockIdx.y into out[3 row]
__global__ void count_fix_batch_kernel(const int8_t* fix, int64_t p, int* out) {
  const int8_t* f = fix + (int64_t)blockIdx.y * p;
  int j1 = 0, jf = 0, bad = 0;
  for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < p; j += (int64_t)gridDim.x * blockDim.x) {
    const int8_t v = f[j];
    j1 += v == 1;
    jf += v == 0;
    bad += (v < -1 || v > 1);
  }
  j1 = warp_sum(j1); jf = warp_sum(jf); bad = warp_sum(bad);
  int* o = out + 3 * blockIdx.y;
  if ((threadIdx.x & 31) == 0) {
    if (j1) atomicAdd(o + 0, j1);
    if (jf) atomicAdd(o + 1, jf);
    if (bad) atomicAdd(o + 2, bad);
  }
}

// loop vectors are FP64; caller vectors are in the handle's dtype
__global__ void init_vectors_kernel(const void* warm, int warm_f64, double* b0, double* b1, double* bb, double* bd,
                                    double* g0, double* g1, int64_t p, double* z0, double* z1, int64_t n) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < p; j += stride) {
    double w = 0.0;
    if (warm) w = warm_f64 ? static_cast<const double*>(warm)[j] : (double)static_cast<const float*>(warm)[j];
    b0[j] = w; b1[j] = w; bb[j] = w; bd[j] = w;
    g0[j] = 0.0; g1[j] = 0.0;
  }
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
    z0[i] = 0.0; z1[i] = 0.0;
  }
}

// init_vectors_kernel for node blockIdx.y of a batch: its vectors at
// vec + nvec node (beta prev, cur; G prev, cur; beta_best, beta_dbest; then
// from 8 p: z prev, cur), the warm start's row `node` (or zeros)
__global__ void init_batch_kernel(const void* warm, int warm_f64, double* vec, int64_t nvec, int64_t p, int64_t n) {
  const int node = blockIdx.y;
  double* v = vec + nvec * node;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < p; j += stride) {
    double w = 0.0;
    if (warm) {
      const int64_t q = (int64_t)node * p + j;
      w = warm_f64 ? static_cast<const double*>(warm)[q] : (double)static_cast<const float*>(warm)[q];
    }
    v[j] = w; v[p + j] = w; v[4 * p + j] = w; v[5 * p + j] = w;
    v[2 * p + j] = 0.0; v[3 * p + j] = 0.0;
  }
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
    v[8 * p + i] = 0.0;
    v[8 * p + n + i] = 0.0;
  }
}

// dst (double) <- src (float or double)
__global__ void to_f64_kernel(const void* src, int src_f64, double* dst, int64_t m) {
  for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < m; j += (int64_t)gridDim.x * blockDim.x)
    dst[j] = src_f64 ? static_cast<const double*>(src)[j] : (double)static_cast<const float*>(src)[j];
}

// dst (float or double) <- src (double)
__global__ void from_f64_kernel(const double* src, void* dst, int dst_f64, int64_t m) {
  for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < m; j += (int64_t)gridDim.x * blockDim.x) {
    if (dst_f64) static_cast<double*>(dst)[j] = src[j];
    else static_cast<float*>(dst)[j] = (float)src[j];
  }
}

template <typename T>
__global__ void fill_kernel(T* v, int64_t p, T val) {
  for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < p; j += (int64_t)gridDim.x * blockDim.x)
    v[j] = val;
}

// out[j] = sum_c part[c*NB*p + j] (fixed order); optional sum of squares
template <typename TA, typename T>
__global__ void reduce_partials_kernel(const TA* part, int ncl, int NB, int64_t p, T* out, double* sq) {
  double s2 = 0.0;
  for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < p; j += (int64_t)gridDim.x * blockDim.x) {
    TA s = (TA)0;
    for (int c = 0; c < ncl; ++c) s += part[(int64_t)c * NB * p + j];
    out[j] = (T)s;
    s2 += (double)s * (double)s;
  }
  if (sq) {
    s2 = warp_sum(s2);
    if ((threadIdx.x & 31) == 0 && s2 != 0.0) atomicAdd(sq, s2);
  }
}

template <typename T>
__global__ void scale_kernel(T* v, int64_t p, const double* sq) {
  const double nrm = sqrt(*sq);
  const T inv = nrm > 0.0 ? (T)(1.0 / nrm) : (T)0;
  for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < p; j += (int64_t)gridDim.x * blockDim.x)
    v[j] *= inv;
}

__global__ void sumsq_kernel(const double* v, int64_t m, double* out) {
  double s = 0.0;
  for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < m; j += (int64_t)gridDim.x * blockDim.x)
    s += v[j] * v[j];
  s = warp_sum(s);
  if ((threadIdx.x & 31) == 0 && s != 0.0) atomicAdd(out, s);
}

// {F(z), -F*(-zeta)} at zeta = -grad F(z) (Eq. 6-7 loss parts), FP64
__global__ void loss_terms_kernel(const double* z, const double* y, int64_t n, int loss, double* out) {
  double f = 0.0, d = 0.0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    if (loss == RELAX_LS) {
      const double r = z[i] - y[i], zeta = -2.0 * r;
      f += r * r;
      d += zeta * y[i] - 0.25 * zeta * zeta;
    } else {
      f += softplus_neg(y[i] * z[i]);
      d += entropy_of(y[i] * z[i]);
    }
  }
  f = warp_sum(f);
  d = warp_sum(d);
  if ((threadIdx.x & 31) == 0) { atomicAdd(out, f); atomicAdd(out + 1, d); }
}

__global__ void nnz_kernel(const double* v, int64_t p, int* out) {
  int c = 0;
  for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < p; j += (int64_t)gridDim.x * blockDim.x)
    c += v[j] != 0.0;
  c = warp_sum(c);
  if ((threadIdx.x & 31) == 0 && c) atomicAdd(out, c);
}

__global__ void colmax_kernel(const float* X, int64_t n, int64_t p, int64_t ldx, unsigned* cmax) {
  const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= p) return;
  const int64_t rows_per = (n + gridDim.y - 1) / gridDim.y;
  const int64_t r0 = (int64_t)blockIdx.y * rows_per;
  const int64_t r1 = std::min<int64_t>(n, r0 + rows_per);
  float m = 0.0f;
  for (int64_t i = r0; i < r1; ++i) m = fmaxf(m, fabsf(X[i * ldx + j]));
  atomicMax(cmax + j, __float_as_uint(m));
}

__global__ void colscale_kernel(const unsigned* cmax, float* scale, int64_t p, float qmax) {
  const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= p) return;
  const float m = __uint_as_float(cmax[j]);
  scale[j] = m > 0.0f ? m / qmax : 1.0f;
}

template <typename TQ>
__global__ void quantize_kernel(const float* X, int64_t n, int64_t p, int64_t ldx, const float* scale,
                                TQ* Xq, int64_t ldq) {
  const int64_t total = n * ldq;
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = t / ldq, j = t - i * ldq;
    float v = 0.0f;
    if (j < p) v = X[i * ldx + j] / (scale ? scale[j] : 1.0f);
    if constexpr (sizeof(TQ) == 2) {
      Xq[t] = __float2bfloat16_rn(v);
    } else {
      __nv_fp8_storage_t s = __nv_cvt_float_to_fp8(v, __NV_SATFINITE, __NV_E4M3);
      Xq[t] = *reinterpret_cast<__nv_fp8_e4m3*>(&s);
    }
  }
}

inline unsigned grid_for(int64_t work, int block = 256) {
  int64_t g = (work + block - 1) / block;
  return (unsigned)std::max<int64_t>(1, std::min<int64_t>(g, 4096));
}

}  // namespace

// ================================================================== handle
// Device memory of relax_solve_batch, kept on the handle between calls
// (grown, never shrunk) together with the CUDA graph of a round for each
// active-set size: the graphs read only these buffers, so a later call with
// no more nodes than `cap` replays them.  Node planes and partials are laid
// out for `cap` nodes.
struct BatchWs {
  int cap = 0;
  IterState* dst = nullptr;
  double* vec = nullptr;
  unsigned long long* acc = nullptr;
  double* bpart = nullptr;
  unsigned long long* bars = nullptr;
  void *Bm = nullptr, *Zm = nullptr, *Rm = nullptr, *Gm = nullptr;   // FP64 data: operands and products
  __nv_bfloat16 *Bp = nullptr, *Rp = nullptr;                      // FP32 data: BF16 planes of B and R
  double *P1 = nullptr, *P2 = nullptr;                              // FP32 data: partial products per slot
  double* part = nullptr;
  int* active_d = nullptr;
  int* done_d = nullptr;
  int8_t* fix = nullptr;          // [cap][p] the call's fixings (zeros without)
  int* cnt = nullptr;             // [cap][3] fixing counts
  PassState* psd = nullptr;       // [cap][2] certificate passes
  double* certd = nullptr;        // [cap][4] certificate values
  std::vector<std::pair<int, cudaGraphExec_t>> graphs;
  bool planned = false, clustered = false;
  PPlan pc;                       // cluster plan of the p-phase (when clustered)
  void release() {
    void* ptrs[] = {dst, vec, acc, bpart, bars, Bm, Zm, Rm, Gm, Bp, Rp, P1, P2, part, active_d, done_d, fix, cnt,
                    psd, certd};
    for (void* q : ptrs) if (q) cudaFree(q);
    for (auto& g : graphs) cudaGraphExecDestroy(g.second);
    graphs.clear();
    *this = BatchWs{planned, clustered, pc};
  }
  BatchWs() = default;
  BatchWs(bool pl, bool cl, PPlan c) : planned(pl), clustered(cl), pc(c) {}
};

struct relax_handle {
  BatchWs bw;                // relax_solve_batch's device memory and graphs
  // batched solves of FP32 data: BF16 planes of X (K = p) and of X' (K = n)
  // for the tensor-core products, built on the first batched call; the K
  // chunks chosen per product and column tile width (BN / 16)
  __nv_bfloat16* bx = nullptr;
  __nv_bfloat16* bxt = nullptr;
  int64_t ldbp = 0, ldbn = 0;
  CUtensorMap tm_bx{}, tm_bxt{};
  cudaEvent_t ev_t[2] = {nullptr, nullptr};   // timing of the first product (relax_batch_xpass)
  cudaEvent_t ev_p[2] = {nullptr, nullptr};   // timing of the second product (relax_batch_xpass)
  int dev = 0;
  cudaStream_t stream = nullptr;
  int64_t n = 0, p = 0;
  int dtype = RELAX_F32;     // X master and vectors
  int loss = RELAX_LS;
  int k = 1;
  double lambda2 = 1.0;
  relax_options opt{};
  double M = 2.0, eta = 0.0;
  int max_iters = 100000, chunk = 32;
  int stall_min = 1000;      // least window of the stall rule (0: off)
  int method = 0, restart_rule = 0, backtrack = 0;   // the convergence study's variants
  double cutoff = INFINITY;  // incumbent objective for the dynamic termination (inf: off)
  uint64_t limit_ns = 4000000000ull;
  bool certify = true;
  double L = 0.0;
  // X
  const void* X = nullptr;   // master (caller's or aligned copy)
  int64_t ldx = 0;
  void* Xown = nullptr;
  void* Xq = nullptr;        // loop copy for BF16/FP8
  int64_t ldq = 0;
  float* colscale = nullptr;
  int xk_loop = XK_F32;
  void* y = nullptr;
  // plans
  XSPlan pl_loop, pl_cert, pl_certz, pl_cert2, pl_ident;
  // The precision ladder of a single solve whose certified gap misses the
  // tolerance on the loop's pass: the FP32 master X (after a BF16 / FP8
  // loop), then float-float products on the master X; the p-phase in FP64.
  XSPlan pl_acc32, pl_ff;
  bool has_acc32 = false, has_ff = false;
  PPlan pp_iter, pp_eval, pp_exact;
  // buffers
  double* xg = nullptr;          // [Gr][2][p] X' r per row group
  double* lterm = nullptr;       // [n][2] certification loss terms
  double* lterm2 = nullptr;      // [n][2] the same at a second dual point
  unsigned* xcnt = nullptr;      // per-pass zeroed area: block counters, max |beta|, fixed-point z
  double rowl1_x = 0.0;          // max_i ||x_i||_1 of X (NaN if X holds a NaN)
  double rowl1_q = 0.0;          // the same for the BF16/FP8 copy (stored values)
  double* colstat = nullptr;     // [2][p]: ||X_j||_2, |corr(X_j, y)| (learned warm start)
  IterState* st = nullptr;
  PassState* ps_aux = nullptr;
  void* vb[16] = {};         // FP64: beta prev/cur, G prev/cur, beta_best, beta_dbest (p);
                             // z prev/cur (n); scratch p, p, n, n; z of the best dual (n);
                             // backtracking: y and its gradient (p, p), X y (n)
  unsigned long long* acc = nullptr;
  double* bpart = nullptr;
  unsigned long long* bar = nullptr;
  unsigned long long* bar_aux = nullptr;
  int* status = nullptr;
  double* dscr = nullptr;    // device scratch doubles
  int* iscr = nullptr;       // device scratch ints
  IterState* h_state = nullptr;  // pinned
  int* h_done = nullptr;         // pinned [2]
  double* h_d = nullptr;         // pinned doubles
  int* h_i = nullptr;            // pinned ints
  // The single-node loop's chunk of `chunk` iterations, captured once as a
  // CUDA graph and replayed by every later solve.  Its kernels read only
  // handle-owned memory (state, buffers, the copy of the solve's fixings in
  // fixbuf), so one graph serves every solve with the same shape of call:
  // with or without fixings, with or without timing events.
  int8_t* fixbuf = nullptr;      // device p: the current solve's fixings
  cudaGraphExec_t gexec = nullptr;
  int g_fix = -1, g_timing = -1; // what gexec was captured for (-1: nothing)
  cudaEvent_t ev[2] = {nullptr, nullptr};   // host polls of the loop
  cudaEvent_t* tev = nullptr;    // [chunk][3] timing events recorded inside gexec
  size_t esz() const { return dtype == RELAX_F64 ? 8 : 4; }
  int f64() const { return dtype == RELAX_F64 ? 1 : 0; }
};

namespace {

void handle_free(relax_handle* h) {
  if (!h) return;
  cudaSetDevice(h->dev);
  cudaStreamSynchronize(h->stream);
  h->bw.release();
  void* ptrs[] = {h->Xown, h->Xq, h->colscale, h->y, h->xg, h->lterm, h->lterm2, h->xcnt, h->st,
                  h->ps_aux, h->acc, h->bpart, h->bar, h->bar_aux, h->status, h->dscr, h->iscr, h->colstat};
  for (void* q : ptrs) if (q) cudaFree(q);
  for (void* q : h->vb) if (q) cudaFree(q);
  if (h->h_state) cudaFreeHost(h->h_state);
  if (h->h_done) cudaFreeHost(h->h_done);
  if (h->h_d) cudaFreeHost(h->h_d);
  if (h->h_i) cudaFreeHost(h->h_i);
  if (h->bx) cudaFree(h->bx);
  if (h->bxt) cudaFree(h->bxt);
  for (cudaEvent_t e : h->ev_t) if (e) cudaEventDestroy(e);
  for (cudaEvent_t e : h->ev_p) if (e) cudaEventDestroy(e);
  if (h->gexec) cudaGraphExecDestroy(h->gexec);
  for (cudaEvent_t e : h->ev) if (e) cudaEventDestroy(e);
  if (h->tev) {
    for (int i = 0; i < 3 * h->chunk; ++i) if (h->tev[i]) cudaEventDestroy(h->tev[i]);
    delete[] h->tev;
  }
  if (h->fixbuf) cudaFree(h->fixbuf);
  delete h;
}

relax_status alloc(void** p, size_t bytes) {
  cudaError_t e = cudaMalloc(p, std::max<size_t>(bytes, 16));
  if (e != cudaSuccess) return map_cuda(e);
  return RELAX_OK;
}

XSArgs pass_args(relax_handle* h, const XSPlan& pl, int link, PassState* ps) {
  XSArgs a{};
  const bool lowp = (pl.xk == XK_BF16 || pl.xk == XK_FP8);
  a.tm = pl.tm;
  a.n = h->n;
  a.p = h->p;
  a.Gc = pl.Gc;
  a.Gr = pl.Gr;
  a.sw = pl.sw;
  a.inner = pl.inner;
  a.nbox = pl.nbox;
  a.boxb = pl.boxb;
  a.B = pl.B;
  a.nblk = pl.nblk;
  a.SA = pl.SA;
  a.SB = pl.SB;
  a.RA = pl.RA;
  a.RB = pl.RB;
  a.lag = pl.lag;
  a.link = link;
  a.y = (const double*)h->y;
  a.colscale = lowp ? h->colscale : nullptr;
  a.ps = ps;
  a.g = h->xg;
  a.lterm = nullptr;
  a.lterm2 = nullptr;
  a.rowl1 = lowp ? h->rowl1_q : h->rowl1_x;
  xstrip_zero_layout(pl, h->xcnt, a);
  a.status = h->status;
  a.limit_ns = h->limit_ns;
  return a;
}

// one fused pass (its block counters are zeroed first)
cudaError_t run_pass(relax_handle* h, const XSPlan& pl, const XSArgs& a, cudaStream_t st) {
  (void)h;
  return xstrip_launch(pl, a, st);
}

PArgs base_pargs(relax_handle* h) {
  PArgs a{};
  a.loss = h->loss;
  a.p = h->p;
  a.k = h->k;
  a.lambda2 = h->lambda2;
  a.M = h->M;
  a.step = 1.0 / h->L;
  a.rho = 2.0 * h->lambda2 / h->L;
  a.eta = h->eta;
  a.max_iters = h->max_iters;
  a.stall_min = h->stall_min;
  a.method = h->method;
  a.restart_rule = h->restart_rule;
  a.backtrack = h->backtrack;
  a.lossp = nullptr;
  a.acc = h->acc;
  a.bpart = h->bpart;
  a.status = h->status;
  a.limit_ns = h->limit_ns;
  a.kc = pconst_make(a.lambda2, a.M, a.step, a.rho);
  return a;
}

// ---- max_i ||x_i||_1 (bound of every dot product a pass forms, with max |beta|)
__device__ __forceinline__ double abs_of(double v) { return fabs(v); }
__device__ __forceinline__ double abs_of(float v) { return fabs((double)v); }
__device__ __forceinline__ double abs_of(__nv_bfloat16 v) { return fabs((double)__bfloat162float(v)); }
__device__ __forceinline__ double abs_of(__nv_fp8_e4m3 v) { return fabs((double)(float)v); }

// one warp per row; FP64 sums; a NaN anywhere makes the result NaN (its bits
// compare above those of every finite value and of +Inf)
template <typename T>
__global__ void rowl1_kernel(const T* X, int64_t n, int64_t p, int64_t ld, unsigned long long* out) {
  const int lane = threadIdx.x & 31;
  const int64_t w0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  unsigned long long mb = 0ull;
  for (int64_t i = w0; i < n; i += nw) {
    double sum = 0.0;
    for (int64_t j = lane; j < p; j += 32) sum += abs_of(X[i * ld + j]);
    sum = warp_sum(sum);
    const unsigned long long bits = (unsigned long long)__double_as_longlong(sum);
    mb = bits > mb ? bits : mb;
  }
  if (lane == 0 && mb) atomicMax(out, mb);
}

template <typename T>
relax_status row_l1(const void* X, int64_t n, int64_t p, int64_t ld, cudaStream_t st, double* out) {
  unsigned long long* d = nullptr;
  relax_status rs = alloc((void**)&d, sizeof(unsigned long long));
  if (rs != RELAX_OK) return rs;
  unsigned long long hb = 0ull;
  cudaError_t e = cudaMemsetAsync(d, 0, sizeof(unsigned long long), st);
  if (e == cudaSuccess) {
    rowl1_kernel<T><<<1024, 256, 0, st>>>(static_cast<const T*>(X), n, p, ld, d);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaMemcpyAsync(&hb, d, sizeof(hb), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  cudaFree(d);
  if (e != cudaSuccess) {
    set_detail("row_l1", e, __LINE__);
    return map_cuda(e);
  }
  double v;
  std::memcpy(&v, &hb, sizeof(v));
  *out = v;
  return RELAX_OK;
}

// ---- Lanczos estimate of ||X||_2^2 (deterministic: fixed grids, fixed-order sums)
constexpr int LZ_BLOCKS = 128;   // blocks of the partial dot products
constexpr int LZ_MAX = 64;       // Lanczos steps at most

// part[b][l] = sum over block b's indices of Q[l][i] * w[i], for l < m
__global__ void mdot_partial_kernel(const double* Q, int m, const double* w, int64_t p, double* part) {
  __shared__ double red[8];
  for (int l = 0; l < m; ++l) {
    double s = 0.0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < p; i += (int64_t)gridDim.x * blockDim.x)
      s += Q[(int64_t)l * p + i] * w[i];
    s = warp_sum(s);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
      double t = 0.0;
      for (int k = 0; k < (int)(blockDim.x >> 5); ++k) t += red[k];
      part[(int64_t)blockIdx.x * m + l] = t;
    }
    __syncthreads();
  }
}
// c[l] = sum_b part[b][l] in block order
__global__ void mdot_final_kernel(const double* part, int nb, int m, double* c) {
  const int l = threadIdx.x;
  if (l < m) {
    double s = 0.0;
    for (int b = 0; b < nb; ++b) s += part[(int64_t)b * m + l];
    c[l] = s;
  }
}
// w -= sum_l c[l] Q[l]
__global__ void msub_kernel(const double* Q, int m, const double* c, double* w, int64_t p) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < p; i += (int64_t)gridDim.x * blockDim.x) {
    double s = w[i];
    for (int l = 0; l < m; ++l) s -= c[l] * Q[(int64_t)l * p + i];
    w[i] = s;
  }
}
// q = w * scale
__global__ void scaled_copy_kernel(const double* w, double scale, double* q, int64_t p) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < p; i += (int64_t)gridDim.x * blockDim.x)
    q[i] = w[i] * scale;
}
// a deterministic start vector with no special structure
__global__ void lanczos_start_kernel(double* q, int64_t p) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < p; i += (int64_t)gridDim.x * blockDim.x)
    q[i] = 1.0 + (double)((uint64_t)(i + 1) * 2654435761ull % 1024ull) / 1024.0;
}

// largest eigenvalue of the symmetric tridiagonal matrix (a[0..m), b[1..m))
// by Sturm-sequence bisection
double tridiag_max_eig(const double* a, const double* b, int m) {
  double lo = a[0], hi = a[0];
  for (int i = 0; i < m; ++i) {
    const double r = (i > 0 ? std::fabs(b[i]) : 0.0) + (i + 1 < m ? std::fabs(b[i + 1]) : 0.0);
    lo = std::min(lo, a[i] - r);
    hi = std::max(hi, a[i] + r);
  }
  auto count_below = [&](double x) {
    int c = 0;
    double d = a[0] - x;
    if (d < 0) ++c;
    for (int i = 1; i < m; ++i) {
      if (d == 0.0) d = 1e-300;
      d = a[i] - x - b[i] * b[i] / d;
      if (d < 0) ++c;
    }
    return c;
  };
  for (int it = 0; it < 200 && hi - lo > 1e-15 * std::max(std::fabs(hi), 1e-300); ++it) {
    const double mid = 0.5 * (lo + hi);
    if (count_below(mid) >= m) hi = mid;   // every eigenvalue below mid
    else lo = mid;
  }
  return hi;
}

// L = c_F * ||X||_2^2: Lanczos on X'X (the operator the loop applies, in the
// loop's storage of X) with full reorthogonalisation; the largest Ritz value
// converges from below, so a 1% margin is added.
relax_status power_iteration(relax_handle* h, double* L_out) {
  const int64_t p = h->p;
  double* w = (double*)h->vb[9];
  double* Q = nullptr;
  double* part = nullptr;
  double* c = nullptr;
  relax_status rs = RELAX_OK;
  if ((rs = alloc((void**)&Q, (size_t)(LZ_MAX + 1) * p * sizeof(double))) != RELAX_OK) return rs;
  if ((rs = alloc((void**)&part, (size_t)LZ_BLOCKS * (LZ_MAX + 1) * sizeof(double))) != RELAX_OK) { cudaFree(Q); return rs; }
  if ((rs = alloc((void**)&c, (size_t)(LZ_MAX + 1) * sizeof(double))) != RELAX_OK) { cudaFree(Q); cudaFree(part); return rs; }
  const unsigned g = grid_for(p);
  double alpha[LZ_MAX + 1] = {}, beta[LZ_MAX + 2] = {};
  double theta = 0.0, theta_prev = 0.0;
  // c[0..m) = Q[0..m)' v (host copy in hc)
  auto mdot = [&](const double* Qb, int m, const double* v, double* hc) -> cudaError_t {
    mdot_partial_kernel<<<LZ_BLOCKS, 256, 0, h->stream>>>(Qb, m, v, p, part);
    mdot_final_kernel<<<1, 128, 0, h->stream>>>(part, LZ_BLOCKS, m, c);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaMemcpyAsync(hc, c, sizeof(double) * m, cudaMemcpyDeviceToHost, h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    return e;
  };
  auto run = [&]() -> relax_status {
    lanczos_start_kernel<<<g, 256, 0, h->stream>>>(Q, p);
    CU(cudaGetLastError());
    double nrm2 = 0.0;
    CU(mdot(Q, 1, Q, &nrm2));
    scaled_copy_kernel<<<g, 256, 0, h->stream>>>(Q, 1.0 / std::sqrt(nrm2), Q, p);
    int m = 0;
    for (int j = 0; j < LZ_MAX; ++j) {
      // w = X'X q_j
      PassState ps{};
      ps.beta = Q + (int64_t)j * p;
      ps.zout = h->vb[10];
      *reinterpret_cast<PassState*>(h->h_d + 1000) = ps;   // staging in pinned memory
      CU(cudaMemcpyAsync(h->ps_aux, h->h_d + 1000, sizeof(PassState), cudaMemcpyHostToDevice, h->stream));
      XSArgs a = pass_args(h, h->pl_ident, LINK_IDENT, h->ps_aux);
      CU(run_pass(h, h->pl_ident, a, h->stream));
      reduce_partials_kernel<double, double><<<g, 256, 0, h->stream>>>(h->xg, h->pl_ident.Gr, 1, p, w, nullptr);
      CU(cudaGetLastError());
      // two rounds of classical Gram-Schmidt against q_0..q_j
      double hc[LZ_MAX + 1], hc2[LZ_MAX + 1];
      CU(mdot(Q, j + 1, w, hc));
      msub_kernel<<<g, 256, 0, h->stream>>>(Q, j + 1, c, w, p);
      CU(mdot(Q, j + 1, w, hc2));
      msub_kernel<<<g, 256, 0, h->stream>>>(Q, j + 1, c, w, p);
      CU(cudaGetLastError());
      int dst = 0;
      CU(cudaMemcpy(&dst, h->status, sizeof(int), cudaMemcpyDeviceToHost));
      if (dst != ST_OK) return map_dev_status(dst);
      alpha[j] = hc[j] + hc2[j];
      double b2 = 0.0;
      CU(mdot(w, 1, w, &b2));
      beta[j + 1] = std::sqrt(std::max(b2, 0.0));
      m = j + 1;
      theta = tridiag_max_eig(alpha, beta, m);
      if (!std::isfinite(theta)) return RELAX_ENUMERIC;
      if (j >= 4 && std::fabs(theta - theta_prev) <= 1e-12 * theta) break;
      if (!(beta[j + 1] > 1e-13 * std::max(theta, 1e-300))) break;   // invariant subspace found
      theta_prev = theta;
      scaled_copy_kernel<<<g, 256, 0, h->stream>>>(w, 1.0 / beta[j + 1], Q + (int64_t)(j + 1) * p, p);
      CU(cudaGetLastError());
    }
    return RELAX_OK;
  };
  rs = run();
  cudaStreamSynchronize(h->stream);
  cudaFree(Q);
  cudaFree(part);
  cudaFree(c);
  if (rs != RELAX_OK) return rs;
  if (!(theta > 0.0) || !std::isfinite(theta)) return RELAX_ENUMERIC;
  const double cf = h->loss == RELAX_LS ? 2.0 : 0.25;
  *L_out = cf * theta * 1.01;   // 1% margin over the Ritz estimate of ||X||^2
  return RELAX_OK;
}

relax_status count_fixings(relax_handle* h, const int8_t* fix, int* j1, int* jf) {
  if (!fix) { *j1 = 0; *jf = (int)h->p; return RELAX_OK; }
  CU(cudaMemsetAsync(h->iscr, 0, 3 * sizeof(int), h->stream));
  count_fix_kernel<<<grid_for(h->p), 256, 0, h->stream>>>(fix, h->p, h->iscr);
  CU(cudaGetLastError());
  CU(cudaMemcpyAsync(h->h_i, h->iscr, 3 * sizeof(int), cudaMemcpyDeviceToHost, h->stream));
  CU(cudaStreamSynchronize(h->stream));
  if (h->h_i[2] != 0) return RELAX_EINVAL;
  *j1 = h->h_i[0];
  *jf = h->h_i[1];
  return RELAX_OK;
}

// FP64 Phi(beta_p) and Psi(zeta) with the master X -> h->h_d[0..1].
// zeta = -grad F(X beta_d) when zd == NULL, else zeta = -grad F(zd) (a dual
// point given by its z).
// Enqueue the FP64 certificate of one point pair on the handle's stream:
// {Phi(bp), Psi(zeta)} into out_dev[0..1], zeta = -grad F(z_d) when the pass
// state names z_d (zprev), else -grad F(X bd).  ps_dev: the pass state in
// device memory (beta = bp, beta2 = bd or NULL, zprev = z_d or NULL).  No
// host synchronisation; consecutive calls share the handle's scratch in
// stream order.
// The dual point of a certificate: the pass state's zprev (DUAL_Z), X beta2
// (DUAL_B2, a second product), or X beta itself (DUAL_SELF, one product).
enum { DUAL_Z = 0, DUAL_B2 = 1, DUAL_SELF = 2 };

relax_status certify_enqueue(relax_handle* h, const int8_t* fix, const void* bp, int dual,
                             PassState* ps_dev, double* out_dev) {
  const XSPlan& pl = dual == DUAL_B2 ? h->pl_cert : h->pl_certz;   // NF = 2 / NF = 1
  const int link = dual == DUAL_Z ? (h->loss == RELAX_LS ? LINK_CERTZ_LS : LINK_CERTZ_LOGI)
                                  : (h->loss == RELAX_LS ? LINK_CERT_LS : LINK_CERT_LOGI);
  XSArgs a = pass_args(h, pl, link, ps_dev);
  a.colscale = nullptr;
  a.lterm = h->lterm;
  CU(run_pass(h, pl, a, h->stream));
  PArgs pa = base_pargs(h);
  pa.mode = PM_EVAL;
  pa.fix = fix;
  pa.part = h->xg;
  pa.ncl = pl.Gr;
  pa.NB = 1;
  pa.st = nullptr;
  pa.vin = bp;
  pa.out = out_dev;
  pa.fast_s1 = 0;
  pa.lossp = h->lterm;
  pa.n = h->n;
  pa.bar = h->bar_aux;
  pa.bar_base = 0;
  CU(cudaMemsetAsync(h->bar_aux, 0, sizeof(unsigned long long), h->stream));
  CU(pphase_launch(h->pp_eval, pa, h->stream));
  return RELAX_OK;
}

// Both certificates of a point in one pass (the X beta product shared): the
// pass state holds beta = beta_best and zprev = the loop's dual-point z.  The
// first evaluation gives (Phi(beta), Psi at the loop's dual point) in
// out_dev[0..1], the second (Phi(beta), Psi at zeta = -grad F(X beta)) in
// out_dev[2..3] -- the values of the two single-certificate calls.
relax_status certify_pair_enqueue(relax_handle* h, const int8_t* fix, const void* bp, PassState* ps_dev,
                                  double* out_dev) {
  const XSPlan& pl = h->pl_cert2;
  XSArgs a = pass_args(h, pl, h->loss == RELAX_LS ? LINK_CERT2_LS : LINK_CERT2_LOGI, ps_dev);
  a.colscale = nullptr;
  a.lterm = h->lterm;
  a.lterm2 = h->lterm2;
  CU(run_pass(h, pl, a, h->stream));
  for (int q = 0; q < 2; ++q) {
    PArgs pa = base_pargs(h);
    pa.mode = PM_EVAL;
    pa.fix = fix;
    pa.part = h->xg + (size_t)q * h->p;    // partials [Gr][2][p]: right-hand side q
    pa.ncl = pl.Gr;
    pa.NB = 2;
    pa.st = nullptr;
    pa.vin = bp;
    pa.out = out_dev + 2 * q;
    pa.fast_s1 = 0;
    pa.lossp = q == 0 ? h->lterm : h->lterm2;
    pa.n = h->n;
    pa.bar = h->bar_aux;
    pa.bar_base = 0;
    CU(cudaMemsetAsync(h->bar_aux, 0, sizeof(unsigned long long), h->stream));
    CU(pphase_launch(h->pp_eval, pa, h->stream));
  }
  return RELAX_OK;
}

relax_status certify(relax_handle* h, const int8_t* fix, const void* bp, const void* bd, const void* zd) {
  PassState ps{};
  ps.beta = bp;
  ps.beta2 = zd ? nullptr : bd;
  ps.zprev = zd;
  *reinterpret_cast<PassState*>(h->h_d + 1000) = ps;
  CU(cudaMemcpyAsync(h->ps_aux, h->h_d + 1000, sizeof(PassState), cudaMemcpyHostToDevice, h->stream));
  const int dual = zd ? DUAL_Z : (bd == bp ? DUAL_SELF : DUAL_B2);
  relax_status rs = certify_enqueue(h, fix, bp, dual, h->ps_aux, h->dscr);
  if (rs != RELAX_OK) return rs;
  CU(cudaMemcpyAsync(h->h_d, h->dscr, 2 * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
  CU(cudaStreamSynchronize(h->stream));
  return RELAX_OK;
}

// certify_pair_enqueue for one point, its four values in h_d[0..3]
relax_status certify_pair(relax_handle* h, const int8_t* fix, const void* bp, const void* zd) {
  PassState ps{};
  ps.beta = bp;
  ps.zprev = zd;
  *reinterpret_cast<PassState*>(h->h_d + 1000) = ps;
  CU(cudaMemcpyAsync(h->ps_aux, h->h_d + 1000, sizeof(PassState), cudaMemcpyHostToDevice, h->stream));
  relax_status rs = certify_pair_enqueue(h, fix, bp, h->ps_aux, h->dscr);
  if (rs != RELAX_OK) return rs;
  CU(cudaMemcpyAsync(h->h_d, h->dscr, 4 * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
  CU(cudaStreamSynchronize(h->stream));
  return RELAX_OK;
}

}  // namespace

extern "C" {

const char* relax_error_detail(void) { return g_detail; }

const char* relax_strerror(relax_status s) {
  switch (s) {
    case RELAX_OK: return "ok";
    case RELAX_EINVAL: return "invalid argument";
    case RELAX_ENOMEM: return "device allocation failed";
    case RELAX_ECUDA: return "CUDA runtime error";
    case RELAX_ENOTCONV: return "iteration limit reached before the gap tolerance";
    case RELAX_ETIMEOUT: return "a bounded device-side wait expired";
    case RELAX_ENUMERIC: return "non-finite value in the data or the iterates";
    case RELAX_EINVALID_BOUND: return "certified dual bound exceeds the certified primal value";
    case RELAX_ENOTSUP: return "shape or option not supported by this library";
    default: return "unknown status";
  }
}

relax_status relax_create(relax_handle** out, const void* X, const void* y, int64_t n, int64_t p, int64_t ldx,
                          int32_t dtype, int32_t loss, int32_t k, double lambda2, const relax_options* opt,
                          void* stream) {
  if (!out || !X || !y || n <= 0 || p <= 0 || ldx < p || k < 1 || !(lambda2 > 0.0) ||
      (dtype != RELAX_F64 && dtype != RELAX_F32) || (loss != RELAX_LS && loss != RELAX_LOGISTIC))
    return RELAX_EINVAL;
  relax_options o{};
  if (opt) o = *opt;
  if (o.M < 0.0 || std::isnan(o.M) || o.eta < 0.0 || o.lipschitz < 0.0 || o.max_iters < 0 ||
      o.watchdog_ms < 0 || o.chunk < 0 || o.method < 0 || o.method > 1 || o.restart < 0 || o.restart > 2 ||
      o.step_rule < 0 || o.step_rule > 1)
    return RELAX_EINVAL;
  const int prec = o.precision == 0 ? dtype : o.precision;
  if (prec != dtype && !((prec == RELAX_BF16 || prec == RELAX_FP8E4M3) && dtype == RELAX_F32))
    return RELAX_EINVAL;
  relax_handle* h = new (std::nothrow) relax_handle();
  if (!h) return RELAX_ENOMEM;
  relax_status rs = RELAX_OK;
#define TRY(x)                          \
  do {                                  \
    rs = (x);                           \
    if (rs != RELAX_OK) goto fail;      \
  } while (0)
#define TRYC(x)                                   \
  do {                                            \
    cudaError_t ec_ = (x);                        \
    if (ec_ != cudaSuccess) {                     \
      set_detail(#x, ec_, __LINE__);              \
      rs = map_cuda(ec_);                         \
      goto fail;                                  \
    }                                             \
  } while (0)
  {
    cudaGetDevice(&h->dev);
    h->stream = (cudaStream_t)stream;
    h->n = n;
    h->p = p;
    h->dtype = dtype;
    h->loss = loss;
    h->k = k;
    h->lambda2 = lambda2;
    h->opt = o;
    h->M = o.M == 0.0 ? 2.0 : o.M;
    h->eta = o.eta == 0.0 ? std::exp(3.0) : o.eta;
    h->max_iters = o.max_iters == 0 ? 100000 : o.max_iters;
    h->chunk = o.chunk == 0 ? 32 : o.chunk;
    h->stall_min = o.stall_window == 0 ? 1000 : std::max(0, o.stall_window);
    h->method = o.method;
    h->restart_rule = o.restart;
    h->backtrack = o.step_rule;
    h->limit_ns = (uint64_t)(o.watchdog_ms == 0 ? 4000 : o.watchdog_ms) * 1000000ull;
    h->certify = o.no_certify == 0;
    const size_t es = h->esz();
    // X: rows must start on 16-byte boundaries for the bulk copies
    if ((reinterpret_cast<uintptr_t>(X) & 15u) == 0 && ((size_t)ldx * es) % 16 == 0) {
      h->X = X;
      h->ldx = ldx;
    } else {
      const int64_t lda = (p * (int64_t)es + 15) / 16 * 16 / (int64_t)es;
      TRY(alloc(&h->Xown, (size_t)n * lda * es));
      TRYC(cudaMemsetAsync(h->Xown, 0, (size_t)n * lda * es, h->stream));
      TRYC(cudaMemcpy2DAsync(h->Xown, lda * es, X, ldx * es, p * es, n, cudaMemcpyDeviceToDevice, h->stream));
      h->X = h->Xown;
      h->ldx = lda;
    }
    TRY(alloc(&h->y, (size_t)n * sizeof(double)));
    to_f64_kernel<<<grid_for(n), 256, 0, h->stream>>>(y, dtype == RELAX_F64 ? 1 : 0, (double*)h->y, n);
    TRYC(cudaGetLastError());
    // low-precision loop copy of X (BF16 unscaled, FP8 with per-column scales)
    h->xk_loop = dtype == RELAX_F64 ? XK_F64 : XK_F32;
    if (prec == RELAX_BF16 || prec == RELAX_FP8E4M3) {
      h->xk_loop = prec == RELAX_BF16 ? XK_BF16 : XK_FP8;
      const int qes = prec == RELAX_BF16 ? 2 : 1;
      h->ldq = (p * qes + 15) / 16 * 16 / qes;
      TRY(alloc(&h->Xq, (size_t)n * h->ldq * qes));
      if (prec == RELAX_FP8E4M3) {
        unsigned* cmax = nullptr;
        TRY(alloc((void**)&cmax, (size_t)p * sizeof(unsigned)));
        TRY(alloc((void**)&h->colscale, (size_t)p * sizeof(float)));
        TRYC(cudaMemsetAsync(cmax, 0, (size_t)p * sizeof(unsigned), h->stream));
        dim3 gr((unsigned)((p + 255) / 256), (unsigned)std::min<int64_t>(256, n));
        colmax_kernel<<<gr, 256, 0, h->stream>>>((const float*)h->X, n, p, h->ldx, cmax);
        colscale_kernel<<<grid_for(p), 256, 0, h->stream>>>(cmax, h->colscale, p, 448.0f);
        quantize_kernel<__nv_fp8_e4m3><<<4096, 256, 0, h->stream>>>((const float*)h->X, n, p, h->ldx, h->colscale,
                                                                  (__nv_fp8_e4m3*)h->Xq, h->ldq);
        TRYC(cudaGetLastError());
        TRYC(cudaStreamSynchronize(h->stream));
        cudaFree(cmax);
      } else {
        quantize_kernel<__nv_bfloat16><<<4096, 256, 0, h->stream>>>((const float*)h->X, n, p, h->ldx, nullptr,
                                                                  (__nv_bfloat16*)h->Xq, h->ldq);
        TRYC(cudaGetLastError());
      }
    }
    const bool vd = dtype == RELAX_F64;
    TRYC(xstrip_plan(h->pl_loop, h->xk_loop, false, 1, loss == RELAX_LS ? 1 : 2, n, p));
    TRYC(xstrip_plan(h->pl_ident, h->xk_loop, false, 1, 1, n, p));
    TRYC(xstrip_plan(h->pl_cert, vd ? XK_F64 : XK_F32, true, 2, 1, n, p));
    TRYC(xstrip_plan(h->pl_certz, vd ? XK_F64 : XK_F32, true, 1, 1, n, p));
    TRYC(xstrip_plan(h->pl_cert2, vd ? XK_F64 : XK_F32, true, 1, 2, n, p));
    if (!vd) {
      const int nbl = loss == RELAX_LS ? 1 : 2;
      TRYC(xstrip_plan(h->pl_ff, XK_F32, true, 1, nbl, n, p));
      h->has_ff = true;
      if (h->xk_loop == XK_BF16 || h->xk_loop == XK_FP8) {
        TRYC(xstrip_plan(h->pl_acc32, XK_F32, false, 1, nbl, n, p));
        h->has_acc32 = true;
      }
    }
    {
      const bool lowp = h->xk_loop == XK_BF16 || h->xk_loop == XK_FP8;
      const void* xl = lowp ? h->Xq : h->X;
      const int64_t ldl = lowp ? h->ldq : h->ldx;
      TRYC(xstrip_bind(h->pl_loop, xl, ldl, n, p));
      TRYC(xstrip_bind(h->pl_ident, xl, ldl, n, p));
      TRYC(xstrip_bind(h->pl_cert, h->X, h->ldx, n, p));
      TRYC(xstrip_bind(h->pl_certz, h->X, h->ldx, n, p));
      TRYC(xstrip_bind(h->pl_cert2, h->X, h->ldx, n, p));
      if (h->has_ff) TRYC(xstrip_bind(h->pl_ff, h->X, h->ldx, n, p));
      if (h->has_acc32) TRYC(xstrip_bind(h->pl_acc32, h->X, h->ldx, n, p));
      if (dtype == RELAX_F64) TRY(row_l1<double>(h->X, n, p, h->ldx, h->stream, &h->rowl1_x));
      else TRY(row_l1<float>(h->X, n, p, h->ldx, h->stream, &h->rowl1_x));
      if (h->xk_loop == XK_BF16) TRY(row_l1<__nv_bfloat16>(h->Xq, n, p, h->ldq, h->stream, &h->rowl1_q));
      if (h->xk_loop == XK_FP8) TRY(row_l1<__nv_fp8_e4m3>(h->Xq, n, p, h->ldq, h->stream, &h->rowl1_q));
    }
    if (std::getenv("RELAX_DEBUG")) {
      const XSPlan& q = h->pl_loop;
      std::fprintf(stderr, "[relax] loop pass: xk=%d Gc=%d Gr=%d sw=%lld (%d x %d) B=%d nblk=%d SA=%d SB=%d RA=%d RB=%d lag=%d threads=%d smem=%zu\n",
                   q.xk, q.Gc, q.Gr, (long long)q.sw, q.nbox, q.inner, q.B, q.nblk, q.SA, q.SB, q.RA, q.RB, q.lag, q.threads,
                   q.smem);
    }
    // FP32, BF16 and FP8 data: the loop's per-coordinate arithmetic in FP32
    // (FP64 at a small fraction of the FP32 rate on this GPU); FP64 data keeps
    // FP64 throughout
    TRYC(pphase_plan(h->pp_iter, true, p, h->backtrack != 0, h->xk_loop != XK_F64 && !h->backtrack));
    // the certificate's evaluation: FP32 per coordinate and FP64 wherever a
    // term of Phi or Psi is nonzero (FP32 data); FP64 throughout for FP64 data
    TRYC(pphase_plan(h->pp_eval, true, p, false, !vd));
    TRYC(pphase_plan(h->pp_exact, true, p, h->backtrack != 0, false));
    {
      const XSPlan* pls[7] = {&h->pl_loop, &h->pl_ident, &h->pl_cert, &h->pl_certz, &h->pl_cert2,
                              h->has_ff ? &h->pl_ff : &h->pl_loop, h->has_acc32 ? &h->pl_acc32 : &h->pl_loop};
      size_t zero_b = 0;
      int gr_max = 1;
      for (const XSPlan* q : pls) {
        zero_b = std::max(zero_b, xstrip_zero_bytes(*q, n));
        gr_max = std::max(gr_max, q->Gr);
      }
      TRY(alloc((void**)&h->xg, (size_t)gr_max * 2 * p * sizeof(double)));
      TRY(alloc((void**)&h->lterm, (size_t)2 * n * sizeof(double)));
      TRY(alloc((void**)&h->lterm2, (size_t)2 * n * sizeof(double)));
      TRY(alloc((void**)&h->xcnt, zero_b));
    }
    TRY(alloc((void**)&h->st, sizeof(IterState)));
    TRY(alloc((void**)&h->ps_aux, sizeof(PassState)));
    for (int i = 0; i < 6; ++i) TRY(alloc(&h->vb[i], (size_t)p * sizeof(double)));
    for (int i = 6; i < 8; ++i) TRY(alloc(&h->vb[i], (size_t)n * sizeof(double)));
    for (int i = 8; i < 10; ++i) TRY(alloc(&h->vb[i], (size_t)p * sizeof(double)));
    for (int i = 10; i < 13; ++i) TRY(alloc(&h->vb[i], (size_t)n * sizeof(double)));
    for (int i = 13; i < 15; ++i) TRY(alloc(&h->vb[i], (size_t)p * sizeof(double)));
    TRY(alloc(&h->vb[15], (size_t)n * sizeof(double)));
    TRY(alloc((void**)&h->acc, 3 * ACC_STRIDE * sizeof(unsigned long long)));
    const int gmax = std::max(std::max(h->pp_iter.grid, h->pp_eval.grid), h->pp_exact.grid);
    TRY(alloc((void**)&h->bpart, (size_t)2 * gmax * NBP * sizeof(double)));
    TRY(alloc((void**)&h->bar, sizeof(unsigned long long)));
    TRY(alloc((void**)&h->bar_aux, sizeof(unsigned long long)));
    TRY(alloc((void**)&h->status, sizeof(int)));
    TRY(alloc((void**)&h->dscr, 16 * sizeof(double)));
    TRY(alloc((void**)&h->iscr, 16 * sizeof(int)));
    TRYC(cudaMemsetAsync(h->acc, 0, 3 * ACC_STRIDE * sizeof(unsigned long long), h->stream));
    TRYC(cudaMemsetAsync(h->status, 0, sizeof(int), h->stream));
    TRYC(cudaHostAlloc((void**)&h->h_state, sizeof(IterState), cudaHostAllocDefault));
    TRYC(cudaHostAlloc((void**)&h->h_done, 2 * sizeof(int), cudaHostAllocDefault));
    TRYC(cudaHostAlloc((void**)&h->h_d, 1024 * sizeof(double), cudaHostAllocDefault));
    TRYC(cudaHostAlloc((void**)&h->h_i, 16 * sizeof(int), cudaHostAllocDefault));
    TRY(alloc((void**)&h->fixbuf, (size_t)p));
    TRYC(cudaEventCreateWithFlags(&h->ev[0], cudaEventDisableTiming));
    TRYC(cudaEventCreateWithFlags(&h->ev[1], cudaEventDisableTiming));
    TRYC(cudaEventCreate(&h->ev_t[0]));
    TRYC(cudaEventCreate(&h->ev_t[1]));
    TRYC(cudaEventCreate(&h->ev_p[0]));
    TRYC(cudaEventCreate(&h->ev_p[1]));
    if (o.lipschitz > 0.0) h->L = o.lipschitz;
    else TRY(power_iteration(h, &h->L));
    TRYC(cudaStreamSynchronize(h->stream));
  }
  *out = h;
  return RELAX_OK;
fail:
  handle_free(h);
  return rs;
#undef TRY
#undef TRYC
}

relax_status relax_destroy(relax_handle* h) {
  if (!h) return RELAX_EINVAL;
  handle_free(h);
  return RELAX_OK;
}

relax_status relax_solve(relax_handle* h, const int8_t* fixings, const void* warm_start, double gap_tol,
                         void* beta_out, relax_result* out) {
  if (!h || !beta_out || !out || !(gap_tol > 0.0)) return RELAX_EINVAL;
  CU(cudaSetDevice(h->dev));
  int j1 = 0, jf = 0;
  relax_status rs = count_fixings(h, fixings, &j1, &jf);
  if (rs != RELAX_OK) return rs;
  if (h->k < j1) return RELAX_EINVAL;
  std::memset(out, 0, sizeof(*out));
  out->lipschitz = h->L;
  // ---- state (loop vectors are FP64)
  const unsigned g = grid_for(std::max(h->p, h->n));
  init_vectors_kernel<<<g, 256, 0, h->stream>>>(warm_start, h->f64(), (double*)h->vb[0], (double*)h->vb[1],
                                                (double*)h->vb[4], (double*)h->vb[5], (double*)h->vb[2],
                                                (double*)h->vb[3], h->p, (double*)h->vb[6], (double*)h->vb[7], h->n);
  CU(cudaGetLastError());
  IterState s{};
  s.beta_prev = h->vb[0];
  s.beta_cur = h->vb[1];
  s.G_prev = h->vb[2];
  s.G_cur = h->vb[3];
  s.beta_best = h->vb[4];
  s.beta_dbest = h->vb[5];
  s.z_dbest = h->vb[12];
  s.z_prev = h->vb[6];
  s.z_cur = h->vb[7];
  s.tau = 1.0;
  s.gap_ref = INFINITY;
  s.phi_best = INFINITY;
  s.psi_best = -INFINITY;
  s.stall_gap = INFINITY;
  s.kbar = h->k - j1;
  s.pbar = jf;
  // With FP32 (or narrower) X the loop's gap is an estimate: aim a little below
  // gap_tol so that the FP64 certificate of the final pair usually confirms it
  // at once.  With FP64 X the loop's gap is the certificate's, to rounding.
  const double tol_exact = (h->dtype == RELAX_F64 && h->xk_loop == XK_F64) ? gap_tol : 0.7 * gap_tol;
  s.tol = tol_exact;
  // A BF16 / FP8 loop converges to the optimum of the problem on the
  // quantized X, whose bound is off the true one by about the format's
  // precision (measured 3e-3 to 5e-3 relative for BF16, 5e-2 to 9e-2 for
  // FP8): converging further buys nothing once the precision ladder's FP32
  // rung takes over, so such a loop stops at a tolerance of that order.
  if ((h->xk_loop == XK_BF16 || h->xk_loop == XK_FP8) && h->has_acc32 && h->certify) {
    double q_tol = h->xk_loop == XK_BF16 ? 1e-3 : 1e-2;
    if (const char* ov = std::getenv("RELAX_QTOL")) q_tol = std::atof(ov);   // tuning runs
    s.tol = std::max(s.tol, q_tol);
  }
  s.ps.beta = s.beta_cur;
  s.ps.zout = s.z_cur;
  s.ps.zprev = s.z_prev;
  s.ps.mom = 0.0;
  s.cutoff_on = std::isfinite(h->cutoff) ? 1 : 0;
  s.cutoff = h->cutoff;
  s.Lk = h->backtrack ? h->L / 64.0 : h->L;   // backtracking starts below the estimate and only grows
  s.rho_last = 2.0 * h->lambda2 / s.Lk;
  s.y_keep = h->vb[13];
  s.gy_keep = h->vb[14];
  s.zy_keep = h->vb[15];
  *h->h_state = s;
  CU(cudaMemcpyAsync(h->st, h->h_state, sizeof(IterState), cudaMemcpyHostToDevice, h->stream));
  CU(cudaMemsetAsync(h->bar, 0, sizeof(unsigned long long), h->stream));
  CU(cudaMemsetAsync(h->status, 0, sizeof(int), h->stream));
  // the loop reads the fixings from the handle's own copy, so that one
  // captured graph serves every solve
  const int8_t* fix_loop = nullptr;
  if (fixings) {
    CU(cudaMemcpyAsync(h->fixbuf, fixings, (size_t)h->p, cudaMemcpyDeviceToDevice, h->stream));
    fix_loop = h->fixbuf;
  }
  // ---- one iteration = fused X-pass + p-phase; enqueue `chunk` per host poll
  XSArgs xa = pass_args(h, h->pl_loop, h->loss == RELAX_LS ? LINK_LS : LINK_LOGISTIC, &h->st->ps);
  PArgs pa = base_pargs(h);
  pa.mode = PM_ITER;
  pa.fix = fix_loop;
  pa.part = h->xg;
  pa.ncl = h->pl_loop.Gr;
  pa.NB = h->pl_loop.NB;
  pa.st = h->st;
  pa.bar = h->bar;
  pa.fast_s1 = h->dtype == RELAX_F32 ? 1 : 0;   // FP32-key top-k select only for FP32 data
  pa.lossp = nullptr;                          // loss terms from z^t (FP64, in the p-phase)
  pa.y = (const double*)h->y;
  pa.n = h->n;
  // Timing mode: event records around every loop kernel (captured into the
  // graph); the host then waits for each chunk before enqueueing the next.
  const bool timing = h->opt.timing != 0;
  const int chunk = h->chunk;
  if (timing && !h->tev) {   // [chunk][3]: before X-pass, after X-pass, after p-phase
    h->tev = new (std::nothrow) cudaEvent_t[(size_t)chunk * 3]();
    if (!h->tev) return RELAX_ENOMEM;
    for (int i = 0; i < chunk * 3; ++i) CU(cudaEventCreate(&h->tev[i]));
  }
  cudaEvent_t* tev = h->tev;
  // the pass and p-phase of the current rung of the precision ladder
  const XSPlan* cur_pl = &h->pl_loop;
  const PPlan* cur_pp = &h->pp_iter;
  XSArgs cur_xa = xa;
  // inside a capture the timing events are recorded as external graph nodes;
  // on direct launches they are plain records
  bool capturing = false;
  auto rec = [&](cudaEvent_t e, cudaStream_t cs) {
    return capturing ? cudaEventRecordWithFlags(e, cs, cudaEventRecordExternal) : cudaEventRecord(e, cs);
  };
  auto enqueue_body = [&](cudaStream_t cs) -> cudaError_t {
    for (int i = 0; i < chunk; ++i) {
      cudaError_t e;
      if (timing && (e = rec(tev[3 * i], cs)) != cudaSuccess) return e;
      if ((e = run_pass(h, *cur_pl, cur_xa, cs)) != cudaSuccess) return e;
      if (timing && (e = rec(tev[3 * i + 1], cs)) != cudaSuccess) return e;
      if ((e = pphase_launch(*cur_pp, pa, cs)) != cudaSuccess) return e;
      if (timing && (e = rec(tev[3 * i + 2], cs)) != cudaSuccess) return e;
    }
    return cudaSuccess;
  };
  // capture the chunk as a graph once per shape of call (falls back to direct launches)
  if (!h->gexec || h->g_fix != (fix_loop ? 1 : 0) || h->g_timing != (timing ? 1 : 0)) {
    if (h->gexec) {
      cudaGraphExecDestroy(h->gexec);
      h->gexec = nullptr;
    }
    cudaGraph_t graph = nullptr;
    cudaStream_t cs = nullptr;
    bool ok = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking) == cudaSuccess;
    if (ok) ok = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal) == cudaSuccess;
    if (ok) {
      capturing = true;
      const bool lok = enqueue_body(cs) == cudaSuccess;
      capturing = false;
      ok = (cudaStreamEndCapture(cs, &graph) == cudaSuccess) && lok && graph;
      if (ok) ok = cudaGraphInstantiate(&h->gexec, graph, 0) == cudaSuccess;
      if (graph) cudaGraphDestroy(graph);
    }
    if (cs) cudaStreamDestroy(cs);
    if (!ok) { h->gexec = nullptr; cudaGetLastError(); }
    h->g_fix = fix_loop ? 1 : 0;
    h->g_timing = timing ? 1 : 0;
  }
  cudaGraphExec_t gexec = h->gexec;
  auto enqueue_chunk = [&]() -> cudaError_t {
    if (gexec && cur_pl == &h->pl_loop) return cudaGraphLaunch(gexec, h->stream);   // the graph is of rung 0
    return enqueue_body(h->stream);
  };
  cudaEvent_t* ev = h->ev;
  const int64_t max_chunks = (int64_t)h->max_iters / chunk + 3;
  cudaError_t err = cudaSuccess;
  int64_t nchunks = 0;
  std::vector<float> xms, pms;   // per launched iteration of the current run (timing mode)
  double xms_work = 0.0, pms_work = 0.0;
  int passes_work = 0;
  auto run_loop = [&](int64_t chunk_budget) {
    xms.clear();
    pms.clear();
    for (int64_t c = 0; c < chunk_budget; ++c) {
      err = enqueue_chunk();
      if (err != cudaSuccess) break;
      ++nchunks;
      cudaMemcpyAsync(&h->h_done[c & 1], &h->st->done, sizeof(int), cudaMemcpyDeviceToHost, h->stream);
      cudaEventRecord(ev[c & 1], h->stream);
      if (timing) {
        cudaEventSynchronize(ev[c & 1]);
        for (int i = 0; i < chunk; ++i) {
          float a = 0.f, b = 0.f;
          cudaEventElapsedTime(&a, tev[3 * i], tev[3 * i + 1]);
          cudaEventElapsedTime(&b, tev[3 * i + 1], tev[3 * i + 2]);
          xms.push_back(a);
          pms.push_back(b);
        }
        if (h->h_done[c & 1]) break;
      } else if (c >= 1) {
        cudaEventSynchronize(ev[(c - 1) & 1]);
        if (h->h_done[(c - 1) & 1]) break;
      }
    }
    cudaStreamSynchronize(h->stream);
  };
  // the first iters_in_run + 1 launches of a run did work; the rest of its last
  // chunk returned at once
  auto account = [&](int it_before, int it_after) {
    const int work = std::min<int>((int)xms.size(), it_after - it_before + 1);
    for (int t = 0; t < work; ++t) { xms_work += xms[t]; pms_work += pms[t]; }
    passes_work += it_after - it_before + 1;
  };
  int it_before = 0;
  run_loop(max_chunks);
  // The loop's gap is tracked in the working precision; when the FP64
  // certificate of the final pair misses gap_tol, continue with a tighter
  // internal tolerance (at most 3 times).
  // Two valid dual points are certified and the better bound is kept: the
  // loop's best dual point (its own z) and zeta = -grad F(X beta_best) with X
  // and the product in FP64.  A resumed run gets at most half as many
  // iterations again, and resuming stops once it no longer helps (and never
  // starts when X is stored in BF16/FP8: that gap is the quantisation's).
  int cert_rounds = 0;
  double cert_primal = 0.0, cert_dual = 0.0, prev_crel = INFINITY, crel = INFINITY;
  bool have_cert = false;
  bool ladder_ok = false;   // the last certification ended for the pass's precision, not a limit
  auto cert_phase = [&]() -> relax_status {
    const bool quantized = cur_pl->xk == XK_BF16 || cur_pl->xk == XK_FP8;
    cert_rounds = 0;
    prev_crel = INFINITY;
    ladder_ok = false;
    for (;;) {
      if (err != cudaSuccess) break;
      CU(cudaMemcpy(h->h_state, h->st, sizeof(IterState), cudaMemcpyDeviceToHost));
      int dst0 = 0;
      CU(cudaMemcpy(&dst0, h->status, sizeof(int), cudaMemcpyDeviceToHost));
      account(it_before, h->h_state->iter);
      if (dst0 != ST_OK || !h->certify) break;
      const IterState& S0 = *h->h_state;
      relax_status r = certify_pair(h, fixings, S0.beta_best, S0.z_dbest);
      if (r != RELAX_OK) return r;
      const double phi = h->h_d[0];
      double psi = h->h_d[1];
      if (h->h_d[3] > psi || !(psi == psi)) psi = h->h_d[3];
      out->launches += 3;
      // every rung's dual bound is valid: the best one stays
      cert_dual = have_cert ? std::max(cert_dual, psi) : psi;
      cert_primal = phi;
      have_cert = true;
      crel = (cert_primal - cert_dual) / std::max(1.0, std::fabs(cert_primal));
      if (crel <= gap_tol || S0.iter >= h->max_iters || !(crel == crel) || S0.cut_rule) break;
      if (quantized || S0.stalled || cert_rounds >= 3 || crel > 0.9 * prev_crel) {
        ladder_ok = true;
        break;
      }
      prev_crel = crel;
      ++cert_rounds;
      double tol_new = S0.tol * 0.25;
      int zero = 0;
      CU(cudaMemcpyAsync(&h->st->tol, &tol_new, sizeof(double), cudaMemcpyHostToDevice, h->stream));
      CU(cudaMemcpyAsync(&h->st->done, &zero, sizeof(int), cudaMemcpyHostToDevice, h->stream));
      CU(cudaMemcpyAsync(&h->st->ps.done, &zero, sizeof(int), cudaMemcpyHostToDevice, h->stream));
      CU(cudaStreamSynchronize(h->stream));
      it_before = S0.iter;
      run_loop(std::max<int64_t>(8, (int64_t)S0.iter / (2 * chunk) + 1));
    }
    return RELAX_OK;
  };
  rs = cert_phase();
  if (rs != RELAX_OK) return rs;
  // the timing covers the loop's own pass (rung 0)
  const double xms_loop = xms_work, pms_loop = pms_work;
  const int passes_loop = passes_work;
  // Precision ladder: when the certified gap misses gap_tol because of the
  // pass's precision (the loop stalled on its arithmetic's floor, or the
  // loop's problem is the BF16 / FP8 copy of X), the loop goes on from
  // beta_best on the FP32 master X, then with float-float products on it,
  // with the FP64 p-phase.
  for (int rung = 0; err == cudaSuccess && ladder_ok && h->certify;) {
    if (rung == 0 && h->has_acc32) { rung = 1; cur_pl = &h->pl_acc32; }
    else if (rung < 2 && h->has_ff) { rung = 2; cur_pl = &h->pl_ff; }
    else break;
    cur_pp = &h->pp_exact;
    cur_xa = pass_args(h, *cur_pl, h->loss == RELAX_LS ? LINK_LS : LINK_LOGISTIC, &h->st->ps);
    pa.ncl = cur_pl->Gr;
    const int it0 = h->h_state->iter;
    if (it0 >= h->max_iters) break;
    // a warm start from beta_best: the first state again, the iteration count kept
    init_vectors_kernel<<<g, 256, 0, h->stream>>>(s.beta_best, 1, (double*)h->vb[0], (double*)h->vb[1],
                                                  (double*)h->vb[4], (double*)h->vb[5], (double*)h->vb[2],
                                                  (double*)h->vb[3], h->p, (double*)h->vb[6], (double*)h->vb[7],
                                                  h->n);
    CU(cudaGetLastError());
    IterState s2 = s;
    s2.iter = it0;
    s2.tol = tol_exact;
    *h->h_state = s2;
    CU(cudaMemcpyAsync(h->st, h->h_state, sizeof(IterState), cudaMemcpyHostToDevice, h->stream));
    CU(cudaMemsetAsync(h->bar, 0, sizeof(unsigned long long), h->stream));
    CU(cudaStreamSynchronize(h->stream));
    out->ladder = rung;
    it_before = it0;
    run_loop(max_chunks);
    rs = cert_phase();
    if (rs != RELAX_OK) return rs;
  }
  if (err != cudaSuccess) {
    set_detail("loop chunk launch", err, __LINE__);
    return map_cuda(err);
  }
  out->launches += (int)(nchunks * chunk * 2) + 1 + (fixings ? 1 : 0);   // loop + init (+ count)
  CU(cudaMemcpy(h->h_state, h->st, sizeof(IterState), cudaMemcpyDeviceToHost));
  int dst = 0;
  CU(cudaMemcpy(&dst, h->status, sizeof(int), cudaMemcpyDeviceToHost));
  const IterState& S = *h->h_state;
  out->iters = S.iter;
  out->xpass_count = passes_loop;
  if (timing) {
    out->xpass_ms = xms_loop;
    out->pphase_ms = pms_loop;
  }
  out->restarts = S.restarts;
  out->stalled = S.stalled;
  out->backtracks = S.backtracks;
  out->lipschitz = S.Lk;
  out->cutoff_rule = S.cut_rule;
  out->primal_loop = S.phi_best;
  out->dual_loop = S.psi_best;
  out->primal = have_cert ? cert_primal : S.phi_best;
  out->dual_bound = have_cert ? cert_dual : S.psi_best;
  relax_status status = map_dev_status(dst);
  out->gap = out->primal - out->dual_bound;
  out->rel_gap = out->gap / std::max(1.0, std::fabs(out->primal));
  from_f64_kernel<<<grid_for(h->p), 256, 0, h->stream>>>((const double*)S.beta_best, beta_out, h->f64(), h->p);
  CU(cudaGetLastError());
  CU(cudaMemsetAsync(h->iscr, 0, sizeof(int), h->stream));
  nnz_kernel<<<grid_for(h->p), 256, 0, h->stream>>>((const double*)S.beta_best, h->p, h->iscr);
  CU(cudaMemcpyAsync(h->h_i, h->iscr, sizeof(int), cudaMemcpyDeviceToHost, h->stream));
  CU(cudaStreamSynchronize(h->stream));
  out->n_nz = h->h_i[0];
  out->launches += 2;
  if (status == RELAX_OK) {
    if (!std::isfinite(out->dual_bound) || std::isnan(out->primal)) status = RELAX_ENUMERIC;
    else if (out->dual_bound > out->primal + 1e-9 * std::max(1.0, std::fabs(out->primal)))
      status = RELAX_EINVALID_BOUND;
    else if (!(out->rel_gap <= gap_tol) && !S.cut_rule)   // the certified gap when certification ran
      status = RELAX_ENOTCONV;
  }
  out->status = status;
  return status;
}

// One CTA takes the library's grid barrier expecting a partner that never
// arrives: the bounded wait must give up after limit_ns and record ST_TIMEOUT.
__global__ void watchdog_probe_kernel(unsigned long long* counter, uint64_t limit_ns, int* status, int* ok) {
  const bool passed = grid_barrier(counter, 2ull, limit_ns, status);
  if (threadIdx.x == 0) *ok = passed ? 1 : 0;
}

relax_status relax_watchdog_probe(int32_t watchdog_ms, double* waited_ms, void* stream) {
  if (watchdog_ms <= 0 || watchdog_ms > 60000) return RELAX_EINVAL;
  cudaStream_t st = (cudaStream_t)stream;
  unsigned char* buf = nullptr;
  relax_status rs = alloc((void**)&buf, 64);
  if (rs != RELAX_OK) return rs;
  unsigned long long* counter = reinterpret_cast<unsigned long long*>(buf);
  int* status = reinterpret_cast<int*>(buf + 16);
  int* ok = reinterpret_cast<int*>(buf + 32);
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaError_t e = cudaMemsetAsync(buf, 0, 64, st);
  if (e == cudaSuccess) e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  if (e == cudaSuccess) e = cudaEventRecord(e0, st);
  if (e == cudaSuccess) {
    watchdog_probe_kernel<<<1, 32, 0, st>>>(counter, (uint64_t)watchdog_ms * 1000000ull, status, ok);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaEventRecord(e1, st);
  int hs[2] = {0, 0};
  if (e == cudaSuccess) e = cudaMemcpyAsync(&hs[0], status, sizeof(int), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(&hs[1], ok, sizeof(int), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  float ms = 0.f;
  if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  cudaFree(buf);
  if (e != cudaSuccess) {
    set_detail("watchdog probe", e, __LINE__);
    return map_cuda(e);
  }
  if (waited_ms) *waited_ms = ms;
  if (hs[1]) return RELAX_OK;                 // cannot happen: nobody else arrives
  return map_dev_status(hs[0]);
}

relax_status relax_set_cutoff(relax_handle* h, double cutoff) {
  if (!h || std::isnan(cutoff)) return RELAX_EINVAL;
  h->cutoff = cutoff;
  return RELAX_OK;
}

relax_status relax_xpass(relax_handle* h, const void* beta, void* z_out, void* g_out, double* loss_host) {
  if (!h || !beta || !g_out) return RELAX_EINVAL;
  CU(cudaSetDevice(h->dev));
  double* b64 = (double*)h->vb[8];
  double* g64 = (double*)h->vb[9];
  double* z64 = (double*)h->vb[10];
  double* zp64 = (double*)h->vb[11];
  to_f64_kernel<<<grid_for(h->p), 256, 0, h->stream>>>(beta, h->f64(), b64, h->p);
  CU(cudaGetLastError());
  PassState ps{};
  ps.beta = b64;
  ps.zout = z64;
  ps.zprev = zp64;
  ps.mom = 0.0;
  *reinterpret_cast<PassState*>(h->h_d + 1000) = ps;
  CU(cudaMemcpyAsync(h->ps_aux, h->h_d + 1000, sizeof(PassState), cudaMemcpyHostToDevice, h->stream));
  CU(cudaMemsetAsync(h->status, 0, sizeof(int), h->stream));
  CU(cudaMemsetAsync(zp64, 0, (size_t)h->n * sizeof(double), h->stream));
  XSArgs a = pass_args(h, h->pl_loop, h->loss == RELAX_LS ? LINK_LS : LINK_LOGISTIC, h->ps_aux);
  CU(run_pass(h, h->pl_loop, a, h->stream));
  const unsigned g = grid_for(h->p);
  reduce_partials_kernel<double, double><<<g, 256, 0, h->stream>>>(h->xg, h->pl_loop.Gr, h->pl_loop.NB, h->p, g64, nullptr);
  from_f64_kernel<<<g, 256, 0, h->stream>>>(g64, g_out, h->f64(), h->p);
  if (z_out) from_f64_kernel<<<grid_for(h->n), 256, 0, h->stream>>>(z64, z_out, h->f64(), h->n);
  CU(cudaMemsetAsync(h->dscr, 0, 2 * sizeof(double), h->stream));
  loss_terms_kernel<<<grid_for(h->n), 256, 0, h->stream>>>(z64, (const double*)h->y, h->n, h->loss, h->dscr);
  CU(cudaGetLastError());
  CU(cudaMemcpyAsync(h->h_d, h->dscr, 2 * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
  CU(cudaStreamSynchronize(h->stream));
  int dst = 0;
  CU(cudaMemcpy(&dst, h->status, sizeof(int), cudaMemcpyDeviceToHost));
  if (loss_host) {
    loss_host[0] = h->h_d[0];
    loss_host[1] = h->h_d[1];
  }
  if (dst != ST_OK) snprintf(g_detail, sizeof(g_detail), "fused pass: device status %d", dst);
  return map_dev_status(dst);
}

relax_status relax_certify(relax_handle* h, const int8_t* fixings, const void* beta_primal, const void* beta_dual,
                           double* out_host) {
  if (!h || !beta_primal || !beta_dual || !out_host) return RELAX_EINVAL;
  CU(cudaSetDevice(h->dev));
  int j1 = 0, jf = 0;
  relax_status rs = count_fixings(h, fixings, &j1, &jf);
  if (rs != RELAX_OK) return rs;
  if (h->k < j1) return RELAX_EINVAL;
  CU(cudaMemsetAsync(h->status, 0, sizeof(int), h->stream));
  to_f64_kernel<<<grid_for(h->p), 256, 0, h->stream>>>(beta_primal, h->f64(), (double*)h->vb[8], h->p);
  to_f64_kernel<<<grid_for(h->p), 256, 0, h->stream>>>(beta_dual, h->f64(), (double*)h->vb[9], h->p);
  CU(cudaGetLastError());
  // one product when both points are the same vector
  rs = certify(h, fixings, h->vb[8], beta_dual == beta_primal ? h->vb[8] : h->vb[9], nullptr);
  if (rs != RELAX_OK) return rs;
  int dst = 0;
  CU(cudaMemcpy(&dst, h->status, sizeof(int), cudaMemcpyDeviceToHost));
  out_host[0] = h->h_d[0];
  out_host[1] = h->h_d[1];
  return map_dev_status(dst);
}

// ------------------------------------------------- standalone regularizer ops
static relax_status standalone(int mode, const void* vin, void* vout, int64_t p, double rho, int32_t k,
                               double lambda2, double M, const int8_t* fix, int32_t dtype, int32_t* counts,
                               double* out_host, cudaStream_t st) {
  if (!vin || p <= 0 || k < 0 || !(M > 0.0) || (dtype != RELAX_F64 && dtype != RELAX_F32)) return RELAX_EINVAL;
  const bool dbl = dtype == RELAX_F64;
  PPlan pl;
  CU(pphase_plan(pl, dbl, p));
  // scratch: round accumulators, block partials, barrier counter, status, output
  const size_t acc_b = 3 * ACC_STRIDE * sizeof(unsigned long long);
  const size_t bp_b = (size_t)2 * pl.grid * NBP * sizeof(double);
  const size_t tot = acc_b + bp_b + 64;
  unsigned char* scr = nullptr;
  CU(cudaMallocAsync((void**)&scr, tot, st));
  cudaError_t e = cudaMemsetAsync(scr, 0, tot, st);
  PArgs a{};
  a.mode = mode;
  a.p = p;
  a.k = k;
  a.lambda2 = lambda2;
  a.M = M;
  a.rho = rho;
  a.kc = pconst_make(lambda2, M, 0.0, rho);
  a.fix = fix;
  a.vin = vin;
  a.vout = vout;
  a.counts = counts;
  a.acc = reinterpret_cast<unsigned long long*>(scr);
  a.bpart = reinterpret_cast<double*>(scr + acc_b);
  a.bar = reinterpret_cast<unsigned long long*>(scr + acc_b + bp_b);
  a.status = reinterpret_cast<int*>(scr + acc_b + bp_b + 8);
  a.out = reinterpret_cast<double*>(scr + acc_b + bp_b + 16);
  a.bar_base = 0;
  a.limit_ns = 4000000000ull;
  if (e == cudaSuccess) e = pphase_launch(pl, a, st);
  relax_status rs = RELAX_OK;
  if (e == cudaSuccess && out_host) {
    double hv[3] = {0, 0, 0};
    int dst = 0;
    e = cudaMemcpyAsync(hv, a.out, sizeof(double), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&dst, a.status, sizeof(int), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e == cudaSuccess) {
      out_host[0] = hv[0];
      rs = map_dev_status(dst);
    }
  }
  cudaFreeAsync(scr, st);
  if (e != cudaSuccess) return map_cuda(e);
  return rs;
}

relax_status prox_persp(const void* beta_in, void* beta_out, int64_t p, double step, int32_t k, double lambda2,
                        double M, const int8_t* fixings, int32_t dtype, int32_t* counts_out, void* stream) {
  if (!beta_out || !(step > 0.0) || !(lambda2 > 0.0)) return RELAX_EINVAL;
  return standalone(PM_PROX, beta_in, beta_out, p, 2.0 * lambda2 * step, k, lambda2, M, fixings, dtype, counts_out,
                    nullptr, (cudaStream_t)stream);
}

relax_status gval_persp(const void* beta, int64_t p, int32_t k, double M, const int8_t* fixings, int32_t dtype,
                        double* out_host, void* stream) {
  if (!out_host) return RELAX_EINVAL;
  return standalone(PM_GVAL, beta, nullptr, p, 1.0, k, 1.0, M, fixings, dtype, nullptr, out_host,
                    (cudaStream_t)stream);
}

relax_status gstar_persp(const void* alpha, int64_t p, int32_t k, double M, const int8_t* fixings, int32_t dtype,
                         double* out_host, void* stream) {
  if (!out_host) return RELAX_EINVAL;
  return standalone(PM_GSTAR, alpha, nullptr, p, 1.0, k, 1.0, M, fixings, dtype, nullptr, out_host,
                    (cudaStream_t)stream);
}

}  // extern "C"

// Error text for this thread's relax_error_detail(), set by other translation
// units of the library.
namespace relax {
void set_error_detail(const char* msg) { snprintf(g_detail, sizeof(g_detail), "%s", msg); }
}  // namespace relax

// ======================================================= batched node solves
// Many node relaxations of one design in lockstep: per iteration the active
// nodes' points form the rows of B, and Z = X B' and G = X' R are two
// products.  FP32 data: the library's tcgen05 kernel (bgemm.cu) on BF16
// planes of X, X' and the operands (FP32-accurate products, FP64 sums of the
// K chunks, fused with the link and the gradient layout).  FP64 data: plain
// tiled FP64 products on the CUDA cores.  The p-phase of every active node
// runs in one segmented launch (one thread-block cluster per node, or
// cooperative waves when p needs more CTAs than a cluster holds).  Converged
// nodes leave the active set every kRetire iterations; each round of kRetire
// iterations is captured as a CUDA graph per active-set size; a node stalled
// on the products' floor is finished by the single-node loop.
namespace {

constexpr int kRetire = 16;
constexpr int kBatchStall = 200;  // least stall window inside a batch (iterations)

// FP64 data: B[s][j] = the next point of node active[s]
__global__ void batch_pack_f64_kernel(const IterState* st, const int* active, int m, int64_t p, double* Bm) {
  const int s = blockIdx.y;
  if (s >= m) return;
  const double* b = static_cast<const double*>(st[active[s]].ps.beta);
  for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < p; j += (int64_t)gridDim.x * blockDim.x)
    Bm[(size_t)s * p + j] = b[j];
}

// FP64 products on the CUDA cores, 64 x 16 outputs per block of 256 threads
// (4 per thread), K in steps of 32 through shared memory:
//   Z[s][i] = sum_j X[i][j] B[s][j]        (rows i of X, points s)
//   G[c][j] = sum_i X[i][j] R[c][i]        (columns j of X, right-hand sides c)
__global__ void zprod_f64_kernel(const double* X, int64_t ldx, int64_t n, int64_t p, const double* B, int m,
                                 double* Z) {
  __shared__ double xs[64][33], bs[16][33];
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;   // 16 x 16
  const int64_t i0 = (int64_t)blockIdx.x * 64;
  const int s0 = blockIdx.y * 16;
  double acc[4] = {0, 0, 0, 0};
  for (int64_t k0 = 0; k0 < p; k0 += 32) {
    for (int t = threadIdx.x; t < 64 * 32; t += 256) {
      const int r = t >> 5, c = t & 31;
      xs[r][c] = (i0 + r < n && k0 + c < p) ? X[(i0 + r) * ldx + k0 + c] : 0.0;
    }
    for (int t = threadIdx.x; t < 16 * 32; t += 256) {
      const int r = t >> 5, c = t & 31;
      bs[r][c] = (s0 + r < m && k0 + c < p) ? B[(int64_t)(s0 + r) * p + k0 + c] : 0.0;
    }
    __syncthreads();
#pragma unroll 8
    for (int c = 0; c < 32; ++c) {
      const double bv = bs[tx][c];
#pragma unroll
      for (int q = 0; q < 4; ++q) acc[q] += xs[ty + 16 * q][c] * bv;
    }
    __syncthreads();
  }
  if (s0 + tx < m)
    for (int q = 0; q < 4; ++q)
      if (i0 + ty + 16 * q < n) Z[(int64_t)(s0 + tx) * n + i0 + ty + 16 * q] = acc[q];
}
__global__ void gprod_f64_kernel(const double* X, int64_t ldx, int64_t n, int64_t p, const double* R, int nc,
                                 double* G) {
  __shared__ double xs[32][65], rs[16][33];
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  const int64_t j0 = (int64_t)blockIdx.x * 64;
  const int c0 = blockIdx.y * 16;
  double acc[4] = {0, 0, 0, 0};
  for (int64_t k0 = 0; k0 < n; k0 += 32) {
    for (int t = threadIdx.x; t < 32 * 64; t += 256) {
      const int r = t >> 6, c = t & 63;
      xs[r][c] = (k0 + r < n && j0 + c < p) ? X[(k0 + r) * ldx + j0 + c] : 0.0;
    }
    for (int t = threadIdx.x; t < 16 * 32; t += 256) {
      const int r = t >> 5, c = t & 31;
      rs[r][c] = (c0 + r < nc && k0 + c < n) ? R[(int64_t)(c0 + r) * n + k0 + c] : 0.0;
    }
    __syncthreads();
#pragma unroll 8
    for (int k = 0; k < 32; ++k) {
      const double rv = rs[tx][k];
#pragma unroll
      for (int q = 0; q < 4; ++q) acc[q] += xs[k][ty + 16 * q] * rv;
    }
    __syncthreads();
  }
  if (c0 + tx < nc)
    for (int q = 0; q < 4; ++q)
      if (j0 + ty + 16 * q < p) G[(int64_t)(c0 + tx) * p + j0 + ty + 16 * q] = acc[q];
}

// FP64 data: z of node active[s] to its state, and the link: R[s] = grad F(z)
// and, for the logistic loop, R[m + s] = grad F at the momentum point
__global__ void batch_link_f64_kernel(const IterState* st, const int* active, int m, int64_t n, const double* Z,
                                      const double* y, int loss, double* R) {
  const int s = blockIdx.y;
  if (s >= m) return;
  const IterState& S = st[active[s]];
  if (S.done) return;
  double* zout = static_cast<double*>(S.ps.zout);
  const double* zprev = static_cast<const double*>(S.ps.zprev);
  const double mom = S.ps.mom;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const double z = Z[(size_t)s * n + i];
    const double yd = y[i];
    zout[i] = z;
    if (loss == RELAX_LS) {
      R[(size_t)s * n + i] = 2.0 * (z - yd);
    } else {
      R[(size_t)s * n + i] = -yd / (1.0 + exp(yd * z));
      const double zy = (1.0 + mom) * z - mom * zprev[i];
      R[(size_t)(m + s) * n + i] = -yd / (1.0 + exp(yd * zy));
    }
  }
}

// FP64 data: part[s][q][j] = G[q m + s][j] (the p-phase's gradient layout)
__global__ void batch_grad_f64_kernel(const double* G, int m, int NB, int64_t p, double* part) {
  const int s = blockIdx.y;
  if (s >= m) return;
  for (int q = 0; q < NB; ++q)
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < p; j += (int64_t)gridDim.x * blockDim.x)
      part[((size_t)s * NB + q) * p + j] = G[(size_t)(q * m + s) * p + j];
}

__global__ void batch_done_kernel(const IterState* st, const int* active, int m, int* done) {
  for (int s = blockIdx.x * blockDim.x + threadIdx.x; s < m; s += gridDim.x * blockDim.x)
    done[s] = st[active[s]].done;
}

// BF16 planes of X and X' for the tensor-core products (built on the first
// batched solve of a handle)
relax_status ensure_planes(relax_handle* h) {
  if (h->bx) return RELAX_OK;
  const int64_t n = h->n, p = h->p;
  h->ldbp = (p + 7) / 8 * 8;
  h->ldbn = (n + 7) / 8 * 8;
  relax_status rs = alloc((void**)&h->bx, sizeof(__nv_bfloat16) * 3 * (size_t)n * h->ldbp);
  if (rs == RELAX_OK) rs = alloc((void**)&h->bxt, sizeof(__nv_bfloat16) * 3 * (size_t)p * h->ldbn);
  if (rs != RELAX_OK) {
    if (h->bx) cudaFree(h->bx);
    h->bx = nullptr;
    return rs;
  }
  CU(bgemm_split_x((const float*)h->X, n, p, h->ldx, false, h->bx, h->ldbp, h->stream));
  CU(bgemm_split_x((const float*)h->X, n, p, h->ldx, true, h->bxt, h->ldbn, h->stream));
  CU(bgemm_encode(&h->tm_bx, h->bx, p, n, h->ldbp, n, BG_BM));
  CU(bgemm_encode(&h->tm_bxt, h->bxt, n, p, h->ldbn, p, BG_BM));
  return RELAX_OK;
}

void fill_bgargs(BGArgs& a, const BGPlan& pl, double* P, int* status, uint64_t limit_ns) {
  a.M = pl.M; a.N = pl.N; a.K = pl.K;
  a.BN = pl.BN; a.NT = pl.NT; a.MT = pl.MT;
  a.nkb = pl.nkb; a.stages = pl.stages;
  a.P = P;
  a.status = status;
  a.limit_ns = limit_ns;
}

}  // namespace

extern "C" relax_status relax_solve_batch(relax_handle* h, int32_t nb, const int8_t* fixings, const void* warm_start,
                                          double gap_tol, void* beta_out, relax_result* out) {
  if (!h || nb <= 0 || !beta_out || !out || !(gap_tol > 0.0)) return RELAX_EINVAL;
  if (h->xk_loop != XK_F32 && h->xk_loop != XK_F64) return RELAX_ENOTSUP;   // BF16/FP8 storage: single solves
  CU(cudaSetDevice(h->dev));
  const int64_t n = h->n, p = h->p;
  const bool f64 = h->xk_loop == XK_F64;
  const size_t es = f64 ? 8 : 4;
  const int NB = h->loss == RELAX_LS ? 1 : 2;
  std::memset(out, 0, sizeof(relax_result) * (size_t)nb);
  BatchWs& W = h->bw;
  // ---- p-phase segments (planned once per handle): one thread-block cluster
  // per node when p fits one cluster (hardware barriers, one launch for every
  // node), else the fewest CTAs that cover p in cooperative waves of
  // co-resident segments
  if (!W.planned) {
    W.clustered = pphase_cluster_plan(W.pc, p, h->backtrack != 0, !f64 && !h->backtrack) == cudaSuccess &&
                  !std::getenv("RELAX_BATCH_WAVES");
    cudaGetLastError();   // a refused cluster plan leaves no sticky error
    W.planned = true;
  }
  PPlan pp = h->pp_iter;
  const PPlan pc = W.pc;
  const bool clustered = W.clustered;
  const int segb = clustered ? pc.seg
                             : (int)std::max<int64_t>(1, (p + (int64_t)PBLOCK * PEPT - 1) / ((int64_t)PBLOCK * PEPT));
  const int wave = std::max(1, pp.maxgrid / segb);
  if (!clustered && segb > pp.maxgrid) return RELAX_ENOTSUP;
  // ---- device memory of the batch (the handle's, grown to nb nodes)
  const size_t nvec = 8 * (size_t)p + 4 * (size_t)n;   // per node: 8 p-vectors, 4 n-vectors (FP64)
  if (nb > W.cap) {
    cudaStreamSynchronize(h->stream);
    W.release();
    const int cap = (nb + 63) / 64 * 64;
    bool ok = true;
    auto get = [&](void** q, size_t bytes) { if (ok && alloc(q, bytes) != RELAX_OK) ok = false; };
    get((void**)&W.dst, sizeof(IterState) * (size_t)cap);
    get((void**)&W.vec, sizeof(double) * nvec * (size_t)cap);
    get((void**)&W.acc, sizeof(unsigned long long) * 3 * ACC_STRIDE * (size_t)cap);
    get((void**)&W.bpart, sizeof(double) * 2 * (size_t)segb * NBP * (size_t)cap);
    get((void**)&W.bars, sizeof(unsigned long long) * (size_t)cap);
    if (f64) {
      get(&W.Bm, es * (size_t)p * cap);
      get(&W.Zm, es * (size_t)n * cap);
      get(&W.Rm, es * (size_t)n * NB * cap);
      get(&W.Gm, es * (size_t)p * NB * cap);
    } else {
      if (ok && ensure_planes(h) != RELAX_OK) ok = false;
      get((void**)&W.Bp, sizeof(__nv_bfloat16) * 3 * (size_t)cap * h->ldbp);
      get((void**)&W.Rp, sizeof(__nv_bfloat16) * 3 * (size_t)NB * cap * h->ldbn);
      get((void**)&W.P1, sizeof(double) * BG_MAXKC * (size_t)cap * n);
      get((void**)&W.P2, sizeof(double) * BG_MAXKC * (size_t)NB * cap * p);
    }
    get((void**)&W.part, sizeof(double) * (size_t)p * NB * cap);
    get((void**)&W.active_d, sizeof(int) * (size_t)cap);
    get((void**)&W.done_d, sizeof(int) * (size_t)cap);
    get((void**)&W.fix, (size_t)p * cap);
    get((void**)&W.cnt, sizeof(int) * 3 * (size_t)cap);
    get((void**)&W.psd, sizeof(PassState) * 2 * (size_t)cap);
    get((void**)&W.certd, sizeof(double) * 4 * (size_t)cap);
    if (!ok) {
      W.release();
      return RELAX_ENOMEM;
    }
    if (!f64) {
      // finite operands everywhere (rows past the active nodes are read by
      // no product, but the planes start defined)
      CU(cudaMemsetAsync(W.Bp, 0, sizeof(__nv_bfloat16) * 3 * (size_t)cap * h->ldbp, h->stream));
      CU(cudaMemsetAsync(W.Rp, 0, sizeof(__nv_bfloat16) * 3 * (size_t)NB * cap * h->ldbn, h->stream));
    }
    W.cap = cap;
  }
  const int cap = W.cap;
  IterState* dst = W.dst;
  double* vec = W.vec;
  unsigned long long* acc = W.acc;
  double* bpart = W.bpart;
  unsigned long long* bars = W.bars;
  void *Bm = W.Bm, *Zm = W.Zm, *Rm = W.Rm, *Gm = W.Gm;
  __nv_bfloat16 *Bp = W.Bp, *Rp = W.Rp;
  double *P1 = W.P1, *P2 = W.P2;
  double* part = W.part;
  int* active_d = W.active_d;
  int* done_d = W.done_d;
  // ---- the call's fixings, in the workspace (the graphs read them there),
  // and their counts per node
  std::vector<int> j1(nb, 0), jf(nb, (int)p);
  if (fixings) {
    CU(cudaMemcpyAsync(W.fix, fixings, (size_t)p * nb, cudaMemcpyDeviceToDevice, h->stream));
    std::vector<int> hc(3 * (size_t)nb);
    CU(cudaMemsetAsync(W.cnt, 0, sizeof(int) * 3 * (size_t)nb, h->stream));
    count_fix_batch_kernel<<<dim3((unsigned)std::min<int64_t>(64, (p + 255) / 256), (unsigned)nb), 256, 0,
                             h->stream>>>(W.fix, p, W.cnt);
    CU(cudaGetLastError());
    CU(cudaMemcpyAsync(hc.data(), W.cnt, sizeof(int) * 3 * (size_t)nb, cudaMemcpyDeviceToHost, h->stream));
    CU(cudaStreamSynchronize(h->stream));
    for (int j = 0; j < nb; ++j) {
      if (hc[3 * j + 2] != 0 || hc[3 * j] > h->k) return RELAX_EINVAL;
      j1[j] = hc[3 * j];
      jf[j] = hc[3 * j + 1];
    }
  } else {
    CU(cudaMemsetAsync(W.fix, 0, (size_t)p * nb, h->stream));
  }
  std::vector<std::pair<int, cudaGraphExec_t>>& graphs = W.graphs;   // one round of iterations per active-set size
  relax_status rs = RELAX_OK;
  auto cleanup = [&]() {};
#define BTRY(x)                    \
  do {                             \
    rs = (x);                      \
    if (rs != RELAX_OK) {          \
      cudaStreamSynchronize(h->stream); \
      cleanup();                   \
      return rs;                   \
    }                              \
  } while (0)
#define BTRYC(x)                                   \
  do {                                             \
    cudaError_t ec_ = (x);                         \
    if (ec_ != cudaSuccess) {                      \
      set_detail(#x, ec_, __LINE__);               \
      cudaStreamSynchronize(h->stream);            \
      cleanup();                                   \
      return map_cuda(ec_);                        \
    }                                              \
  } while (0)
  BTRYC(cudaMemsetAsync(acc, 0, sizeof(unsigned long long) * 3 * ACC_STRIDE * (size_t)nb, h->stream));
  BTRYC(cudaMemsetAsync(bars, 0, sizeof(unsigned long long) * (size_t)nb, h->stream));
  BTRYC(cudaMemsetAsync(h->status, 0, sizeof(int), h->stream));
  // ---- node states
  std::vector<IterState> hs(nb);
  const double loop_tol = f64 ? gap_tol : 0.7 * gap_tol;
  for (int j = 0; j < nb; ++j) {
    double* v = vec + nvec * (size_t)j;
    IterState s{};
    s.beta_prev = v;
    s.beta_cur = v + p;
    s.G_prev = v + 2 * p;
    s.G_cur = v + 3 * p;
    s.beta_best = v + 4 * p;
    s.beta_dbest = v + 5 * p;
    s.y_keep = v + 6 * p;
    s.gy_keep = v + 7 * p;
    s.z_prev = v + 8 * p;
    s.z_cur = v + 8 * p + n;
    s.z_dbest = v + 8 * p + 2 * n;
    s.zy_keep = v + 8 * p + 3 * n;
    s.tau = 1.0;
    s.gap_ref = INFINITY;
    s.phi_best = INFINITY;
    s.psi_best = -INFINITY;
    s.stall_gap = INFINITY;
    s.kbar = h->k - j1[j];
    s.pbar = jf[j];
    s.tol = loop_tol;
    s.cutoff_on = std::isfinite(h->cutoff) ? 1 : 0;
    s.cutoff = h->cutoff;
    s.Lk = h->backtrack ? h->L / 64.0 : h->L;
    s.rho_last = 2.0 * h->lambda2 / s.Lk;
    s.ps.beta = s.beta_cur;
    s.ps.zout = s.z_cur;
    s.ps.zprev = s.z_prev;
    s.ps.mom = 0.0;
    hs[j] = s;
  }
  init_batch_kernel<<<dim3((unsigned)std::min<int64_t>(64, (std::max(p, n) + 255) / 256), (unsigned)nb), 256, 0,
                      h->stream>>>(warm_start, f64 ? 1 : 0, vec, (int64_t)nvec, p, n);
  BTRYC(cudaGetLastError());
  BTRYC(cudaMemcpyAsync(dst, hs.data(), sizeof(IterState) * (size_t)nb, cudaMemcpyHostToDevice, h->stream));
  // ---- p-phase arguments (segmented)
  PArgs pa = base_pargs(h);
  pa.mode = PM_ITER;
  pa.fix = W.fix;
  pa.fix_stride = p;
  pa.part = part;
  pa.part_stride = (int64_t)NB * p;
  pa.ncl = 1;
  pa.NB = NB;
  pa.st = dst;
  pa.bar = bars;
  pa.acc = acc;
  pa.bpart = bpart;
  pa.fast_s1 = h->dtype == RELAX_F32 ? 1 : 0;
  pa.lossp = nullptr;
  pa.y = (const double*)h->y;
  pa.n = n;
  pa.seg_blocks = segb;
  // a node on the floor of the products hands over to the single-node finish
  // after a shorter stall than a single solve waits
  if (pa.stall_min > kBatchStall) pa.stall_min = kBatchStall;
  // ---- the loop
  std::vector<int> active(nb), hdone(nb);
  for (int j = 0; j < nb; ++j) active[j] = j;
  const int max_rounds = h->max_iters / kRetire + 2;
  int launches = 0;
  for (int round = 0; round < max_rounds && !active.empty(); ++round) {
    const int m = (int)active.size();
    BTRYC(cudaMemcpyAsync(active_d, active.data(), sizeof(int) * (size_t)m, cudaMemcpyHostToDevice, h->stream));
    // products of this round's active-set size
    BGPlan pl1, pl2;
    BGArgs a1{}, a2{};
    BatchIo io{};
    if (!f64) {
      BTRYC(bgemm_plan(pl1, (int)n, m, (int)p));
      BTRYC(bgemm_plan(pl2, (int)p, NB * m, (int)n));
      a1.tmA = h->tm_bx;
      a2.tmA = h->tm_bxt;
      BTRYC(bgemm_encode(&a1.tmB, Bp, p, m, h->ldbp, cap, pl1.BN));
      BTRYC(bgemm_encode(&a2.tmB, Rp, n, (int64_t)NB * m, h->ldbn, (int64_t)NB * cap, pl2.BN));
      fill_bgargs(a1, pl1, P1, h->status, h->limit_ns);
      fill_bgargs(a2, pl2, P2, h->status, h->limit_ns);
      io.st = dst;
      io.active = active_d;
      io.m = m;
      io.nb = cap;
      io.n = n;
      io.p = p;
      io.ldp = h->ldbp;
      io.ldn = h->ldbn;
      io.NB = NB;
      io.loss = h->loss;
      io.y = (const double*)h->y;
      io.Bp = Bp;
      io.Rp = Rp;
      io.P1 = P1;
      io.s1 = pl1.split();
      io.P2 = P2;
      io.s2 = pl2.split();
      io.part = part;
    }
    const dim3 gp((unsigned)std::min<int64_t>(64, (p + 255) / 256), (unsigned)m);
    const dim3 gn((unsigned)std::min<int64_t>(64, (n + 255) / 256), (unsigned)m);
    const dim3 gz((unsigned)((n + 63) / 64), (unsigned)((m + 15) / 16));
    const dim3 gg((unsigned)((p + 63) / 64), (unsigned)((NB * m + 15) / 16));
    int round_launches = 0;
    auto enqueue_round = [&](cudaStream_t cs) -> cudaError_t {
      round_launches = 0;
      for (int it = 0; it < kRetire; ++it) {
        cudaError_t e;
        if (f64) {
          batch_pack_f64_kernel<<<gp, 256, 0, cs>>>(dst, active_d, m, p, (double*)Bm);
          zprod_f64_kernel<<<gz, 256, 0, cs>>>((const double*)h->X, h->ldx, n, p, (const double*)Bm, m, (double*)Zm);
          batch_link_f64_kernel<<<gn, 256, 0, cs>>>(dst, active_d, m, n, (const double*)Zm, (const double*)h->y,
                                                    h->loss, (double*)Rm);
          gprod_f64_kernel<<<gg, 256, 0, cs>>>((const double*)h->X, h->ldx, n, p, (const double*)Rm, NB * m,
                                               (double*)Gm);
          batch_grad_f64_kernel<<<gp, 256, 0, cs>>>((const double*)Gm, m, NB, p, part);
          if ((e = cudaGetLastError()) != cudaSuccess) return e;
        } else {
          if ((e = batch_pack(io, cs)) != cudaSuccess) return e;
          if ((e = bgemm_launch(pl1, a1, cs)) != cudaSuccess) return e;
          if ((e = batch_reduce_link(io, cs)) != cudaSuccess) return e;
          if ((e = bgemm_launch(pl2, a2, cs)) != cudaSuccess) return e;
          if ((e = batch_reduce_grad(io, cs)) != cudaSuccess) return e;
        }
        round_launches += 5;
        if (clustered) {
          PArgs pw = pa;
          pw.seg_node = active_d;
          pw.cluster = 1;
          if ((e = pphase_launch_clusters(pc, pw, m, cs)) != cudaSuccess) return e;
          ++round_launches;
        } else {
          for (int w0 = 0; w0 < m; w0 += wave) {
            PArgs pw = pa;
            pw.seg_node = active_d + w0;
            pw.part = part + (size_t)w0 * NB * p;
            const int cnt = std::min(wave, m - w0);
            if ((e = pphase_launch_grid(pp, pw, cnt * segb, cs)) != cudaSuccess) return e;
            ++round_launches;
          }
        }
      }
      return cudaSuccess;
    };
    // one graph per active-set size, captured on its first round
    cudaGraphExec_t gx = nullptr;
    for (auto& g : graphs)
      if (g.first == m) gx = g.second;
    if (!gx) {
      cudaGraph_t graph = nullptr;
      cudaStream_t cs = nullptr;
      bool ok = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking) == cudaSuccess;
      if (ok) ok = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal) == cudaSuccess;
      if (ok) {
        const bool lok = enqueue_round(cs) == cudaSuccess;
        ok = (cudaStreamEndCapture(cs, &graph) == cudaSuccess) && lok && graph;
        if (ok) ok = cudaGraphInstantiate(&gx, graph, 0) == cudaSuccess;
        if (graph) cudaGraphDestroy(graph);
      }
      if (cs) cudaStreamDestroy(cs);
      if (ok) graphs.emplace_back(m, gx);
      else { gx = nullptr; cudaGetLastError(); }
    }
    if (gx) {
      BTRYC(cudaGraphLaunch(gx, h->stream));
    } else {
      BTRYC(enqueue_round(h->stream));
    }
    launches += round_launches;
    batch_done_kernel<<<1, 256, 0, h->stream>>>(dst, active_d, m, done_d);
    BTRYC(cudaGetLastError());
    BTRYC(cudaMemcpyAsync(hdone.data(), done_d, sizeof(int) * (size_t)m, cudaMemcpyDeviceToHost, h->stream));
    BTRYC(cudaStreamSynchronize(h->stream));
    int dstat = 0;
    BTRYC(cudaMemcpy(&dstat, h->status, sizeof(int), cudaMemcpyDeviceToHost));
    if (dstat != ST_OK) break;
    std::vector<int> still;
    for (int s = 0; s < m; ++s)
      if (!hdone[s]) still.push_back(active[s]);
    active.swap(still);
  }
  BTRYC(cudaMemcpyAsync(hs.data(), dst, sizeof(IterState) * (size_t)nb, cudaMemcpyDeviceToHost, h->stream));
  BTRYC(cudaStreamSynchronize(h->stream));
  int dstat = 0;
  BTRYC(cudaMemcpy(&dstat, h->status, sizeof(int), cudaMemcpyDeviceToHost));
  // ---- FP64 certificate of every node (two dual points, the better bound):
  // all passes enqueued back to back, one synchronisation
  std::vector<double> cert(4 * (size_t)nb, 0.0);
  if (h->certify && map_dev_status(dstat) == RELAX_OK) {
    PassState* psd = W.psd;
    double* certd = W.certd;
    std::vector<PassState> pss(2 * (size_t)nb);
    for (int j = 0; j < nb; ++j) {
      PassState a{};
      a.beta = hs[j].beta_best;            // Phi(beta_best); Psi at the loop's dual point
      a.zprev = hs[j].z_dbest;             // and at zeta = -grad F(X beta_best)
      pss[2 * j] = a;
    }
    auto chk = [&](cudaError_t e, const char* what, int line) {
      if (e == cudaSuccess) return RELAX_OK;
      set_detail(what, e, line);
      return map_cuda(e);
    };
    relax_status rc = chk(cudaMemcpyAsync(psd, pss.data(), sizeof(PassState) * 2 * (size_t)nb,
                                          cudaMemcpyHostToDevice, h->stream), "pass states to device", __LINE__);
    for (int j = 0; j < nb && rc == RELAX_OK; ++j) {
      const int8_t* fx = fixings ? W.fix + (size_t)j * p : nullptr;
      rc = certify_pair_enqueue(h, fx, hs[j].beta_best, psd + 2 * j, certd + 4 * j);
    }
    if (rc == RELAX_OK)
      rc = chk(cudaMemcpyAsync(cert.data(), certd, sizeof(double) * 4 * (size_t)nb, cudaMemcpyDeviceToHost,
                               h->stream), "certificates to host", __LINE__);
    if (rc == RELAX_OK) rc = chk(cudaStreamSynchronize(h->stream), "certificate passes", __LINE__);
    cudaStreamSynchronize(h->stream);
    BTRY(rc);
    // a non-finite certificate shows in that node's own values (judged below)
  }
  for (int j = 0; j < nb; ++j) {
    const IterState& S = hs[j];
    const int8_t* fx = fixings ? fixings + (size_t)j * p : nullptr;
    relax_result& o = out[j];
    o.lipschitz = h->L;
    o.iters = S.iter;
    o.restarts = S.restarts;
    o.backtracks = S.backtracks;
    o.lipschitz = S.Lk;
    o.primal_loop = S.phi_best;
    o.dual_loop = S.psi_best;
    o.launches = launches + (h->certify ? 4 * nb : 0);
    relax_status st_j = map_dev_status(dstat);
    if (h->certify && st_j == RELAX_OK) {
      const double phi = cert[4 * (size_t)j];
      double psi = cert[4 * (size_t)j + 1];
      const double psi2 = cert[4 * (size_t)j + 3];
      if (psi2 > psi || !(psi == psi)) psi = psi2;
      o.primal = phi;
      o.dual_bound = psi;
    } else {
      o.primal = S.phi_best;
      o.dual_bound = S.psi_best;
    }
    o.gap = o.primal - o.dual_bound;
    o.rel_gap = o.gap / std::max(1.0, std::fabs(o.primal));
    from_f64_kernel<<<grid_for(p), 256, 0, h->stream>>>((const double*)S.beta_best,
                                                         static_cast<unsigned char*>(beta_out) + es * (size_t)p * j,
                                                         f64 ? 1 : 0, p);
    o.stalled = S.stalled;
    o.cutoff_rule = S.cut_rule;
    auto judge = [&](relax_status s0) {
      if (s0 != RELAX_OK) return s0;
      if (!std::isfinite(o.dual_bound) || std::isnan(o.primal)) return RELAX_ENUMERIC;
      if (o.dual_bound > o.primal + 1e-9 * std::max(1.0, std::fabs(o.primal))) return RELAX_EINVALID_BOUND;
      if (!(o.rel_gap <= gap_tol) && !o.cutoff_rule) return RELAX_ENOTCONV;
      return RELAX_OK;
    };
    st_j = judge(st_j);
    if (st_j == RELAX_ENOTCONV && S.stalled && h->certify) {
      // The node stalled on the floor of the batch's GEMM products (FP32
      // accumulation over n or p terms): finish it with the single-node loop,
      // whose fused pass forms the products with compensated sums, from the
      // node's best point.  Both dual bounds are valid; the better one stays.
      void* bj = static_cast<unsigned char*>(beta_out) + es * (size_t)p * j;
      relax_result o2;
      const relax_status r2 = relax_solve(h, fx, bj, gap_tol, bj, &o2);
      if (r2 == RELAX_ECUDA || r2 == RELAX_ENOMEM || r2 == RELAX_ETIMEOUT || r2 == RELAX_EINVAL) {
        cudaStreamSynchronize(h->stream);
        cleanup();
        return r2;
      }
      o.polish_iters = o2.iters;
      o.launches += o2.launches;
      if (r2 == RELAX_OK || r2 == RELAX_ENOTCONV) {
        o.primal = o2.primal;            // Phi of the beta now in beta_out
        o.dual_bound = std::max(o.dual_bound, o2.dual_bound);
        o.stalled = o2.stalled;
        o.gap = o.primal - o.dual_bound;
        o.rel_gap = o.gap / std::max(1.0, std::fabs(o.primal));
        st_j = judge(RELAX_OK);
      } else {
        st_j = r2;
      }
    }
    o.status = st_j;
  }
  BTRYC(cudaGetLastError());
  BTRYC(cudaStreamSynchronize(h->stream));
  cleanup();
#undef BTRY
#undef BTRYC
  relax_status worst = RELAX_OK;
  for (int j = 0; j < nb; ++j)
    if (out[j].status != RELAX_OK && worst == RELAX_OK) worst = (relax_status)out[j].status;
  return worst;
}

// ================================================= learned warm start: features
namespace {

// per column j (one thread each; rows read in order, coalesced across j):
// ||X_j||_2 and |corr(X_j, y)| from centred FP64 sums (two passes over X)
template <typename T>
__global__ void colstat_kernel(const T* X, int64_t n, int64_t p, int64_t ld, const double* y, double* out) {
  const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= p) return;
  double sx = 0.0, sy = 0.0;
  for (int64_t i = 0; i < n; ++i) {
    sx += (double)X[i * ld + j];
    sy += y[i];
  }
  const double mx = sx / (double)n, my = sy / (double)n;
  double sxx = 0.0, cxx = 0.0, cyy = 0.0, cxy = 0.0;
  for (int64_t i = 0; i < n; ++i) {
    const double x = (double)X[i * ld + j];
    const double dx = x - mx, dy = y[i] - my;
    sxx += x * x;
    cxx += dx * dx;
    cyy += dy * dy;
    cxy += dx * dy;
  }
  const double den = sqrt(cxx) * sqrt(cyy);
  out[j] = sqrt(sxx);
  out[p + j] = den > 0.0 ? fabs(cxy) / den : 0.0;
}

// b = beta^P with the child's J0 set to zero
template <typename T>
__global__ void project_parent_kernel(const T* beta, const int8_t* fix, int64_t p, T* b) {
  for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < p; j += (int64_t)gridDim.x * blockDim.x)
    b[j] = (fix && fix[j] < 0) ? (T)0 : beta[j];
}

template <typename T>
__global__ void features_kernel(const T* beta, const T* g, const int8_t* fix, const double* colstat, int64_t p,
                                float* feat) {
  for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < p; j += (int64_t)gridDim.x * blockDim.x) {
    float* f = feat + j * 5;
    f[0] = (float)beta[j];
    f[1] = (float)g[j];
    f[2] = fix ? (float)fix[j] : 0.f;
    f[3] = (float)colstat[j];
    f[4] = (float)colstat[p + j];
  }
}

}  // namespace

extern "C" relax_status relax_mlp_features(relax_handle* h, const void* beta_parent, const int8_t* fixings,
                                           float* feat_out) {
  if (!h || !beta_parent || !feat_out) return RELAX_EINVAL;
  CU(cudaSetDevice(h->dev));
  const int64_t p = h->p;
  if (!h->colstat) {
    relax_status rs = alloc((void**)&h->colstat, sizeof(double) * 2 * (size_t)p);
    if (rs != RELAX_OK) return rs;
    const unsigned g = (unsigned)((p + 127) / 128);
    if (h->dtype == RELAX_F64)
      colstat_kernel<double><<<g, 128, 0, h->stream>>>((const double*)h->X, h->n, p, h->ldx, (const double*)h->y, h->colstat);
    else
      colstat_kernel<float><<<g, 128, 0, h->stream>>>((const float*)h->X, h->n, p, h->ldx, (const double*)h->y, h->colstat);
    CU(cudaGetLastError());
  }
  // b (the parent on the child's set) and X' grad F(X b): one fused pass
  void* gbuf = nullptr;
  relax_status rs = alloc(&gbuf, 2 * h->esz() * (size_t)p);
  if (rs != RELAX_OK) return rs;
  void* bbuf = static_cast<unsigned char*>(gbuf) + h->esz() * (size_t)p;
  if (h->dtype == RELAX_F64)
    project_parent_kernel<double><<<grid_for(p), 256, 0, h->stream>>>((const double*)beta_parent, fixings, p, (double*)bbuf);
  else
    project_parent_kernel<float><<<grid_for(p), 256, 0, h->stream>>>((const float*)beta_parent, fixings, p, (float*)bbuf);
  {
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
      set_detail("project_parent_kernel", e, __LINE__);
      rs = map_cuda(e);
    }
  }
  if (rs == RELAX_OK) rs = relax_xpass(h, bbuf, nullptr, gbuf, nullptr);
  if (rs == RELAX_OK) {
    if (h->dtype == RELAX_F64)
      features_kernel<double><<<grid_for(p), 256, 0, h->stream>>>((const double*)bbuf, (const double*)gbuf,
                                                                  fixings, h->colstat, p, feat_out);
    else
      features_kernel<float><<<grid_for(p), 256, 0, h->stream>>>((const float*)bbuf, (const float*)gbuf,
                                                                 fixings, h->colstat, p, feat_out);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) { set_detail("features", e, __LINE__); rs = map_cuda(e); }
  }
  cudaStreamSynchronize(h->stream);
  cudaFree(gbuf);
  return rs;
}

// ================================================ batched products (diagnostic)
extern "C" relax_status relax_certify_batch(relax_handle* h, int32_t nb, const int8_t* fixings, const void* points,
                                            double* out_host) {
  if (!h || nb <= 0 || !points || !out_host) return RELAX_EINVAL;
  CU(cudaSetDevice(h->dev));
  const int64_t p = h->p;
  // scratch: the points in FP64, their pass states, the values, the fixing counts
  const size_t b64 = sizeof(double) * (size_t)nb * p;
  const size_t bps = sizeof(PassState) * (size_t)nb;
  const size_t bout = sizeof(double) * 2 * (size_t)nb;
  const size_t bcnt = sizeof(int) * 3 * (size_t)nb;
  auto al = [](size_t x) { return (x + 255) / 256 * 256; };
  unsigned char* scr = nullptr;
  relax_status rs = alloc((void**)&scr, al(b64) + al(bps) + al(bout) + al(bcnt));
  if (rs != RELAX_OK) return rs;
  double* pts = reinterpret_cast<double*>(scr);
  PassState* psd = reinterpret_cast<PassState*>(scr + al(b64));
  double* outd = reinterpret_cast<double*>(scr + al(b64) + al(bps));
  int* cnt = reinterpret_cast<int*>(scr + al(b64) + al(bps) + al(bout));
  auto run = [&]() -> relax_status {
    if (fixings) {
      std::vector<int> hc(3 * (size_t)nb);
      CU(cudaMemsetAsync(cnt, 0, bcnt, h->stream));
      count_fix_batch_kernel<<<dim3((unsigned)std::min<int64_t>(64, (p + 255) / 256), (unsigned)nb), 256, 0,
                               h->stream>>>(fixings, p, cnt);
      CU(cudaGetLastError());
      CU(cudaMemcpyAsync(hc.data(), cnt, bcnt, cudaMemcpyDeviceToHost, h->stream));
      CU(cudaStreamSynchronize(h->stream));
      for (int j = 0; j < nb; ++j)
        if (hc[3 * j + 2] != 0 || hc[3 * j] > h->k) return RELAX_EINVAL;
    }
    CU(cudaMemsetAsync(h->status, 0, sizeof(int), h->stream));
    to_f64_kernel<<<grid_for((int64_t)nb * p), 256, 0, h->stream>>>(points, h->f64(), pts, (int64_t)nb * p);
    CU(cudaGetLastError());
    std::vector<PassState> pss((size_t)nb);
    for (int j = 0; j < nb; ++j) {
      PassState b{};
      b.beta = pts + (size_t)j * p;   // Phi(b) and Psi at zeta = -grad F(X b)
      pss[j] = b;
    }
    CU(cudaMemcpyAsync(psd, pss.data(), bps, cudaMemcpyHostToDevice, h->stream));
    for (int j = 0; j < nb; ++j) {
      const relax_status r = certify_enqueue(h, fixings ? fixings + (size_t)j * p : nullptr, pts + (size_t)j * p,
                                             DUAL_SELF, psd + j, outd + 2 * j);
      if (r != RELAX_OK) return r;
    }
    CU(cudaMemcpyAsync(out_host, outd, bout, cudaMemcpyDeviceToHost, h->stream));
    CU(cudaStreamSynchronize(h->stream));
    int dst = 0;
    CU(cudaMemcpy(&dst, h->status, sizeof(int), cudaMemcpyDeviceToHost));
    return map_dev_status(dst);
  };
  rs = run();
  cudaStreamSynchronize(h->stream);
  cudaFree(scr);
  return rs;
}

extern "C" relax_status relax_batch_xpass(relax_handle* h, int32_t nb, const void* points, double* z_out,
                                          double* g_out, double* products_ms) {
  if (!h || nb <= 0 || !points || !z_out || !g_out) return RELAX_EINVAL;
  if (h->xk_loop != XK_F32 && h->xk_loop != XK_F64) return RELAX_ENOTSUP;
  CU(cudaSetDevice(h->dev));
  const int64_t n = h->n, p = h->p;
  const dim3 gz((unsigned)((n + 63) / 64), (unsigned)((nb + 15) / 16));
  const dim3 gg((unsigned)((p + 63) / 64), (unsigned)((nb + 15) / 16));
  CU(cudaMemsetAsync(h->status, 0, sizeof(int), h->stream));
  if (h->xk_loop == XK_F64) {
    zprod_f64_kernel<<<gz, 256, 0, h->stream>>>((const double*)h->X, h->ldx, n, p, (const double*)points, nb, z_out);
    gprod_f64_kernel<<<gg, 256, 0, h->stream>>>((const double*)h->X, h->ldx, n, p, z_out, nb, g_out);
    CU(cudaGetLastError());
    CU(cudaStreamSynchronize(h->stream));
    return RELAX_OK;
  }
  relax_status rs = ensure_planes(h);
  if (rs != RELAX_OK) return rs;
  // scratch: the points in FP64, B and R planes, the partials of both products
  const size_t b64 = sizeof(double) * (size_t)nb * p;
  const size_t bpb = sizeof(__nv_bfloat16) * 3 * (size_t)nb * h->ldbp;
  const size_t rpb = sizeof(__nv_bfloat16) * 3 * (size_t)nb * h->ldbn;
  const size_t p1b = sizeof(double) * BG_MAXKC * (size_t)nb * n;
  const size_t p2b = sizeof(double) * BG_MAXKC * (size_t)nb * p;
  unsigned char* scr = nullptr;
  rs = alloc((void**)&scr, b64 + bpb + rpb + p1b + p2b + 4 * 256);
  if (rs != RELAX_OK) return rs;
  auto al = [](size_t x) { return (x + 255) / 256 * 256; };
  double* bsrc = reinterpret_cast<double*>(scr);
  __nv_bfloat16* Bp = reinterpret_cast<__nv_bfloat16*>(scr + al(b64));
  __nv_bfloat16* Rp = reinterpret_cast<__nv_bfloat16*>(scr + al(b64) + al(bpb));
  double* P1 = reinterpret_cast<double*>(scr + al(b64) + al(bpb) + al(rpb));
  double* P2 = reinterpret_cast<double*>(scr + al(b64) + al(bpb) + al(rpb) + al(p1b));
  auto run = [&]() -> relax_status {
    to_f64_kernel<<<grid_for((int64_t)nb * p), 256, 0, h->stream>>>(points, 0, bsrc, (int64_t)nb * p);
    CU(cudaGetLastError());
    BGPlan pl1, pl2;
    CU(bgemm_plan(pl1, (int)n, nb, (int)p));
    CU(bgemm_plan(pl2, (int)p, nb, (int)n));
    BGArgs a1{}, a2{};
    a1.tmA = h->tm_bx;
    a2.tmA = h->tm_bxt;
    CU(bgemm_encode(&a1.tmB, Bp, p, nb, h->ldbp, nb, pl1.BN));
    CU(bgemm_encode(&a2.tmB, Rp, n, nb, h->ldbn, nb, pl2.BN));
    fill_bgargs(a1, pl1, P1, h->status, h->limit_ns);
    fill_bgargs(a2, pl2, P2, h->status, h->limit_ns);
    BatchIo io{};
    io.m = nb;
    io.nb = nb;
    io.n = n;
    io.p = p;
    io.ldp = h->ldbp;
    io.ldn = h->ldbn;
    io.NB = 1;
    io.loss = -1;                 // identity link: the second product is X' z
    io.bsrc = bsrc;
    io.zdst = z_out;
    io.Bp = Bp;
    io.Rp = Rp;
    io.P1 = P1;
    io.s1 = pl1.split();
    io.P2 = P2;
    io.s2 = pl2.split();
    io.part = g_out;              // NB = 1: part[s][0][j] = g_out[s * p + j]
    CU(batch_pack(io, h->stream));
    CU(cudaEventRecord(h->ev_t[0], h->stream));
    CU(bgemm_launch(pl1, a1, h->stream));
    CU(cudaEventRecord(h->ev_t[1], h->stream));
    CU(batch_reduce_link(io, h->stream));
    CU(cudaEventRecord(h->ev_p[0], h->stream));
    CU(bgemm_launch(pl2, a2, h->stream));
    CU(cudaEventRecord(h->ev_p[1], h->stream));
    CU(batch_reduce_grad(io, h->stream));
    CU(cudaStreamSynchronize(h->stream));
    if (products_ms) {
      float t1 = 0.f, t2 = 0.f;
      CU(cudaEventElapsedTime(&t1, h->ev_t[0], h->ev_t[1]));
      CU(cudaEventElapsedTime(&t2, h->ev_p[0], h->ev_p[1]));
      products_ms[0] = t1;
      products_ms[1] = t2;
    }
    int dst = 0;
    CU(cudaMemcpy(&dst, h->status, sizeof(int), cudaMemcpyDeviceToHost));
    if (dst != ST_OK) snprintf(g_detail, sizeof(g_detail), "batched products: device status %d", dst);
    return map_dev_status(dst);
  };
  rs = run();
  cudaStreamSynchronize(h->stream);
  cudaFree(scr);
  return rs;
}
