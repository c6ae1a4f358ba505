// C ABI of the library (include/relax.h): handle lifecycle, the solve loop,
// FP64 certification and the standalone regularizer entry points.
#include <cuda_bf16.h>
#include <cuda_fp8.h>

#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <new>
#include <vector>

#include "launch.cuh"
#include "relax.h"

using namespace relax;

namespace {

#define CU(call)                                  \
  do {                                            \
    cudaError_t e_ = (call);                      \
    if (e_ != cudaSuccess) return map_cuda(e_);   \
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

template <typename T>
__global__ void init_vectors_kernel(const T* warm, T* b0, T* b1, T* bb, T* bd, T* g0, T* g1, int64_t p,
                                    T* z0, T* z1, int64_t n) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < p; j += stride) {
    const T w = warm ? warm[j] : (T)0;
    b0[j] = w; b1[j] = w; bb[j] = w; bd[j] = w;
    g0[j] = (T)0; g1[j] = (T)0;
  }
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
    z0[i] = (T)0; z1[i] = (T)0;
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

template <typename T>
__global__ void nnz_kernel(const T* v, int64_t p, int* out) {
  int c = 0;
  for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < p; j += (int64_t)gridDim.x * blockDim.x)
    c += v[j] != (T)0;
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
struct relax_handle {
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
  XPlan pl_loop, pl_cert, pl_ident;
  PPlan pp_iter, pp_eval;
  // buffers
  void* part_loop = nullptr;
  void* part_cert = nullptr;
  double* lossp = nullptr;
  IterState* st = nullptr;
  PassState* ps_aux = nullptr;
  void* vb[8] = {};          // beta prev/cur, G prev/cur, beta_best, beta_dbest, z prev/cur
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
  size_t esz() const { return dtype == RELAX_F64 ? 8 : 4; }
};

namespace {

void handle_free(relax_handle* h) {
  if (!h) return;
  cudaSetDevice(h->dev);
  cudaStreamSynchronize(h->stream);
  void* ptrs[] = {h->Xown, h->Xq, h->colscale, h->y, h->part_loop, h->part_cert, h->lossp, h->st,
                  h->ps_aux, h->acc, h->bpart, h->bar, h->bar_aux, h->status, h->dscr, h->iscr};
  for (void* q : ptrs) if (q) cudaFree(q);
  for (void* q : h->vb) if (q) cudaFree(q);
  if (h->h_state) cudaFreeHost(h->h_state);
  if (h->h_done) cudaFreeHost(h->h_done);
  if (h->h_d) cudaFreeHost(h->h_d);
  if (h->h_i) cudaFreeHost(h->h_i);
  delete h;
}

relax_status alloc(void** p, size_t bytes) {
  cudaError_t e = cudaMalloc(p, std::max<size_t>(bytes, 16));
  if (e != cudaSuccess) return map_cuda(e);
  return RELAX_OK;
}

XPassArgs pass_args(relax_handle* h, const XPlan& pl, int link, PassState* ps, void* part) {
  XPassArgs a{};
  const bool lowp = (pl.xk == XK_BF16 || pl.xk == XK_FP8);
  a.X = lowp ? h->Xq : h->X;
  a.ldx = lowp ? h->ldq : h->ldx;
  a.n = h->n;
  a.p = h->p;
  a.slice = pl.slice;
  a.C = pl.C;
  a.R = pl.R;
  a.S = pl.S;
  a.slot_bytes = pl.slot_bytes;
  a.link = link;
  a.y = h->y;
  a.colscale = lowp ? h->colscale : nullptr;
  a.ps = ps;
  a.part = part;
  a.lossp = h->lossp;
  a.status = h->status;
  a.limit_ns = h->limit_ns;
  return a;
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
  a.lossp = h->lossp;
  a.acc = h->acc;
  a.bpart = h->bpart;
  a.status = h->status;
  a.limit_ns = h->limit_ns;
  return a;
}

// L = c_f * ||X||_2^2 by power iteration on the operator the loop uses
relax_status power_iteration(relax_handle* h, double* L_out) {
  const bool dbl = h->dtype == RELAX_F64;
  void* v = h->vb[0];
  void* w = h->vb[1];
  const unsigned g = grid_for(h->p);
  const double v0 = 1.0 / std::sqrt((double)h->p);
  if (dbl) fill_kernel<double><<<g, 256, 0, h->stream>>>((double*)v, h->p, v0);
  else fill_kernel<float><<<g, 256, 0, h->stream>>>((float*)v, h->p, (float)v0);
  CU(cudaGetLastError());
  double ray_prev = 0.0, ray = 0.0;
  for (int it = 0; it < 500; ++it) {
    PassState ps{};
    ps.beta = v;
    *reinterpret_cast<PassState*>(h->h_d + 1000) = ps;   // staging in pinned memory
    CU(cudaMemcpyAsync(h->ps_aux, h->h_d + 1000, sizeof(PassState), cudaMemcpyHostToDevice, h->stream));
    XPassArgs a = pass_args(h, h->pl_ident, LINK_IDENT, h->ps_aux, h->part_loop);
    CU(xpass_launch(h->pl_ident, a, h->stream));
    CU(cudaMemsetAsync(h->dscr, 0, sizeof(double), h->stream));
    if (dbl)
      reduce_partials_kernel<double, double><<<g, 256, 0, h->stream>>>((const double*)h->part_loop, h->pl_ident.ncl, 1,
                                                                       h->p, (double*)w, h->dscr);
    else
      reduce_partials_kernel<float, float><<<g, 256, 0, h->stream>>>((const float*)h->part_loop, h->pl_ident.ncl, 1,
                                                                     h->p, (float*)w, h->dscr);
    CU(cudaGetLastError());
    CU(cudaMemcpyAsync(h->h_d, h->lossp, sizeof(double) * 2 * h->pl_ident.ncl, cudaMemcpyDeviceToHost, h->stream));
    CU(cudaStreamSynchronize(h->stream));
    int dst = 0;
    CU(cudaMemcpy(&dst, h->status, sizeof(int), cudaMemcpyDeviceToHost));
    if (dst != ST_OK) return map_dev_status(dst);
    ray = 0.0;
    for (int c = 0; c < h->pl_ident.ncl; ++c) ray += h->h_d[2 * c];   // ||X v||^2 with ||v|| = 1
    if (dbl) scale_kernel<double><<<g, 256, 0, h->stream>>>((double*)w, h->p, h->dscr);
    else scale_kernel<float><<<g, 256, 0, h->stream>>>((float*)w, h->p, h->dscr);
    CU(cudaGetLastError());
    std::swap(v, w);
    if (it > 3 && std::fabs(ray - ray_prev) <= 1e-7 * ray) break;
    ray_prev = ray;
  }
  if (!(ray > 0.0) || !std::isfinite(ray)) return RELAX_ENUMERIC;
  const double cf = h->loss == RELAX_LS ? 2.0 : 0.25;
  *L_out = cf * ray * 1.01;   // 1% margin over the Rayleigh estimate of ||X||^2
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

// FP64 Phi(beta_p), Psi(zeta(beta_d)) with the master X -> h->h_d[0..1]
relax_status certify(relax_handle* h, const int8_t* fix, const void* bp, const void* bd) {
  PassState ps{};
  ps.beta = bp;
  ps.beta2 = bd;
  *reinterpret_cast<PassState*>(h->h_d + 1000) = ps;
  CU(cudaMemcpyAsync(h->ps_aux, h->h_d + 1000, sizeof(PassState), cudaMemcpyHostToDevice, h->stream));
  XPassArgs a = pass_args(h, h->pl_cert, h->loss == RELAX_LS ? LINK_CERT_LS : LINK_CERT_LOGI, h->ps_aux,
                          h->part_cert);
  a.X = h->X;
  a.ldx = h->ldx;
  a.colscale = nullptr;
  CU(xpass_launch(h->pl_cert, a, h->stream));
  PArgs pa = base_pargs(h);
  pa.mode = PM_EVAL;
  pa.fix = fix;
  pa.part = h->part_cert;
  pa.ncl = h->pl_cert.ncl;
  pa.NB = 1;
  pa.st = nullptr;
  pa.vin = bp;
  pa.out = h->dscr;
  pa.bar = h->bar_aux;
  pa.bar_base = 0;
  CU(cudaMemsetAsync(h->bar_aux, 0, sizeof(unsigned long long), h->stream));
  CU(pphase_launch(h->pp_eval, pa, h->stream));
  CU(cudaMemcpyAsync(h->h_d, h->dscr, 2 * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
  CU(cudaStreamSynchronize(h->stream));
  return RELAX_OK;
}

}  // namespace

extern "C" {

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
    case RELAX_ENOTSUP: return "shape or option not supported by this build";
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
      o.watchdog_ms < 0 || o.chunk < 0)
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
#define TRYC(x) TRY(((x) == cudaSuccess) ? RELAX_OK : map_cuda(cudaGetLastError()))
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
    TRY(alloc(&h->y, (size_t)n * es));
    TRYC(cudaMemcpyAsync(h->y, y, (size_t)n * es, cudaMemcpyDeviceToDevice, h->stream));
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
    TRYC(xpass_plan(h->pl_loop, h->xk_loop, vd, false, 1, loss == RELAX_LS ? 1 : 2, n, p));
    TRYC(xpass_plan(h->pl_ident, h->xk_loop, vd, false, 1, 1, n, p));
    TRYC(xpass_plan(h->pl_cert, vd ? XK_F64 : XK_F32, vd, true, 2, 1, n, p));
    TRYC(pphase_plan(h->pp_iter, vd, vd, p));
    TRYC(pphase_plan(h->pp_eval, vd, true, p));
    const int ncl_max = std::max(std::max(h->pl_loop.ncl, h->pl_ident.ncl), h->pl_cert.ncl);
    TRY(alloc(&h->part_loop, (size_t)h->pl_loop.ncl * h->pl_loop.NB * p * es +
                                 (size_t)h->pl_ident.ncl * p * es));
    TRY(alloc(&h->part_cert, (size_t)h->pl_cert.ncl * p * sizeof(double)));
    TRY(alloc((void**)&h->lossp, (size_t)ncl_max * 2 * sizeof(double)));
    TRY(alloc((void**)&h->st, sizeof(IterState)));
    TRY(alloc((void**)&h->ps_aux, sizeof(PassState)));
    for (int i = 0; i < 6; ++i) TRY(alloc(&h->vb[i], (size_t)p * es));
    for (int i = 6; i < 8; ++i) TRY(alloc(&h->vb[i], (size_t)n * es));
    TRY(alloc((void**)&h->acc, 3 * ACC_STRIDE * sizeof(unsigned long long)));
    const int gmax = std::max(h->pp_iter.grid, h->pp_eval.grid);
    TRY(alloc((void**)&h->bpart, (size_t)2 * gmax * NBP * sizeof(double)));
    TRY(alloc((void**)&h->bar, sizeof(unsigned long long)));
    TRY(alloc((void**)&h->bar_aux, sizeof(unsigned long long)));
    TRY(alloc((void**)&h->status, sizeof(int)));
    TRY(alloc((void**)&h->dscr, 16 * sizeof(double)));
    TRY(alloc((void**)&h->iscr, 16 * sizeof(int)));
    TRYC(cudaMemsetAsync(h->acc, 0, 3 * ACC_STRIDE * sizeof(unsigned long long), h->stream));
    TRYC(cudaMemsetAsync(h->status, 0, sizeof(int), h->stream));
    TRYC(cudaMemsetAsync(h->lossp, 0, (size_t)ncl_max * 2 * sizeof(double), h->stream));
    TRYC(cudaHostAlloc((void**)&h->h_state, sizeof(IterState), cudaHostAllocDefault));
    TRYC(cudaHostAlloc((void**)&h->h_done, 2 * sizeof(int), cudaHostAllocDefault));
    TRYC(cudaHostAlloc((void**)&h->h_d, 1024 * sizeof(double), cudaHostAllocDefault));
    TRYC(cudaHostAlloc((void**)&h->h_i, 16 * sizeof(int), cudaHostAllocDefault));
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
  const bool dbl = h->dtype == RELAX_F64;
  const size_t es = h->esz();
  std::memset(out, 0, sizeof(*out));
  out->lipschitz = h->L;
  // ---- state
  const unsigned g = grid_for(std::max(h->p, h->n));
  if (dbl)
    init_vectors_kernel<double><<<g, 256, 0, h->stream>>>((const double*)warm_start, (double*)h->vb[0],
                                                          (double*)h->vb[1], (double*)h->vb[4], (double*)h->vb[5],
                                                          (double*)h->vb[2], (double*)h->vb[3], h->p,
                                                          (double*)h->vb[6], (double*)h->vb[7], h->n);
  else
    init_vectors_kernel<float><<<g, 256, 0, h->stream>>>((const float*)warm_start, (float*)h->vb[0],
                                                         (float*)h->vb[1], (float*)h->vb[4], (float*)h->vb[5],
                                                         (float*)h->vb[2], (float*)h->vb[3], h->p, (float*)h->vb[6],
                                                         (float*)h->vb[7], h->n);
  CU(cudaGetLastError());
  IterState s{};
  s.beta_prev = h->vb[0];
  s.beta_cur = h->vb[1];
  s.G_prev = h->vb[2];
  s.G_cur = h->vb[3];
  s.beta_best = h->vb[4];
  s.beta_dbest = h->vb[5];
  s.z_prev = h->vb[6];
  s.z_cur = h->vb[7];
  s.tau = 1.0;
  s.gap_ref = INFINITY;
  s.phi_best = INFINITY;
  s.psi_best = -INFINITY;
  s.kbar = h->k - j1;
  s.pbar = jf;
  s.ps.beta = s.beta_cur;
  s.ps.zout = h->loss == RELAX_LOGISTIC ? s.z_cur : nullptr;
  s.ps.zprev = s.z_prev;
  s.ps.mom = 0.0;
  *h->h_state = s;
  CU(cudaMemcpyAsync(h->st, h->h_state, sizeof(IterState), cudaMemcpyHostToDevice, h->stream));
  CU(cudaMemsetAsync(h->bar, 0, sizeof(unsigned long long), h->stream));
  CU(cudaMemsetAsync(h->status, 0, sizeof(int), h->stream));
  // ---- one iteration = fused X-pass + p-phase; enqueue `chunk` per host poll
  XPassArgs xa = pass_args(h, h->pl_loop, h->loss == RELAX_LS ? LINK_LS : LINK_LOGISTIC, &h->st->ps, h->part_loop);
  PArgs pa = base_pargs(h);
  pa.mode = PM_ITER;
  pa.fix = fixings;
  pa.part = h->part_loop;
  pa.ncl = h->pl_loop.ncl;
  pa.NB = h->pl_loop.NB;
  pa.st = h->st;
  pa.bar = h->bar;
  pa.tol = gap_tol;
  // Timing mode: event records around every loop kernel (captured into the
  // graph); the host then waits for each chunk before enqueueing the next.
  const bool timing = h->opt.timing != 0;
  const int chunk = h->chunk;
  cudaEvent_t* tev = nullptr;   // [chunk][3]: before X-pass, after X-pass, after p-phase
  if (timing) {
    tev = new (std::nothrow) cudaEvent_t[(size_t)chunk * 3];
    if (!tev) return RELAX_ENOMEM;
    for (int i = 0; i < chunk * 3; ++i) cudaEventCreate(&tev[i]);
  }
  auto enqueue_body = [&](cudaStream_t cs) -> cudaError_t {
    for (int i = 0; i < chunk; ++i) {
      cudaError_t e;
      if (timing && (e = cudaEventRecord(tev[3 * i], cs)) != cudaSuccess) return e;
      if ((e = xpass_launch(h->pl_loop, xa, cs)) != cudaSuccess) return e;
      if (timing && (e = cudaEventRecord(tev[3 * i + 1], cs)) != cudaSuccess) return e;
      if ((e = pphase_launch(h->pp_iter, pa, cs)) != cudaSuccess) return e;
      if (timing && (e = cudaEventRecord(tev[3 * i + 2], cs)) != cudaSuccess) return e;
    }
    return cudaSuccess;
  };
  // capture the chunk as a graph (falls back to direct launches)
  cudaGraphExec_t gexec = nullptr;
  {
    cudaGraph_t graph = nullptr;
    cudaStream_t cs = nullptr;
    bool ok = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking) == cudaSuccess;
    if (ok) ok = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal) == cudaSuccess;
    if (ok) {
      const bool lok = enqueue_body(cs) == cudaSuccess;
      ok = (cudaStreamEndCapture(cs, &graph) == cudaSuccess) && lok && graph;
      if (ok) ok = cudaGraphInstantiate(&gexec, graph, 0) == cudaSuccess;
      if (graph) cudaGraphDestroy(graph);
    }
    if (cs) cudaStreamDestroy(cs);
    if (!ok) { gexec = nullptr; cudaGetLastError(); }
  }
  auto enqueue_chunk = [&]() -> cudaError_t {
    if (gexec) return cudaGraphLaunch(gexec, h->stream);
    return enqueue_body(h->stream);
  };
  cudaEvent_t ev[2];
  cudaEventCreateWithFlags(&ev[0], cudaEventDisableTiming);
  cudaEventCreateWithFlags(&ev[1], cudaEventDisableTiming);
  const int64_t max_chunks = (int64_t)h->max_iters / chunk + 3;
  cudaError_t err = cudaSuccess;
  int64_t nchunks = 0;
  std::vector<float> xms, pms;   // per launched iteration (timing mode)
  for (int64_t c = 0; c < max_chunks; ++c) {
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
  cudaEventDestroy(ev[0]);
  cudaEventDestroy(ev[1]);
  if (tev) {
    for (int i = 0; i < chunk * 3; ++i) cudaEventDestroy(tev[i]);
    delete[] tev;
  }
  if (gexec) cudaGraphExecDestroy(gexec);
  if (err != cudaSuccess) return map_cuda(err);
  out->launches = (int)(nchunks * chunk * 2) + 1 + (fixings ? 1 : 0);   // loop + init (+ count)
  CU(cudaMemcpy(h->h_state, h->st, sizeof(IterState), cudaMemcpyDeviceToHost));
  int dst = 0;
  CU(cudaMemcpy(&dst, h->status, sizeof(int), cudaMemcpyDeviceToHost));
  const IterState& S = *h->h_state;
  out->iters = S.iter;
  out->xpass_count = S.iter + 1;
  if (timing) {
    // the pass at beta^t and the p-phase that follows it, for t = 0..iters
    for (int t = 0; t <= S.iter && t < (int)xms.size(); ++t) {
      out->xpass_ms += xms[t];
      out->pphase_ms += pms[t];
    }
  }
  out->restarts = S.restarts;
  out->primal_loop = S.phi_best;
  out->dual_loop = S.psi_best;
  out->primal = S.phi_best;
  out->dual_bound = S.psi_best;
  relax_status status = map_dev_status(dst);
  if (status == RELAX_OK && h->certify) {
    rs = certify(h, fixings, S.beta_best, S.beta_dbest);
    if (rs != RELAX_OK) return rs;
    out->launches += 2;
    CU(cudaMemcpy(&dst, h->status, sizeof(int), cudaMemcpyDeviceToHost));
    status = map_dev_status(dst);
    out->primal = h->h_d[0];
    out->dual_bound = h->h_d[1];
  }
  out->gap = out->primal - out->dual_bound;
  out->rel_gap = out->gap / std::max(1.0, std::fabs(out->primal));
  CU(cudaMemcpyAsync(beta_out, S.beta_best, (size_t)h->p * es, cudaMemcpyDeviceToDevice, h->stream));
  CU(cudaMemsetAsync(h->iscr, 0, sizeof(int), h->stream));
  if (dbl) nnz_kernel<double><<<grid_for(h->p), 256, 0, h->stream>>>((const double*)S.beta_best, h->p, h->iscr);
  else nnz_kernel<float><<<grid_for(h->p), 256, 0, h->stream>>>((const float*)S.beta_best, h->p, h->iscr);
  CU(cudaMemcpyAsync(h->h_i, h->iscr, sizeof(int), cudaMemcpyDeviceToHost, h->stream));
  CU(cudaStreamSynchronize(h->stream));
  out->n_nz = h->h_i[0];
  out->launches += 1;
  if (status == RELAX_OK) {
    if (!std::isfinite(out->dual_bound) || std::isnan(out->primal)) status = RELAX_ENUMERIC;
    else if (out->dual_bound > out->primal + 1e-9 * std::max(1.0, std::fabs(out->primal)))
      status = RELAX_EINVALID_BOUND;
    else if (!(S.phi_best - S.psi_best <= gap_tol * std::max(1.0, std::fabs(S.phi_best))))
      status = RELAX_ENOTCONV;
  }
  out->status = status;
  return status;
}

relax_status relax_xpass(relax_handle* h, const void* beta, void* z_out, void* g_out, double* loss_host) {
  if (!h || !beta || !g_out) return RELAX_EINVAL;
  CU(cudaSetDevice(h->dev));
  PassState ps{};
  ps.beta = beta;
  ps.zout = z_out;
  ps.zprev = h->vb[6];
  ps.mom = 0.0;
  *reinterpret_cast<PassState*>(h->h_d + 1000) = ps;
  CU(cudaMemcpyAsync(h->ps_aux, h->h_d + 1000, sizeof(PassState), cudaMemcpyHostToDevice, h->stream));
  CU(cudaMemsetAsync(h->status, 0, sizeof(int), h->stream));
  CU(cudaMemsetAsync(h->vb[6], 0, (size_t)h->n * h->esz(), h->stream));
  XPassArgs a = pass_args(h, h->pl_loop, h->loss == RELAX_LS ? LINK_LS : LINK_LOGISTIC, h->ps_aux, h->part_loop);
  CU(xpass_launch(h->pl_loop, a, h->stream));
  const unsigned g = grid_for(h->p);
  if (h->dtype == RELAX_F64)
    reduce_partials_kernel<double, double><<<g, 256, 0, h->stream>>>((const double*)h->part_loop, h->pl_loop.ncl,
                                                                     h->pl_loop.NB, h->p, (double*)g_out, nullptr);
  else
    reduce_partials_kernel<float, float><<<g, 256, 0, h->stream>>>((const float*)h->part_loop, h->pl_loop.ncl,
                                                                   h->pl_loop.NB, h->p, (float*)g_out, nullptr);
  CU(cudaGetLastError());
  CU(cudaMemcpyAsync(h->h_d, h->lossp, sizeof(double) * 2 * h->pl_loop.ncl, cudaMemcpyDeviceToHost, h->stream));
  CU(cudaStreamSynchronize(h->stream));
  int dst = 0;
  CU(cudaMemcpy(&dst, h->status, sizeof(int), cudaMemcpyDeviceToHost));
  if (loss_host) {
    double f = 0.0, d = 0.0;
    for (int c = 0; c < h->pl_loop.ncl; ++c) { f += h->h_d[2 * c]; d += h->h_d[2 * c + 1]; }
    loss_host[0] = f;
    loss_host[1] = d;
  }
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
  rs = certify(h, fixings, beta_primal, beta_dual);
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
  CU(pphase_plan(pl, dbl, dbl, p));
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
