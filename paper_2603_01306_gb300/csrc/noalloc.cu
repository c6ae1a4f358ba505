// prox_persp_noalloc: the prox of prox_persp with its scratch in a fixed
// device array instead of stream-ordered allocations.
//
// Some callers cannot allocate device memory while they work: a solver
// embedded in a host framework whose memory pool already owns the whole GPU
// (an allocation from outside the pool fails or steals from it), or a node
// loop with a hard latency budget, where an allocator call may block, may
// synchronize the device, or may fail late under memory pressure.  For them
// this entry point takes its scratch from the array below and calls no
// allocation routine at all.
#include <cstdio>
#include <mutex>

#include "launch.cuh"
#include "relax.h"

namespace relax {
void set_error_detail(const char* msg);   // api.cu
}  // namespace relax

using namespace relax;

namespace {

// Scratch of one prox launch: the threshold rounds' accumulators, the
// per-block partial sums, the grid barrier counter, a status word and one
// output value.  64 KiB; every GPU that loads this library holds it until the
// process exits.  In host code this name is only a stand-in: the device
// address comes from cudaGetSymbolAddress.
constexpr size_t kScratchBytes = 64 * 1024;
static __device__ __align__(256) unsigned char g_prox_scratch[kScratchBytes];
// Each block of the launch takes 160 bytes of partials, after 3 * 256 * 8
// bytes of accumulators and 64 bytes of counters.  kMaxP is the largest p for
// which ceil(p / 512) blocks fit; the launch's own grid (one element per
// thread while all its blocks fit the GPU at once, else more) is checked
// against the array again before the launch.
constexpr int64_t kMaxP = (int64_t)((kScratchBytes - 3 * ACC_STRIDE * 8 - 64) / (2 * NBP * 8)) * (2 * PBLOCK);

constexpr int kMaxDevices = 64;
void* g_scratch_dev[kMaxDevices] = {};   // device address of g_prox_scratch, per device
std::mutex g_scratch_mu;

// Device address of the scratch array on the current device, looked up once
// per device (with that device current) and remembered.
cudaError_t scratch_address(void** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_scratch_mu);
  if (!g_scratch_dev[dev]) {
    void* ptr = nullptr;
    e = cudaGetSymbolAddress(&ptr, g_prox_scratch);
    if (e != cudaSuccess) return e;
    g_scratch_dev[dev] = ptr;
  }
  *out = g_scratch_dev[dev];
  return cudaSuccess;
}

relax_status cuda_failure(const char* what, cudaError_t e) {
  char msg[256];
  std::snprintf(msg, sizeof(msg), "%s failed: %s (noalloc.cu)", what, cudaGetErrorString(e));
  set_error_detail(msg);
  (void)cudaGetLastError();
  return e == cudaErrorMemoryAllocation ? RELAX_ENOMEM : RELAX_ECUDA;
}

}  // namespace

extern "C" relax_status prox_persp_noalloc(const void* beta_in, void* beta_out, int64_t p, double step, int32_t k,
                                           double lambda2, double M, const int8_t* fixings, int32_t dtype,
                                           int32_t* counts_out, void* stream) {
  if (!beta_in || !beta_out || p <= 0 || k < 0 || !(step > 0.0) || !(lambda2 > 0.0) || !(M > 0.0) ||
      (dtype != RELAX_F64 && dtype != RELAX_F32))
    return RELAX_EINVAL;
  if (p > kMaxP) {
    char msg[256];
    std::snprintf(msg, sizeof(msg), "prox_persp_noalloc: p = %lld exceeds %lld, the most its fixed %zu-byte scratch serves",
                  (long long)p, (long long)kMaxP, kScratchBytes);
    set_error_detail(msg);
    return RELAX_ENOTSUP;
  }
  const cudaStream_t st = static_cast<cudaStream_t>(stream);
  PPlan pl;
  cudaError_t e = pphase_plan(pl, dtype == RELAX_F64, p);
  if (e == cudaErrorNotSupported) return RELAX_ENOTSUP;
  if (e != cudaSuccess) return cuda_failure("pphase_plan", e);
  // the same layout as the allocating entry point: accumulators | block partials | counter, status, output
  const size_t acc_b = 3 * ACC_STRIDE * sizeof(unsigned long long);
  const size_t bp_b = (size_t)2 * pl.grid * NBP * sizeof(double);
  const size_t need = acc_b + bp_b + 64;
  if (need > kScratchBytes) {
    char msg[256];
    std::snprintf(msg, sizeof(msg),
                  "prox_persp_noalloc: p = %lld needs %zu bytes of scratch (%d blocks); the fixed array holds %zu",
                  (long long)p, need, pl.grid, kScratchBytes);
    set_error_detail(msg);
    return RELAX_ENOTSUP;
  }
  void* scr_v = nullptr;
  e = scratch_address(&scr_v);
  if (e != cudaSuccess) return cuda_failure("cudaGetSymbolAddress", e);
  unsigned char* scr = static_cast<unsigned char*>(scr_v);
  // the array keeps the previous call's contents: zero everything the kernel counts from zero
  e = cudaMemsetAsync(scr, 0, need, st);
  if (e != cudaSuccess) return cuda_failure("cudaMemsetAsync", e);
  PArgs a{};
  a.mode = PM_PROX;
  a.p = p;
  a.k = k;
  a.lambda2 = lambda2;
  a.M = M;
  a.rho = 2.0 * lambda2 * step;
  a.kc = pconst_make(lambda2, M, step, a.rho);
  a.fix = fixings;
  a.vin = beta_in;
  a.vout = beta_out;
  a.counts = counts_out;
  a.acc = reinterpret_cast<unsigned long long*>(scr);
  a.bpart = reinterpret_cast<double*>(scr + acc_b);
  a.bar = reinterpret_cast<unsigned long long*>(scr + acc_b + bp_b);
  a.status = reinterpret_cast<int*>(scr + acc_b + bp_b + 8);
  a.out = reinterpret_cast<double*>(scr + acc_b + bp_b + 16);
  a.bar_base = 0;
  a.limit_ns = 4000000000ull;
  e = pphase_launch(pl, a, st);
  if (e != cudaSuccess) return cuda_failure("pphase_launch", e);
  return RELAX_OK;
}
