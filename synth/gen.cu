// Seeded synthetic-input generator on the device (no arithmetic of the
// relaxation method lives here).  Same definitions as synth/__init__.py:
//   * Philox4x64-10 (Salmon et al., SC'11): raw value r of stream (k0, k1) is
//     lane r % 4 of the block for counter (r / 4 + 1, 0, 0, 0);
//   * Box-Muller on raw pairs (2s, 2s+1): u1 = ((raw >> 11) + 1) 2^-53,
//     u2 = (raw >> 11) 2^-53, normal 2s = sqrt(-2 log u1) cos(2 pi u2),
//     normal 2s+1 = ... sin(2 pi u2);
//   * design rows by the AR(1) recursion x_{i,0} = e, x_{i,j} = rho x_{i,j-1} + c e
//     in FP64 with explicitly rounded products and sums, then cast.
#include <cstdint>
#include <cuda_runtime.h>

namespace {

__device__ __forceinline__ void philox4x64_10(uint64_t c[4], uint64_t k0, uint64_t k1) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    const uint64_t m0 = 0xD2E7470EE14C6C93ull, m1 = 0xCA5A826395121157ull;
    uint64_t lo0 = m0 * c[0], hi0 = __umul64hi(m0, c[0]);
    uint64_t lo1 = m1 * c[2], hi1 = __umul64hi(m1, c[2]);
    uint64_t n0 = hi1 ^ c[1] ^ k0, n2 = hi0 ^ c[3] ^ k1;
    c[0] = n0; c[1] = lo1; c[2] = n2; c[3] = lo0;
    k0 += 0x9E3779B97F4A7C15ull;
    k1 += 0xBB67AE8584CAA73Bull;
  }
}

// normals 4m .. 4m+3 of the stream
__device__ __forceinline__ void normal_block(uint64_t m, uint64_t k0, uint64_t k1, double out[4]) {
  uint64_t c[4] = {m + 1ull, 0ull, 0ull, 0ull};
  philox4x64_10(c, k0, k1);
  const double twopi = 6.283185307179586;
#pragma unroll
  for (int h = 0; h < 2; ++h) {
    double u1 = __dmul_rn((double)((c[2 * h] >> 11) + 1ull), 1.1102230246251565e-16);
    double u2 = __dmul_rn((double)(c[2 * h + 1] >> 11), 1.1102230246251565e-16);
    double r = sqrt(__dmul_rn(-2.0, log(u1)));
    double t = __dmul_rn(twopi, u2);
    double s, co;
    sincos(t, &s, &co);
    out[2 * h] = __dmul_rn(r, co);
    out[2 * h + 1] = __dmul_rn(r, s);
  }
}

template <typename T>
__global__ void __launch_bounds__(128) ar1_kernel(T* __restrict__ X, int64_t n, int64_t p, int64_t ldx,
                                                  double rho, double cc, uint64_t k0, uint64_t k1) {
  __shared__ T tile[4][32][33];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t row0 = ((int64_t)blockIdx.x * 4 + warp) * 32;
  if (row0 >= n) return;
  const int64_t i = row0 + lane;
  const bool live = i < n;
  double x = 0.0;
  uint64_t cached = ~0ull;
  double nb[4] = {0, 0, 0, 0};
  for (int64_t j0 = 0; j0 < p; j0 += 32) {
    const int64_t jn = (p - j0) < 32 ? (p - j0) : 32;
    if (live) {
      for (int64_t jj = 0; jj < jn; ++jj) {
        const int64_t j = j0 + jj;
        const uint64_t q = (uint64_t)i * (uint64_t)p + (uint64_t)j;
        const uint64_t m = q >> 2;
        if (m != cached) { normal_block(m, k0, k1, nb); cached = m; }
        const double e = nb[q & 3];
        x = (j == 0) ? e : __dadd_rn(__dmul_rn(rho, x), __dmul_rn(cc, e));
        tile[warp][lane][jj] = (T)x;
      }
    }
    __syncwarp();
    for (int r = 0; r < 32; ++r) {
      const int64_t row = row0 + r;
      if (row < n && lane < jn) X[row * ldx + j0 + lane] = tile[warp][r][lane];
    }
    __syncwarp();
  }
}

template <typename T>
__global__ void signal_kernel(const T* __restrict__ X, int64_t n, int64_t ldx, int k,
                              const int64_t* __restrict__ sup, double* __restrict__ s) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  double acc = 0.0;
  for (int t = 0; t < k; ++t) acc = __dadd_rn(acc, (double)X[i * ldx + sup[t]]);
  s[i] = acc;
}

}  // namespace

extern "C" {

// dtype: 0 = float64, 1 = float32.  Returns a cudaError_t value.
int synth_ar1_design(void* X, int64_t n, int64_t p, int64_t ldx, double rho, uint64_t seed,
                     uint64_t stream_id, int dtype, void* stream) {
  if (n <= 0 || p <= 0 || ldx < p) return (int)cudaErrorInvalidValue;
  const double cc = sqrt(1.0 - rho * rho);
  const int64_t warps = (n + 31) / 32;
  const unsigned grid = (unsigned)((warps + 3) / 4);
  cudaStream_t st = (cudaStream_t)stream;
  if (dtype == 0)
    ar1_kernel<double><<<grid, 128, 0, st>>>((double*)X, n, p, ldx, rho, cc, seed, stream_id);
  else if (dtype == 1)
    ar1_kernel<float><<<grid, 128, 0, st>>>((float*)X, n, p, ldx, rho, cc, seed, stream_id);
  else
    return (int)cudaErrorInvalidValue;
  return (int)cudaGetLastError();
}

int synth_signal(const void* X, int64_t n, int64_t p, int64_t ldx, int dtype, int64_t k,
                 const void* support, void* s) {
  (void)p;
  const unsigned grid = (unsigned)((n + 255) / 256);
  if (dtype == 0)
    signal_kernel<double><<<grid, 256>>>((const double*)X, n, ldx, (int)k, (const int64_t*)support,
                                         (double*)s);
  else if (dtype == 1)
    signal_kernel<float><<<grid, 256>>>((const float*)X, n, ldx, (int)k, (const int64_t*)support,
                                        (double*)s);
  else
    return (int)cudaErrorInvalidValue;
  return (int)cudaGetLastError();
}

}  // extern "C"
