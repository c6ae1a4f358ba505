// Shared pieces of the fused pass over X: link modes, the pass's view of the
// solver state, 16-byte vector loads of every storage type of X, and the
// compensated FP32 pair arithmetic used for dot products and accumulations.
#pragma once
#include <cuda_bf16.h>
#include <cuda_fp8.h>

#include "common.cuh"

namespace relax {

enum Link : int {
  LINK_LS = 0,         // NF=1 NB=1: r = 2(z - y)
  LINK_LOGISTIC = 1,   // NF=1 NB=2: r = grad at z, r_y = grad at (1+mu) z - mu z_prev
  LINK_IDENT = 2,      // NF=1 NB=1: r = z             (power iteration on X'X)
  LINK_CERT_LS = 3,    // NF=2 NB=1: F at z0, r = 2(z1 - y)
  LINK_CERT_LOGI = 4,  // NF=2 NB=1: F at z0, r = grad at z1
  LINK_CERTZ_LS = 5,   // NF=1 NB=1: F at z0, r = 2(zd - y) with zd = ps.zprev (given dual point)
  LINK_CERTZ_LOGI = 6, // NF=1 NB=1: F at z0, r = grad at zd
  // both dual points of a certificate in one pass: NF=1 NB=2, F at z0,
  // r0 = the link at zd = ps.zprev (the loop's best dual point), r1 = the link
  // at z0 (zeta = -grad F(X beta)); lterm gets {F, dual term at zd}, lterm2
  // {F, dual term at z0}
  LINK_CERT2_LS = 7,
  LINK_CERT2_LOGI = 8,
};

// Device-resident solver state that the pass reads (pointers rotate between
// iterations, so a captured graph can replay the same launches).
struct PassState {
  const void* beta;      // forward vector 0 (beta^t)
  const void* beta2;     // forward vector 1 (certification)
  void* zout;            // z^t output (logistic; NULL otherwise)
  const void* zprev;     // z^{t-1} (logistic)
  double mom;            // tentative momentum mu for z_y
  int done;              // solver finished: pass returns immediately
};

template <typename TX> struct XTraits;
// 16-byte vectors of X: load from shared memory (load), from global memory
// keeping the line in L2 for a later re-read (load_global: ld.global.cg), or
// from global memory as its last use (load_global_last: ld.global.cs).
template <> struct XTraits<double> {
  static constexpr int VEC = 2;
  template <typename TA> __device__ static void cvt(const double2 v, TA* o) { o[0] = (TA)v.x; o[1] = (TA)v.y; }
  template <typename TA> __device__ static void load(const double* p, TA* o) { cvt(*reinterpret_cast<const double2*>(p), o); }
  template <typename TA> __device__ static void load_global(const double* p, TA* o) { cvt(__ldcg(reinterpret_cast<const double2*>(p)), o); }
  template <typename TA> __device__ static void load_global_last(const double* p, TA* o) { cvt(__ldcs(reinterpret_cast<const double2*>(p)), o); }
};
template <> struct XTraits<float> {
  static constexpr int VEC = 4;
  template <typename TA> __device__ static void cvt(const float4 v, TA* o) {
    o[0] = (TA)v.x; o[1] = (TA)v.y; o[2] = (TA)v.z; o[3] = (TA)v.w;
  }
  template <typename TA> __device__ static void load(const float* p, TA* o) { cvt(*reinterpret_cast<const float4*>(p), o); }
  template <typename TA> __device__ static void load_global(const float* p, TA* o) { cvt(__ldcg(reinterpret_cast<const float4*>(p)), o); }
  template <typename TA> __device__ static void load_global_last(const float* p, TA* o) { cvt(__ldcs(reinterpret_cast<const float4*>(p)), o); }
};
template <> struct XTraits<__nv_bfloat16> {
  static constexpr int VEC = 8;
  template <typename TA> __device__ static void cvt(const uint4 v, TA* o) {
    const __nv_bfloat162* h = reinterpret_cast<const __nv_bfloat162*>(&v);
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      float2 f = __bfloat1622float2(h[i]);
      o[2 * i] = (TA)f.x; o[2 * i + 1] = (TA)f.y;
    }
  }
  template <typename TA> __device__ static void load(const __nv_bfloat16* p, TA* o) { cvt(*reinterpret_cast<const uint4*>(p), o); }
  template <typename TA> __device__ static void load_global(const __nv_bfloat16* p, TA* o) { cvt(__ldcg(reinterpret_cast<const uint4*>(p)), o); }
  template <typename TA> __device__ static void load_global_last(const __nv_bfloat16* p, TA* o) { cvt(__ldcs(reinterpret_cast<const uint4*>(p)), o); }
};
template <> struct XTraits<__nv_fp8_e4m3> {
  static constexpr int VEC = 16;
  template <typename TA> __device__ static void cvt(const uint4 v, TA* o) {
    const __nv_fp8x2_storage_t* h = reinterpret_cast<const __nv_fp8x2_storage_t*>(&v);
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      __half2_raw hr = __nv_cvt_fp8x2_to_halfraw2(h[i], __NV_E4M3);
      float2 f = __half22float2(*reinterpret_cast<__half2*>(&hr));
      o[2 * i] = (TA)f.x; o[2 * i + 1] = (TA)f.y;
    }
  }
  template <typename TA> __device__ static void load(const __nv_fp8_e4m3* p, TA* o) { cvt(*reinterpret_cast<const uint4*>(p), o); }
  template <typename TA> __device__ static void load_global(const __nv_fp8_e4m3* p, TA* o) { cvt(__ldcg(reinterpret_cast<const uint4*>(p)), o); }
  template <typename TA> __device__ static void load_global_last(const __nv_fp8_e4m3* p, TA* o) { cvt(__ldcs(reinterpret_cast<const uint4*>(p)), o); }
};

// log(1 + exp(-t)) computed stably, in double
__device__ __forceinline__ double softplus_neg(double t) {
  return fmax(-t, 0.0) + log1p(exp(-fabs(t)));
}
// -(u log u + (1-u) log(1-u)) with u = 1/(1+exp(t)), in double
__device__ __forceinline__ double entropy_of(double t) {
  const double u = 1.0 / (1.0 + exp(t));
  const double v = 1.0 / (1.0 + exp(-t));
  double h = 0.0;
  if (u > 0.0) h -= u * log(u);
  if (v > 0.0) h -= v * log(v);
  return h;
}

// Compensated accumulation of FP32 partial sums into an (hi, lo) FP32 pair
// (Knuth's TwoSum): hi + lo carries the running sum to about twice the FP32
// precision without FP64 arithmetic.
// Packed FP32 pairs: Blackwell's f32x2 add / sub / fma issue one instruction
// for two independent FP32 operations, each rounded exactly as the scalar
// instruction rounds it (IEEE round to nearest even).
__device__ __forceinline__ unsigned long long f2_bits(float2 v) {
  return ((unsigned long long)__float_as_uint(v.y) << 32) | __float_as_uint(v.x);
}
__device__ __forceinline__ float2 f2_of(unsigned long long b) {
  return make_float2(__uint_as_float((unsigned)b), __uint_as_float((unsigned)(b >> 32)));
}
// a * b + c per half
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) {
  unsigned long long r;
  asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(r) : "l"(f2_bits(a)), "l"(f2_bits(b)), "l"(f2_bits(c)));
  return f2_of(r);
}
__device__ __forceinline__ float2 add2(float2 a, float2 b) {
  unsigned long long r;
  asm("add.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(f2_bits(a)), "l"(f2_bits(b)));
  return f2_of(r);
}
__device__ __forceinline__ float2 sub2(float2 a, float2 b) {
  unsigned long long r;
  asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(f2_bits(a)), "l"(f2_bits(b)));
  return f2_of(r);
}
// two_sum_acc (below) on both halves of a pair
__device__ __forceinline__ void two_sum_acc2(float2& hi, float2& lo, float2 a) {
  const float2 s = add2(hi, a);
  const float2 bp = sub2(s, hi);
  const float2 err = add2(sub2(hi, sub2(s, bp)), sub2(a, bp));
  hi = s;
  lo = add2(lo, err);
}

__device__ __forceinline__ void two_sum_acc(float& hi, float& lo, float a) {
  const float s = hi + a;
  const float bp = s - hi;
  const float err = (hi - (s - bp)) + (a - bp);
  hi = s;
  lo += err;
}

// A (hi, lo) FP32 pair travels through the exchange as the bits of a double.
__device__ __forceinline__ double pack_pair(float hi, float lo) {
  return __hiloint2double(__float_as_int(hi), __float_as_int(lo));
}
__device__ __forceinline__ void add_pair(float& hi, float& lo, double packed) {
  const float ph = __int_as_float(__double2hiint(packed));
  const float pl = __int_as_float(__double2loint(packed));
  two_sum_acc(hi, lo, ph);
  lo += pl;
}
__device__ __forceinline__ float exp_t(float t) { return expf(t); }
__device__ __forceinline__ double exp_t(double t) { return exp(t); }

// Warp sum of (hi, lo) FP32 pairs: each butterfly step adds the partner's pair
// with TwoSum, keeping about 44 bits; FP32 pipe only.
__device__ __forceinline__ void warp_sum_pair(float& hi, float& lo) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const float oh = __shfl_xor_sync(0xffffffffu, hi, o);
    const float ol = __shfl_xor_sync(0xffffffffu, lo, o);
    float h = hi, l = 0.f;
    two_sum_acc(h, l, oh);
    hi = h;
    lo = lo + ol + l;
  }
}

}  // namespace relax
