// Fused pass over X: for each row tile, z = X_tile beta (per-row dot products),
// r = link(z) (GLM gradient / residual), then acc += X_tile' r -- with the tile
// resident in shared memory, so X is read from HBM exactly once per pass.
//
// This is the matrix-vector work that dominates the method (Sec. 5.2.3).  The
// induced dual point zeta = -grad F(X beta) (Sec. 3.3) comes out of the same
// pass: zeta = -r.
//
// Layout and schedule (sm_103a):
//  * X row-major n x ldx.  A cluster of C CTAs splits the p columns into C
//    slices; CTA rank q owns columns [q*slice, q*slice + W_q).
//  * A producer warp streams R-row tiles of its slice into an S-stage shared
//    ring with 1-D bulk copies (cp.async.bulk, completion on an mbarrier with
//    transaction bytes).  Consumer warps keep the beta slice and the X'r
//    accumulators in registers.
//  * Per tile: partial row dots -> block reduction -> each CTA writes its R
//    partials into every peer's exchange slot (DSMEM) and arrives on the
//    peer's mbarrier; after all C partials are in, every CTA sums them in the
//    same order (so all CTAs see bit-identical z), applies the link and
//    accumulates X' r from the still-resident tile.  The dot products of tile
//    k+1 are computed before waiting on tile k's exchange, hiding its latency.
//  * Clusters take row tiles round-robin; each writes its X' r partial to
//    part[cluster][b][:]; the p-phase sums the partials in a fixed order.
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

struct XPassArgs {
  const void* X;
  int64_t ldx, n, p;
  int64_t slice;          // columns per cluster rank (multiple of VEC)
  int C, R, S;            // cluster size, rows per tile, stages
  uint32_t slot_bytes;    // bytes per row slot in the ring (>= round16(slice*esize))
  int link;
  const void* y;          // n, storage type of the vectors (TB)
  const float* colscale;  // per-column scale for quantized X (NULL = 1)
  PassState* ps;          // pointers/scalars (device)
  void* part;             // [ncl][NB][p] of TA
  double* lossp;          // [ncl][2]: {F, -F*(-zeta)} partial sums
  int* status;
  uint64_t limit_ns;
};

template <typename TX> struct XTraits;
template <> struct XTraits<double> {
  static constexpr int VEC = 2;
  template <typename TA> __device__ static void load(const double* p, TA* o) {
    double2 v = *reinterpret_cast<const double2*>(p);
    o[0] = (TA)v.x; o[1] = (TA)v.y;
  }
};
template <> struct XTraits<float> {
  static constexpr int VEC = 4;
  template <typename TA> __device__ static void load(const float* p, TA* o) {
    float4 v = *reinterpret_cast<const float4*>(p);
    o[0] = (TA)v.x; o[1] = (TA)v.y; o[2] = (TA)v.z; o[3] = (TA)v.w;
  }
};
template <> struct XTraits<__nv_bfloat16> {
  static constexpr int VEC = 8;
  template <typename TA> __device__ static void load(const __nv_bfloat16* p, TA* o) {
    uint4 v = *reinterpret_cast<const uint4*>(p);
    const __nv_bfloat162* h = reinterpret_cast<const __nv_bfloat162*>(&v);
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      float2 f = __bfloat1622float2(h[i]);
      o[2 * i] = (TA)f.x; o[2 * i + 1] = (TA)f.y;
    }
  }
};
template <> struct XTraits<__nv_fp8_e4m3> {
  static constexpr int VEC = 16;
  template <typename TA> __device__ static void load(const __nv_fp8_e4m3* p, TA* o) {
    uint4 v = *reinterpret_cast<const uint4*>(p);
    const __nv_fp8x2_storage_t* h = reinterpret_cast<const __nv_fp8x2_storage_t*>(&v);
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      __half2_raw hr = __nv_cvt_fp8x2_to_halfraw2(h[i], __NV_E4M3);
      float2 f = __half22float2(*reinterpret_cast<__half2*>(&hr));
      o[2 * i] = (TA)f.x; o[2 * i + 1] = (TA)f.y;
    }
  }
};

template <typename TA>
__device__ __forceinline__ TA sigmoid_neg(TA t);  // 1 / (1 + exp(t))
template <> __device__ __forceinline__ float sigmoid_neg(float t) { return 1.0f / (1.0f + expf(t)); }
template <> __device__ __forceinline__ double sigmoid_neg(double t) { return 1.0 / (1.0 + exp(t)); }

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

template <typename TX, typename TB, typename TA, int NF, int NB, int BLOCK, int NV, int R>
__global__ void __launch_bounds__(BLOCK + 32, 1) xpass_kernel(const XPassArgs a) {
  constexpr int VEC = XTraits<TX>::VEC;
  constexpr int NWARP = BLOCK / 32;
  constexpr int NRF = R * NF;
  constexpr int NXS = 4;  // exchange slots (see the reuse argument below)
  extern __shared__ __align__(128) unsigned char smem[];

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int C = a.C, S = a.S;
  const uint32_t rank = cluster_ctarank();
  const uint32_t cid = cluster_id_x();
  const uint32_t ncl = nclusters_x();

  // ---- shared layout
  unsigned char* ring = smem;
  const size_t ring_bytes = (size_t)S * R * a.slot_bytes;
  uint64_t* full = reinterpret_cast<uint64_t*>(smem + ring_bytes);
  uint64_t* empty = full + S;
  uint64_t* xfull = empty + S;
  TA* xch = reinterpret_cast<TA*>(xfull + NXS);        // [NXS][C][NRF]
  TA* red = xch + NXS * C * NRF;                       // [2][NWARP][NRF]
  __shared__ volatile int tmo;   // a bounded wait expired: stop waiting, keep the barrier sequence
  __shared__ int skip;

  if (tid == 0) {
    tmo = 0;
    skip = a.ps->done;
    for (int s = 0; s < S; ++s) { mbar_init(&full[s], 1); mbar_init(&empty[s], NWARP); }
    for (int s = 0; s < NXS; ++s) mbar_init(&xfull[s], C);
    fence_mbar_init_cluster();
  }
  __syncthreads();
  cluster_sync_all();
  if (skip) { cluster_sync_all(); return; }   // uniform across the cluster (same flag)

  const int64_t c0 = (int64_t)rank * a.slice;
  const int64_t W = (a.p - c0) < a.slice ? (a.p - c0) : a.slice;
  const int nvec = (int)((W + VEC - 1) / VEC);
  const uint32_t row_bytes = (uint32_t)(((W * (int64_t)sizeof(TX)) + 15) & ~(int64_t)15);
  const int64_t ntiles = (a.n + R - 1) / R;
  const int K = (int64_t)cid < ntiles ? (int)((ntiles - cid + ncl - 1) / ncl) : 0;
  const TX* X = static_cast<const TX*>(a.X);
  auto tile_ptr = [&](int s, int r) -> const TX* {
    return reinterpret_cast<const TX*>(ring + ((size_t)s * R + r) * a.slot_bytes);
  };
  auto tile_rows = [&](int k) -> int {
    const int64_t row0 = ((int64_t)cid + (int64_t)k * ncl) * R;
    const int64_t left = a.n - row0;
    return left < R ? (int)left : R;
  };

  if (warp == NWARP) {
    // ------------------------------------------------------------ producer
    if (lane == 0) {
      const uint64_t pol = policy_evict_first();
      int issued = 0;
      for (int k = 0; k < K; ++k) {
        const int s = k % S;
        if (k >= S) {
          if (tmo || !mbar_wait<false>(&empty[s], (uint32_t)(((k / S) - 1) & 1), a.limit_ns, a.status)) {
            tmo = 1;
            break;
          }
        }
        const int rows = tile_rows(k);
        const int64_t row0 = ((int64_t)cid + (int64_t)k * ncl) * R;
        mbar_arrive_expect_tx(&full[s], (uint32_t)rows * row_bytes);
        for (int r = 0; r < rows; ++r)
          bulk_g2s((void*)tile_ptr(s, r), X + (row0 + r) * a.ldx + c0, row_bytes, &full[s], pol);
        ++issued;
      }
      // never leave with copies in flight into this CTA's shared memory
      for (int k = issued > S ? issued - S : 0; k < issued; ++k)
        mbar_wait<false>(&full[k % S], (uint32_t)((k / S) & 1), a.limit_ns, a.status);
    }
    __syncwarp();
    cluster_sync_all();
    return;
  }

  // -------------------------------------------------------------- consumers
  const PassState* ps = a.ps;
  const TB* bvec[2] = {static_cast<const TB*>(ps->beta), static_cast<const TB*>(ps->beta2)};
  const TB* yv = static_cast<const TB*>(a.y);
  const TB* zprev = static_cast<const TB*>(ps->zprev);
  TB* zout = static_cast<TB*>(ps->zout);
  const TA mom = (TA)ps->mom;

  TA u[NF][NV * VEC];
  TA acc[NB][NV * VEC];
#pragma unroll
  for (int iv = 0; iv < NV; ++iv) {
    const int v = tid + BLOCK * iv;
#pragma unroll
    for (int l = 0; l < VEC; ++l) {
      const int64_t col = c0 + (int64_t)v * VEC + l;
      const bool ok = v < nvec && col < a.p;
      const TA sc = (ok && a.colscale) ? (TA)a.colscale[col] : (TA)1;
#pragma unroll
      for (int f = 0; f < NF; ++f) u[f][iv * VEC + l] = ok ? (TA)bvec[f][col] * sc : (TA)0;
#pragma unroll
      for (int b = 0; b < NB; ++b) acc[b][iv * VEC + l] = (TA)0;
    }
  }

  // After an expired wait (tmo) nothing waits any more, but every consumer
  // still runs the same sequence of named barriers and exchanges, so no
  // thread of the cluster is left blocked; the status word reports the error.
  auto wait_full = [&](int k) {
    if (!tmo && !mbar_wait<false>(&full[k % S], (uint32_t)((k / S) & 1), a.limit_ns, a.status))
      tmo = 1;
  };

  // partial dots of tile k; X entries past column p are masked to zero
  auto dots = [&](int k, TA (&d)[R][NF]) {
    const int s = k % S;
    const int rows = tile_rows(k);
#pragma unroll
    for (int r = 0; r < R; ++r) {
#pragma unroll
      for (int f = 0; f < NF; ++f) d[r][f] = (TA)0;
      if (r < rows) {
        const TX* t = tile_ptr(s, r);
#pragma unroll
        for (int iv = 0; iv < NV; ++iv) {
          const int v = tid + BLOCK * iv;
          if (v < nvec) {
            TA x[VEC];
            XTraits<TX>::load(t + (size_t)v * VEC, x);
            const int64_t colv = c0 + (int64_t)v * VEC;
            if (colv + VEC > a.p) {   // row padding past column p: may hold anything
#pragma unroll
              for (int l = 0; l < VEC; ++l)
                if (colv + l >= a.p) x[l] = (TA)0;
            }
#pragma unroll
            for (int l = 0; l < VEC; ++l) {
#pragma unroll
              for (int f = 0; f < NF; ++f) d[r][f] += x[l] * u[f][iv * VEC + l];
            }
          }
        }
      }
    }
  };

  // Block-reduce the R*NF partials of tile k and publish them to every CTA of
  // the cluster.  Exchange slot k % 4: a peer that is still reading slot
  // (k-4) % 4 cannot exist, because our sending of tile k happens after our
  // wait on tile k-2, which needs every peer's tile k-2 partial, which each
  // peer sends only after it finished reading tile k-4's slot.
  auto publish = [&](int k, TA (&d)[R][NF]) {
    TA* rb = red + (k & 1) * NWARP * NRF;
#pragma unroll
    for (int r = 0; r < R; ++r)
#pragma unroll
      for (int f = 0; f < NF; ++f) {
        TA v = warp_sum(d[r][f]);
        if (lane == 0) rb[warp * NRF + r * NF + f] = v;
      }
    named_sync(1, BLOCK);
    if (tid == 0) {
      const int slot = k % NXS;
      for (int i = 0; i < NRF; ++i) {
        TA s = (TA)0;
        for (int w = 0; w < NWARP; ++w) s += rb[w * NRF + i];
        TA* dst = xch + (slot * C + (int)rank) * NRF + i;
        for (int q = 0; q < C; ++q) st_cluster(mapa(dst, (uint32_t)q), s);
      }
      for (int q = 0; q < C; ++q) mbar_arrive_remote(mapa(&xfull[slot], (uint32_t)q));
    }
  };

  double lossF = 0.0, lossD = 0.0;
  TA dn[R][NF];
  if (K > 0) {
    wait_full(0);
    dots(0, dn);
    publish(0, dn);
  }
  for (int k = 0; k < K; ++k) {
    const int s = k % S;
    const int rows = tile_rows(k);
    if (k + 1 < K) {
      wait_full(k + 1);
      dots(k + 1, dn);
      publish(k + 1, dn);
    }
    const int slot = k % NXS;
    if (!tmo && !mbar_wait<true>(&xfull[slot], (uint32_t)((k / NXS) & 1), a.limit_ns, a.status))
      tmo = 1;
    // every CTA sums the C partials in rank order -> identical z in all CTAs
    TA w[R][NB];
    const int64_t row0 = ((int64_t)cid + (int64_t)k * ncl) * R;
#pragma unroll
    for (int r = 0; r < R; ++r) {
#pragma unroll
      for (int b = 0; b < NB; ++b) w[r][b] = (TA)0;
      if (r < rows) {
        TA z[NF];
#pragma unroll
        for (int f = 0; f < NF; ++f) {
          TA acc_z = (TA)0;
          for (int q = 0; q < C; ++q) acc_z += xch[(slot * C + q) * NRF + r * NF + f];
          z[f] = acc_z;
        }
        const int64_t i = row0 + r;
        const bool lead = (rank == 0 && tid == 0);
        switch (a.link) {
          case LINK_LS: {
            const TA yi = (TA)yv[i];
            w[r][0] = (TA)2 * (z[0] - yi);
            if (lead) {
              const double d = (double)z[0] - (double)yi;
              const double zeta = -2.0 * d;
              lossF += d * d;
              lossD += zeta * (double)yi - 0.25 * zeta * zeta;
            }
            break;
          }
          case LINK_LOGISTIC: {
            const TA yi = (TA)yv[i];
            w[r][0] = -yi * sigmoid_neg<TA>(yi * z[0]);
            if (NB > 1) {
              const TA zy = ((TA)1 + mom) * z[0] - mom * (TA)zprev[i];
              w[r][NB - 1] = -yi * sigmoid_neg<TA>(yi * zy);
            }
            if (lead) {
              const double t = (double)yi * (double)z[0];
              lossF += softplus_neg(t);
              lossD += entropy_of(t);
              if (zout) zout[i] = (TB)z[0];
            }
            break;
          }
          case LINK_IDENT: {
            w[r][0] = z[0];
            if (lead) lossF += (double)z[0] * (double)z[0];
            break;
          }
          case LINK_CERT_LS: {
            const TA yi = (TA)yv[i];
            w[r][0] = (TA)2 * (z[NF - 1] - yi);
            if (lead) {
              const double d0 = (double)z[0] - (double)yi;
              const double d1 = (double)z[NF - 1] - (double)yi;
              const double zeta = -2.0 * d1;
              lossF += d0 * d0;
              lossD += zeta * (double)yi - 0.25 * zeta * zeta;
            }
            break;
          }
          case LINK_CERT_LOGI: {
            const TA yi = (TA)yv[i];
            w[r][0] = -yi * sigmoid_neg<TA>(yi * z[NF - 1]);
            if (lead) {
              lossF += softplus_neg((double)yi * (double)z[0]);
              lossD += entropy_of((double)yi * (double)z[NF - 1]);
            }
            break;
          }
          default: break;
        }
        if (lead && zout && a.link != LINK_LOGISTIC) zout[i] = (TB)z[0];
      }
    }
    // acc += X_tile' w from the resident tile
#pragma unroll
    for (int r = 0; r < R; ++r) {
      if (r < rows) {
        const TX* t = tile_ptr(s, r);
#pragma unroll
        for (int iv = 0; iv < NV; ++iv) {
          const int v = tid + BLOCK * iv;
          if (v < nvec) {
            TA x[VEC];
            XTraits<TX>::load(t + (size_t)v * VEC, x);
#pragma unroll
            for (int l = 0; l < VEC; ++l)
#pragma unroll
              for (int b = 0; b < NB; ++b) acc[b][iv * VEC + l] += w[r][b] * x[l];
          }
        }
      }
    }
    __syncwarp();
    if (lane == 0) mbar_arrive(&empty[s]);
  }

  // ---- write this cluster's X' r partial (columns of this rank's slice)
  TA* part = static_cast<TA*>(a.part);
#pragma unroll
  for (int iv = 0; iv < NV; ++iv) {
    const int v = tid + BLOCK * iv;
    if (v < nvec) {
#pragma unroll
      for (int l = 0; l < VEC; ++l) {
        const int64_t col = c0 + (int64_t)v * VEC + l;
        if (col < a.p) {
          const TA sc = a.colscale ? (TA)a.colscale[col] : (TA)1;
#pragma unroll
          for (int b = 0; b < NB; ++b)
            part[((int64_t)cid * NB + b) * a.p + col] = acc[b][iv * VEC + l] * sc;
        }
      }
    }
  }
  if (rank == 0 && tid == 0) {
    a.lossp[cid * 2 + 0] = lossF;
    a.lossp[cid * 2 + 1] = lossD;
  }
  cluster_sync_all();
}

}  // namespace relax
