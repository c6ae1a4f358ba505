// Batched products of many node relaxations sharing X on the 5th-generation
// tensor cores: D = A B^T with A (M x K) and B (N x K) both K-major, each
// stored as three BF16 planes whose sum is the FP32 value exactly (8 + 8 + 8
// significand bits).  Six BF16 products per element pair (the pairs of planes
// whose significance sums to at most the third plane's) reproduce FP32
// products to within 2^-23 relative.
//
// Accumulation.  X' r cancels by several orders of magnitude near a node's
// optimum (the gradient is small against the sum of the magnitudes of its
// terms), and the tensor cores' FP32 accumulation loses about half an ulp of
// the running sum per MMA (measured: its error grows like truncation, not
// like rounding), so one FP32 accumulator over thousands of terms put the
// duality gap's floor above 1e-6.  Two measures keep it near the fused
// pass's: the main product (first planes of both operands) accumulates alone
// in one TMEM accumulator, the five correction products (2^-8 smaller and
// below, so their accumulation error is negligible) in a second one; and
// both hold only BG_DRAIN K blocks (128 elements) before the epilogue warps
// drain them into FP32 registers (round to nearest) while the MMAs fill the
// other of two TMEM buffer pairs.
//
// Schedule.  The iteration space (tile, K block), tiles in order with the
// N-tiles innermost, is cut into one contiguous range per CTA of equal length
// (to one K block), so every SM gets the same work whatever the tile count.
// A range covers the end of one tile, whole tiles, the start of another; each
// piece writes its partial tile in FP64 to slot (CTA - first CTA of the
// tile), and a reduction kernel sums a tile's slots in FP64 in slot order
// (deterministic), fused with what consumes the product: the link of the
// loss (Z = X B) or the per-node gradient layout of the p-phase (G = X' R).
#pragma once
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include "pphase.cuh"

namespace relax {

constexpr int BG_BM = 128;          // rows of A per tile (the MMA's M)
constexpr int BG_SW = 64;           // bytes per tile row in shared memory (64-byte swizzle)
constexpr int BG_BK = BG_SW / 2;    // K elements (BF16) per pipeline stage
constexpr int BG_MAXN = 128;        // columns of D per tile (one MMA's N) at most
constexpr int BG_NBUF = 2;          // TMEM buffer pairs (main, corrections) of BG_MAXN columns each
constexpr int BG_DRAIN = 4;         // K blocks accumulated in TMEM between drains
constexpr int BG_PLANES = 3;
constexpr int BG_MAXS = 8;          // pipeline stages at most
constexpr int BG_THREADS = 320;     // producer warp, MMA warp, eight epilogue warps
constexpr int BG_MAXKC = 16;        // partial slots per tile at most (partials are KC x N x M doubles)

// The split of the iteration space: MT x NT tiles of nkb K blocks over `grid`
// CTAs; CTA c takes [c T / grid, (c + 1) T / grid), T = MT NT nkb.
struct BGSplit {
  int MT = 1, NT = 1, BN = 16, nkb = 1, grid = 1;
};
// the CTA whose range holds iteration i
__host__ __device__ inline int64_t bg_owner(int64_t i, int64_t T, int grid) { return ((i + 1) * grid - 1) / T; }
// first CTA of tile t and its number of slots (CTAs whose range meets the tile)
__host__ __device__ inline int bg_first(const BGSplit& s, int t) {
  const int64_t T = (int64_t)s.MT * s.NT * s.nkb;
  return (int)bg_owner((int64_t)t * s.nkb, T, s.grid);
}
__host__ __device__ inline int bg_slots(const BGSplit& s, int t) {
  const int64_t T = (int64_t)s.MT * s.NT * s.nkb;
  return (int)(bg_owner((int64_t)(t + 1) * s.nkb - 1, T, s.grid) - bg_owner((int64_t)t * s.nkb, T, s.grid)) + 1;
}

struct BGArgs {
  CUtensorMap tmA;        // planes of A: dims {K, M, 3}, box {BG_BK, 128, 3}
  CUtensorMap tmB;        // planes of B: dims {K, N, 3}, box {BG_BK, BN, 3}
  int M, N, K;
  int BN, NT, MT;         // tile columns, N-tiles, M-tiles
  int nkb;                // K blocks (of BG_BK) over K
  int stages;
  double* P;              // [slot][N][M] partial products (FP64)
  int* status;
  uint64_t limit_ns;
};

struct BGPlan {
  int M = 0, N = 0, K = 0;
  int BN = 16, NT = 1, MT = 1, KC = 1, nkb = 1, stages = 2, grid = 1;   // KC: slots per tile at most
  size_t smem = 0;
  BGSplit split() const {
    BGSplit s;
    s.MT = MT; s.NT = NT; s.BN = BN; s.nkb = nkb; s.grid = grid;
    return s;
  }
};

// Tile plan of D (M x N) = A B^T over K: BN and the N-tiles from N, the
// stages from shared memory, one CTA per SM (fewer when the tiles' slots
// would exceed BG_MAXKC or there are fewer K blocks than SMs).
cudaError_t bgemm_plan(BGPlan& pl, int M, int N, int K);
// Tensor map of three BF16 planes [3][rows][ld] with `rows` rows of K valid
// elements (ld >= K, a multiple of 8), box {BG_BK, box_rows, 3}, 64-byte swizzle.
cudaError_t bgemm_encode(CUtensorMap* tm, const void* planes, int64_t K, int64_t rows, int64_t ld,
                         int64_t plane_rows, int box_rows);
cudaError_t bgemm_launch(const BGPlan& pl, const BGArgs& a, cudaStream_t st);
// planes[3][rows][ld] of FP32 X (n x p, leading dimension ldx): rows = n,
// K = p (transpose = false) or rows = p, K = n (transpose = true); padding
// columns are zero.
cudaError_t bgemm_split_x(const float* X, int64_t n, int64_t p, int64_t ldx, bool transpose, __nv_bfloat16* planes,
                          int64_t ld, cudaStream_t st);

// Per-iteration kernels of the batched solve around the two products.
struct BatchIo {
  const IterState* st;   // node states (NULL: the points are bsrc and z goes to zdst)
  const int* active;     // active node of each column slot
  int m;                 // active nodes
  int nb;                // node slots allocated (plane row stride of B)
  int64_t n, p;
  int64_t ldp, ldn;      // plane leading dimensions (K = p, K = n)
  int NB;                // right-hand sides per node (1 LS, 2 logistic)
  int loss;              // RELAX_LS, RELAX_LOGISTIC, or -1: the identity link (R = Z)
  const double* bsrc;    // st == NULL: the points, [m][p]
  double* zdst;          // st == NULL: z of every point, [m][n]
  const double* y;
  __nv_bfloat16* Bp;     // [3][nb][ldp] planes of the node points
  __nv_bfloat16* Rp;     // [3][NB nb][ldn] planes of the link (the second product's B)
  const double* P1;      // [slot][m][n] partials of Z = X B
  BGSplit s1;
  const double* P2;      // [slot][NB m][p] partials of G = X' R
  BGSplit s2;
  double* part;          // [m][NB][p] gradients per node (p-phase layout)
};
// B planes of the active nodes' next points
cudaError_t batch_pack(const BatchIo& io, cudaStream_t st);
// z = sum of the Z partials (FP64): each node's z^t, and the planes of
// grad F at z (and at the momentum point for the logistic loop)
cudaError_t batch_reduce_link(const BatchIo& io, cudaStream_t st);
// the gradients X' grad F of every node, summed over the chunks in FP64
cudaError_t batch_reduce_grad(const BatchIo& io, cudaStream_t st);

}  // namespace relax
