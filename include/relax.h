/*
 * relax.h -- C ABI of the GB300 (sm_103a) library that computes branch-and-bound
 * node lower bounds for cardinality-constrained GLMs (arxiv 2603.01306).
 *
 * Problem (Sec. 2.3, Eq. 1):  min_beta f(X beta, y) + lambda2 ||beta||^2
 *                              s.t. ||beta||_inf <= M, ||beta||_0 <= k.
 * At a node N with fixings J0 (z = 0), J1 (z = 1) and free Jf, the library solves
 * the perspective relaxation (Eq. 3-4) in its composite form (Eq. 6)
 *     Phi(beta) = F(X beta) + 2 lambda2 g_N(beta)
 * with FISTA and the duality-gap restart of Sec. 3.4, and returns
 *     Psi(zeta) = -F*(-zeta) - G*(X' zeta)   (Eq. 7),  zeta = -grad F(X beta),
 * which is a valid lower bound for the node by weak duality.
 *
 * Losses (the paper's formulas are in its missing appendix; this library's reading):
 *   RELAX_LS:       F(z) = ||y - z||^2
 *   RELAX_LOGISTIC: F(z) = sum_i log(1 + exp(-y_i z_i)),  y_i in {-1, +1}
 *
 * Conventions shared by every entry point
 *  - Pointers marked "device" are CUDA device pointers owned by the caller
 *    (e.g. torch.Tensor.data_ptr()); the library never frees them.  Pointers
 *    marked "host" are ordinary host memory.
 *  - X is row-major with leading dimension ldx (elements), ldx >= p.
 *  - fixings: device int8[p], -1 = J0, 0 = free (Jf), +1 = J1; NULL = root node.
 *  - All device work is enqueued on the caller's stream (a cudaStream_t passed as
 *    void*; NULL = legacy default stream).  Entry points that return values in
 *    host memory synchronize that stream before returning.
 *  - Errors are returned as relax_status codes; nothing aborts or exits.  Invalid
 *    arguments (k < |J1|, k < 0, lambda2 <= 0, M <= 0, n or p <= 0, null required
 *    pointers) give RELAX_EINVAL and leave outputs untouched.
 *  - Device-side waits are bounded by options.watchdog_ms; on expiry the kernel
 *    records RELAX_ETIMEOUT and returns instead of spinning.
 */
#ifndef RELAX_H
#define RELAX_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct relax_handle relax_handle;

typedef enum { RELAX_LS = 0, RELAX_LOGISTIC = 1 } relax_loss;

typedef enum {
  RELAX_F64 = 0,     /* double */
  RELAX_F32 = 1,     /* float */
  RELAX_BF16 = 2,    /* bfloat16 storage of X (FP32's exponent range: no scales), FP32 accumulation */
  RELAX_FP8E4M3 = 3  /* fp8 e4m3 storage of X, per-column FP32 scales, FP32 accumulation */
} relax_dtype;

typedef enum {
  RELAX_OK = 0,
  RELAX_EINVAL = 1,          /* invalid argument */
  RELAX_ENOMEM = 2,          /* device allocation failed */
  RELAX_ECUDA = 3,           /* a CUDA runtime call failed */
  RELAX_ENOTCONV = 4,        /* max_iters reached before gap_tol (bounds still valid) */
  RELAX_ETIMEOUT = 5,        /* a bounded device-side wait expired */
  RELAX_ENUMERIC = 6,        /* NaN/Inf met in the data or the iterates */
  RELAX_EINVALID_BOUND = 7,  /* certified dual bound above certified primal beyond rounding */
  RELAX_ENOTSUP = 8          /* shape or option outside what this library supports */
} relax_status;

/* Solver options.  A zero-initialised struct means "all defaults". */
typedef struct {
  double M;            /* box bound of Eq. 1; 0 -> 2.0; +INFINITY allowed (no box) */
  double eta;          /* restart factor of Sec. 3.4; 0 -> e^3 */
  double lipschitz;    /* L of beta -> F(X beta); 0 -> Lanczos estimate at create */
  int32_t max_iters;   /* 0 -> 100000 */
  int32_t precision;   /* storage used for the in-loop X reads: 0 -> dtype of X;
                          RELAX_BF16 / RELAX_FP8E4M3 require X in RELAX_F32 and make the
                          handle keep a quantized copy that the loop reads; the FP64
                          certificate of each solve reads the FP32 X */
  int32_t watchdog_ms; /* bound on any device-side wait; 0 -> 4000 */
  int32_t no_certify;  /* 0 -> final FP64 evaluation of the bounds with the full X */
  int32_t chunk;       /* iterations enqueued per host poll; 0 -> 32 */
  int32_t timing;      /* 1 -> time every loop kernel with CUDA events on the handle's
                          stream (fills xpass_ms / pphase_ms of relax_result); the host
                          then waits for each chunk before enqueueing the next */
  int32_t stall_window; /* stall rule: the loop stops once its best duality gap has not
                          fallen by 10% over the last quarter of its iterations and over
                          at least this many; 0 -> 1000, < 0 -> off */
  /* The methods of the convergence study (Sec. 5.2).  Defaults: FISTA with
   * the duality-gap restart of Sec. 3.4 and the fixed step 1/L. */
  int32_t method;      /* 0 FISTA (Beck 2017 Sec. 10.7), 1 proximal gradient (Sec. 10.2) */
  int32_t restart;     /* FISTA only: 0 duality gap (Sec. 3.4), 1 function value
                          (restart when Phi rises, O'Donoghue and Candes), 2 none */
  int32_t step_rule;   /* 0 fixed 1/L; 1 backtracking (Beck Sec. 10.4.2): from L/64, L
                          doubles until F(X x) <= F(y) + <grad F(y), x - y> + L/2 ||x - y||^2
                          (+ 1e-12 |F(y)| for rounding); each retry costs one more
                          fused pass and p-phase, and L never decreases */
  int32_t reserved[2];
} relax_options;

typedef struct {
  double primal;       /* min Phi over the iterates (FP64-certified unless no_certify) */
  double dual_bound;   /* max Psi: valid lower bound for the node (FP64-certified) */
  double gap;          /* primal - dual_bound */
  double rel_gap;      /* gap / max(1, |primal|) */
  double primal_loop;  /* the same two values as tracked inside the loop, in the */
  double dual_loop;    /* working precision of X */
  double lipschitz;    /* L used (step = 1/L) */
  int32_t iters;       /* prox steps taken */
  int32_t restarts;    /* gap-based restarts */
  int32_t status;      /* relax_status of the solve */
  int32_t n_nz;        /* nonzeros of the returned beta */
  int32_t launches;    /* CUDA kernels this call launched (incl. no-op tail of a chunk) */
  int32_t xpass_count; /* fused X-passes on the loop's own stored X that did work (iters + 1
                          before any rung of the precision ladder) */
  double xpass_ms;     /* options.timing: summed device time of those X-passes */
  double pphase_ms;    /* options.timing: summed device time of their p-phase launches */
  int32_t stalled;     /* 1: the loop stopped on the stall rule (see stall_window) */
  int32_t polish_iters; /* relax_solve_batch: iterations of the single-node finish that a
                          node stalled in the batch received (0: none) */
  int32_t cutoff_rule; /* dynamic termination (relax_set_cutoff): 0 none, 1 the loop's Phi
                          fell to the cutoff (branch), 2 its Psi reached it (prune) */
  int32_t backtracks;  /* step_rule 1: rejected trial points (each doubled L); lipschitz
                          is then the final L */
  int32_t ladder;      /* relax_solve: rungs of the precision ladder taken after the loop's
                          own pass missed gap_tol on its arithmetic's floor (0: none; 1 the
                          FP32 master X after a BF16 / FP8 loop; 2 float-float products on
                          the master X).  Each rung restarts from beta_best; iters counts
                          every rung's iterations; dual_bound is the best over the rungs. */
} relax_result;

/* Create a solver handle bound to one design X and response y (Sec. 2.3).
 *   X: device, row-major n x ldx, element type `dtype` (RELAX_F64 or RELAX_F32);
 *      must stay alive and unchanged for the life of the handle.  Rows are read
 *      with 16-byte bulk copies; when ldx*sizeof(elem) or X is not 16-byte
 *      aligned the handle keeps an aligned internal copy.
 *   y: device, n elements of `dtype` (copied into the handle).
 *   k >= 1, lambda2 > 0; opt may be NULL (defaults).
 * Computes L = c_f ||X||_2^2 (c_f = 2 for LS, 1/4 for logistic) unless
 * opt->lipschitz > 0: the largest Ritz value of a Lanczos run on X'X (full
 * reorthogonalisation, deterministic reductions) plus a 1% margin.
 * Synchronizes `stream`. */
relax_status relax_create(relax_handle** h, const void* X, const void* y, int64_t n,
                          int64_t p, int64_t ldx, int32_t dtype, int32_t loss, int32_t k,
                          double lambda2, const relax_options* opt, void* stream);

/* Solve the node relaxation (Eq. 3-4) to gap_tol relative duality gap
 * ((Phi_best - Psi_best) / max(1, |Phi_best|)) with FISTA + gap restart (Sec. 3.4).
 *   fixings: device int8[p] or NULL (root).
 *   warm_start: device p elements of the handle's dtype or NULL (zero); any
 *      vector is accepted (outside dom g_N the reference gap is taken at the
 *      first iterate).
 *   beta_out: device p elements of the handle's dtype: the primal point with the
 *      smallest Phi seen.
 *   out: host; filled on every return path after argument validation, including
 *      RELAX_ENOTCONV / RELAX_ETIMEOUT (dual_bound stays a valid bound).
 * The loop stops when its own gap estimate reaches gap_tol (0.7 gap_tol when X
 * is FP32 or narrower, where that estimate is not FP64; a loop on BF16 / FP8
 * storage stops at 1e-3 / 1e-2, about its format's effect on the bound).  The
 * certificate then evaluates Phi at the best primal iterate and Psi at two
 * dual points (the loop's best one, and zeta = -grad F(X beta_best)) in one
 * pass over the full-precision X (FP64 for FP64 data, float-float for FP32
 * data) and keeps the better bound; it decides the status.  When it misses
 * gap_tol the loop resumes with a 4x tighter target for at most half as many
 * iterations again, at most 3 times and only while the certified gap keeps
 * shrinking.  When the loop's arithmetic is what stops it (the loop stalled,
 * or it read the BF16 / FP8 copy), the solve climbs the precision ladder
 * (relax_result.ladder): the loop goes on from beta_best on the FP32 X, then
 * with float-float products; a gap still above gap_tol after that is
 * reported through RELAX_ENOTCONV with a valid bound.
 * Synchronizes the handle's stream. */
relax_status relax_solve(relax_handle* h, const int8_t* fixings, const void* warm_start,
                         double gap_tol, void* beta_out, relax_result* out);

/* Solve nb node relaxations of the handle's design together: the batched
 * form of relax_solve for the nodes of one branch-and-bound tree, which all
 * share X (Sec. 2.3 node sets; FISTA with gap restart, Sec. 3.4, per node).
 *   fixings: device int8[nb][p] (row j: node j's J0/Jf/J1 as in relax_solve),
 *      or NULL (every node the root).
 *   warm_start: device [nb][p] of the handle's dtype, or NULL (zero).
 *   beta_out: device [nb][p] of the handle's dtype: each node's best primal point.
 *   out: host relax_result[nb], filled per node.
 * Per iteration the active nodes' points are the rows of a matrix B;
 * Z = X B' and G = X' R run as two products (FP32 X: the library's
 * tensor-core kernel on BF16 planes of X, X', B and R, FP32-accurate products
 * summed over K chunks in FP64; FP64 X: FP64 products), and each node's
 * prox / g / g* / gap / restart step runs in its own segment of one launch.
 * Nodes converge after uneven iteration counts and leave the batch every 16
 * iterations (each round of 16 is one CUDA graph per active-set size); the
 * stall rule's window is at most 200 inside a batch, and a node that stalls
 * above gap_tol is finished by relax_solve's loop from its best point
 * (out[j].polish_iters).  The first batched call of a FP32 handle builds the
 * BF16 planes of X and X' (six bytes per element of X each) and times a few
 * K-chunk choices per product, keeping the fastest for the handle.  Each node's bound is
 * certified in FP64 as in relax_solve (without resuming).  Needs FP32 or
 * FP64 storage of X (RELAX_ENOTSUP for BF16/FP8).  Returns RELAX_OK when every
 * node certified gap_tol, else the first failing node's status (out[j].status
 * holds each node's).  Synchronizes the handle's stream. */
relax_status relax_solve_batch(relax_handle* h, int32_t nb, const int8_t* fixings,
                               const void* warm_start, double gap_tol, void* beta_out,
                               relax_result* out);

/* The two products of a batched iteration on their own, with the identity
 * link: for nb points b_s (the rows of `points`), z_s = X b_s and
 * g_s = X' z_s, i.e. the operator X'X of the power iteration, through exactly
 * the kernels relax_solve_batch uses (the matrix-vector products that
 * dominate the method, Sec. 5.2; stacked as matrix products for many nodes).
 *   points: device [nb][p] of the handle's dtype.
 *   z_out: device double [nb][n]; g_out: device double [nb][p].
 * FP32 X: tensor-core products on BF16 planes (FP32-accurate products, FP64
 * sums of the K chunks); FP64 X: FP64 products.  Needs FP32 or FP64 storage
 * (RELAX_ENOTSUP otherwise).
 *   products_ms: host double[2] or NULL: FP32 X, the device time of the two
 *      tensor-core launches (z, then g), from CUDA events on the handle's stream.
 * Synchronizes the handle's stream. */
relax_status relax_batch_xpass(relax_handle* h, int32_t nb, const void* points, double* z_out,
                               double* g_out, double* products_ms);

/* Dynamic termination of Sec. 5.3 for the handle's later solves (single and
 * batched): with cutoff = f(X b) + lambda2 ||b||^2 of the incumbent b, a
 * node's loop stops as soon as its Phi falls to the cutoff (the node will be
 * branched: result.cutoff_rule = 1) or its Psi reaches it (the node can be
 * pruned: cutoff_rule = 2).  Such a solve is RELAX_OK whatever its gap; the
 * certified bound is valid as always.  cutoff = +inf turns it off (the
 * default); NaN is RELAX_EINVAL. */
relax_status relax_set_cutoff(relax_handle* h, double cutoff);

/* Diagnostic of the failure detection: one block takes the library's grid
 * barrier expecting a partner that never arrives, so its bounded wait must
 * give up after watchdog_ms (1..60000) and record a timeout, as every device
 * wait of the library does when its bound expires.  Returns RELAX_ETIMEOUT
 * when it did, with the wait's device time in *waited_ms (host double, or
 * NULL).  No GPU fault, no copy in flight; the context stays usable.
 * Synchronizes `stream`. */
relax_status relax_watchdog_probe(int32_t watchdog_ms, double* waited_ms, void* stream);

/* One fused pass over X (the matrix-vector products of Sec. 5.2.3 that dominate
 * the method): z = X beta, r = grad F(z), g = X' r, read of X once.
 *   beta: device p (handle dtype), z_out: device n (handle dtype),
 *   g_out: device p (handle dtype), loss_host: host double[2] or NULL:
 *   {F(z), -F*(r)} i.e. the primal loss and the loss part of Psi at zeta = -r.
 * Synchronizes the handle's stream. */
relax_status relax_xpass(relax_handle* h, const void* beta, void* z_out, void* g_out,
                         double* loss_host);

/* FP64-grade evaluation of Phi(beta_primal) (Eq. 6) and Psi(zeta) (Eq. 7) at
 * zeta = -grad F(X beta_dual), with the full-precision X (certification:
 * FP64 passes for FP64 data, float-float products and sums for FP32 data).
 *   beta_primal, beta_dual: device p (handle dtype); fixings as in relax_solve.
 *   The same pointer for both points takes one product of X instead of two.
 *   out_host: host double[2] = {Phi, Psi}.  Phi is +inf when beta_primal is
 *   outside dom g_N.  Synchronizes the handle's stream. */
relax_status relax_certify(relax_handle* h, const int8_t* fixings, const void* beta_primal,
                           const void* beta_dual, double* out_host);

/* relax_certify for nb points at once (the learned warm start's fallback
 * test in a batched BnB): out_host[2 s], out_host[2 s + 1] = {Phi(b_s),
 * Psi(-grad F(X b_s))} for the rows b_s of points.
 *   points: device nb x p (handle dtype), row-major; fixings: device nb x p
 *   int8 (row s for point s) or NULL; out_host: host double[2 nb].
 * The passes of every point are enqueued back to back and the stream is
 * synchronized once.  RELAX_EINVAL for a row of fixings with more than k
 * coordinates in J1 or a value outside {-1, 0, 1}. */
relax_status relax_certify_batch(relax_handle* h, int32_t nb, const int8_t* fixings, const void* points,
                                 double* out_host);

/* Release the handle and everything it allocated (not X, y, or caller buffers). */
relax_status relax_destroy(relax_handle* h);

/* prox of rho*g_N with rho = 2*lambda2*step (Algorithm 2 + Eq. prox:gN, Thm 4.5):
 *   beta_out = argmin_u 0.5||u - beta_in||^2 + rho g_N(u).
 *   beta_in, beta_out: device p elements of dtype (RELAX_F64 or RELAX_F32); may alias.
 *   counts_out: device int32[2] or NULL: {n_top, n_nz} = free coordinates with
 *      z_j = 1 (placed before the pooled block of Algorithm 2) and nonzero free
 *      outputs.
 * Uses stream-ordered scratch (cudaMallocAsync) on `stream`; does not synchronize,
 * so a failure inside the kernel cannot change the returned status.  It shows
 * in the outputs instead: a NaN or Inf in beta_in, or a bounded device wait
 * that expired, makes beta_out all NaN (every coordinate the failing blocks
 * own, all of them for a non-finite input) and counts_out {-1, -1}. */
relax_status prox_persp(const void* beta_in, void* beta_out, int64_t p, double step,
                        int32_t k, double lambda2, double M, const int8_t* fixings,
                        int32_t dtype, int32_t* counts_out, void* stream);

/* prox_persp without any allocation.  The paper has no counterpart: this is a
 * library convenience.  Some callers cannot allocate device memory while they
 * work: a solver embedded in a framework whose memory pool owns the whole GPU,
 * or a node loop with a hard latency budget where an allocator call may block,
 * synchronize or fail.  This call computes exactly what prox_persp computes
 * (same arguments, layouts and results) but takes its scratch from one
 * 64 KiB array in device memory that every GPU which loads the library holds
 * until the process exits; it calls no allocation routine.
 *   Limit: p must need at most 64 KiB of scratch (3 * 256 * 8 bytes of
 *   accumulators + 160 bytes per block of the launch, which admits every
 *   p <= 189440 for either dtype).  Beyond it: RELAX_ENOTSUP, with the sizes in
 *   relax_error_detail(), and nothing is launched.
 *   The first call on a device looks up the array's device address
 *   (cudaGetSymbolAddress) with that device current; make that first call
 *   before any stream capture.
 *   Every call shares the one array and leaves its contents behind (each call
 *   zeroes what it needs at its start): calls that overlap on the GPU, e.g. on
 *   two streams without ordering between them, race and give wrong results.
 *   Does not synchronize; failures inside the kernel show in the outputs as
 *   for prox_persp (NaN in beta_out, counts_out {-1, -1}), since the next call
 *   clears the array's status word. */
relax_status prox_persp_noalloc(const void* beta_in, void* beta_out, int64_t p, double step,
                                int32_t k, double lambda2, double M, const int8_t* fixings,
                                int32_t dtype, int32_t* counts_out, void* stream);

/* g_N(beta) (Eq. 5; value of Algorithm 1 / Thm 4.4) into out_host[0]; +inf when
 * beta is outside dom g_N: a J0 coordinate nonzero, |beta_j| > M (1 + 1e-6), or
 * sum_Jf |beta_j| > M kbar (1 + 1e-6) (the relative slack admits boundary points
 * rounded to FP32 or FP64).
 *   beta: device p of dtype.  Synchronizes `stream`. */
relax_status gval_persp(const void* beta, int64_t p, int32_t k, double M,
                        const int8_t* fixings, int32_t dtype, double* out_host,
                        void* stream);

/* g_N*(alpha) = sum_J1 H_M(alpha_j) + TopSum_{k-|J1|} H_M(alpha_Jf)  (Lemma 4.2)
 * into out_host[0].  alpha: device p of dtype.  Synchronizes `stream`. */
relax_status gstar_persp(const void* alpha, int64_t p, int32_t k, double M,
                         const int8_t* fixings, int32_t dtype, double* out_host,
                         void* stream);

/* Static, human-readable message for a status code. */
const char* relax_strerror(relax_status s);

/* Thread-local description of the last failing CUDA runtime call made by this
 * library in the calling thread (empty when none); valid until the next call. */
const char* relax_error_detail(void);

#ifdef __cplusplus
}
#endif

#endif /* RELAX_H */
