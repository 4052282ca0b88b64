/*
 * ttutv.h -- C ABI of the GB300 (sm_103a) TT-UTV library.
 *
 * Implements the tensor-train decompositions of "Effective algorithms for
 * tensor-train decomposition via the UTV framework" (arXiv 2501.07904):
 * TT-URV right-to-left (Alg. 3 and its prescribed-accuracy analogue,
 * Sec. 3.2), TT-ULV left-to-right (Alg. 1 and Alg. 2, Sec. 3.1), and TT-SVD
 * (the paper's comparison method, Sec. 4), plus contraction of a TT back to a
 * full tensor (Eq. TT), orthogonalization of TT cores (Def. 2.2), and masked
 * evaluation of a TT with its gradient and the tangent-space projection of
 * the Riemannian gradient (the observation operator P_Omega and the solver
 * of the completion experiment, Sec. 4.2.2).
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 * - Tensors and cores are dense, row-major (C order; the last index is
 *   fastest).  Core k is an array [r_{k-1}][I_k][r_k] with r_0 = r_d = 1.
 *   Row-major order permutes the rows and columns of every unfolding
 *   (Def. 2.1) relative to the paper's reverse-lexicographic ivec; ranks,
 *   truncation errors and the represented tensor are unchanged.
 * - "device" pointers are CUDA global memory of the current device; "host"
 *   pointers are ordinary (preferably pinned) host memory.
 * - `stream` is a cudaStream_t passed as void* (NULL = legacy default stream).
 *   All work is enqueued on it.  tt_utv / tt_svd synchronize that stream
 *   once per sweep step to read the chosen rank (the next step's shapes
 *   depend on it), and tt_eval_plan_create (and the one-shot masked
 *   evaluations built on it) once to read its index check; the other calls
 *   are asynchronous.
 * - Every function returns a tt_status; on failure tt_last_error() returns a
 *   thread-local message.  No function aborts or traps.
 */
#ifndef TTUTV_H
#define TTUTV_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define TT_MAXD 16

typedef enum {
  TT_OK = 0,
  TT_EINVAL = 1,        /* bad argument: d < 2, a dim <= 0, eps <= 0, rank < 1, NULL pointer */
  TT_ENONFINITE = 2,    /* the input holds a NaN or an Inf (||A||_F^2 is not finite) */
  TT_ENOMEM = 3,        /* the allocator returned NULL */
  TT_ECUDA = 4,         /* a CUDA runtime call failed (message has the CUDA error) */
  TT_ENOCONV = 5,       /* Jacobi (TT-SVD) did not converge within its sweep cap */
  TT_ETIMEOUT = 6,      /* a bounded wait inside a tensor-core kernel ran out (2 s); the
                           kernel unwound and released its resources, the context stays usable */
  TT_EUNSUPPORTED = 7   /* valid request outside what the library implements */
} tt_status;

typedef enum { TT_F32 = 0, TT_F64 = 1 } tt_dtype;
typedef enum { TT_URV = 0, TT_ULV = 1 } tt_variant;
typedef enum { TT_RL = 0, TT_LR = 1 } tt_direction;

/* Arithmetic of the sweep.
 *  TT_P_FP64 : everything in FP64 (an FP32 input is widened first).
 *  TT_P_FP32 : FP32 data and FFMA products; FP64 for every cross-block sum,
 *              Gram matrix, norm and truncation-error accumulation.
 *  TT_P_MIXED: FP32 data, products on the tcgen05 tensor cores with FP32
 *              accumulation.  The Gram matrix of an exact step (the one
 *              product that only ranks directions) rounds its operands to
 *              TF32; every other product carries each FP32 operand as two
 *              TF32 terms (~2^-22 relative), so the sketch, Cholesky-QR,
 *              projection, carry and core match the FP32 form to within a
 *              few 1e-6.  Tight steps (see TT_SMALL_AUTO) find their range
 *              (Grams, sketch, projection) on the FP32 SIMT path and form
 *              carry and core on the tensor cores; products whose leading
 *              dimensions are not multiples of 4 run on the SIMT path. */
typedef enum { TT_P_FP64 = 0, TT_P_FP32 = 1, TT_P_MIXED = 2 } tt_precision;

/* Arithmetic of the small (<= 256 x 256) factorizations:
 *  TT_SMALL_AUTO picks FP32 when eps^2 w_k^2 >= 2 n u_fp32 (the Gram-based
 *  truncation error is then resolved with margin) or the ranks are fixed,
 *  FP64 otherwise; TT_SMALL_FP32 / TT_SMALL_FP64 force one.  TT_SMALL_DF
 *  (FP32 data only) takes the FP64 choices everywhere but runs factors of
 *  n <= 64 in double-float arithmetic (an FP32 pair, ~2^-48 unit roundoff,
 *  at FP32 instruction rates; GB300 issues FP64 at 1/64 of them); larger
 *  factors stay FP64. */
typedef enum {
  TT_SMALL_AUTO = 0,
  TT_SMALL_FP32 = 1,
  TT_SMALL_FP64 = 2,
  TT_SMALL_DF = 3
} tt_small_precision;

/* Phases timed when tt_opts.phase_ms is set (device time from CUDA events
 * recorded on the sweep's stream). */
typedef enum {
  TT_PH_GRAM = 0,     /* exact path: Gram of the basis side */
  TT_PH_SMALL = 1,    /* small factorization (QLP / Jacobi) */
  TT_PH_CARRY = 2,    /* carry product (the next unfolding) */
  TT_PH_CORE = 3,     /* core formation */
  TT_PH_SKETCH = 4,   /* sketch matrix and Y = C^T Omega / C Omega */
  TT_PH_ORTH = 5,     /* Cholesky-QR3 of Y */
  TT_PH_PROJECT = 6,  /* B = C W / C^T W and its Gram */
  TT_NPHASES = 8
} tt_phase;

typedef struct {
  int32_t precision;        /* tt_precision, default TT_P_FP32 */
  int32_t small_precision;  /* tt_small_precision, default TT_SMALL_AUTO */
  int32_t oversample;       /* sketch oversampling p, default 16 */
  int32_t l_full;           /* basis side <= l_full columns -> exact Gram path, default 256 (max 256) */
  uint64_t seed;            /* Philox key of the Rademacher sketch, default 0 */
  const double* weights;    /* host, d-1 error weights w_k with sum w_k^2 = 1; NULL = equal 1/sqrt(d-1) */
  int32_t orth_precision;   /* tt_small_precision of the Cholesky-QR passes of a sketched step;
                               default TT_SMALL_AUTO = FP64 for FP64 data or a tight step, else FP32 */
  int32_t reverse;          /* 1: factor the index-reversed tensor A'(i_d..i_1) = A(i_1..i_d) and
                               read its cores back as cores of A (Remark after Thm 3.2): TT-URV
                               right-to-left then gives left-orthogonal cores of A, TT-ULV
                               left-to-right right-orthogonal ones.  Costs one device copy of A
                               (reversed in a tiled transposition kernel).  Weights, fixed ranks
                               and every per-unfolding result refer to the unfoldings of A.
                               Default 0. */
  double* phase_ms;         /* host, TT_MAXD * TT_NPHASES doubles [sweep step][tt_phase], or NULL.
                               Milliseconds of device time are ADDED to it; the sweep step index is
                               0 for the first factored unfolding. */
  int32_t power_iters;      /* q in [0, 8]: power (subspace) iterations of a sketched step's range,
                               Y <- X^T X Q with Q an orthonormal basis of the previous Y (the
                               randomized range finder behind randUTV, Sec. 2.2); no effect when
                               Omega = I.  Default 0. */
  int32_t inner;            /* tt_inner: the small rank-revealing factor of tt_utv, default
                               TT_INNER_QLP; ignored by tt_svd */
  int32_t usvp_iters;       /* TT_INNER_USVP, TT_INNER_LURV: power iterations per basis vector,
                               in [0, 64], default 8 */
  int32_t lhat;             /* tt_lhat: the kept middle block of TT-ULV right-to-left (the
                               appendix's Alg. 4), default TT_LHAT_FULL */
  int32_t direct_tails;     /* 0 or 1 (default 0).  1: every step that would report
                               ||C||^2 - ||carry||^2 (exact or sketched, tolerance not tight, not
                               an identity sketch) reports instead its error ||E_k||_F^2 (the
                               summands of Thm 3.1's equality) summed directly from the residual
                               E_k = C - carry Z_1^T (TT-URV; TT-ULV: C - Z_1 carry), formed slab
                               by slab of C's rows and summed in FP64: one more pass over the
                               unfolding and a product per slab.  The difference of two squared
                               norms carries the products' rounding (~1e-6 of ||C||^2 on the
                               tensor cores), the size of a sketched step's range miss.  Ranks
                               and cores are unchanged; ignored with TT_LHAT_L11. */
} tt_opts;

/* Middle block kept by TT-ULV right-to-left (appendix, Alg. 4), whose inner
 * factor is the ULV form C ~ U L V^T of the pivoted QLP:
 *  TT_LHAT_FULL : [L_11; L_21]: carry U L(:, 1:r) = C V_1, residual
 *                 U_2 L_22 V_2^T orthogonal to V_1 (the bounds of Thm 3.1);
 *                 computes exactly the TT-URV right-to-left sweep.
 *  TT_LHAT_L11  : L_11 alone (Alg. 4 as printed): carry U_1 L_11, step error
 *                 mu^2 + ||L||_F^2 - ||L_11||_F^2, errors adding in norm (the
 *                 appendix's Proposition: ||A - A_hat|| <= sum_k eps_k), so the
 *                 default weights are w_k = 1/(d-1) and given weights must sum
 *                 to 1.  Only with TT_ULV, TT_RL and TT_INNER_QLP (else
 *                 TT_EINVAL); its small factors run on the generic kernel. */
typedef enum { TT_LHAT_FULL = 0, TT_LHAT_L11 = 1 } tt_lhat;

/* Inner factor of each tt_utv step, applied to the Gram matrix of the basis
 * side (or of the range-projected matrix on a sketched step):
 *  TT_INNER_QLP  : Stewart's pivoted QLP (the default, see tt_utv);
 *  TT_INNER_USVP : USV-plus-style deflation (the rank-revealing decomposition
 *                  the paper runs inside TT-ULV in Sec. 4, with its stopping
 *                  rule adapted to fixed ranks and to Alg. 2): basis vectors
 *                  one at a time, each started from the column of largest norm
 *                  of the deflated matrix D = X (I - V V^T) and refined by
 *                  usvp_iters power iterations on D^T D, re-orthogonalized
 *                  twice against the basis; the error of keeping i vectors is
 *                  ||X - X V_i V_i^T||_F^2 (plus the sketch's range miss); the
 *                  rank is fixed or the first i with error <= eps_k^2.  One CTA,
 *                  sequential in the rank: slower than the QLP.
 *  TT_INNER_LURV : low-rank revealing URV with Givens rotations (the
 *                  Fierro-Hansen family the paper runs inside TT-URV in Sec. 4),
 *                  warm-started from the column-pivoted QR X Pi = Q R (V = Pi):
 *                  for i = 0, 1, ... the dominant right singular vector of the
 *                  trailing block R(i:, i:) is estimated (its column of largest
 *                  norm, then usvp_iters power iterations), rotated onto e_i by
 *                  Givens rotations on adjacent columns of R and V, and the fill
 *                  below the diagonal removed by rotations of adjacent rows; the
 *                  error of keeping i vectors is ||R(:, i:)||_F^2 (plus the
 *                  sketch's range miss); the rank is fixed or the first i with
 *                  error <= eps_k^2.  One CTA, sequential in the rank. */
typedef enum { TT_INNER_QLP = 0, TT_INNER_USVP = 1, TT_INNER_LURV = 2 } tt_inner;

/* Fill *o with the defaults listed above. */
void tt_opts_default(tt_opts* o);

/* Caller-supplied stream-ordered allocator (e.g. PyTorch's caching
 * allocator).  alloc returns device memory of at least `bytes` bytes usable
 * on `stream`, or NULL; free releases it after the work already enqueued on
 * `stream`.  Passing NULL for both selects cudaMallocAsync / cudaFreeAsync. */
typedef void* (*tt_alloc_fn)(size_t bytes, void* stream, void* ctx);
typedef void (*tt_free_fn)(void* ptr, void* stream, void* ctx);

/* Result of a sweep.  Filled by tt_utv / tt_svd; cores are device memory
 * obtained from the caller's allocator, released by tt_result_free (or by
 * the caller directly, core by core, through its own allocator). */
typedef struct {
  int32_t d;
  int32_t dtype;                 /* tt_dtype of the cores */
  int32_t orth;                  /* 0 = right-orthogonal cores 2..d (RL), 1 = left-orthogonal 1..d-1 (LR) */
  int32_t pad_;
  int64_t dims[TT_MAXD];
  int64_t ranks[TT_MAXD + 1];    /* r_0 .. r_d, r_0 = r_d = 1 */
  void* cores[TT_MAXD];          /* device, row-major [r_{k-1}][I_k][r_k] */
  double norm_sq;                /* ||A||_F^2 (FP64) */
  double tail_sq[TT_MAXD];       /* per unfolding k = 1..d-1 (index k-1): ||E_k||_F^2 of its truncation:
                                    for a tight step the small factor's estimate (compensated Gram,
                                    FP64 factorization), otherwise ||C_k||^2 - ||carry||^2 summed in
                                    FP64 over the stored values (FP32 data: accurate to a few
                                    n u_fp32 ||C_k||^2) */
  double delta_sq[TT_MAXD];      /* per unfolding: the tolerance eps_k^2 (0 for fixed ranks) */
  int32_t sketch_l[TT_MAXD];     /* per unfolding: 0 = exact Gram path, else sketch width l */
  int32_t small_fp64[TT_MAXD];   /* per unfolding: 1 if its small factor ran in FP64 */
} tt_result;

/* TT-UTV decomposition (Sec. 3).
 *   A          device, prod(dims) elements of `dtype`, row-major.
 *   d, dims    order 2 <= d <= TT_MAXD and mode sizes I_1..I_d (host).
 *   eps        prescribed relative accuracy (Alg. 2): each unfolding k is cut
 *              at the smallest rank with ||E_k||_F <= w_k eps ||A||_F, which
 *              by Cor. 3.1 / Thm 3.2 gives ||A - A_hat||_F <= eps ||A||_F.
 *              Ignored when fixed_ranks != NULL.
 *   fixed_ranks host, d-1 ranks r_1..r_{d-1} (Alg. 1 / Alg. 3), or NULL.  A
 *              rank above the size of its unfolding is clamped; the ranks
 *              actually used are returned.
 *   variant/direction  TT_URV with TT_RL (Alg. 3) or TT_ULV with TT_LR
 *              (Alg. 1/2).  TT_ULV with TT_RL is the appendix's Alg. 4 with
 *              the middle block [L_11; L_21] kept (its first case, for which
 *              the bounds of Thm 3.1 / Cor. 3.1 hold); with the pivoted-QLP
 *              inner factor it computes exactly the TT_URV / TT_RL sweep, and
 *              TT_URV with TT_LR ([R_11 R_12] kept) exactly the TT_ULV / TT_LR
 *              one.  Alg. 4's L_11-only carry: tt_opts.lhat.
 *   opts       host, may be NULL (defaults).
 * Each unfolding step: if the basis side (columns for URV, rows for ULV) has
 * at most l_full entries, its Gram matrix is factored exactly; otherwise a
 * Rademacher sketch of width l (grown if the rank needs it) gives an
 * orthonormal range basis first.  The small factor is Stewart's pivoted QLP
 * (a rank-revealing UTV, Sec. 2.2) of the projected matrix.
 * out receives cores, ranks and per-step truncation errors. */
tt_status tt_utv(const void* A, int32_t dtype, int32_t d, const int64_t* dims, double eps,
                 const int64_t* fixed_ranks, int32_t variant, int32_t direction,
                 const tt_opts* opts, tt_alloc_fn alloc, tt_free_fn free_fn, void* alloc_ctx,
                 void* stream, tt_result* out);

/* One tensor decomposed by P processes (one GPU each), every process holding
 * an equal slab of one mode: mode 1 for the right-to-left sweep (TT-URV,
 * Alg. 3), whose unfoldings C_k = [I_1..I_{k-1}, I_k r_k] keep i_1 as their
 * slowest row index, and mode d for the left-to-right sweep (TT-ULV, Alg. 1/2),
 * whose unfoldings keep i_d as their fastest column index (Def. 2.1) -- so
 * every carry stays within its slab.  Per step the Gram matrix (exact path)
 * or the sketch, the projection's Gram B^T B and the squared norms are
 * partial sums over the slabs, summed over ranks by `allreduce` (FP64, in
 * place); the small factorizations then run identically on every rank, the
 * sketch rows a slab draws are those of its own rows of the whole unfolding,
 * and the carries stay local.  A step whose sketch is the identity gathers
 * its whole unfolding by `allgather` and the rest of the sweep runs on every
 * rank alike; the partitioned last core is gathered.  Every rank returns the
 * same ranks, errors and (whole) cores, equal to tt_utv of the whole tensor
 * up to the summation order of the partial sums. */

/* Sum of `count` doubles of device memory over all ranks, in place.  Every
 * rank makes the same calls in the same order.  The work that produces buf
 * is already enqueued on `stream`; the callee orders its communication after
 * it and the library's later work after the result (e.g. a NCCL all-reduce
 * on that stream, or a synchronize, a host-staged sum and a copy back).
 * Returns 0 or a tt_status. */
typedef int32_t (*tt_allreduce_fn)(double* buf, int64_t count, void* stream, void* ctx);
/* Concatenation in rank order: every rank contributes `bytes` bytes of
 * device memory from send; recv (nranks * bytes) receives rank 0's block
 * first.  Same ordering rules as tt_allreduce_fn. */
typedef int32_t (*tt_allgather_fn)(const void* send, void* recv, int64_t bytes, void* stream,
                                   void* ctx);

typedef struct {
  int32_t nranks;             /* P >= 1 (1: no partition, tt_utv) */
  int32_t rank;               /* this process, 0 .. P-1; its slab is rank * I_p / P .. */
  tt_allreduce_fn allreduce;  /* required when P > 1 */
  tt_allgather_fn allgather;  /* required when P > 1 */
  void* ctx;                  /* passed to both */
} tt_shard;

/* tt_utv over a partitioned tensor.
 *   A_local  device (or host), this rank's slab: dims with mode 1 (TT_RL) or
 *            mode d (TT_LR) replaced by dims[p] / P, row-major
 *   dims     the WHOLE tensor's mode sizes; dims[p] must be a multiple of P
 *   the rest as tt_utv (TT_URV/TT_RL or TT_ULV/TT_LR and their Alg. 4
 *   pairings); opts->reverse and TT-SVD return TT_EUNSUPPORTED.
 * Every rank receives the whole result in *out. */
tt_status tt_utv_sharded(const void* A_local, int32_t dtype, int32_t d, const int64_t* dims,
                         double eps, const int64_t* fixed_ranks, int32_t variant, int32_t direction,
                         const tt_opts* opts, tt_alloc_fn alloc, tt_free_fn free_fn, void* alloc_ctx,
                         void* stream, const tt_shard* shard, tt_result* out);

/* TT-SVD (the comparison method of Sec. 4) through the same sweep: the small
 * factor is a Jacobi eigen-decomposition of the Gram matrix, so the kept
 * basis is the leading singular subspace and ||E_k||^2 = sum of the dropped
 * sigma_i^2.  direction TT_LR (left-orthogonal, as in the paper) or TT_RL.
 * A step whose basis side exceeds l_full takes the sweep's sketch: the
 * Jacobi SVD is then that of the projection C P_W onto the Rademacher
 * sketch's range (the identity when the other side is at most 256), the
 * range miss ||C||^2 - ||C P_W||^2 is part of ||E_k||^2, and the sketch is
 * widened (up to 256 columns) until the kept rank leaves the oversampling
 * margin and the tail meets the tolerance; beyond that, TT_EUNSUPPORTED. */
tt_status tt_svd(const void* A, int32_t dtype, int32_t d, const int64_t* dims, double eps,
                 const int64_t* fixed_ranks, int32_t direction, const tt_opts* opts,
                 tt_alloc_fn alloc, tt_free_fn free_fn, void* alloc_ctx, void* stream,
                 tt_result* out);

/* Release the cores of *r through free_fn (NULL = cudaFreeAsync) and zero it. */
void tt_result_free(tt_result* r, tt_free_fn free_fn, void* alloc_ctx, void* stream);

/* Contract TT cores into the full tensor (Eq. TT).
 *   d, dims, ranks  host (ranks has d+1 entries, r_0 = r_d = 1);
 *   cores           host array of d device pointers, each [r_{k-1}][I_k][r_k] of `dtype`;
 *   out             device, prod(dims) elements of `dtype` (caller-allocated);
 *   work            device scratch of at least tt_full_work_bytes(...) bytes. */
size_t tt_full_work_bytes(int32_t d, const int64_t* dims, const int64_t* ranks, int32_t dtype);
tt_status tt_full(int32_t d, const int64_t* dims, const int64_t* ranks, const void* const* cores,
                  int32_t dtype, void* out, void* work, void* stream);

/* Orthogonalize TT cores (Def. 2.2): the same tensor with left-orthogonal
 * cores 1..d-1 (side = 1: each left unfolding [r_{k-1} I_k] x [r_k] has
 * orthonormal columns, core d carries the norm) or right-orthogonal cores
 * 2..d (side = 0: each right unfolding [r_{k-1}] x [I_k r_k] has orthonormal
 * rows, core 1 carries the norm), the frames of the tangent space in which
 * the Riemannian gradient of Sec. 4.2.2 is written.  Left: for k = 1..d-1 the
 * unfolding of R_{k-1} G_k (R_0 = 1) is factored by Cholesky-QR2 with FP64
 * Gram matrices, Q_k R_k, Q_k becomes core k and R_k = Q_k^T (R_{k-1} G_k) is
 * multiplied into core k+1; right: mirrored from core d down to 2.  The two
 * passes leave the columns orthonormal to the data's rounding when each
 * unfolding's condition number is below ~1e6 (the first pass's Gram is shifted
 * by 4 r u_64 of its trace, so a numerically rank-deficient unfolding still
 * factors, with columns that are then orthonormal only to ~1e-8).
 *   d, dims, ranks  host; ranks r_0 = r_d = 1, each r_k <= 256, and
 *                   r_k <= r_{k-1} I_k (left) / r_{k-1} <= I_k r_k (right),
 *                   else TT_EINVAL;
 *   cores           host array of d device pointers [r_{k-1}][I_k][r_k] of `dtype`;
 *   out             host array of d device pointers of the same shapes, none of
 *                   them one of the input cores (TT_EINVAL);
 *   work            device scratch of tt_orthogonalize_work_bytes(...) bytes.
 * Asynchronous on `stream`; a NaN in the input gives NaN cores (not checked). */
size_t tt_orthogonalize_work_bytes(int32_t d, const int64_t* dims, const int64_t* ranks,
                                   int32_t dtype);
tt_status tt_orthogonalize(int32_t d, const int64_t* dims, const int64_t* ranks,
                           const void* const* cores, int32_t dtype, int32_t side, void* const* out,
                           void* work, void* stream);

/* tt_full without any device allocation, for callers that cannot allocate
 * device memory during the call: code running with every byte of device
 * memory already owned by another allocator's pool, or a latency-critical
 * loop that must not hit cudaMalloc's implicit device synchronization.  (The
 * paper has no counterpart; this is a service of the library.)
 * Same arguments and result as tt_full, without `work`: the scratch is a
 * fixed array of tt_full_noalloc_max_work_bytes() = 32 MiB of static device
 * memory.  A contraction needing more (tt_full_work_bytes) returns TT_EINVAL.
 * The array is reserved on a device when the CUDA runtime first loads the
 * module that holds it there -- under the default lazy module loading, at the
 * first tt_full_noalloc call on that device -- and stays reserved until the
 * process exits.  That first call also looks up the array's device address
 * (with the device current) and caches it, so it may allocate and
 * synchronize: make it before another allocator's pool takes the device's
 * memory and before any stream capture on the device.  Later calls allocate
 * nothing.  All calls share the one array and nothing in it needs to start at
 * zero, but two calls whose work overlaps on the GPU (other streams, other
 * host threads) race on it: serialize them. */
size_t tt_full_noalloc_max_work_bytes(void);
tt_status tt_full_noalloc(int32_t d, const int64_t* dims, const int64_t* ranks,
                          const void* const* cores, int32_t dtype, void* out, void* stream);

/* Reconstruction error of a TT against a full tensor, streamed: the TT is
 * contracted one slab of the first mode at a time into scratch (as tt_full
 * does) and compared with the matching slab of A, so the full TT tensor is
 * never formed.  The relative error of Sec. 4 (RSE) is sqrt(out[0] / out[1]).
 *   d, dims, ranks, cores, dtype  as for tt_full (cores device, [r_{k-1}][I_k][r_k]);
 *   A      device, prod(dims) elements of `dtype`, row-major;
 *   work   device scratch of at least tt_rse_work_bytes(...) bytes (a slab of
 *          at most 2^24 entries, or one slice of the first mode if larger,
 *          plus the contraction's scratch);
 *   out    device double[2]: out[0] = ||A - A_TT||_F^2, out[1] = ||A||_F^2,
 *          both summed in FP64 in a fixed order (deterministic).
 * Asynchronous on `stream`. */
size_t tt_rse_work_bytes(int32_t d, const int64_t* dims, const int64_t* ranks, int32_t dtype);
tt_status tt_rse(int32_t d, const int64_t* dims, const int64_t* ranks, const void* const* cores,
                 int32_t dtype, const void* A, void* work, double* out, void* stream);

/* Masked TT evaluation (the observation operator P_Omega of the completion
 * experiment, Sec. 4.2.2): x_e = G_1[i_1] G_2[:, i_2, :] ... G_d[:, i_d] at n
 * row-major linear indices idx[e] of a tensor of shape dims, and the core
 * gradients of sum_e gout_e x_e,
 *   dG_k[:, i_k, :] += gout_e (G_1[i_1]..G_{k-1}[i_{k-1}])^T (G_{k+1}[i_{k+1}]..G_d[i_d])^T,
 * the left and right interface products recomputed per entry (nothing is
 * stored between calls).  FP32 cores, values and gradients; d in [1, 16],
 * ranks in [1, 64] with r_0 = r_d = 1, dims in [1, 2^31), n in [0, 2^31).
 *
 * A plan holds what depends only on the index set: the decoded mode indices
 * and, for every core, the entries ordered stably by that core's index (ties
 * by a neighbouring core's).  Device bytes: 8 d n (indices and orders),
 * 5 d ceil(n/128) (chunk flags and slice ends), 2 ceil(n/128)
 * max_k(round4(r_{k-1}) round4(r_k)) * 4 (per-chunk gradient partials),
 * 4 n + 4 * 256 ceil(n/2048) (sort scratch).
 *
 * Gradients are summed in a fixed order with no floating-point atomics: a
 * plan gives bitwise-equal results on every call (and two plans built from
 * the same idx give the same results).  One call at a time per plan (the
 * backward writes the plan's partials): calls on one stream are ordered. */
typedef struct tt_eval_plan tt_eval_plan;

/* Build a plan for idx (device int64[n]).  Device memory comes from `alloc`
 * (or cudaMallocAsync on `stream` when alloc and free_fn are both NULL) and
 * goes back through free_fn in tt_eval_plan_destroy.  Synchronizes `stream`
 * once to read the index check: an index outside [0, prod(dims)) returns
 * TT_EINVAL (the kernels read no core memory for it) and no plan.  *out is
 * a host handle. */
tt_status tt_eval_plan_create(int32_t d, const int64_t* dims, const int64_t* ranks,
                              const int64_t* idx, int64_t n, tt_alloc_fn alloc, tt_free_fn free_fn,
                              void* alloc_ctx, void* stream, tt_eval_plan** out);
/* Release the plan (its device block is freed stream-ordered on `stream`). */
void tt_eval_plan_destroy(tt_eval_plan* plan, void* stream);
/* Bytes of the plan's device block. */
size_t tt_eval_plan_device_bytes(const tt_eval_plan* plan);

/* x_e for the plan's indices.  cores: host array of d device pointers, core
 * k an FP32 array [r_{k-1}][I_k][r_k] with the plan's dims and ranks;
 * out: device float[n].  Asynchronous; 1 kernel launch. */
tt_status tt_eval_plan_at(const tt_eval_plan* plan, const float* const* cores, float* out,
                          void* stream);
/* Gradients of sum_e gout_e x_e (gout: device float[n]), ACCUMULATED into
 * grads (host array of d device pointers shaped like the cores, distinct
 * buffers; zero them first for a plain gradient).  Asynchronous; 2 d launches. */
tt_status tt_eval_plan_backward(tt_eval_plan* plan, const float* const* cores, const float* gout,
                                float* const* grads, void* stream);
/* The same gradients with the interfaces taken from two sets of cores:
 *   grads_k[:, i, :] += sum_{e: i_k(e) = i} gout_e (L_1[i_1] .. L_{k-1}[i_{k-1}])^T
 *                                                (R_{k+1}[i_{k+1}] .. R_d[i_d])^T
 * with L = left and R = right (host arrays of d device pointers, shaped like
 * the plan's cores).  left = right is tt_eval_plan_backward.  With left the
 * left-orthogonal and right the right-orthogonal cores of one TT tensor X,
 * grads_k is U_{<k}^T Z_(k) V_{>k}^T for the zero-filled tensor Z of gout on
 * the index set: the first part of the tangent-space projection of the
 * Riemannian gradient (Sec. 4.2.2).  Asynchronous; 2 d launches. */
tt_status tt_eval_plan_backward_mixed(tt_eval_plan* plan, const float* const* left,
                                      const float* const* right, const float* gout,
                                      float* const* grads, void* stream);
/* Projection of P_Omega Z onto the tangent space at X of the manifold of TT
 * tensors of the plan's ranks (the Riemannian gradient of Sec. 4.2.2 when z
 * is the residual X - M on the index set).  U: the left-orthogonal cores of X
 * (U_1 .. U_{d-1} with orthonormal left unfoldings [r_{k-1} I_k] x [r_k], U_d
 * carrying the norm); V: the right-orthogonal cores of the same X (V_2 .. V_d
 * with orthonormal right unfoldings).  z: device float[n], the values of Z on
 * the plan's indices.  dU (host array of d device pointers shaped like the
 * cores, distinct buffers) is OVERWRITTEN with
 *   Y_k  = tt_eval_plan_backward_mixed(U, V, z)_k,
 *   dU_k = Y_k - U_k (U_k^T Y_k)   (left unfoldings, k < d; FP64 sums),
 *   dU_d = Y_d,
 * so that P_T(P_Omega Z) = sum_k U_1 .. U_{k-1} dU_k V_{k+1} .. V_d with the
 * gauge U_k^T dU_k = 0.  The result is only meaningful when U and V are
 * orthogonal frames of one tensor; that is not checked.  Asynchronous;
 * d memsets and 2 d + 3 (d - 1) launches. */
tt_status tt_tangent_project(tt_eval_plan* plan, const float* const* U, const float* const* V,
                             const float* z, float* const* dU, void* stream);
/* The tangent vector xi = sum_k U_1 .. U_{k-1} dU_k V_{k+1} .. V_d at the
 * plan's indices (P_Omega xi, for the step size of Sec. 4.2.2):
 *   out_e = sum_k (U_1[i_1] .. U_{k-1}[i_{k-1}]) dU_k[:, i_k, :] (V_{k+1}[i_{k+1}] .. V_d[i_d]).
 * U, V as for tt_tangent_project, dU shaped like the cores (host arrays of d
 * device pointers); out: device float[n], overwritten.  The terms are added
 * in the order k = 1..d, so the result is deterministic.  Works at the
 * plan's own ranks (no rank-2r block TT).  Asynchronous; d launches. */
tt_status tt_tangent_eval(const tt_eval_plan* plan, const float* const* U, const float* const* V,
                          const float* const* dU, float* out, void* stream);

/* One-shot forms: build a plan (cudaMallocAsync), run, destroy.  Each
 * synchronizes `stream` once (the index check); TT_EINVAL for an index
 * outside [0, prod(dims)). */
tt_status tt_eval_at(int32_t d, const int64_t* dims, const int64_t* ranks,
                     const float* const* cores, const int64_t* idx, int64_t n, float* out,
                     void* stream);
tt_status tt_eval_at_backward(int32_t d, const int64_t* dims, const int64_t* ranks,
                              const float* const* cores, const int64_t* idx, int64_t n,
                              const float* gout, float* const* grads, void* stream);

/* Diagnostics used by the tests: write the Rademacher sketch matrix of sweep
 * step `step` (rows x cols, +-1 as `dtype`, row-major, device) exactly as the
 * sweep draws it. */
tt_status tt_sketch_matrix(int64_t rows, int64_t cols, uint64_t seed, int32_t step, int32_t dtype,
                           void* out, void* stream);

/* Diagnostic used by the tests: run the bounded mbarrier wait of the
 * tensor-core kernels, with the given limit (nanoseconds, at most 1e10), on a
 * shared-memory barrier of one arrival that one thread completes
 * (arrive != 0) or that nothing completes.  TT_OK when the wait returns,
 * TT_ETIMEOUT when it ran out (the kernel then returns normally and the
 * context stays usable).  Synchronizes `stream`. */
tt_status tt_wait_selftest(int32_t arrive, int64_t limit_ns, void* stream);

/* Bounds-checked build (compiled with -DTT_BOUNDS_CHECK; build.py --checked
 * makes libttutv_bc.so): every checked device access whose index falls
 * outside its buffer is skipped and counted instead of performed (indices
 * read from data -- the masked evaluation's decoded indices, permutations
 * and positions -- core slices, tensor-map coordinates and their 16-byte
 * alignment, gathered copies).  Returns the number of violations counted
 * since the last reset (the device counters of every translation unit,
 * read with a synchronizing copy), the source line of the first in
 * *first_line (may be NULL), and zeroes the counters when reset != 0.
 * Returns -1 from the normal build. */
int64_t tt_bounds_violations(int32_t* first_line, int32_t reset);

/* Number of kernels this library has launched in the process so far
 * (all threads); a diagnostic for counting launches per call. */
uint64_t tt_kernel_launches(void);

/* Thread-local message of the last failure ("" if none). */
const char* tt_last_error(void);

/* Library version string. */
const char* tt_version(void);

#ifdef __cplusplus
}
#endif
#endif /* TTUTV_H */
