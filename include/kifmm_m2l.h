/*
 * kifmm_m2l.h -- C ABI of the SVD-compressed KIFMM M2L translation on GB300.
 *
 * The library implements the multipole-to-local (M2L) translation of the
 * kernel-independent FMM compressed by the SVD, after Cao, Wen & Rong,
 * "A SVD accelerated kernel-independent fast multipole method and its
 * application to BEM" (arXiv 1211.2517):
 *
 *   dense M2L            p^{t,d} = sum_{s in I^t} K(t,s) q^{s,u}        (Eq. (4))
 *   compressed M2L       p^{t,d} = U~ [ s_l sum_{s in I^t} K~_{t-s} (R~^T q^{s,u}) ]
 *                                                     (Eqs. (13), (14))
 *
 * with K(t,s)_ij = G(x_i^{t,d}, y_j^{s,u}), G = 1/(4 pi |x-y|) (Sec. 4), the
 * target's downward check surface x^{t,d} and the source's upward equivalent
 * surface y^{s,u} both at half-width (1+d) h (Sec. 2.1), I^t the
 * interaction field (Sec. 2.1), the 316 unit-level cores
 * K~_o = U~^T K_o R~ from the SVDs of K_fat and K_thin (Sec. 3.1), and the
 * level scale s_l = (r0 / 2^l)^(-1) from homogeneity (Sec. 3.1).  A
 * non-homogeneous kernel (the Yukawa kernel exp(-kappa r) / (4 pi r)) takes
 * one plan per level instead (Sec. 3.1's O(L) case, KIFMM_KERNEL_YUKAWA).
 *
 * Around the M2L: the second compression stage (Sec. 3.2), batched
 * multi-instance launches, a tile autotuner, and the complete potential
 * evaluation of a point cloud (kifmm_fmm_*: near field plus the compressed
 * passes S~, M~, L~, T~ of Sec. 3.3; point charges or dipoles, the double
 * layer of Sec. 4).
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 *  - Every function returns an int status: KIFMM_OK (0) or a negative
 *    KIFMM_ERR_* code.  No C++ exception crosses this boundary.  The message
 *    of the last failure on the calling thread is kifmm_m2l_last_error().
 *  - Surface points: the p^3 - (p-2)^3 = 6(p-1)^2+2 = n grid points
 *    c + h (1+d) (2 (i,j,k)/(p-1) - 1) with min(i,j,k) = 0 or
 *    max(i,j,k) = p-1, in lexicographic (i,j,k) order.
 *  - Offsets: the 316 vectors o in {-3..3}^3 with max|o_i| >= 2, in
 *    lexicographic order; a pair (t, s) has offset o = t - s (box units).
 *  - Boxes of a level are given by integer coordinates box_ijk[b] =
 *    (i,j,k), 0 <= i,j,k < 2^level, int32, row-major [n_boxes][3], no
 *    duplicates.  Their order is the caller's and indexes the density arrays.
 *  - Density arrays are float32, row-major [n_boxes][nrhs][n], contiguous.
 *  - Device pointers must be CUDA device (or managed) memory on the device
 *    that was current when the plan was made; host pointers are ordinary
 *    host memory.
 *  - Streams are passed as a cudaStream_t cast to void* (NULL = legacy
 *    default stream).  Device work is asynchronous on that stream; argument
 *    errors are reported synchronously, CUDA launch errors at the call that
 *    launched, device-side faults at the next synchronising call.
 *  - A plan is not thread-safe: calls on one plan must be serialised by the
 *    caller, and work on one (instance, level) state must not run on two
 *    streams at once (they share the plan's scratch buffers).
 */
#ifndef KIFMM_M2L_H
#define KIFMM_M2L_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ------------------------------------------------------ */
#define KIFMM_OK               0
#define KIFMM_ERR_INVALID_ARG  (-1) /* a pointer, size or enum is out of range        */
#define KIFMM_ERR_UNSUPPORTED  (-2) /* a valid request this build does not implement  */
#define KIFMM_ERR_CUDA         (-3) /* a CUDA runtime/driver call failed              */
#define KIFMM_ERR_OOM          (-4) /* host or device allocation failed               */
#define KIFMM_ERR_TIMEOUT      (-5) /* a bounded device wait ran out                   */
#define KIFMM_ERR_STATE        (-6) /* call order violated (e.g. apply before set_level) */

/* ---- enums ------------------------------------------------------------- */
#define KIFMM_KERNEL_LAPLACE   0    /* G(x,y) = 1 / (4 pi |x - y|), Sec. 4 */
#define KIFMM_KERNEL_YUKAWA    1    /* G(x,y) = exp(-kappa |x - y|) / (4 pi |x - y|): radial
                                       (translation invariant, K_o^T = K_{-o}) but not
                                       homogeneous, so its compressed operators depend on the
                                       box size (Sec. 3.1's O(L) case): a plan serves the boxes
                                       of one half-width, box_halfwidth, and L levels take L
                                       plans.  The plan's unit operator is
                                       h G(h (2 o + (1+d)(u_i - u_j))) = exp(-kappa h r) /
                                       (4 pi r), so the level scale 2^l / r0 = 1 / h applies as
                                       for the Laplace kernel.  M2L only: point-source
                                       evaluation and the pass operators are Laplace. */

/* Arithmetic of the core products sum_o K~_o q~ (Sec. 3.1).  Vt compression
 * and U expansion are FP32 in every mode. */
#define KIFMM_PREC_FP32        0    /* FP32 CUDA-core FMA                                  */
#define KIFMM_PREC_BF16        1    /* tcgen05 BF16 x BF16, FP32 accumulate (1 product)    */
#define KIFMM_PREC_SPLIT3      2    /* 2-piece BF16 split, 3 products (hi*hi+hi*lo+lo*hi)  */
#define KIFMM_PREC_SPLIT6      3    /* 3-piece BF16 split, 6 products (all terms <= 2^-16)  */
#define KIFMM_PREC_F16X3       4    /* 2-piece FP16 split with per-box scaling, 3 products:
                                       every q~ row is scaled by a power of two that keeps
                                       its entries below 2^15 (from sqrt(n) max|q| >= |q|
                                       >= |q~_i|; the point-source passes use q~'s largest
                                       entry), the cores by one that puts their largest
                                       entry in [2^13, 2^14), so both FP16 pieces stay
                                       normal where they matter; dropped terms <= 2^-22.
                                       apply, apply_levels (and adjoints), apply_batch,
                                       stage 2 (its factors and the rank-k_o intermediate
                                       scaled the same way) and point-source evaluation;
                                       not apply_noalloc */

#define KIFMM_N_OFFSETS        316  /* unique M2L offsets per level, Sec. 3.1 */

/* ---- types ------------------------------------------------------------- */
typedef struct kifmm_m2l_params {
    int    kernel_id;  /* KIFMM_KERNEL_LAPLACE or KIFMM_KERNEL_YUKAWA                  */
    int    p;          /* points per cube edge, 2 <= p <= 12; n = 6(p-1)^2+2             */
    double eps;        /* rank cutoff eps_1: keep sigma_i >= eps * sigma_0 (Sec. 3.1);
                          1e-12 <= eps < 1, or eps <= 0 to keep all n                    */
    double d;          /* surface ratio: surfaces at half-width (1+d) h, 0 <= d <= 2/3   */
    int    precision;  /* KIFMM_PREC_*                                                   */
    double kappa;      /* KIFMM_KERNEL_YUKAWA: screening constant, kappa > 0 (1 / length);
                          ignored for the Laplace kernel                                 */
    double box_halfwidth; /* KIFMM_KERNEL_YUKAWA: half-width h of the boxes the plan serves,
                          h > 0, kappa h <= 64; kifmm_m2l_set_level accepts only levels
                          with root_halfwidth / 2^level = h (relative 1e-12); ignored for
                          the Laplace kernel                                             */
} kifmm_m2l_params;

typedef struct kifmm_m2l_plan_s* kifmm_m2l_plan;   /* opaque; owned by the library */

/* ---- plan lifetime ----------------------------------------------------- */

/* Build the translation operators for `params` (Sec. 3.1, Step 1.4 of the
 * paper's algorithm): forms the 316 unit-level K_o, takes the SVD of K_fat
 * in FP64 on the host (TSQR, then the preconditioned one-sided Jacobi
 * method: column-pivoted QR, Jacobi on the transposed factor), truncates at
 * eps (a cut through a cluster of equal singular values moves past the
 * cluster: values within 1e-13 sigma_0 count as equal), sets R~ = U~
 * (K_o^T = K_{-o} for both radial kernels, so the thin SVD's right basis
 * spans U~'s space), forms K~_o = U~^T K_o U~ in FP64 for one offset of
 * every (o, -o) pair (the other is its transpose; the identity is checked
 * on sampled pairs and the plan refused above 1e-10 relative) and uploads
 * FP32 / BF16 / FP16-split copies to the current CUDA device.  The FP64 factors are cached on disk under
 * $KIFMM_M2L_CACHE (default: no cache) keyed by (kernel, p, d, eps, kappa h).
 * On success *out owns device memory until kifmm_m2l_destroy(). */
int kifmm_m2l_precompute(const kifmm_m2l_params* params, kifmm_m2l_plan* out);

/* Release every host and device resource of the plan (NULL is a no-op).
 * The caller must have synchronised streams that used it.
 * Library lifetime; no passage of the paper. */
int kifmm_m2l_destroy(kifmm_m2l_plan plan);

/* Rank introspection: *r = retained rank, *r_pad = r rounded up to a
 * multiple of 16 (device layout; the extra columns are zero), *n = surface
 * points.  Any output pointer may be NULL.
 * r is the rank kept by the truncation of Sec. 3.1 (Eqs. (8), (10)). */
int kifmm_m2l_plan_rank(kifmm_m2l_plan plan, int* r, int* r_pad, int* n);

/* ---- per-level state --------------------------------------------------- */

/* Register the non-empty boxes of one octree level of one FMM instance
 * (Step 1.2: interaction lists).  `box_ijk` is HOST memory [n_boxes][3]
 * int32, copied.  `root_halfwidth` is r0 (> 0); boxes of this level have
 * half-width r0 / 2^level.  Builds the interaction-list pairs grouped by
 * offset on the host and uploads them.  Replaces an earlier registration of
 * the same (instance, level).  0 <= level <= 20, n_boxes >= 0, coordinates
 * in [0, 2^level), instance >= 0.  A KIFMM_KERNEL_YUKAWA plan accepts only
 * levels whose boxes have its box_halfwidth (KIFMM_ERR_INVALID_ARG
 * otherwise). */
int kifmm_m2l_set_level(kifmm_m2l_plan plan, int instance, int level, double root_halfwidth,
                        int n_boxes, const int32_t* box_ijk);

/* Number of M2L pairs (target, source) of a registered level.
 * The pairs are those of the interaction fields I^t (Sec. 2.1, Step 1.2). */
int kifmm_m2l_level_pairs(kifmm_m2l_plan plan, int instance, int level, int64_t* n_pairs);

/* ---- the translation --------------------------------------------------- */

/* Compressed M2L of one registered level (Eq. (14) restricted to M2L):
 *   q~ = R~^T q_up ;  p~^t = s_l sum_{s in I^t} K~_{t-s} q~^s ;
 *   p_down = beta * p_down + U~ p~
 * q_up, p_down: DEVICE float32 [n_boxes][nrhs][n]; they must not overlap.
 * beta is 0 (overwrite; p_down need not be initialised) or any value
 * (accumulate, Step 3.1 "add to the downward check potentials").
 * nrhs >= 1.  Runs on `stream`.
 * Reproducibility: the core adds every pair's contribution into its
 * target's p~ row with global atomic or TMA bulk reductions, whose order is
 * not fixed, so two calls on the same input can differ in the last bits
 * (well inside the stated error; an iterative solver or an adjoint check
 * that needs bit-identical repeats must not rely on them). */
int kifmm_m2l_apply(kifmm_m2l_plan plan, int instance, int level, int nrhs,
                    const float* q_up, float* p_down, float beta, void* stream);

/* Adjoint (transpose) of kifmm_m2l_apply's linear map:
 *   p~bar = U~^T pbar_down ;  q~bar^s = s_l sum_{t: s in I^t} K~_{t-s}^T p~bar^t ;
 *   qbar_up = beta * qbar_up + R~ q~bar
 * applied as the core of the reversed offset, K~_o^T = K~_{-o} (which holds
 * to FP64 rounding because K_o^T = K_{-o} and R~ = U~; checked at
 * precompute).  Same layouts and rules as kifmm_m2l_apply.
 * The transpose of Eq. (14) (Sec. 3.1), formed with K~_o^T = K~_{-o}. */
int kifmm_m2l_apply_adjoint(kifmm_m2l_plan plan, int instance, int level, int nrhs,
                            const float* pbar_down, float* qbar_up, float beta, void* stream);

/* Compressed M2L of the consecutive registered levels level_lo..level_hi
 * of one instance as one batch (Step 3.1 over the downward pass's M2L
 * levels): the same result as kifmm_m2l_apply on each level, in five
 * kernel launches for all levels together (split into BF16 pieces and
 * compression of every row, one core over the levels' pairs merged by
 * offset, split and expansion of every row).
 * q_up and p_down hold the levels' arrays back to back in level order:
 * [n_boxes(level_lo)][nrhs][n], then level_lo + 1, ...  DEVICE float32.
 * 0 <= level_lo <= level_hi < level_lo + 32; the merged pair list is built
 * on the first call for (instance, level_lo, level_hi) and rebuilt after a
 * kifmm_m2l_set_level of any of these levels. */
int kifmm_m2l_apply_levels(kifmm_m2l_plan plan, int instance, int level_lo, int level_hi, int nrhs,
                           const float* q_up, float* p_down, float beta, void* stream);

/* Adjoint of kifmm_m2l_apply_levels (see kifmm_m2l_apply_adjoint).
 * The transpose of Eq. (14) (Sec. 3.1) over several levels. */
int kifmm_m2l_apply_levels_adjoint(kifmm_m2l_plan plan, int instance, int level_lo, int level_hi, int nrhs,
                                   const float* pbar_down, float* qbar_up, float beta, void* stream);

/* kifmm_m2l_apply_levels (Eq. (14), Sec. 3.1, over several levels) on HOST
 * buffers: q_up_host and p_down_host are HOST float32 arrays laid out as the
 * device buffers of kifmm_m2l_apply_levels (page-locked memory lets the
 * copies run asynchronously; pageable memory works, with synchronous
 * copies).  The rows travel in up to four chunks of whole 128-row tiles on
 * a copy stream of the plan; each chunk's split and compression start as
 * soon as it has landed, and each chunk of the expansion's output goes back
 * as soon as it is written, so the copies overlap the compression and the
 * expansion.  Every copy and kernel is ordered on `stream`: p_down_host is
 * complete when work enqueued on `stream` afterwards starts, or after
 * kifmm_m2l_sync.  beta != 0 first copies p_down_host in.  The plan keeps
 * device copies of both arrays (2 x rows x n floats) until destroyed.  The
 * host arrays must stay valid until the stream has passed the call. */
int kifmm_m2l_apply_levels_host(kifmm_m2l_plan plan, int instance, int level_lo, int level_hi, int nrhs,
                                const float* q_up_host, float* p_down_host, float beta, void* stream);

/* One FMM instance's share of a batch: levels level_lo..level_hi of
 * `instance` of `plan`, nrhs right-hand sides, DEVICE buffers laid out as
 * for kifmm_m2l_apply_levels, p_down = beta * p_down + M2L(q_up). */
typedef struct kifmm_m2l_batch_item {
    kifmm_m2l_plan plan;
    int instance;
    int level_lo, level_hi;
    int nrhs;
    const float* q_up;
    float* p_down;
    float beta;
} kifmm_m2l_batch_item;

/* Compressed M2L of many FMM instances of uneven sizes (and of several
 * operators, e.g. different p) in one batch (Step 3.1 for every instance).
 * Items are grouped by plan; for each plan one split and one persistent
 * compression launch and one split and one expansion launch cover all its
 * items, and the cores of all plans are one launch (each plan a group with
 * its own cores, rank and offset-ordered tile list merged over its items and
 * levels; the launch's CTAs split the summed work) when the plans share an
 * arithmetic with 1 or 2 pieces (bf16, split3, f16x3), use no stage 2 and
 * number at most 8; otherwise one core launch per plan.  A bounded-wait
 * timeout of a grouped core launch is reported by kifmm_m2l_sync of the
 * first plan in item order.  Tables and
 * scratch of a batch are built on its first call and cached by the batch's
 * signature (plans, instances, levels, nrhs, pointers, beta); the cached
 * batches of a plan are dropped by kifmm_m2l_set_level and by
 * kifmm_m2l_destroy on that plan.  With use_graph != 0 the launches of
 * the batch are captured once into a CUDA graph (after one eager pass,
 * which produces that call's result) and later calls with the same
 * signature replay the graph on `stream`.  Plans must use a tensor-core
 * precision (KIFMM_PREC_FP32 plans: KIFMM_ERR_UNSUPPORTED).  Items of one
 * plan must not write overlapping p_down buffers. */
int kifmm_m2l_apply_batch(int n_items, const kifmm_m2l_batch_item* items, int use_graph, void* stream);

/* Uncompressed M2L (Eq. (4)), the baseline the compression is compared
 * with:  p_down = beta * p_down + s_l sum_{s in I^t} K_{t-s} q^s  with the
 * FP32 unit-level K_o (formed on first use; 316 n^2 floats of device
 * memory).  Always FP32 CUDA-core arithmetic, accumulated with atomic adds
 * (summation order not fixed).  Same layouts and rules. */
int kifmm_m2l_apply_dense(kifmm_m2l_plan plan, int instance, int level, int nrhs,
                          const float* q_up, float* p_down, float beta, void* stream);

/* The same uncompressed M2L (Eq. (4)) on the tensor cores, in the plan's
 * f16x3 arithmetic: the q_up rows as two FP16 pieces after per-row
 * power-of-two scaling, K_o as two FP16 pieces of tau K_o, the products
 * hi*lo + lo*hi + hi*hi accumulated in FP32 (the compressed core's kernel
 * with K = N = n_pad), so that compressed and uncompressed M2L compare at
 * equal accuracy on equal hardware.  The first call forms the FP16 pieces
 * of K_o (2 * 316 * n_pad^2 halfs, 117 MB at p = 8) and its operand buffers
 * grow with the level's rows like kifmm_m2l_apply's.  Same layouts and beta
 * rule as kifmm_m2l_apply; rows reduced with TMA bulk additions (summation
 * order not fixed).  Errors: KIFMM_ERR_UNSUPPORTED unless the plan's
 * precision is KIFMM_PREC_F16X3 and its kernel Laplace. */
int kifmm_m2l_apply_dense_tc(kifmm_m2l_plan plan, int instance, int level, int nrhs,
                             const float* q_up, float* p_down, float beta, void* stream);

/* Synchronise `stream` and report device-side failures of earlier applies
 * on this plan: KIFMM_ERR_TIMEOUT when a bounded wait inside the
 * tensor-core kernel ran out (results of that apply are invalid; the flag
 * is cleared), KIFMM_ERR_CUDA on an asynchronous CUDA error.
 * Library utility; no passage of the paper. */
int kifmm_m2l_sync(kifmm_m2l_plan plan, void* stream);

/* Bound, in nanoseconds, of every mbarrier wait inside this plan's core
 * kernels from the next apply on (0 restores the default of 2 s).  A wait
 * that runs out sets the plan's device error flag, the kernel stops all its
 * roles, waits for its copies and MMAs in flight and frees its tensor
 * memory, and the next kifmm_m2l_sync returns KIFMM_ERR_TIMEOUT; the plan
 * stays usable.  A very short bound (a few ns) makes the first wait that is
 * not already complete give up, which is how the failure path is tested
 * without faulting the GPU.  Library utility (failure detection):
 * no passage of the paper.  Errors: KIFMM_ERR_INVALID_ARG for a NULL plan. */
int kifmm_m2l_set_wait_limit(kifmm_m2l_plan plan, unsigned long long ns);

/* ---- allocation-free apply ------------------------------------------------ */

/* kifmm_m2l_apply without any device allocation.  The paper has no
 * counterpart; this is an interface for callers of the library.
 *
 * kifmm_m2l_apply grows plan-owned scratch buffers with cudaMalloc the
 * first time a level or an nrhs needs them.  Callers that must not
 * allocate device memory once their run has started use this entry point
 * instead: applications whose memory manager reserved the device up front,
 * solvers held to a fixed memory budget, and latency-critical loops that
 * cannot take the device-wide synchronisation of cudaMalloc / cudaFree.
 * It computes what kifmm_m2l_apply computes (same layouts, beta rule and
 * precision modes, except KIFMM_PREC_F16X3, which it rejects with
 * KIFMM_ERR_UNSUPPORTED) and calls no allocating routine.  The core runs
 * the plan's core variant (the one kifmm_m2l_autotune chose, if any); the
 * compression and expansion split the FP32 rows into BF16 pieces inside
 * their GEMMs instead of through the separate split kernel, which saves the
 * split buffer.  Its
 * scratch is one static device array of KIFMM_NOALLOC_SCRATCH_BYTES
 * (64 MiB) that every GPU which loads this part of the library keeps until
 * the process exits.
 *  - The first call on a device (and the first after that device's
 *    context was destroyed and created again) looks up the array's device
 *    address, with that device current; make that first call before any
 *    stream capture.
 *  - A level and nrhs whose scratch would not fit is rejected with
 *    KIFMM_ERR_INVALID_ARG before anything is launched; the message gives
 *    the bytes needed.  The need is about n_boxes * nrhs * r_pad bytes
 *    times (2 * pieces + 4) (split modes; 8 for KIFMM_PREC_FP32), plus
 *    about 1 KB per 128 (pair, rhs) rows (tile and row tables).
 *  - Every call, from any plan, reuses the same array and overwrites it
 *    (the call clears what must start at zero).  Calls whose device work
 *    overlaps, e.g. on two streams at once, race and give wrong results:
 *    serialise them.
 * Same argument rules as kifmm_m2l_apply.
 * no passage of the paper (an allocation-free variant of kifmm_m2l_apply). */
#define KIFMM_NOALLOC_SCRATCH_BYTES ((size_t)64 << 20)
int kifmm_m2l_apply_noalloc(kifmm_m2l_plan plan, int instance, int level, int nrhs,
                            const float* q_up, float* p_down, float beta, void* stream);

/* ---- stage 2: per-offset low-rank cores (Sec. 3.2) ----------------------- */

/* Switch the plan's core to the second compression stage of Sec. 3.2
 * (Eq. (17)): each unit-level core is factored in FP64 on the host,
 * K~_o = U_o S_o Q_o^T, and truncated to the k_o singular values with
 * sigma >= eps2 * sigma_0(K_fat), eps2 = c2 * eps / r (Eq. (18), with
 * eps = the plan's eps_1 and r its rank); then
 *   p~^t += s_l Uhat_o (Vhat_o q~^s),  Uhat_o = U_o[:, :k_o] (r x k_o),
 *                                      Vhat_o = S_o Q_o^T restricted (k_o x r),
 * two skinny GEMMs per tile on the tensor cores instead of one r x r product.
 * Applies to every later apply / apply_adjoint / apply_levels / apply_batch /
 * apply_noalloc on this plan (the adjoint uses the reversed offset's factors).
 * c2 <= 0 switches back to the single-stage cores.  Tensor-core precisions
 * only (KIFMM_PREC_FP32: KIFMM_ERR_UNSUPPORTED); every k_o must be <= 96 and
 * r_pad <= 320 (else KIFMM_ERR_UNSUPPORTED: take a larger c2).  In
 * KIFMM_PREC_F16X3 the factors are two FP16 pieces of tau_V Vhat and tau_U
 * Uhat (powers of two, largest entry in [2^13, 2^14)) and each row of the
 * intermediate Vhat_o q~ is split into two FP16 pieces after its own power
 * of two; the output row undoes all of them.  Drops this plan's cached
 * batches.  Host work: the FP64 factors (from the plan's cache if
 * $KIFMM_M2L_CACHE is set, else recomputed) and 316 r x r SVDs; device
 * memory: 2 x 3 x 316 x 96 x r_pad 2-byte values. */
int kifmm_m2l_set_stage2(kifmm_m2l_plan plan, double c2);

/* The per-offset ranks k_o of stage 2 (k[316], HOST memory, offsets in the
 * lexicographic order above).  KIFMM_ERR_STATE when stage 2 is off.
 * Stage 2 is Sec. 3.2 (Eqs. (17), (18)). */
int kifmm_m2l_stage2_ranks(kifmm_m2l_plan plan, int* k);

/* Host-only stage 2 (no GPU needed): the FP64 precompute of
 * kifmm_m2l_precompute followed by the factoring of kifmm_m2l_set_stage2;
 * writes the 316 ranks to k and, if core is not NULL, the truncated cores
 * Uhat_o Vhat_o to core[316][r][r] (row-major, r from kifmm_m2l_factors_host).
 * Stage 2 is Sec. 3.2 (Eqs. (17), (18)). */
int kifmm_m2l_stage2_host(const kifmm_m2l_params* params, double c2, int* k, double* core);

/* ---- tracing ------------------------------------------------------------ */

/* Per-stage timing (enable != 0 turns it on, 0 off; off by default).  While
 * on, every apply / apply_adjoint records CUDA events on the caller's
 * stream around its compression, core and expansion kernels.  Recording
 * costs a few microseconds per stage; leave it off for throughput runs.
 * Library utility; no passage of the paper. */
int kifmm_m2l_profile_enable(kifmm_m2l_plan plan, int enable);

/* Read and clear the stage times recorded since the last read: waits for
 * the recorded events, writes ms[0..2] = summed milliseconds of the
 * compression, core and expansion kernels, and *launches = the number of
 * this library's kernel launches inside those intervals.  Either output
 * may be NULL.
 * Library utility; no passage of the paper. */
int kifmm_m2l_profile_read(kifmm_m2l_plan plan, double* ms, int64_t* launches);

/* ---- autotuning ---------------------------------------------------------- */

/* The choice kifmm_m2l_autotune kept: n_chunk = N columns of K~_o per core
 * work item, contiguous = 1 if each CTA takes one contiguous run of work
 * items (0: items dealt round-robin), variant = the split6 / f16x3 core
 * variant (0: hi and lo accumulators per tile, epilogue after the tile's
 * MMAs; 1 (split6 only): each tile's rows of q~ resident in shared memory,
 * K~_o streamed in column blocks, n_chunk then does not apply; 2 / 3:
 * partial sums of two / one K-chunks drained into registers while the next
 * partial's MMAs run; 4 / 5: as 2 / 3 with the output rows reduced into p~
 * by TMA bulk reductions; 6 (f16x3 only): partials of three K-chunks;
 * 9 / 10 / 11 (f16x3; 9 also split6): as 2 / 6 / 6 with two / two / three
 * K-chunks of a partial issued per MMA step; 12 (f16x3 only): as 11 with
 * every epilogue lane reducing its own row into p~ without a transpose;
 * other precisions: 0), core_ms = the core launch's
 * mean time (ms) under that choice, from_cache = 1 if read back from the
 * cache file. */
typedef struct kifmm_m2l_tune_result {
    int n_chunk;
    int contiguous;
    int variant;
    double core_ms;
    int from_cache;
} kifmm_m2l_tune_result;

/* Tile autotuner of the core GEMM (Step 3.1's per-offset products, on the
 * tensor cores).  The paper fixes no launch shape; the candidates here
 * change how the core's work is tiled and spread over the persistent CTAs
 * (N per work item, round-robin or contiguous work) and, for split6 and
 * f16x3, where partial sums are kept and how rows reach p~ (the variants
 * above).  The piece products
 * are the same for every candidate; the split6 variants differ in how the
 * FP32 partial sums are grouped (each stays within the split6 tolerance),
 * the others only in atomic accumulation order, which is never fixed.  Runs
 * kifmm_m2l_apply_levels(plan, instance, level_lo, level_hi, nrhs, q_up,
 * p_down, beta = 0, stream) once plus `reps` times (1 <= reps <= 1000) per
 * candidate, times the core launch with CUDA events, keeps the fastest in
 * the plan (used from then on by apply, apply_levels and apply_batch on this
 * plan) and writes it to *result (may be NULL).  p_down is overwritten with
 * the M2L of q_up.  Synchronises `stream`; drops pending tracing records.
 * If the environment variable KIFMM_M2L_AUTOTUNE_CACHE names a file, a
 * previous result for the same operator, device and workload (levels, nrhs,
 * box and pair counts) is read from it and applied without timing, and a
 * new result is added to it (a JSON object, one entry per line).
 * KIFMM_PREC_FP32 plans: KIFMM_ERR_UNSUPPORTED. */
int kifmm_m2l_autotune(kifmm_m2l_plan plan, int instance, int level_lo, int level_hi, int nrhs,
                       const float* q_up, float* p_down, int reps, kifmm_m2l_tune_result* result, void* stream);

/* ---- complete potential evaluation for point sources ------------------- */

/* The potential of a point cloud on itself, p_i = sum_{j != i} G(x_i, x_j) q_j
 * (Eq. (1)), evaluated as in the complete algorithm of Sec. 4 with the
 * compressed upward and downward passes of Sec. 3.3:
 *   near field  direct sums over the leaves sharing at least one vertex
 *               with the point's leaf, that leaf included (Sec. 2.1);
 *   far field   S~ = R~^T S at the leaves, M~ = R~^T M R~ up the tree, the
 *               plan's compressed M2L cores on levels 2..depth, L~ = U~^T L U~
 *               down the tree, T~ = T U~ at the leaves (Eqs. (2) ..
 *               (6) with Sec. 3.3's operators).
 * S, M, L, T are the KIFMM check / equivalent surface translations of
 * Sec. 2.1: upward equivalent and downward check surfaces at half-width
 * (1+d) h, upward check and downward equivalent surfaces at (3-2d) h; the
 * check-to-equivalent solves use the pseudo-inverse that drops singular
 * values below 1e-9 of the largest.  Every leaf sits at `depth`; the passes
 * run on the tensor cores in the split6 arithmetic, the M2L core in the
 * plan's precision, the leaf sums on the CUDA cores in FP32 with point
 * coordinates relative to their leaf's centre. */
typedef struct kifmm_fmm_s* kifmm_fmm;

#define KIFMM_FMM_NEAR 1  /* near-field part (S2T)          */
#define KIFMM_FMM_FAR  2  /* far-field part (S2M .. L2T)    */
#define KIFMM_FMM_ALL  3

/* Build the octree of a point cloud for `plan` (tensor-core precisions;
 * KIFMM_PREC_FP32: KIFMM_ERR_UNSUPPORTED; n > 512, i.e. p > 10:
 * KIFMM_ERR_UNSUPPORTED).
 *   points   HOST float64 [n_points][3], 1 <= n_points < 2^30; copied.
 *   depth    2..20; every leaf is a box of this level.
 *   centre   HOST float64 [3], root cube centre, with r0 > 0 its half-width;
 *            r0 <= 0 (centre may be NULL) takes the bounding box's midpoint
 *            and half-width max half-extent * (1 + 2^-20).
 * A point's box per coordinate is min(max(floor((x - (c - r0)) / (2 r0)
 * 2^depth), 0), 2^depth - 1); empty boxes are skipped.  The first call on a
 * plan also computes the pass operators (host FP64, about a second).  The
 * tree registers its levels on the plan under instances >= 2^30; destroy
 * every tree of a plan before the plan.  Errors: KIFMM_ERR_INVALID_ARG
 * (NULL pointer, sizes, non-finite coordinates), KIFMM_ERR_OOM,
 * KIFMM_ERR_CUDA.
 * The octree and lists of Sec. 2.1 and the setup of Sec. 4. */
int kifmm_fmm_create(kifmm_m2l_plan plan, int64_t n_points, const double* points, int depth,
                     const double* centre, double r0, kifmm_fmm* out);

/* potential[i] = the parts (KIFMM_FMM_NEAR | KIFMM_FMM_FAR) of the
 * potential at point i from the densities q.  q and potential: DEVICE
 * float32 [n_points] in the caller's point order; potential is overwritten.
 * Asynchronous on `stream`; calls on one tree (and on trees of one plan)
 * must be serialised.  Errors: KIFMM_ERR_INVALID_ARG (NULL, parts out of
 * 1..3), KIFMM_ERR_CUDA.
 * Eq. (1) by the complete algorithm of Sec. 4 with the compressed passes of Sec. 3.3. */
int kifmm_fmm_evaluate(kifmm_fmm fmm, const float* q, float* potential, int parts, void* stream);

/* Double layer (Sec. 4, Eq. (26)): with normals set, the sources are
 * dipoles and evaluate computes
 *   p_i = sum_{j != i} dG(x_i, x_j)/dn(x_j) q_j,
 *   dG(x, y)/dn(y) = n(y) . (x - y) / (4 pi |x - y|^3),
 * with dG/dn in the near field (S2T) and in the leaf check potentials (the
 * first step of S2M); the equivalent densities and every later step are
 * single layer, as for point charges.  The adjoint is a different operator
 * (the evaluation is not symmetric in this mode).
 *   normals  HOST float64 [n_points][3] in the caller's point order (n_j as
 *            given: unit normals for a double-layer integral); copied to the
 *            device in leaf order (synchronous: no evaluate of this tree may
 *            be in flight).  NULL returns the tree to single layer.
 * Errors: KIFMM_ERR_INVALID_ARG (NULL fmm, non-finite entries),
 * KIFMM_ERR_OOM, KIFMM_ERR_CUDA. */
int kifmm_fmm_set_normals(kifmm_fmm fmm, const double* normals);

/* Sizes of a tree: depth, leaves, boxes on levels 2..depth, M2L pairs over
 * those levels, and (target point, source point) pairs of the near field
 * (the point itself excluded).  Any output may be NULL.
 * Sizes of the Sec. 2.1 tree and lists. */
int kifmm_fmm_info(kifmm_fmm fmm, int* depth, int64_t* n_leaves, int64_t* n_boxes, int64_t* n_m2l_pairs,
                   int64_t* n_near_pairs);

/* Release a tree and its levels on the plan.  NULL is a no-op.
 * Library lifetime; no passage of the paper. */
int kifmm_fmm_destroy(kifmm_fmm fmm);

/* ---- host-side introspection (no GPU needed) ----------------------------- */

/* Run the FP64 precompute of kifmm_m2l_precompute on the host only and copy
 * out its results.  n and r are returned in *n, *r (either may be NULL).
 * sigma: [n] singular values of K_fat, descending (or NULL);
 * U: [n][r] row-major retained left basis U~ (or NULL);
 * C: [316][r][r] row-major unit-level cores K~_o (or NULL).
 * Call once with the arrays NULL to learn n and r.
 * The factors of Sec. 3.1 (Eqs. (8), (10), (13)). */
int kifmm_m2l_factors_host(const kifmm_m2l_params* params, int* n, int* r,
                           double* sigma, double* U, double* C);

/* The compressed pass operators of Sec. 3.3 that kifmm_fmm_create uses,
 * computed on the host in FP64 for a unit parent box with the basis U~ of
 * kifmm_m2l_factors_host (R~ = U~):
 *   Ws [r][n]      U~^T E_u, E_u the pseudo-inverse of K(x^u, y^u) keeping
 *                  singular values >= rcond * sigma_0 (*kept of them);
 *                  S~ of a leaf of half-width h is h Ws K(x^u, points)
 *   Mt [8][r][r]   U~^T E_u K(x^u, y^u of child c) U~ = M~ of the child in
 *                  octant c = 4 b_x + 2 b_y + b_z (centre (2b - 1)/2)
 * The downward operators are the transposes (T~'s factor Ws^T, L~_c =
 * Mt[c]^T).  Any output may be NULL.  0 < rcond < 1. */
int kifmm_m2l_pass_ops_host(const kifmm_m2l_params* params, double rcond, int* kept, double* Ws, double* Mt);

/* Interaction-list pairs of a box set on the host (Sec. 2.1): for every
 * target t and source s in I^t, one entry (t, s, offset index of t - s).
 * Entries are sorted by offset index, then target.  Call with
 * targets == NULL to get the count in *n_pairs; then with arrays of that
 * length.  Same box rules as kifmm_m2l_set_level. */
int kifmm_m2l_pairs_host(int level, int n_boxes, const int32_t* box_ijk, int64_t* n_pairs,
                         int32_t* targets, int32_t* sources, int32_t* offsets);

/* Message of the last failed call on this thread ("" if none).
 * Library utility; no passage of the paper. */
const char* kifmm_m2l_last_error(void);

/* Library version string.
 * Library utility; no passage of the paper. */
const char* kifmm_m2l_version(void);

#ifdef __cplusplus
}
#endif

#endif /* KIFMM_M2L_H */
