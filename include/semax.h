/*
 * semax.h -- C ABI of libsemax, the element-local spectral-element Laplacian
 * operator ("Ax") for one NVIDIA GB300 (sm_103a).
 *
 * The operation.  For every hexahedral element e of polynomial order N
 * (n = N+1 Gauss-Lobatto-Legendre nodes per direction) the library computes
 *
 *     w_e = sum_{a,b in {r,s,t}} D_a^T diag(G_e,ab) D_b u_e
 *
 * with D_r = I(x)I(x)D, D_s = I(x)D(x)I, D_t = D(x)I(x)I acting on the node
 * index (k*n + j)*n + i, i.e. the sum-factorised sequence
 *     ur = sum_l D[i][l] u[k][j][l],  us = sum_l D[j][l] u[k][l][i],
 *     ut = sum_l D[k][l] u[l][j][i];  [wr ws wt] = G_p [ur us ut];
 *     w  = sum_l D[l][i] wr[k][j][l] + D[l][j] ws[k][l][i] + D[l][k] wt[l][j][i].
 * This is the textbook weak-form Laplacian of the spectral-element method
 * (Deville, Fischer & Mund 2002, Sec. 4.4).  The paper (Kloeckner, "Loo.py:
 * From Fortran to performance via transformation and substitution rules",
 * ARRAY'15) does not print this operator: its Section 1 names PDE-solver
 * kernels and autotuning search spaces as the system's use cases, its
 * Section 3 ingests Fortran array subroutines of exactly this shape (arrays
 * u(i,j,k,e) passed by the caller, loop bounds as arguments), and its
 * Section 5.2 blocks a matrix-matrix product, the form each contraction above
 * takes ((n x n) times (n x n^2)).
 *
 * Layouts (all row-major C order, i fastest = Fortran u(i,j,k,e)):
 *   u, w   [E][n][n][n]
 *   G      [E][6][n][n][n], components (rr, rs, rt, ss, st, tt) of the
 *          symmetric 3x3 factor det(J) w_i w_j w_k J^{-1} J^{-T}
 *   D      [n][n], D[i][l] = derivative of the l-th Lagrange polynomial at
 *          node i
 *
 * Conventions shared by every entry point:
 *   - All array pointers are owned by the caller and must be accessible from
 *     the device at the address given: device memory, or host memory pinned
 *     with cudaHostAlloc/cudaHostRegister (on NVLink-C2C systems such as
 *     GB300 the kernel then streams the arrays over the coherent link with no
 *     staging copy).  The operator calls (sem_ax, sem_ax_* apart from the
 *     plan functions) never allocate, free or synchronise; work is queued
 *     on `stream` (a cudaStream_t, NULL = legacy default stream) and the
 *     call returns before it finishes.  Plans, the gather-scatter and the
 *     PCG solver state what they allocate or wait for.
 *   - 1 <= N <= 15 (n <= 16), else SEMAX_EUNSUPPORTED_N.
 *   - E == 0 is a no-op returning SEMAX_OK (pointers are not inspected).
 *     E < 0 or a NULL pointer with E > 0 returns SEMAX_EINVAL.
 *   - u, G and w must be 16-byte aligned (128-bit vector access), else
 *     SEMAX_EALIGN.  D needs only its natural alignment.
 *   - w must not overlap u, G or D, else SEMAX_EALIAS.
 *   - A failed kernel launch returns SEMAX_ECUDA; semax_last_cuda_error()
 *     then gives the cudaError_t of the failing call on this host thread.
 *   - On any error nothing has been queued and w is untouched.
 */
#ifndef SEMAX_H
#define SEMAX_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    SEMAX_OK = 0,
    SEMAX_EINVAL = -1,          /* bad count, NULL pointer, bad argument        */
    SEMAX_EUNSUPPORTED_N = -2,  /* N outside 1..15                              */
    SEMAX_EALIGN = -3,          /* u, G or w not 16-byte aligned                */
    SEMAX_EALIAS = -4,          /* output overlaps an input                     */
    SEMAX_ECUDA = -5,           /* a CUDA runtime call failed                   */
    SEMAX_ETIMEOUT = -6,        /* a bounded device-side wait gave up           */
    SEMAX_ENOPLAN = -7,         /* NULL or destroyed plan                       */
    SEMAX_EWORKSPACE = -8,      /* workspace missing or too small               */
    SEMAX_EIO = -9              /* tuning cache could not be read or written    */
} semax_status;

typedef enum { SEMAX_F64 = 0, SEMAX_F32 = 1 } semax_prec;

/* ---------------------------------------------------------------- plain forms */

/* FP64 Ax.  Loads u and G once, stores w once; computes in double. */
int sem_ax(int64_t E, int N, const double *u, const double *G, const double *D,
           double *w, void *stream);

/* Helmholtz form of the operator, FP64:
 *     w = h1 A u + h2 B u,
 * B [E][n][n][n] the diagonal GLL mass matrix (det(J) w_i w_j w_k per node),
 * h1, h2 scalars.  The SEM Helmholtz operator of implicit time stepping and
 * of the pressure/velocity solvers that apply Ax (Deville, Fischer & Mund
 * 2002, Sec. 4.4); one extra read of B and two FP64 operations per node on
 * top of Ax, fused into the same pass.  B follows the alignment and aliasing
 * rules of G.  With h1 = 1, h2 = 0 it returns sem_ax's values. */
int sem_ax_helmholtz(int64_t E, int N, const double *u, const double *G, const double *B,
                     const double *D, double h1, double h2, double *w, void *stream);

/* FP64 inputs and outputs, FP64-accurate result; the six contractions run
 * in double-float arithmetic (each value an unevaluated sum of two floats,
 * ~47 significant bits) on the FP32 pipe, which GB300 issues 62.5 times
 * faster than FP64, and the geometric-factor multiply in FP64.  Each
 * element's u and its intermediate [wr ws wt] are scaled by powers of two
 * (exact) so that their largest entry lies in [1, 2); entries more than
 * 2^126 times smaller than their element's largest count as zero.  Error
 * against the FP64 definition ~1e-14 of ||w||_inf.  Even n with a
 * centro-antisymmetric D (the GLL derivative); other orders and matrices
 * are computed by the FP64 kernel of sem_ax. */
int sem_ax_f64x(int64_t E, int N, const double *u, const double *G, const double *D,
                double *w, void *stream);

/* FP64 inputs and outputs, FP64-accurate result; the six contractions run
 * on FP16 tensor cores by exact slicing (the Ozaki scheme).  Per element, u
 * and the intermediate [wr ws wt] are scaled by a power of two and written
 * as five balanced base-1024 digits (integers of magnitude <= 528, exact in
 * FP16), D likewise once per call; the digit products of levels 0..4 (15
 * pairs per contraction) are summed on tensor cores in FP32 accumulators
 * (exact: below 2^24 at n = 8, and for levels 0..2 at n = 16, whose levels
 * 3 and 4 weigh 2^-30 and 2^-40), and the level sums are combined in
 * double-float.  The geometric-factor multiply runs in double-float with G
 * split by bit operations after a per-node power-of-two scale.  Error
 * against the FP64 definition ~1e-13 of ||w||_inf or less; entries more
 * than ~2^48 times smaller than their element's largest count only to that
 * precision.  An element with an Inf or NaN input returns NaN in every
 * entry.  Orders N = 7 (n = 8) and N = 15 (n = 16) on tensor cores, any
 * D; other orders are computed by sem_ax_f64x.  N = 15 launches one
 * persistent 512-thread block per SM with 207 KB of shared memory.  N = 7
 * is launched as a programmatic dependent of the previous kernel in the
 * stream (its blocks may become resident while that kernel finishes), and
 * reads no global memory before that kernel has completed, so stream order
 * holds as for any launch. */
int sem_ax_f64tc(int64_t E, int N, const double *u, const double *G, const double *D,
                 double *w, void *stream);

/* The Helmholtz form w = h1 A u + h2 B u (as sem_ax_helmholtz) with A u
 * computed FP64-accurately on tensor cores as in sem_ax_f64tc and the mass
 * term added in FP64: 72 bytes per node moved, like the FP64 form, without
 * its FP64-pipe limit (N = 15 reads u a second time for the mass term, 80
 * bytes per node).  N = 7 and N = 15 on tensor cores; other orders are
 * computed by sem_ax_helmholtz.  B follows the alignment and aliasing rules
 * of G. */
int sem_ax_helmholtz_f64tc(int64_t E, int N, const double *u, const double *G, const double *B,
                           const double *D, double h1, double h2, double *w, void *stream);

/* sem_ax_f64tc with a status word for its bounded device-side waits.  The
 * tensor-core kernels of orders 7 and 15 stage each element's u and G in
 * shared memory with TMA bulk copies that complete on an mbarrier, and wait
 * for them with a bounded number of polls (2^20 by default; each poll may
 * suspend the thread briefly).  A copy that never completes is a failure of
 * the device, not a property of any input.  If a wait gives up, its CTA
 * stores SEMAX_ETIMEOUT in *status, writes NaN to every output element it
 * has not yet written, waits once more (bounded, with the default limit) for
 * its copies in flight, and exits; other CTAs carry on.  (Should that second
 * wait give up too, the CTA exits with a copy still in flight, which may then
 * land in shared memory the CTA no longer owns: the device is failing.)  `status` is a
 * device int (4-byte aligned) that the kernels write only on a timeout: set
 * it to SEMAX_OK before the call and read it once `stream` has reached the
 * call's end.  NULL reports nothing (exactly sem_ax_f64tc).  Orders other
 * than 7 and 15 run the double-float tile, which has no waits, and never
 * write it.  The status is not the call's return value because the call
 * returns before the kernel runs. */
int sem_ax_f64tc_status(int64_t E, int N, const double *u, const double *G, const double *D,
                        double *w, int *status, void *stream);

/* The tensor-core FP64-accurate Ax with the geometric factor prepared once
 * (for repeated applications with the same G, as in an iterative solver).
 * sem_ax_f64tc_prepare splits G's entries into (hi, lo) float pairs against
 * one power-of-two scale per element, kept in a 16-byte record with the
 * element's split pairs: E * 24592 bytes at N = 7 (64 bytes per node plus 16
 * per element, the same HBM traffic per call as FP64 G) and E * 196624 at
 * N = 15 (sem_ax_f64tc_prepare_size).  sem_ax_f64tc_prepared then computes,
 * bit for bit, what sem_ax_f64tc computes from G, without the split:
 * sem_ax_f64tc splits per node (at N = 15 per node and half of G), which
 * gives the same digits unless an element's G entries span more than about
 * 2^100, far beyond any mesh, where the per-element split flushes entries
 * below 2^-126 of the element's largest to zero.  N = 7 and N = 15
 * (SEMAX_EUNSUPPORTED_N otherwise).  Gp: device memory, 16-byte aligned,
 * owned by the caller, not overlapping G or w, and prepared for the same E
 * and N (its size is not checked, like G's in sem_ax). */
int sem_ax_f64tc_prepare_size(int64_t E, int N, size_t *bytes);
int sem_ax_f64tc_prepare(int64_t E, int N, const double *G, void *Gp, void *stream);
int sem_ax_f64tc_prepared(int64_t E, int N, const double *u, const void *Gp, const double *D,
                          double *w, void *stream);
/* sem_ax_f64tc_prepared with the status word of sem_ax_f64tc_status. */
int sem_ax_f64tc_prepared_status(int64_t E, int N, const double *u, const void *Gp, const double *D,
                                 double *w, int *status, void *stream);

/* FP32 storage and FP32 compute.  G_scale is NULL or [E] per-element factors
 * s_e: the kernel then treats the stored G as G_e / s_e and multiplies the
 * element's result by s_e (use powers of two so that this is exact). */
int sem_ax_f32(int64_t E, int N, const float *u, const float *G, const float *D,
               float *w, const float *G_scale, void *stream);

/* FP32 storage; the six derivative contractions run on tensor cores in BF16
 * with FP32 accumulation, each FP32 operand x split as x0 + x1 (+ x2) with
 * x0 = bf16(x), x1 = bf16(x - x0), x2 = bf16(x - x0 - x1).  terms = 3 keeps
 * the products x0 y0 + x0 y1 + x1 y0 ("bf16x3", ~16 significant bits);
 * terms = 6 also keeps x0 y2 + x1 y1 + x2 y0 (~24 bits).  The geometric
 * factor multiply is FP32.  G_scale as in sem_ax_f32.  Order N = 15 only
 * (n = 16, one 16 x 16 tensor-core tile per plane); other orders return
 * SEMAX_EUNSUPPORTED_N. */
int sem_ax_bf16x3(int64_t E, int N, const float *u, const float *G, const float *D,
                  float *w, const float *G_scale, int terms, void *stream);

/* The split tensor-core form with FP16 pieces and three products: each
 * operand x is scaled by a power of two s (exact) and split as x s = x0 + x1,
 * x0 = fp16(x s), x1 = fp16(x s - x0), ~22 significant bits against BF16's
 * 16, and the products x0 y0 + x0 y1 + x1 y0 are accumulated in FP32 on the
 * tensor cores.  FP16's exponent range is narrow, so the scales are chosen
 * to put each group's largest magnitude in [1, 2): u and the intermediate wt
 * per element, D once, wr and ws per plane of the element (their
 * contractions stay inside a plane); they are undone on the output.  Values
 * more than 2^24 below their group's largest keep an absolute accuracy of
 * 2^-25 of it.  The geometric factor multiply is FP32; G_scale as in
 * sem_ax_f32.  Error against the FP64 definition ~1e-6 of ||w||_inf.
 * Orders N = 7 and N = 15 (others: SEMAX_EUNSUPPORTED_N); at N = 7 wr and
 * ws are scaled per pair of planes (the planes a warp owns). */
int sem_ax_f16x3(int64_t E, int N, const float *u, const float *G, const float *D, float *w,
                 const float *G_scale, void *stream);

/* The BF16-split tensor-core form with the geometric factor recomputed at
 * every node instead of read: X [E][8][3] holds each element's vertices
 * (FP32; vertex v = a + 2b + 4c at reference corner ((-1)^(a+1), (-1)^(b+1),
 * (-1)^(c+1))), the map is trilinear, and G = w_i w_j w_k adj(J) adj(J)^T /
 * det(J) is formed in FP32 from the map's coefficients.  xi_wq [32] (device)
 * holds the 16 GLL nodes then the 16 GLL weights.  A call reads 8 bytes per
 * node (u, w) plus 96 bytes per element instead of 32 bytes per node.  This
 * is the paper's store-versus-recompute trade-off (Section 4.1, turning a
 * stored temporary back into a substitution rule that is recomputed where it
 * is used).  N = 15 only; terms as in sem_ax_bf16x3. */
int sem_ax_bf16x3_geo(int64_t E, int N, const float *u, const float *X, const float *xi_wq,
                      const float *D, float *w, int terms, void *stream);

/* ---------------------------------------------------------------- batched form */

/* One group of E elements of order N (FP64), with its own arrays. */
typedef struct {
    int N;
    int64_t E;
    const double *u;
    const double *G;
    const double *D;
    double *w;
} semax_group;

/* Bytes of device workspace sem_ax_batched needs for these groups. */
int sem_ax_batched_workspace_size(const semax_group *groups, int ngroups, size_t *bytes);

/* All groups in ONE persistent kernel launch: tiles of elements are handed out
 * longest-first (cost ~ n^4 per element) through a device work counter held
 * in `workspace` (device memory, >= the size above, caller-owned).  At most
 * 32 groups (else SEMAX_EINVAL); the group table travels in the kernel
 * parameters, so the call queues only a reset of the counter and the kernel,
 * and `groups` may be reused as soon as it returns.  Calls sharing one
 * workspace must not overlap on the GPU.  Tile sizes and thread mapping use
 * built-in defaults (see the plan API for tuned choices). */
int sem_ax_batched(const semax_group *groups, int ngroups, void *workspace,
                   size_t ws_bytes, void *stream);

/* A plan owns a device work counter and a captured CUDA graph that resets the
 * counter and launches the persistent kernel (and, with SEMAX_PLAN_F64TC,
 * the groups launched apart beside it, on up to eight forked streams joined
 * before the graph ends, longest first).  Creating a plan allocates device memory; executing it does
 * not.
 *   tune = 0: use the tuning cache entry if present, else defaults;
 *   tune = 1: time the candidate (elements per tile, thread mapping) pairs for
 *             every order present on the current device and keep the fastest;
 *             the choice is written to cache_path (JSON) if not NULL.
 *   flags = SEMAX_PLAN_F64X: even orders take the double-float FP64-accurate
 *             tile (error ~1e-14 of ||w||_inf) instead of the FP64 tiles and
 *             are not tuned; odd orders are unaffected.
 *   flags |= SEMAX_PLAN_F64TC: groups of order N = 7 and N = 15 leave the
 *             persistent launch and run sem_ax_f64tc (FP64-accurate on tensor
 *             cores), bit for bit that call's result.  With SEMAX_PLAN_F64X
 *             as well, every group with even n = N + 1 leaves it (the others
 *             run sem_ax_f64x, bit for bit), each in a launch of its own, so
 *             that groups too small to fill the GPU alone run side by side.
 *   flags |= SEMAX_PLAN_F64TC_PREPARED (with SEMAX_PLAN_F64TC): the groups of
 *             order 7 and 15 run sem_ax_f64tc_prepared on their G split once
 *             at plan creation (sem_ax_f64tc_prepare, into device buffers the
 *             plan owns), bit for bit sem_ax_f64tc: G's values are read then,
 *             so a later change to them does not reach the plan.
 * The group arrays are bound into the plan: they must stay valid while the
 * plan is used (tuning runs the kernel on them, overwriting their w). */
typedef struct semax_plan semax_plan;
enum {
    SEMAX_PLAN_F64X = 1,    /* even n: the double-float FP64-accurate tile of sem_ax_f64x */
    SEMAX_PLAN_F64TC = 2,   /* N = 7, 15: sem_ax_f64tc beside the persistent kernel (with F64X: every even n apart) */
    SEMAX_PLAN_F64TC_PREPARED = 4   /* with F64TC: N = 7, 15 on G prepared at plan creation */
};
int sem_ax_plan_create(semax_plan **plan, const semax_group *groups, int ngroups,
                       int tune, const char *cache_path, int flags);
int sem_ax_plan_exec(semax_plan *plan, void *stream);
int sem_ax_plan_destroy(semax_plan *plan);
/* SEMAX_ETIMEOUT if, in an execution of the plan since the last call, a
 * staging wait of its tensor-core launches (SEMAX_PLAN_F64TC) gave up (see
 * sem_ax_f64tc_status), else SEMAX_OK; clears the plan's status word.
 * Blocks the host until the work queued on `stream` so far has finished. */
int sem_ax_plan_status(semax_plan *plan, void *stream);
/* The configuration the plan uses for order N: elements per tile and thread
 * mapping (0 = one thread per node, 1 = one thread per (i,j) column,
 * 2 = one thread per line with the even/odd split of D, even n only,
 * 3 = the double-float tile of sem_ax_f64x, chosen by SEMAX_PLAN_F64X,
 * 4 = sem_ax_f64tc in its own launch, chosen by SEMAX_PLAN_F64TC; elements
 * per tile is then 1; the other orders launched apart report 3 and the
 * double-float tile's elements per tile).  Returns SEMAX_EINVAL if N is not in the plan. */
int sem_ax_plan_config(const semax_plan *plan, int N, int *elems_per_tile, int *mapping);

/* ---------------------------------------------------------------- solver around Ax */

/* Direct stiffness summation (gather-scatter) on vectors in local element
 * form: every local value becomes the sum of the local values that share its
 * global node (Q Q^T in the usual notation; Deville, Fischer & Mund 2002,
 * Sec. 4.5).  local_to_global (HOST array, nlocal entries in [0, nglobal))
 * gives each local node's global node; dirichlet (HOST, nglobal bytes, or
 * NULL) marks global nodes held at zero when apply_mask is set.  The sums use
 * a fixed order, so the result is deterministic.  Creating the handle
 * allocates device memory; applying it does not. */
typedef struct semax_gs semax_gs;
int semax_gs_create(semax_gs **gs, int64_t nlocal, const int64_t *local_to_global, int64_t nglobal,
                    const unsigned char *dirichlet);
int semax_gs_apply(const semax_gs *gs, double *v, int apply_mask, void *stream);
int semax_gs_destroy(semax_gs *gs);

/* diag(A_e) of every element (FP64, layout of u): the Jacobi preconditioner's
 * element part. */
int sem_ax_diag(int64_t E, int N, const double *G, const double *D, double *diag, void *stream);

/* Jacobi-preconditioned conjugate gradients for Q A_L Q^T x = b with the
 * homogeneous Dirichlet nodes of gs held at zero -- the PDE solve that
 * applies Ax once per iteration.  Vectors are continuous local vectors (E n^3
 * doubles, equal copies at shared nodes); b must already be summed (gs) and
 * masked.  Create allocates the work vectors and computes the preconditioner;
 * G, D and gs stay bound to the solver; flags = 0 applies A with the FP64
 * kernel of sem_ax, SEMAX_PCG_F64X with that of sem_ax_f64x, SEMAX_PCG_F64TC
 * with that of sem_ax_f64tc (at most one of the two flags; at N = 7 from G
 * prepared once at create, sem_ax_f64tc_prepared, E * 24592 bytes more
 * device memory, the same results bit for bit).  SEMAX_PCG_MIXED
 * (combinable with either) is mixed-precision iterative refinement: each
 * outer step computes the true residual r = b - A x with the FP64-accurate
 * operator, solves A d = r from d = 0 by PCG whose recurrences are FP64 but
 * whose A is the FP32 kernel (FP32 copies of G and D made at create; the
 * search direction converted to FP32 and the product back), to a relative
 * reduction max(1e-5, rtol / 2 / current residual), and adds d to x.  The
 * reported residual is the true one; the solve also stops when an outer
 * step fails to halve it (the FP64-accurate operator's own floor); iters
 * counts the inner iterations.  Solve starts from x (in/out) and
 * stops when ||r|| <= rtol ||r_0|| (norms weighted by 1/multiplicity) or after
 * max_iter iterations, checked every 10 iterations: a block of 10 iterations
 * is one CUDA-graph launch with all scalars in device memory.  Solve blocks
 * the host until it returns; it is ordered after earlier work on `stream` and
 * later work on `stream` is ordered after it.  With SEMAX_PCG_F64TC it
 * returns SEMAX_ETIMEOUT (x then holds NaN) if a staging wait of the
 * tensor-core operator gave up (see sem_ax_f64tc_status). */
typedef struct semax_pcg semax_pcg;
enum { SEMAX_PCG_F64X = 1,     /* apply A with sem_ax_f64x (double-float, FP64-accurate) */
       SEMAX_PCG_F64TC = 2,     /* apply A with sem_ax_f64tc (tensor-core digit slicing, FP64-accurate) */
       SEMAX_PCG_MIXED = 4 };   /* FP32 operator inside, FP64 residuals outside (iterative refinement) */
int sem_pcg_create(semax_pcg **pcg, int64_t E, int N, const double *G, const double *D, const semax_gs *gs,
                   int flags);
int sem_pcg_solve(semax_pcg *pcg, const double *b, double *x, int max_iter, double rtol, int *iters,
                  double *rel_res, void *stream);
int sem_pcg_destroy(semax_pcg *pcg);

/* ---------------------------------------------------------------- FP64 checks */

/* FP64 reductions over `count` entries, on the GPU:
 *   out[0] = max_i |a_i - b_i|,  out[1] = max_i |b_i|,  out[2] = sum_i a_i b_i
 * a and b are FP64 or FP32 (a_prec, b_prec in semax_prec), widened to double
 * before any arithmetic.  `out` is a device pointer to 3 doubles.  Uses
 * `workspace` (device, >= semax_reduce_workspace_size bytes) for per-block
 * partial results; the result does not depend on the launch order. */
int semax_reduce_workspace_size(int64_t count, size_t *bytes);
int semax_reduce(int64_t count, const void *a, int a_prec, const void *b, int b_prec,
                 double *out, void *workspace, size_t ws_bytes, void *stream);

/* Same reduction as semax_reduce for callers that cannot allocate device
 * memory (a legacy solver that owns every allocation and passes the library
 * only its own arrays, or code where the allocator must not be called), so it
 * takes no workspace.  The paper has no counterpart: this is a deployment
 * convenience of this library.  Its per-block partials live in a file-scope
 * device array of 1024 x 3 doubles (24 KiB) that every GPU which loads the
 * library holds until the process exits.  The fixed partition of
 * semax_reduce never needs more than those 1024 blocks, so every count >= 0
 * fits and the result equals semax_reduce's bit for bit; a partition that
 * needed more would be rejected with SEMAX_EWORKSPACE.  Nothing in the array
 * has to start at zero (pass 1 writes every partial that pass 2 reads).
 * The first call on a device looks up the array's device address
 * (cudaGetSymbolAddress, with that device current) and caches it for the
 * device's current context; make that first call before any stream capture.
 * After a device reset (cudaDeviceReset) the next call, in the new context,
 * looks the address up again.  Every call on a device shares the one array and
 * it keeps the last call's partials: calls that can overlap on the GPU (on
 * different streams, or from several host threads) race on it and must be
 * ordered by the caller.  No cudaMalloc, cudaFree or allocating library call
 * is made. */
int semax_reduce_noalloc(int64_t count, const void *a, int a_prec, const void *b, int b_prec,
                         double *out, void *stream);

/* ---------------------------------------------------------------- errors */

const char *semax_strerror(int status);
/* cudaError_t of the last failing CUDA call made by libsemax on this thread. */
int semax_last_cuda_error(void);

/* Diagnostic: the FMA pipe's throughput, the peak that the plain FP64 and
 * FP32 kernels are graded against.  Launches `blocks` blocks of 256 threads,
 * each thread running 4 (FP64, prec = SEMAX_F64) or 8 (FP32, SEMAX_F32)
 * independent chains of `iters` (a multiple of 4, else SEMAX_EINVAL)
 * dependent fused multiply-adds and storing one value per thread in `sink`
 * (device, blocks * 256 elements of that type); *flops (host) receives the
 * floating-point operations the launch performs (an FMA counts 2).  Time it with events on `stream`.  The paper
 * has no counterpart; this measures the machine. */
int semax_fma_probe(int prec, int blocks, int iters, void *sink, double *flops, void *stream);

/* Diagnostic: the number of polls the first staging wait of each element in
 * the tensor-core kernels (sem_ax_f64tc and its variants) makes before it
 * gives up, for launches queued after this call from any host thread;
 * polls < 0 restores the default (2^20).  Launches already queued or
 * captured into a graph keep the limit they were made with.  polls = 0
 * makes every such wait give up at once, which drives the timeout path of
 * sem_ax_f64tc_status on ordinary inputs: the CTA's copies are still
 * drained by the second wait, which keeps the default limit.  The paper has
 * no counterpart; this exists to test the status reporting. */
int semax_set_wait_polls(int polls);

#ifdef __cplusplus
}
#endif

#endif /* SEMAX_H */
