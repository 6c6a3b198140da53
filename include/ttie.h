/*
 * ttie.h -- C ABI of the GB300 triangle-triangle intersection energy (TTIE) library.
 *
 * The library evaluates, for a triangle mesh, the energy of "Differentiable 3D
 * Triangle-Triangle Intersection Energy" (arXiv 2606.06511) and drives the mesh
 * towards an intersection-free state with an inexact Newton method:
 *
 *   ttie_build_bvh    broad phase: candidate triangle pairs (LBVH or brute force)
 *   ttie_eval_pairs   narrow phase + energy: Möller reduction to the intervals
 *                     I_a, I_b, the Minkowski interval I_c (Eq. 1), the energy
 *                     T = (t_c^0 t_c^1)^2 (Eq. 2), its gradient (Eq. 3) and the
 *                     inexact Hessian (Eq. 4) made PSD by its eigen-analysis (§1.1)
 *   ttie_assemble     3x3 block-CSR Hessian and per-vertex gradient
 *   ttie_newton_step  one inexact Newton iteration (PCG + backtracking line search)
 *   ttie_solve        Newton iterations until no pair intersects
 *
 * Conventions for every call:
 *   - Pointers named d_* are CUDA device pointers on the context's device;
 *     pointers without the prefix are host pointers.  Caller-owned buffers are
 *     only borrowed for the duration of the call.
 *   - All work is enqueued on the context's stream.  Calls that return host
 *     values synchronise that stream.
 *   - Every call returns a ttie_status.  Arguments are checked before anything
 *     is launched; on error nothing of the caller's memory has been written
 *     unless stated.  ttie_last_error(ctx) describes the last failure.
 *   - Nothing aborts, traps or waits without a bound.
 *   - A context is not thread-safe; use one per host thread.
 */
#ifndef TTIE_H
#define TTIE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    TTIE_OK = 0,
    TTIE_ERR_INVALID = 1,        /* bad argument (null pointer, size, index out of range) */
    TTIE_ERR_CUDA = 2,           /* a CUDA runtime call failed */
    TTIE_ERR_OOM = 3,            /* a device allocation failed */
    TTIE_ERR_CAPACITY = 4,       /* a bounded structure overflowed (BVH stack, max_candidates) */
    TTIE_ERR_NONFINITE = 5,      /* NaN or Inf in positions, energy or solver residual */
    TTIE_ERR_NOT_CONVERGED = 6,  /* iteration limit reached */
    TTIE_ERR_STATE = 7           /* calls made out of order (e.g. eval before build) */
} ttie_status;

/* Arithmetic of the per-pair evaluation.
 * TTIE_F32: positions float32, FP32 evaluation; every sign that decides the
 *           intersection test is certified (FP32 filter -> FP64 -> exact).
 * TTIE_F64: positions float64, FP64 evaluation, same certified signs.        */
typedef enum { TTIE_F32 = 0, TTIE_F64 = 1 } ttie_precision;

/* Which triangle pairs are considered.  Topologically adjacent pairs (sharing a
 * vertex index) are always excluded (§1).                                    */
typedef enum {
    TTIE_PAIRS_SELF = 0,         /* every non-adjacent pair i<j                   */
    TTIE_PAIRS_INTER_GROUP = 1,  /* only pairs with group[i] != group[j]          */
    TTIE_PAIRS_INTRA_GROUP = 2   /* only pairs with group[i] == group[j]          */
} ttie_pair_mode;

/* OR-ed into pair_mode: enumerate every pair of the mode instead of the LBVH
 * candidates (no bounding-box test). */
#define TTIE_PAIRS_BRUTE 4

/* OR-ed into pair_mode: candidates from a uniform spatial hash grid (the broad phase §1.2
 * names) instead of the LBVH; the same candidate set (closed box overlap, no shared vertex,
 * i < j), in another deterministic order.  Not used by the batched-instance solve. */
#define TTIE_PAIRS_HASH 8

/* PSD projection of the Eq. 4 Hessian (eigen-analysis of §1.1).
 * PER_PART:   parts 1 and 2 kept, part 3 keeps its non-negative eigenpair.
 * DROP_CROSS: parts 1 and 2 only.
 * WHOLE:      the sum of the three parts with its negative eigenvalue set to
 *             zero (rank one: Eq. 4 has one positive and one negative
 *             eigenvalue on every intersecting pair).                       */
typedef enum { TTIE_PSD_PER_PART = 0, TTIE_PSD_DROP_CROSS = 1, TTIE_PSD_WHOLE = 2 } ttie_psd_mode;

typedef struct {
    int precision;        /* ttie_precision                                        */
    int pair_mode;        /* ttie_pair_mode, optionally | TTIE_PAIRS_BRUTE          */
    int psd_mode;         /* ttie_psd_mode                                         */
    double tc_scale;      /* t_c = tc_scale * (Eq. 1); 1.0 = Eq. 1, 0.5 = appendix */
    double mu_rel;        /* Newton regulariser: mu = mu_rel * mean diag(H+)       */
    double pcg_rtol;      /* PCG stops at |r| <= pcg_rtol |r0|                     */
    int pcg_max_it;
    int newton_max_it;
    int ls_max_halvings;  /* line search tries 1+push_eta, 1, 1/2, ... 2^-this      */
    double armijo_c;
    double push_eta;      /* first trial step 1 + push_eta (overshoot past touching) */
    int exact_only;       /* test switch: 1 decides every sign with exact arithmetic
                             (float32 points in 256-bit integers where their span fits,
                             else expansions), 2 with expansion arithmetic only         */
    int profile;          /* record per-stage GPU times in ttie_step_info          */
    double max_step;      /* Newton step cap: largest vertex move per iteration, in
                             mean edge lengths of the mesh (0 = no cap)            */
    int64_t max_candidates; /* cap on a candidate list (0 = 64 F + 1e6); a larger
                             list is refused with TTIE_ERR_CAPACITY               */
    int inst_threads;     /* batched instances: threads per instance block (128, 256,
                             512 or 1024); 0 = chosen per size bucket by timing the
                             candidates on the first step (results do not depend on it) */
    int test_withhold;    /* test switch (0 in use): block 0 of the shared-memory PCG never
                             publishes its partial sums, so every block's bounded wait for
                             them runs out (about a second) and the call returns
                             TTIE_ERR_CUDA with the context still usable               */
    int pcg_precond;      /* preconditioner (TTIE_PCG_*) of the shared-memory PCG and of
                             the batched-instance PCG (AUTO there: Chebyshev for the
                             instances whose rows fit a block's shared memory); the
                             global-memory and streamed PCGs use 3x3 block Jacobi      */
    int pcg_cheb_degree;  /* TTIE_PCG_CHEBYSHEV: degree k of the polynomial, 1..8 (0 = 2) */
    int traversal_mode;   /* TTIE_TRAVERSAL_*: how the LBVH walk lists candidates; both give
                             the same list in the same order                              */
    int ls_rule;          /* TTIE_LS_*: which line-search trials are accepted            */
    double push_eta_max;  /* adaptive overshoot (TTIE_LS_FEWER): when a step took the
                             overshoot trial 1 + eta and left as many intersecting pairs,
                             eta doubles for the next step, up to this (<= push_eta: no
                             growth); it returns to push_eta when a step lowers the count.
                             Not used by batched instances.                           */
    int pcg_kernel;       /* TTIE_PCG_KERNEL_*: which kernels run the PCG                */
} ttie_params;

/* PCG kernels (same recurrence, same stopping test; results agree to rounding).
 * AUTO:     RESIDENT when every solver block's rows fit its shared memory (with the matrix
 *           rows too when they fit, else in the lean layout that reads them from global
 *           memory), else STREAMED.
 * RESIDENT: one cooperative launch, each block's rows (and, when they fit, matrix rows) held in
 *           shared memory for the whole solve, blocks exchanging through tagged words.
 * STREAMED: two kernels per iteration replayed from a CUDA graph, the matrix streamed from
 *           global memory and u read through the read-only path; block Jacobi only (with
 *           pcg_precond CHEBYSHEV the resident kernel runs).
 * RESIDENT_UNCACHED: RESIDENT with the matrix rows read from global memory on every product
 *           even where they would fit shared memory (the product that systems too large for
 *           shared memory get, on any system).                                           */
enum {
    TTIE_PCG_KERNEL_AUTO = 0,
    TTIE_PCG_KERNEL_RESIDENT = 1,
    TTIE_PCG_KERNEL_STREAMED = 2,
    TTIE_PCG_KERNEL_RESIDENT_UNCACHED = 3
};

/* Line-search acceptance (the paper states no line search; these are readings of its inexact
 * Newton route).  E: energy, n: intersecting pairs, at x and at the trial x + a d.
 * ARMIJO: accept when Armijo's condition holds or no pair intersects at the trial.
 * FEWER:  ARMIJO, or fewer intersecting pairs with E not above E(x); with the adaptive
 *         overshoot of push_eta_max.
 * With either rule the last (smallest) trial of the ladder is taken when none is accepted.  */
enum { TTIE_LS_ARMIJO = 0, TTIE_LS_FEWER = 1 };

/* LBVH traversal (one thread per leaf, depth-first walk over rope links).
 * TWO_WALKS: a counting walk from the root keeps each leaf's first 16 partners; leaves with
 *            more walk again to write them.
 * ONE_WALK:  the walk starts after leaf lo - 1 of the leaf's window (its rope) and stops past
 *            the window; partners past the first 16 go to 32-pair chunks taken from a pool
 *            and linked per leaf, then copied in walk order.  When the pool is exhausted the
 *            second walk writes those leaves instead.                                       */
enum { TTIE_TRAVERSAL_TWO_WALKS = 0, TTIE_TRAVERSAL_ONE_WALK = 1 };


/* PCG preconditioners.
 * BLOCK_JACOBI: M^-1 = D^-1, the inverses of the 3x3 diagonal blocks of H+ + mu I.
 * CHEBYSHEV:    after 6 block-Jacobi iterations, lambda_max of D^-1 (H+ + mu I) is
 *               estimated from the Lanczos tridiagonal of those iterations' alpha and beta
 *               (times 1.1), and CG restarts from the current x with M^-1 = p_k(D^-1 A) D^-1,
 *               the Chebyshev iteration polynomial of degree k on [lambda_max / 10,
 *               lambda_max]: k extra products per iteration, no extra reduction.  An even k
 *               keeps M^-1 positive definite whatever the estimate; with an odd k a
 *               lambda_max above the estimate can make it indefinite, which ends the solve
 *               at the breakdown test with the iterate so far.                           */
enum { TTIE_PCG_BLOCK_JACOBI = 0, TTIE_PCG_CHEBYSHEV = 1, TTIE_PCG_AUTO = 2 };
/* AUTO: CHEBYSHEV whenever the block-resident kernel holds the system's rows (with their
 * matrix rows in shared memory, or streaming them from global memory in the lean layout): it
 * needs about as many products as block Jacobi but a third of the reductions, and reaches the
 * tolerance where block Jacobi stops at the iteration cap (the 2,097,152-triangle noisy
 * sphere's first Newton system: 68 iterations to 1e-3 against 200 capped at 3.7e-3, 15.5
 * against 15.0 ms); BLOCK_JACOBI in the global-memory and streamed kernels. */

typedef struct ttie_ctx ttie_ctx;

/* Fills *p with the defaults: F32, SELF, PER_PART, tc_scale 1, mu_rel 1e-3,
 * pcg_rtol 1e-3, pcg_max_it 200, newton_max_it 200, ls_max_halvings 20,
 * armijo_c 1e-4, push_eta 0.5, exact_only 0, profile 0, max_step 1,
 * max_candidates 0, inst_threads 0, test_withhold 0, pcg_precond AUTO,
 * pcg_cheb_degree 0, traversal_mode ONE_WALK, ls_rule ARMIJO,
 * push_eta_max 1.5, pcg_kernel AUTO. */
void ttie_default_params(ttie_params *p);

/* Creates a context on the current CUDA device.  stream: a cudaStream_t or NULL
 * for the legacy default stream.  The context owns every internal buffer (pair
 * lists, BVH, BSR, solver vectors); they grow on demand. */
ttie_status ttie_create(ttie_ctx **out, const ttie_params *p, void *stream);
void ttie_destroy(ttie_ctx *ctx);
/* Message of the last failed call on ctx (never NULL; valid until the next call). */
const char *ttie_last_error(const ttie_ctx *ctx);
ttie_status ttie_set_params(ttie_ctx *ctx, const ttie_params *p);

/*
 * Broad phase (§1.2 uses a spatial structure "to eliminate redundant
 * computations"; this library uses an LBVH).
 *   d_x      V x x_stride positions (float for F32, double for F64), x_stride 3 or 4
 *   d_tri    F x 3 int32 vertex indices in [0, V)
 *   d_group  F int32 group ids in [0, 2^20) or NULL (required by the group modes)
 *   n_candidates (host out) number of candidate pairs: non-adjacent pairs i<j of
 *            the pair mode whose closed axis-aligned bounding boxes overlap
 *            (every pair of the mode with TTIE_PAIRS_BRUTE).
 * Records the topology (tri, group, V) in the context for the calls below.
 * Errors: INVALID (sizes, indices), NONFINITE (positions), CAPACITY, OOM, CUDA. */
ttie_status ttie_build_bvh(ttie_ctx *ctx, const void *d_x, int64_t V, int x_stride,
                           const int32_t *d_tri, int64_t F, const int32_t *d_group,
                           int64_t *n_candidates);

/* Evaluation flags. */
#define TTIE_EVAL_E 1u   /* energy sum T (Eq. 2)                                  */
#define TTIE_EVAL_G 2u   /* gradient (Eq. 3), scattered per vertex                 */
#define TTIE_EVAL_H 4u   /* per-pair PSD Hessian factors (Eq. 4, §1.1) for ttie_assemble */

/*
 * Narrow phase and energy over the candidates of the last ttie_build_bvh, at
 * positions d_x (same V, stride and dtype as the build; may differ in value).
 *   energy   (host out, nullable) sum over intersecting pairs of T, FP64 sum
 *   n_active (host out, nullable) number of intersecting pairs: both triangles
 *            straddle the other's plane and 0 lies strictly inside I_c (§1)
 *   d_grad   (device out, nullable) V x 3 gradient of the energy (same dtype as
 *            the positions); rows of vertices in no intersecting pair are zero.
 * Errors: STATE (no build), INVALID, NONFINITE, OOM, CUDA.
 */
ttie_status ttie_eval_pairs(ttie_ctx *ctx, const void *d_x, unsigned what, double *energy,
                            int64_t *n_active, void *d_grad);

/* Device views into context memory, valid until the next mutating call. */
typedef struct {
    int64_t n_rows;              /* active vertices (in at least one intersecting pair) */
    int64_t nnzb;                /* stored 3x3 blocks                                    */
    const int32_t *row_ptr;      /* n_rows + 1                                          */
    const int32_t *col_idx;      /* nnzb, compact row ids, ascending within a row        */
    const void *val;             /* nnzb x 9, row-major 3x3 blocks of H+ (positions' dtype) */
    const int32_t *vertex_of_row;/* n_rows, ascending global vertex ids                  */
    const void *grad;            /* n_rows x 3 assembled gradient (positions' dtype)      */
} ttie_bsr_view;

/*
 * Assembles the PSD Hessian H+ and the gradient of the last ttie_eval_pairs
 * (which must have included TTIE_EVAL_H) over the active vertices.  Each pair
 * contributes its gradient (Eq. 3) and its Eq. 4 Hessian projected as §1.1's
 * eigen-analysis prescribes (params.psd_mode); the Newton system of the inexact
 * Newton route (abstract, §1.2) is the sum over pairs.  The block
 * pattern is the union of the 6x6 vertex blocks of the intersecting pairs; the
 * sums run in a fixed order (sorted keys), so the result is deterministic.
 * Errors: STATE, OOM, CUDA.
 */
ttie_status ttie_assemble(ttie_ctx *ctx, ttie_bsr_view *out);

/* Copies the last assembled system into caller-owned device buffers sized from the
 * ttie_assemble view: row_ptr n_rows + 1, col_idx nnzb, val nnzb x 9,
 * vertex_of_row n_rows, grad n_rows x 3.  Any pointer may be NULL.
 * Errors: STATE (nothing assembled), CUDA. */
ttie_status ttie_copy_bsr(ttie_ctx *ctx, int32_t *d_row_ptr, int32_t *d_col_idx, void *d_val,
                         int32_t *d_vertex_of_row, void *d_grad);

/*
 * Preconditioned conjugate gradients on the last assembled system:
 * (H+ + mu I) d = rhs with mu = mu_rel * mean diag(H+), block-Jacobi (3x3)
 * preconditioner, FP64 dot products.  d_rhs, d_out: n_rows x 3 device arrays
 * of the positions' dtype.  Stops at |r| <= rtol |rhs| or max_it iterations.
 * iters, rel_residual: host outs (nullable).
 */
ttie_status ttie_pcg(ttie_ctx *ctx, const void *d_rhs, void *d_out, double rtol, int max_it,
                     int *iters, double *rel_residual);

/*
 * Hessian-vector product of the energy at the positions of the last ttie_eval_pairs (which
 * must have included TTIE_EVAL_G or TTIE_EVAL_H), restricted to its intersecting pairs:
 *   exact = 1: the full Hessian of sum T (Eq. 2) applied to v, by forward-mode
 *              differentiation of the per-pair gradient (Eq. 3) along v (dual numbers, the
 *              way Appendix A obtains derivatives); d_x must be the evaluated positions,
 *              V x x_stride as given to ttie_build_bvh (borrowed for the call).
 *   exact = 0: the PSD Hessian H+ (Eq. 4 projected per §1.1) as assembled by ttie_assemble
 *              (assembled here if needed); d_x is ignored.
 * d_v, d_out: V x 3 device arrays of the positions' dtype; rows of vertices in no
 * intersecting pair are zero.  Per-vertex sums run in a fixed order (deterministic).
 * Errors: STATE, INVALID, NONFINITE, CUDA.
 */
ttie_status ttie_hvp(ttie_ctx *ctx, const void *d_x, const void *d_v, void *d_out, int exact);

/*
 * Gradients of t_c^0 and t_c^1 of every intersecting pair of the last ttie_eval_pairs, by
 * forward-mode dual numbers in FP64 (the route Appendix A takes to the derivatives; an
 * independent check of the analytic chain rule that ttie_eval_pairs uses).  d_x: the evaluated
 * positions, V x x_stride as given to ttie_build_bvh.  d_out: n_active x 36 doubles (device),
 * [d t_c^0 (18), d t_c^1 (18)] per pair in the order of ttie_get_active, coordinates of
 * [A0 A1 A2 B0 B1 B2].  Errors: STATE (no evaluation), INVALID (null pointer), CUDA.
 */
ttie_status ttie_dual_gradients(ttie_ctx *ctx, const void *d_x, double *d_out);

typedef struct {
    int64_t n_candidates;        /* candidate pairs at x                              */
    int64_t n_active;            /* intersecting pairs at x                           */
    int64_t n_rows, nnzb;        /* assembled system size                             */
    double energy;               /* E(x)                                               */
    double energy_new;           /* E at the accepted point                           */
    int64_t n_active_new;        /* intersecting pairs at the accepted point          */
    double alpha;                /* accepted step length                               */
    double grad_dot_dir;         /* g . d                                              */
    int pcg_iters;
    double pcg_rel_residual;
    int ls_trials;               /* trial steps evaluated                              */
    int64_t n_candidates_swept;  /* candidates of the line-search sweep [x, x+a_max d] */
    float ms_build, ms_eval, ms_assemble, ms_pcg, ms_line_search;  /* if params.profile */
    float ms_classify;           /* classification kernel of the evaluation at x (profile) */
    float ms_pcg_kernel;         /* persistent PCG kernel (profile)                          */
    int64_t pcg_block_iters;     /* sum over the PCG's products of the 3x3 blocks multiplied
                                    (one product per iteration; k + 1 with the Chebyshev
                                    preconditioner after its restart)                      */
    int64_t pcg_row_iters;       /* sum over the PCG's products of the rows updated           */
    double energy_elastic;       /* elastic term's part of energy (0 without one)             */
    int pcg_kernel;              /* the PCG kernels that ran: TTIE_PCG_KERNEL_RESIDENT,
                                    _STREAMED or _RESIDENT_UNCACHED; 0 when no PCG ran or with
                                    batched instances (their own solver)                      */
    int64_t stage_launches[5];   /* kernels launched by the step per stage: build, evaluation,
                                    assembly, PCG, line search (graph replays count each of
                                    their kernels)                                            */
    int inst_threads;            /* batched instances: the PCG schedule that ran (threads per
                                    block, blocks per SM requested, instance order 0 largest
                                    first / 1 as numbered); 0 otherwise                        */
    int inst_blocks_per_sm;
    int inst_order;
} ttie_step_info;

/*
 * Elastic term of the quasi-static simulation (Fig. 2: a simulation with the energy that
 * evolves from an invalid state to a valid one; the paper does not state its elastic model,
 * so this is a mass-spring term):
 *   E_el(x) = sum_e k_edge/2 (|x_i - x_j| - rest_e)^2 + sum_a k_anchor/2 |x_a - target_a|^2.
 * Once set, ttie_newton_step and ttie_solve minimise E_el + sum T: the gradient and the
 * PSD-projected Hessian of both terms are assembled into one block-CSR system whose rows are
 * the vertices of intersecting pairs, springs and anchors (mu from its mean diagonal), and
 * the line search tests E_el + sum T.  A step at a state with no intersecting pair does
 * nothing (the state is valid), so ttie_solve stops there as without the term.
 * ttie_eval_pairs and ttie_assemble stay the pairs' alone.  Not with batched instances
 * (pair_mode TTIE_PAIRS_INTRA_GROUP over an LBVH).
 */
typedef struct {
    const int32_t *edges;        /* device, n_edges x 2 vertex ids, distinct, each in [0, V) */
    const void *rest;            /* device, n_edges rest lengths, float or double as the
                                    context's precision                                    */
    int64_t n_edges;
    double k_edge;               /* spring stiffness, >= 0                                  */
    const int32_t *anchors;      /* device, n_anchors vertex ids in [0, V); NULL if none    */
    const void *targets;         /* device, n_anchors x 3 anchor points (context precision) */
    int64_t n_anchors;
    double k_anchor;             /* anchor stiffness, >= 0                                  */
} ttie_elastic;

/*
 * Sets (or, with el NULL or no springs and no anchors, removes) the elastic term for the mesh
 * of the last ttie_build_bvh.  The arrays are copied into the context during the call (stream
 * ordered), so the caller's buffers may be reused after it.  Errors: STATE (no mesh built),
 * INVALID (negative counts or stiffness, null arrays with nonzero counts, a vertex id out of
 * range or a spring with equal endpoints, batched-instance mode), OOM, CUDA.  A later
 * ttie_build_bvh with another vertex count removes the term.
 */
ttie_status ttie_set_elastic(ttie_ctx *ctx, const ttie_elastic *el);

/*
 * One iteration of the inexact Newton method the abstract and §1.2 name for
 * driving a mesh to an intersection-free state ("GPU-based inexact Newton"; its
 * tolerances, regulariser and line search are not stated there and are this
 * library's parameters) on the mesh recorded by ttie_build_bvh:
 * candidates and evaluation at x, assembly, PCG for d, then a backtracking line
 * search over the trial steps 1+push_eta, 1, 1/2, ... on candidates from the
 * boxes swept between x and x + (1+push_eta) d; a trial is accepted when it
 * meets Armijo's condition or leaves no intersecting pair.  d_x_inout is
 * updated in place (unchanged when x has no intersecting pair).
 */
/*
 * With pair_mode TTIE_PAIRS_INTRA_GROUP (LBVH) every group is an independent problem and one
 * call steps all of them at once but independently: one PCG per group (one thread block per
 * group, in a single launch; mu and the stopping test per group), the step cap per group
 * (max_step x the group's mean edge length at ttie_build_bvh), and the line search per group
 * (each group takes the first trial of the shared ladder that meets its own Armijo test or
 * leaves it without intersecting pairs).  Every vertex must belong to one group and each
 * group's vertices must be numbered contiguously (else TTIE_ERR_INVALID).  In this mode info
 * reports alpha = the smallest accepted step, pcg_iters and pcg_rel_residual = the largest
 * over the groups, grad_dot_dir = the sum over the groups.
 */
ttie_status ttie_newton_step(ttie_ctx *ctx, void *d_x_inout, ttie_step_info *info);

typedef struct {
    int iterations;
    int converged;               /* 1 when the final x has no intersecting pair        */
    int64_t n_active_initial, n_active_final;
    double energy_initial, energy_final;
    double seconds;              /* wall time of the solve                              */
} ttie_solve_info;

/* Newton iterations until no pair intersects or params.newton_max_it: the paper's
 * use of the energy, from an intersecting start to a valid state (abstract, §1.2,
 * Fig. 2); "intersects" is the exact test of ttie_eval_pairs (§1).
 * Returns NOT_CONVERGED (with d_x_inout holding the last iterate) at the limit. */
ttie_status ttie_solve(ttie_ctx *ctx, void *d_x_inout, ttie_solve_info *info);

/* ---- inspection (tests, tools) ------------------------------------------------ */

/* Copies the candidate pairs of the last build (n x 2 int32, i<j, deterministic
 * order) into d_out (capacity pairs).  *n receives the count. */
ttie_status ttie_get_candidates(ttie_ctx *ctx, int32_t *d_out, int64_t capacity, int64_t *n);

/* Copies the intersecting pairs of the last ttie_eval_pairs in candidate order:
 * d_pairs n x 2 int32 (nullable); d_tc n x 2 (t_c^0, t_c^1) and d_dtc n x 36
 * (gradients of t_c^0 then t_c^1 w.r.t. [A0 A1 A2 B0 B1 B2], A = first triangle)
 * in the positions' dtype, both nullable (require TTIE_EVAL_G or TTIE_EVAL_H). */
ttie_status ttie_get_active(ttie_ctx *ctx, int32_t *d_pairs, void *d_tc, void *d_dtc,
                            int64_t capacity, int64_t *n);

/* Copies the last Newton direction (V x 3, positions' dtype) into d_out. */
ttie_status ttie_get_direction(ttie_ctx *ctx, void *d_out);

/* Counters of the last ttie_eval_pairs (host out array of 3): signs decided by the FP32
 * filter in the pass over all candidates (FP32 positions); then, in the pass over the pairs
 * that left a sign undecided, signs decided by the second stage (FP32 positions: the exact
 * sign in 128/256-bit integers where the coordinates' span fits; otherwise the FP64 filter
 * and its zero certificates); then signs decided by the last pass's exact arithmetic. */
ttie_status ttie_get_filter_stats(ttie_ctx *ctx, int64_t *out3);

/* sizeof of the public structs, so that a binding can check its layouts against this build:
 * out5 (host, 5 entries) = ttie_params, ttie_bsr_view, ttie_step_info, ttie_elastic,
 * ttie_solve_info.  Needs no GPU and no context. */
void ttie_struct_sizes(int64_t *out5);

/* ---- solve without allocating -------------------------------------------------- */

/* Largest system ttie_pcg_static accepts (rows of 3x3 blocks). */
#define TTIE_PCG_STATIC_MAX_ROWS 16384

/*
 * The block-Jacobi PCG solve of ttie_pcg, (H + mu I) d = rhs on a 3x3 block-CSR matrix
 * (layout as ttie_bsr_view: row_ptr n_rows + 1, col_idx nnzb ascending per row, val
 * nnzb x 9 row-major, float32), for callers that cannot allocate device memory: a host
 * whose device-memory budget is planned up front (a plugin or embedded runtime that
 * hands out no cudaMalloc), or a loop that cannot afford the device-wide
 * synchronisation an allocation implies.  It needs no context and allocates nothing:
 * no cudaMalloc, cudaFree or allocating library call.  The paper has no counterpart;
 * this is a service of the library.
 *
 * All inputs and the output d_out (n_rows x 3) are the caller's device buffers.  The
 * work vectors live in one static device array sized for TTIE_PCG_STATIC_MAX_ROWS rows
 * (about 1.4 MB), which every GPU that loads the library holds until the process exits.
 * n_rows beyond that limit is refused with TTIE_ERR_INVALID before any work.
 *
 * The first call on a device looks up the array's device address (once per device, with
 * that device current).  Every call reuses the same array and clears the parts that must
 * start at zero; two calls whose work overlaps on the GPU (other streams, other host
 * threads, the same device) race on it, so serialise them.  Work is enqueued on `stream`
 * (NULL: legacy default stream); every call copies host values to the device and
 * synchronises that stream before returning iters and rel_residual (host outs, nullable),
 * so it cannot be called on a stream that is being captured into a CUDA graph.
 * Errors: INVALID (arguments; also, in a self-checking build, arrays that fail its bounds
 * checks), CUDA (a runtime call failed, or the solver's bounded grid-barrier wait ran out),
 * NONFINITE.
 */
ttie_status ttie_pcg_static(const int32_t *d_row_ptr, const int32_t *d_col_idx, const float *d_val,
                            int64_t n_rows, double mu, const float *d_rhs, float *d_out, double rtol,
                            int max_it, void *stream, int *iters, double *rel_residual);

/* Number of CUDA kernels the context has launched since ttie_create (host out). */
ttie_status ttie_get_launch_count(ttie_ctx *ctx, int64_t *n);

#ifdef __cplusplus
}
#endif

#endif /* TTIE_H */
