/*
 * fe_hotpath.h -- C ABI of the GB300 implicit finite-element time step.
 *
 * The library implements the hot path of Zeng & Courtecuisse, "Efficient
 * parallelization strategy for real-time FE simulations" (arXiv 2306.05893):
 *
 *   per-element hyperelastic force and tangent (Section 3.1)
 *   -> fast assembly of A and b through a triplet->CSR map C computed once
 *      per topology (Section 4, Algorithm 1, Table "build pattern")
 *   -> preconditioned CG on A a = b with
 *        A = (1 + h alpha) M + h (beta + h) K          (Eq. "dynamic equation2")
 *        b = p - f - (alpha M + (beta + h) K) v        (Eq. "dynamic equation1",
 *                                                       Rayleigh B = alpha M + beta K)
 *      and a lagged LDL^T preconditioner P = A_t = L D L^T
 *      (Eq. "asynchronous preconditioner", Section 3.3) applied level by level
 *      over nested-dissection sub-domains (Section 6.1, Eq. "regional problem")
 *   -> backward Euler v+ = v + h a, q+ = q + h v+     (Eq. "implicit integration").
 *
 * Conventions shared by every call:
 *   - every call returns an fe_status; none throws or aborts;
 *   - a message for the last failure of a context is in fe_last_error();
 *   - after a non-zero status other than FE_ERR_CUDA the context stays usable;
 *   - DOF numbering: DOF = 3 * node + component, node-major;
 *   - the caller owns every buffer it passes; fe_create copies all inputs;
 *   - "host or device" buffers: when fe_options.device_ptrs is 1 the state
 *     and force pointers of fe_set_state / fe_get_state / fe_step /
 *     fe_element_eval / fe_assemble are device pointers used on
 *     fe_options.stream; otherwise they are host pointers and the call copies
 *     through the library's own pinned staging buffers.
 */
#ifndef FE_HOTPATH_H
#define FE_HOTPATH_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct fe_ctx fe_ctx; /* opaque, owned by the library */

typedef enum {
  FE_OK = 0,
  FE_ERR_ARG = 1,             /* invalid argument (sizes, pointers, ids)       */
  FE_ERR_CUDA = 2,            /* CUDA runtime error; context must be destroyed */
  FE_ERR_OOM = 3,             /* device or host allocation failed              */
  FE_ERR_PATTERN_CHANGED = 4, /* topology differs from the one the map C holds */
  FE_ERR_NOT_CONVERGED = 5,   /* PCG hit max_iters                             */
  FE_ERR_BREAKDOWN = 6,       /* p^T A p <= 0 in CG or an LDL^T pivot <= 0     */
  FE_ERR_INVERTED = 7,        /* an element has det F <= 0                     */
  FE_ERR_TIMEOUT = 8,         /* the lagged factor was not ready in time       */
  FE_ERR_STATE = 9            /* calls out of order (e.g. step before pattern) */
} fe_status;

enum { FE_TET4 = 0, FE_HEX8 = 1 };
enum { FE_SVK = 0, FE_NEOHOOKE = 1, FE_MOONEY_RIVLIN = 2, FE_COROTATIONAL = 3 };
enum { FE_FP64 = 0, FE_MIXED = 1 };

/* Mesh (Section 3.1).  Local node order of a hex: a = dx + 2 dy + 4 dz.
 * rest_xyz [n_nodes * 3] (host), conn [n_elems * npe] (host, npe = 4 or 8),
 * fixed_nodes [n_fixed] (host): nodes held by projective constraints
 * (Section 5.1): their rows and columns are cleared with 1 on the diagonal. */
typedef struct {
  int32_t elem_type;
  int64_t n_nodes;
  int64_t n_elems;
  const double *rest_xyz;
  const int32_t *conn;
  int64_t n_fixed;
  const int32_t *fixed_nodes;
} fe_mesh;

/* Material (Section 3.1): params are (mu, lambda, unused) for St Venant-
 * Kirchhoff, neo-Hookean and co-rotational linear elasticity, (C10, C01,
 * kappa) for Mooney-Rivlin; one triple for the whole mesh, or one per element
 * when per_element = 1 ([n_elems * 3], element-major).  rho is the mass
 * density.  Co-rotational elements (Eq. "eqmodel": int B^T D B rotated by the
 * polar decomposition of the element's mean deformation gradient) have no
 * energy and a tangent without the rotation's derivative, so fe_adjoint
 * refuses them (and keep_checkpoints with them). */
typedef struct {
  int32_t model;
  double rho;
  const double *params;
  int32_t per_element;
} fe_material;

typedef struct {
  int32_t precision;      /* FE_FP64: all FP64.  FE_MIXED: FP32 element
                             tangents K_e, inner PCG (SpMV, vectors), factor
                             and triangular solves; FP64-accurate element
                             forces f_e, assembly sums and residual in
                             double-float (pairs of floats, about 2^-46 per
                             operation: A is kept as float pairs for the
                             residual and in FP32 for the inner solves), FP64
                             right-hand side b, dot products, and pivots summed
                             in double-float; iterative refinement to tol.   */
  double tol;             /* stop when ||b - A a||_2 <= tol ||b||_2           */
  int32_t max_iters;      /* PCG iterations per step (all refinement sweeps)  */
  int32_t refactor_every; /* R: factor A_s at steps s = 0 mod R on the side
                             stream; that factor preconditions steps
                             s+k .. s+k+R-1 (k = factor_lag); steps 0 .. k+R-1
                             use the factor of A_0, made synchronously at
                             step 0.  R = 1: the exact factor of the step's
                             own A every step (synchronous).                 */
  int32_t device_ptrs;    /* 1: state/force buffers are device pointers       */
  void *stream;           /* cudaStream_t for device_ptrs = 1 (NULL: the
                             library's own stream, created at the highest
                             priority).  The lagged factorisation runs on a
                             library stream at the lowest priority: a
                             caller's stream should have a higher one.      */
  int32_t keep_checkpoints; /* store (q_t, v_t) of every step for fe_adjoint  */
  int32_t nd_leaf_nodes;  /* nested-dissection leaf size in nodes (0: 64)     */
  double inner_tol;       /* FE_MIXED inner PCG tolerance per sweep (0: 1e-4) */
  double factor_timeout_s;/* how long the step that first uses a lagged
                             factor waits for it on the host before
                             returning FE_ERR_TIMEOUT (0: 30 s); a
                             synchronous factorisation (step 0, R = 1,
                             fe_factor_now) waits up to max(this, 300 s)     */
  int32_t use_graph;      /* 1: the PCG iterations run as a CUDA graph of
                             kGraphIters iterations, replayed until the
                             device-side convergence flag is set (one host
                             read per replay; iterations after convergence
                             exit at once, so results are bit-identical)      */
  int32_t profile_stages; /* 1: time every stage with CUDA events on its own
                             stream (read with fe_get_stage_times)          */
  int32_t newton_iters;   /* Newton iterations per step (0 or 1: the paper's
                             single linearisation).  Iteration k > 1 solves
                             A(q_k) d = p - f(q_k) - (alpha M + beta K(q_k)) v_k
                             - M a_k at q_k = q + h v + h^2 a_k, v_k = v + h a_k,
                             then a_{k+1} = a_k + d (lagged preconditioner).
                             Not combinable with keep_checkpoints.            */
  double newton_tol;      /* stop the iterations once ||d|| <= newton_tol ||a||
                             (0: run all newton_iters)                        */
  int32_t factor_tf32;    /* FE_MIXED: 0 = the factor's trailing updates keep
                             FP32 accuracy (3xTF32 split on the tensor
                             cores), 1 = plain TF32 products (faster; a
                             coarser preconditioner, same final tolerance)   */
  int32_t precond_fp16;   /* FE_MIXED: 1 = the preconditioner applies a binary16
                             copy of Y (made from the FP32 factor once per
                             factorisation; entries rounded to nearest and
                             clamped to +-65504), halving the bytes each PCG
                             iteration streams; arithmetic stays FP32 and the
                             solve is still refined to tol in FP64.  The copy
                             keeps M^{-1} = Y^T D^{-1} Y symmetric positive
                             definite.  Ignored for FE_FP64.                  */
  int32_t contact_sweeps; /* projected Gauss-Seidel sweeps at most per step with
                             contacts (fe_set_contacts); default 200         */
  double contact_tol;     /* stop when a sweep changes no multiplier by more
                             than contact_tol * max |lambda|; default 1e-12  */
  int32_t factor_lag;     /* k, 1 <= k <= R (0: 1): steps between the
                             snapshot of A_s and the first step its factor
                             preconditions (Eq. "asynchronous
                             preconditioner": the factor becomes available
                             several steps after the matrix it inverts).  A
                             larger k gives the side stream k steps of the
                             main stream's time to finish the factorisation,
                             at the price of an older preconditioner.  The
                             schedule is fixed, so iteration counts do not
                             depend on timing.  Ignored when R = 1.          */
  double dep_wait_s;      /* limit of every bounded dependency wait inside
                             the preconditioner application's kernels
                             (0: 1 s); a wait that runs out stops the
                             application and the call reports FE_ERR_TIMEOUT */
  int32_t element_fp64;   /* FE_MIXED only: 1 = the element kernel computes
                             and stores the tangents K_e and forces in FP64
                             too, so the FP64-accurate copy of A carries the
                             FP64 path's sums and the refined solution reaches
                             tol against the FP64 system; the inner PCG,
                             factor and solves stay
                             FP32 (0: FP32 tangents, see precision)          */
  int32_t warm_start;     /* 1: a step's PCG starts from the previous step's
                             acceleration instead of 0 (the stopping test
                             ||b - A a|| <= tol ||b|| is unchanged, so the
                             result differs from a cold start only within the
                             tolerance); fe_set_state resets the guess to 0.
                             Single meshes; batches start from 0.            */
  int32_t spmv_variant;   /* -1 (default): the first solve times the SpMV
                             variants on the assembled matrix and keeps the
                             fastest (batches: one kernel per size class).
                             0-3: the node-block kernel with 4, 8, 16 or 32
                             lanes per node; 4, 5: CSR with 8 or 16 threads
                             per row (for batches: every size class uses
                             that kernel).  Variants sum each row in a
                             different order, so runs that must agree bit
                             for bit across contexts fix one.                */
  double apply_sm_share;  /* 0 (default) to 0.9: while a lagged factorisation
                             is in flight, the preconditioner application's
                             persistent kernels launch this fraction fewer
                             CTAs, leaving room on the SMs for the factor's
                             kernels (the application is bound by its tree's
                             dependency chains more than by its CTA count).
                             The result does not depend on it.               */
  int32_t update_bf16;    /* FE_MIXED: 1 (default) applies each superpanel's
                             deferred trailing update (the rank-512 updates
                             of the rest of a front, the bulk of the factor's
                             flops) on the tensor cores with BF16 operands and
                             FP32 accumulation (tcgen05 kind::f16), read by
                             TMA from K-major BF16 copies of W = L D, L and
                             the pivot rows of Y that the panel and diagonal
                             kernels write beside their FP32 results; 0 keeps
                             them in the TF32 kernel (factor_tf32).  The
                             factor is a preconditioner: operands rounded to
                             BF16 (relative 2^-9) leave the PCG iteration
                             counts of the bench mesh unchanged, and the solve
                             is refined to tol in FP64 either way.  Ignored
                             for FE_FP64.                                    */
} fe_options;

typedef struct {
  int32_t iters;          /* PCG iterations of the step (all sweeps)          */
  int32_t refinements;    /* outer FP64 residual sweeps (FE_MIXED), else 1    */
  int32_t factor_age;     /* steps since the preconditioner's matrix          */
  double rel_residual;    /* final ||b - A a|| / ||b|| (FP64) of the last
                             linear solve                                     */
  int32_t newton;         /* Newton iterations done (1: the paper's step)      */
  double newton_correction; /* ||d|| / ||a|| of the last Newton correction    */
} fe_step_info;

/* Fills *opt with defaults: FP64, tol 1e-8, max_iters 1000, R = 1, host
 * pointers, no checkpoints. */
int fe_options_default(fe_options *opt);

/* Copies mesh, material, h, Rayleigh (alpha, beta) and options into a new
 * context (Section 3.2).  Touches no GPU.  *out is NULL on failure.
 * FE_ERR_ARG: a NULL or empty mesh, an unknown element type or model, a
 * node index out of range, h not finite and positive, rho not positive,
 * alpha or beta negative or not finite (Rayleigh damping B = alpha M +
 * beta K), or a non-finite rest coordinate or material parameter. */
int fe_create(const fe_mesh *mesh, const fe_material *mat, double h, double alpha,
              double beta, const fe_options *opt, fe_ctx **out);

/* Batched context: nb independent meshes (same element type and density,
 * any models) stepped together as one block-diagonal system.  Every stage is
 * one launch over all members (one element launch per material model); the
 * CG keeps per-member scalars, so member k converges on its own test
 * ||r_k|| <= tol ||b_k||.  Members are stored grouped by model: member
 * order, node offsets [nb+1] and element offsets [nb+1] of the concatenated
 * state come from fe_get_batch_layout; state and force vectors passed to
 * the other calls are concatenations in that order. */
int fe_create_batch(int32_t nb, const fe_mesh *meshes, const fe_material *mats, double h,
                    double alpha, double beta, const fe_options *opt, fe_ctx **out);
int fe_get_batch_layout(fe_ctx *ctx, int32_t *nb, const int32_t **member,
                        const int64_t **node_off, const int64_t **elem_off);
/* Per-member PCG iterations and final relative residuals of the last step
 * ([nb] each, stored order; NULL to skip). */
int fe_get_batch_stats(fe_ctx *ctx, int32_t *iters, double *rel_residual);

/* Setup once per topology (Section 4.2, Table "build pattern"; Section 5.1;
 * Section 6.1): the triplet (row, col) stream in fill order
 *   t = ((e * npe + a) * npe + b) * 9 + 3 i + k   (value K_e[3a+i][3b+k]),
 * the CSR pattern that two transposes of that stream give, with fixed
 * rows/columns skipped (built row by row on the host's cores), the map C
 * (triplet -> CSR slot, -1 when dropped) and its inverse (per slot, its
 * triplets ascending), the consistent mass on that pattern, a nested-
 * dissection ordering of the free nodes, the multifrontal symbolic analysis
 * and the level schedule.  Host work only; device buffers are created at the
 * first call that needs the GPU.  Must precede every call below.
 * FE_ERR_ARG: a free node that belongs to no element (its row would be
 * empty and A singular); fix such nodes or drop them from the mesh.
 * The host part runs on all cores; the environment variable FE_HOST_THREADS
 * (a positive integer) caps the threads.  The products do not depend on it. */
int fe_build_pattern(fe_ctx *ctx);

/* Borrowed host views of the setup products, valid until fe_destroy:
 * rowptr [n+1], colind [nnz], scatter = C [ntrip]. */
int fe_get_pattern(fe_ctx *ctx, int64_t *n, int64_t *nnz, const int32_t **rowptr,
                   const int32_t **colind, int64_t *ntrip, const int32_t **scatter);

/* Inverse of C: slot s gathers triplets slot_src[slot_ptr[s] .. slot_ptr[s+1])
 * (ascending).  Borrowed host views. */
int fe_get_inverse_map(fe_ctx *ctx, const int64_t **slot_ptr, const int32_t **slot_src);

/* Consistent-mass values on the CSR pattern (host, [nnz], fixed rows 0). */
int fe_get_mass(fe_ctx *ctx, const double **mass_vals);

/* Nested-dissection result (Section 6.1): perm [n_free_dofs] lists the
 * original DOF of each new position; fronts: n_fronts, and per front its
 * first pivot (new numbering), pivot count, update-row count, parent (-1 for
 * a root) and level (0 = leaves).  Borrowed host views. */
int fe_get_ordering(fe_ctx *ctx, int64_t *n_free, const int32_t **perm, int64_t *n_fronts,
                    const int32_t **front_first, const int32_t **front_npiv,
                    const int32_t **front_nupd, const int32_t **front_parent,
                    const int32_t **front_level);

/* Update rows (original DOF numbers, ascending in the new order) of a front. */
int fe_get_front_rows(fe_ctx *ctx, int64_t front, int64_t *n_upd, const int32_t **rows);

/* Sets the state (positions q and velocities v, [n] each; NULL keeps the
 * current value).  Default state: q = rest positions, v = 0.  v must vanish
 * on fixed DOFs.  Host arrays (device_ptrs = 0) are checked before any
 * device work: FE_ERR_ARG for a non-finite entry or a non-zero velocity on a
 * fixed DOF. */
int fe_set_state(fe_ctx *ctx, const double *q, const double *v);
int fe_get_state(fe_ctx *ctx, double *q, double *v);

/* Element kernel alone at positions q ([n], NULL: current state):
 * f_e [n_elems * 3npe] and K_e [n_elems * (3npe)^2] in fill order (FP64
 * outputs; FP32 tangents are widened, double-float forces summed to FP64).
 * Either output may be NULL. */
int fe_element_eval(fe_ctx *ctx, const double *q, double *f_e, double *K_e);

/* Element kernel + fast assembly at the current state with external force
 * p_ext [n] (NULL = 0): A_vals [nnz] on the CSR pattern (the FP64-accurate
 * matrix the residual uses: FP64, or double-float with FE_MIXED, sums of the
 * element tangents) and b [n]
 * (Eq. "dynamic equation2"; fixed rows: A_ii = 1, b_i = 0).  Either output
 * may be NULL. */
int fe_assemble(fe_ctx *ctx, const double *p_ext, double *A_vals, double *b);

/* Numeric LDL^T of the current A (Eq. "asynchronous preconditioner") on the
 * factor stream, and one application z = P^{-1} r ([n] each, FP64 in/out).
 * For tests of the factor and of the level-scheduled solves. */
int fe_factor_now(fe_ctx *ctx);
int fe_apply_preconditioner(fe_ctx *ctx, const double *r, double *z);

/* Allocation-free variant of fe_apply_preconditioner, for callers that
 * cannot call cudaMalloc: an interactive simulator's real-time loop, where an
 * allocation's implicit device synchronisation and latency would break the
 * frame budget, or a host whose device memory is already fully reserved by
 * another allocator.  (The paper has no counterpart; this is a library
 * convenience.)
 *   r, z: DEVICE pointers to [n] FP64 vectors (z = P^{-1} r), whatever
 *         fe_options.device_ptrs says; stream: cudaStream_t (NULL: legacy).
 * The call is asynchronous on `stream` and allocates nothing: its work
 * vectors live in one file-scope device array of 64 MiB that every GPU
 * loading the library holds until exit.  A mesh needing more
 * (fe_info.noalloc_bytes: (2 n + update rows + free DOFs) x 4 or 8 bytes
 * plus the split application tasks' partial sums, two to three times the
 * vectors alone; 16.9 MB mixed and 33.5 MB FP64 at 348,843 DOF) is
 * rejected with FE_ERR_ARG before any GPU work.  The context must
 * already hold a factor (fe_factor_now or fe_step) and its device must be
 * current.  The first call on a device looks the array's address up
 * (cudaGetSymbolAddress); make that first call before any stream capture.
 * All calls share the array and it keeps the last call's contents (the call
 * clears what must start at zero): calls that overlap on the GPU, on any
 * stream or context, race.
 * Ordering with the context's own work: the call also uses the context's
 * per-front counters and reads its current factor, so it starts on `stream`
 * only after the work already queued on the context's stream (events, no
 * allocation), and the context's later calls (steps, refactorisations,
 * applications) wait for it.  If one of its bounded dependency waits runs
 * out (fe_options.dep_wait_s), z is incomplete; the context's next fe_step
 * or fe_apply_preconditioner then returns FE_ERR_TIMEOUT naming this call
 * (once; the state is unchanged and the call can be repeated). */
int fe_apply_preconditioner_noalloc(fe_ctx *ctx, const double *r, double *z, void *stream);

/* Frictionless contacts against rigid planes, by Lagrange multipliers
 * (Section "Lagrangian multipliers", Eq. "KKT"), for every following step
 * until replaced: constraint i asks that node nodes[i] end the step on the
 * positive side of its plane, normals[3i..3i+2] . x >= offsets[i] (x the
 * node's end-of-step position; the normal need not be unit length).  A step
 * with contacts solves the free motion A a_free = b (the usual PCG), builds
 * the compliance W = H P^{-1} H^T with the step's preconditioner P (the
 * lagged factor; the exact A^{-1} when refactor_every = 1), one
 * preconditioner application per constraint, solves the LCP
 * lambda >= 0, W lambda >= delta - H a_free, complementary, by projected
 * Gauss-Seidel (contact_sweeps, contact_tol), and corrects
 * a = a_free + P^{-1} H^T lambda before integrating.  Constraints on fixed
 * nodes keep lambda = 0.  Host arrays, copied; m = 0 removes the contacts;
 * m <= 4096.  FE_ERR_ARG for a node out of range or a zero normal;
 * FE_ERR_STATE with keep_checkpoints (the adjoint does not cover contacts)
 * or newton_iters > 1. */
int fe_set_contacts(fe_ctx *ctx, int32_t m, const int32_t *nodes, const double *normals,
                    const double *offsets);

/* The multipliers lambda [m] of the last step with contacts (host array):
 * the contact force on the node is lambda_i times the normal, in the
 * units of the equation of motion's right-hand side (N). */
int fe_get_contact_forces(fe_ctx *ctx, double *lambda);

/* One implicit step with external nodal forces p_ext [n] (NULL = 0), one
 * Newton iteration (Eq. "taylor expansion").  Writes the new q, v when the
 * pointers are non-NULL; info may be NULL. */
int fe_step(fe_ctx *ctx, const double *p_ext, double *q_out, double *v_out,
            fe_step_info *info);

/* Sizes of the setup products. */
typedef struct {
  int64_t n, nnz, ntrip;  /* DOFs, CSR slots, triplets                       */
  int64_t n_free;         /* DOFs not held by projective constraints         */
  int64_t n_fronts, n_levels;
  int64_t y_nnz;          /* stored nonzeros of the fronts' apply operators
                             (lower-trapezoidal m x p blocks; the analogue of
                             nnz(L) read twice per preconditioner application) */
  double factor_flops;    /* flops of one numeric factorisation              */
  int64_t device_bytes;   /* device memory held by the context (0 before use) */
  int64_t noalloc_bytes;  /* scratch bytes fe_apply_preconditioner_noalloc
                             needs for this mesh (its limit is 64 MiB)       */
  int64_t ntrip_kept;     /* triplets the assembly gathers (C[t] >= 0)       */
  int64_t n_blocks;       /* 3x3 node blocks of the free rows (nnz of the
                             free rows / 9): the assembly's gather units     */
} fe_info;
int fe_get_info(fe_ctx *ctx, fe_info *info);

/* Stage timings gathered when fe_options.profile_stages = 1: for each stage
 * the summed CUDA-event time in ms (measured on the stream that runs it) and
 * the number of timed calls, plus the library's kernel launches since the
 * last reset.  Arrays have FE_STAGE_COUNT entries; any pointer may be NULL. */
enum {
  FE_STAGE_ELEMENT = 0, FE_STAGE_ASSEMBLY, FE_STAGE_FACTOR, FE_STAGE_APPLY,
  FE_STAGE_SPMV, FE_STAGE_VECTOR, FE_STAGE_RESIDUAL, FE_STAGE_INTEGRATE,
  FE_STAGE_FACTOR_UPDATE, /* the factor's trailing-update launches only */
  FE_STAGE_PCG_GRAPH,     /* PCG iterations replayed as CUDA graphs (use_graph) */
  FE_STAGE_CONTACT,       /* constraint resolution and motion correction      */
  FE_STAGE_FACTOR_UPDATE_BF16, /* the superpanels' BF16 trailing-update launches
                                  (update_bf16); FE_STAGE_FACTOR_UPDATE then
                                  times the other update launches        */
  FE_STAGE_COUNT
};
int fe_get_stage_times(fe_ctx *ctx, double *ms, int64_t *calls, int64_t *kernel_launches);
/* Algorithmic flops of the trailing-update launches timed so far (lower
 * triangle of the Schur updates plus the apply-operator updates). */
int fe_get_update_flops(fe_ctx *ctx, double *flops);
/* The same for the launches timed as FE_STAGE_FACTOR_UPDATE_BF16. */
int fe_get_update_bf16_flops(fe_ctx *ctx, double *flops);
/* The 128 x 128 output tiles of those launches (each read and written once
 * by a TMA reduce-add: 128 KB of DRAM traffic for F or Y per tile). */
int fe_get_update_bf16_tiles(fe_ctx *ctx, int64_t *tiles);
int fe_reset_stage_times(fe_ctx *ctx);

/* Replaces the material parameters ([n_elems * 3], element-major, the layout
 * of fe_material with per_element = 1) without redoing the setup. */
int fe_set_params(fe_ctx *ctx, const double *params);

/* Discrete adjoint of the rollout recorded since the last
 * fe_clear_checkpoints (fe_step stores (q_t, v_t, a_t) when
 * fe_options.keep_checkpoints = 1).  Given dL/dq_T and dL/dv_T ([n] each;
 * dL_dvT may be NULL = 0), sweeps the steps backwards: per step it rebuilds
 * A_t, solves A_t lambda = h v_bar + h^2 q_bar with the PCG (A_t symmetric,
 * lambda = 0 on fixed DOFs; lagged factor of the sweep refreshed every
 * refactor_every steps), and updates
 *   q_bar -= c_K dK[lambda] a + (beta + h) dK[lambda] v + K lambda,
 *   v_bar += h q_bar - (alpha M + (beta + h) K) lambda,
 *   s_bar_e -= lambda_e . (c_K K_e a_e + f_e + (beta + h) K_e v_e).
 * Outputs: dL_ds [n_elems], the derivative with respect to a scale s_e of
 * element e's energy (its material parameters all multiplied by s_e; for a
 * per-element Young's modulus at fixed nu, dL/dE_e = dL_ds[e] / E_e), and
 * dL_dp [T * n] (step-major; NULL to skip), the derivative with respect to
 * the external forces of every step.  Pointers follow device_ptrs. */
int fe_adjoint(fe_ctx *ctx, const double *dL_dqT, const double *dL_dvT, double *dL_ds, double *dL_dp);
int fe_clear_checkpoints(fe_ctx *ctx);
int fe_num_checkpoints(fe_ctx *ctx, int64_t *count);

/* Test hook for failure detection without a GPU fault (not part of the
 * paper's method): before the context's next preconditioner application,
 * front `front` (0 <= front < n_fronts of fe_get_ordering) gets `extra` > 0
 * more pending children than it has, so its forward tasks wait on a count
 * that nothing reaches.  That wait runs out after fe_options.dep_wait_s; the
 * application's kernels then stop taking tasks and the call that ran the
 * application (fe_step, fe_apply_preconditioner) returns FE_ERR_TIMEOUT with
 * the state unchanged.  The hold lasts one application: the backward launch
 * resets every counter, so the next call runs normally. */
int fe_debug_hold_front(fe_ctx *ctx, int64_t front, int32_t extra);

/* Message of the last failure on ctx ("" if none). */
const char *fe_last_error(const fe_ctx *ctx);

/* Frees every host and device resource of ctx (NULL is a no-op). */
void fe_destroy(fe_ctx *ctx);

/* ------------------------------------------------------------------------
 * Generic triplet ingestion (Section 4.2, "Collect data", "Build matrix
 * pattern", Algorithm "add"): any caller-side FE code hands over, every
 * step, its stream of (row, col, value) contributions to an n x n matrix in
 * its own filling order.  When the (row, col) stream equals the previous
 * call's element by element and in length (the filling-order test), the
 * CSR pattern and the map C are kept and only the values are merged on the
 * GPU: slot s = sum of its triplets in ascending stream order, one thread
 * per slot, no atomics (bit-reproducible).  Otherwise the pattern is
 * rebuilt on the host by two counting-sort transposes ("full assembly") and
 * uploaded.  The handle owns its device memory; one device, one caller
 * thread at a time.
 * ---------------------------------------------------------------------- */
typedef struct fe_trip fe_trip;

/* New handle for n x n matrices (n >= 1) on the current device. */
int fe_trip_create(int64_t n, fe_trip **out);

/* Merges the stream: rows, cols [ntrip] int32 in [0, n), vals [ntrip]
 * FP64.  device_ptrs = 0: host arrays (compared with the previous stream on
 * the host); 1: device arrays on stream `stream` (compared on the device,
 * one flag read back).  *rebuilt (may be NULL) = 1 when the pattern was
 * (re)built.  An index outside [0, n) is FE_ERR_ARG (checked whenever the
 * pattern is built; an unchanged stream was checked when first seen).
 * ntrip = 0 gives an empty pattern.  The merged values stay on the device
 * until the next call (fe_trip_values, fe_trip_device_csr). */
int fe_trip_assemble(fe_trip *t, int64_t ntrip, const int32_t *rows, const int32_t *cols, const double *vals,
                     int32_t device_ptrs, void *stream, int32_t *rebuilt);

/* Borrowed host views of the pattern (valid until the next rebuild or
 * fe_trip_destroy): rowptr [n + 1], colind [nnz], scatter = C [ntrip]. */
int fe_trip_pattern(fe_trip *t, int64_t *nnz, const int32_t **rowptr, const int32_t **colind,
                    const int32_t **scatter);

/* Copies the merged values [nnz] to `out` (host, or device when
 * device_ptrs = 1) on `stream`; host copies are complete on return. */
int fe_trip_values(fe_trip *t, double *out, int32_t device_ptrs, void *stream);

/* Borrowed device views of the CSR matrix (valid until the next
 * fe_trip_assemble or fe_trip_destroy). */
int fe_trip_device_csr(fe_trip *t, const int32_t **rowptr, const int32_t **colind, const double **vals);

/* Message of the last failure on t ("" if none). */
const char *fe_trip_last_error(const fe_trip *t);

/* Frees the handle (NULL is a no-op). */
void fe_trip_destroy(fe_trip *t);

#ifdef __cplusplus
}
#endif
#endif /* FE_HOTPATH_H */
