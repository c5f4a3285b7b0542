// Device-side declarations shared by the CUDA translation units.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <vector>

#include "fe_ctx.h"

namespace fe {

#define FE_CUDA_TRY(call)                                                         \
  do {                                                                            \
    cudaError_t e_ = (call);                                                      \
    if (e_ != cudaSuccess)                                                        \
      return set_error(c, FE_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
  } while (0)

// Front descriptor as the kernels see it.
struct DFront {
  int32_t first, npiv, nupd, m;
  int32_t child_begin, child_end;    // into child_list
  int32_t ldy, parent;               // parent front (-1: a root)
  int32_t nfwd, nbwd;                // tasks of this front in the dataflow application lists
  int32_t ldf;                       // leading dimension of the front's F (multiple of 4)
  int16_t fcols, brows;              // application task sizes: forward pivot columns, backward rows
  int64_t f_off, y_off, w_off, u_off, rows_off, fac_off;
};

// Error flags raised by kernels (bit mask in DeviceState::flags[0]; an
// allocation-free application raises its own in flags[1], which stays set
// until a later call of the context reports it).
enum { FLAG_INVERTED = 1, FLAG_PIVOT = 2, FLAG_BREAKDOWN = 4, FLAG_WAIT_TIMEOUT = 8, FLAG_APPLY_TIMEOUT = 16 };

// Scalars of the PCG kept on the device (double).
enum {
  S_RZ = 0, S_RZ_NEW, S_PQ, S_ALPHA, S_BETA, S_RR, S_BB, S_TOL2, S_DONE, S_ITERS,
  S_ORR, S_OTOL2, S_ODONE, S_NDELTA, S_NA, S_SWEEPS,
  S_COUNT = 16
};

// Per-member scalars of a batched solve (double [nseg][B_COUNT]).
enum { B_RZ = 0, B_PQ, B_ALPHA, B_BETA, B_RR, B_BB, B_TOL2, B_DONE, B_ITERS, B_ORR, B_OTOL2, B_ODONE, B_COUNT = 12 };
enum { SEG_PQ = 0, SEG_RR, SEG_RZ_FIRST, SEG_RZ, SEG_INIT_OUTER, SEG_INIT_INNER, SEG_ORR };

struct Buf {
  void *p = nullptr;
  size_t bytes = 0;
};

struct DeviceState {
  int device = 0;
  cudaStream_t stream = nullptr;   // main stream (caller's or own)
  cudaStream_t fstream = nullptr;  // factor side stream
  bool own_stream = false;
  cudaEvent_t ev_assembled = nullptr, ev_factored = nullptr, ev_apply_done = nullptr;
  // ordering of fe_apply_preconditioner_noalloc on a caller's stream against
  // the context's own stream, both ways (created with the device state)
  cudaEvent_t ev_main_tail = nullptr, ev_noalloc_done = nullptr;
  std::vector<void *> allocs;

  // mesh / setup
  int32_t *conn = nullptr;
  double *rest = nullptr, *params = nullptr, *X = nullptr;
  int32_t *rowptr = nullptr, *colind = nullptr, *slot_ptr = nullptr, *slot_src = nullptr;
  double *mass = nullptr;
  int8_t *fixed_row = nullptr;
  int32_t *node_ptr = nullptr, *node_src = nullptr;
  int32_t *bptr = nullptr, *bcol = nullptr, *bsrc_ptr = nullptr, *bsrc = nullptr;
  double *bmass = nullptr;
  float2 *bmass2 = nullptr;        // mixed path: bmass as float pairs (the assembly's double-float mass)

  // state
  double *q = nullptr, *v = nullptr, *pext = nullptr, *acc = nullptr;
  double *a_prev = nullptr;        // the last step's acceleration (warm start; 0 after fe_set_state)
  double *stage_in = nullptr, *stage_out = nullptr;  // pinned host staging [n]
  double *stage_big = nullptr; size_t stage_big_bytes = 0;

  // element outputs: forces f_e in FP64, or as float pairs (double-float)
  // in the mixed path with FP32 tangents; tangents K_e in FP64, or FP32 in
  // the mixed path (unless element_fp64)
  double *fe = nullptr;
  // that path's inputs as float pairs: rest data and parameters (made at
  // setup and by fe_set_params), the displacement q - X (per launch)
  float2 *rest2 = nullptr, *params2 = nullptr, *u2 = nullptr;
  void *Ke = nullptr;
  // system: A in the matrix type (FP64, or FP32 in the mixed path: the inner
  // SpMV and the snapshot the factor reads), b in FP64.  The refinement
  // residual's FP64-accurate A: A64 = A in the FP64 path; in the mixed path
  // A2, the values as float pairs (hi, lo; fe_df.cuh), read by double-float
  // residual kernels, and A64 null
  void *A = nullptr;
  double *A64 = nullptr;
  float2 *A2 = nullptr;
  void *Afac = nullptr;
  double *b = nullptr;

  // PCG vectors (FP64 outer) and inner vectors (matrix type)
  double *x = nullptr, *r = nullptr;
  // mixed path: the refinement iterate x as float pairs, written with x by
  // the outer init and every refinement update, read by the residual
  float2 *x2 = nullptr;
  void *vz = nullptr, *vp = nullptr, *vq = nullptr, *vr = nullptr, *vd = nullptr;
  double *scal = nullptr;          // [S_COUNT] device scalars
  double *partials = nullptr;      // [kMaxBlocks]
  unsigned int *ticket = nullptr;  // last-block counters [4]
  int *flags = nullptr;            // device error flags
  int *h_flags = nullptr;          // pinned mirror
  double *h_scal = nullptr;        // pinned mirror of scal

  // multifrontal factor
  DFront *fronts = nullptr;
  int32_t *perm = nullptr, *upd_rows_old = nullptr, *rmap = nullptr, *child_list = nullptr;
  int32_t *fa_slot = nullptr, *fa_off = nullptr;
  int32_t *wsrc_ptr = nullptr, *wsrc = nullptr;
  int64_t *fa_colptr = nullptr;
  int32_t *tasks = nullptr;        // all task lists, concatenated
  void *F = nullptr;               // front scratch (factor type)
  void *Y[2] = {nullptr, nullptr}; // apply operators (double-buffered for the lag)
  void *Yh[2] = {nullptr, nullptr};  // their binary16 copies (precond_fp16)
  // TMA tensor maps of the FP32 factor (128-byte CUtensorMap objects, 64-byte
  // aligned): [0, nf) one per front over F, [nf, 3 nf) one per front over
  // the pivot rows of Y[0] then Y[1] (4 x 128 boxes), [3 nf, 5 nf) one per
  // front over all rows of Y[0] then Y[1] (128 x 16 boxes); null for the
  // FP64 factor
  void *tmaps = nullptr;
  // update_bf16: K-major BF16 copies of the current superpanel, [rows][256]
  // (Wt, Lt: W = L D and L, row w_off + r of a front; Yk: the pivot rows of
  // Y, row first + c for column c), and their three tensor maps
  void *bt_w = nullptr, *bt_l = nullptr, *bt_y = nullptr;
  void *bmaps = nullptr;
  // contacts (fe_contact.cu): constraint data, forward solves G, compliance
  // W (m x m), PGS right-hand side and multipliers
  int32_t *c_node = nullptr;
  double *c_normal = nullptr, *c_off = nullptr, *c_W = nullptr, *c_rhs = nullptr, *c_lam = nullptr;
  void *c_G = nullptr;  // forward solves D^{-1} L^{-1} H^T e_i, [m][n_free] in the solve's precision
  // the fronts on the constraints' paths to the root: their forward tasks
  // (topological order, each repeated for the c_nrhs right-hand sides of a
  // launch) and their children's forward tasks on the paths; per right-hand side
  // of a launch: input vectors, update vectors, partial sums, tickets,
  // counters; the launch's control words
  int32_t *c_tasks = nullptr;
  int *c_pend = nullptr, *c_pendm = nullptr, *c_bdm = nullptr, *c_ctl = nullptr, *c_tick = nullptr;
  void *c_r = nullptr, *c_u = nullptr, *c_part = nullptr;
  int64_t c_ntask = 0, c_nrhs = 0;
  size_t c_bytes[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};  // capacities of the per-set buffers above
  int64_t c_cap = 0, c_m = 0;
  bool c_dirty = true;  // the context's constraint set changed since the last upload
  double *D[2] = {nullptr, nullptr};
  void *wbuf = nullptr, *ubuf = nullptr, *yperm = nullptr;  // apply work vectors
  double *na = nullptr, *nq = nullptr, *nv = nullptr;       // Newton iterate a_k, q_k, v_k
  // whole-step graphs (use_graph): the solve (PCG, refinement) and the
  // integration of a step as one graph with device-side WHILE loops, one
  // per factor buffer the applications read; kernels per prologue, inner
  // iteration and refinement sweep (launch counting)
  struct StepGraph {
    int cur = -1;
    cudaGraphExec_t exec = nullptr;
    int64_t k_pro = 0, k_inner = 0, k_outer = 0;
  };
  StepGraph step_graph[4];         // [2 * cur + (a factorisation in flight)]
  void *part_f = nullptr, *part_b = nullptr;                // partial sums of split apply tasks
  int *tick_f = nullptr, *tick_b = nullptr;                 // their tickets (zero between launches)
  // dataflow application: task lists, per-front counters (forward: children
  // still pending; backward: tasks done), task queues and the abort flag
  int32_t *apply_fwd = nullptr, *apply_bwd = nullptr;
  int64_t n_apply_fwd = 0, n_apply_bwd = 0;
  int *df_pend = nullptr, *df_pend0 = nullptr, *df_bdone = nullptr, *df_ctl = nullptr;
  int df_grid = 0;                                          // resident CTAs of the application kernels
  mutable int df_hold = -1;        // fe_debug_hold_front: front held for the next application, or -1
  int df_hold_extra = 0;
  int cur = 0;                     // buffer the solver reads
  int factor_pending = -1;         // buffer being written on fstream, or -1
  int64_t pending_step = -1;       // step whose A the pending factor holds
  int64_t cur_step = -1;           // step whose A the current factor holds
  bool have_factor = false;

  // task list offsets: per level {asm, per step: diag, panel, trail}, fwd, bwd
  struct LevelTasks {
    int64_t asm_off = 0, asm_n = 0;
    std::vector<int64_t> diag_off, diag_n, panel_off, panel_n, trail_off, trail_n, tend_off, tend_n;
    std::vector<double> trail_flops, tend_flops;
    int64_t fwd_off = 0, fwd_n = 0, bwd_off = 0, bwd_n = 0;
    int64_t nfronts = 0, fronts_off = 0;
  };
  std::vector<LevelTasks> lt;
  int32_t *level_fronts = nullptr;

  int64_t step_index = 0;
  size_t bytes_total = 0;

  // live stage timing (fe_options.profile_stages) and launch counting
  struct StageRec { int stage; cudaEvent_t a, b; };
  std::vector<StageRec> recs;
  std::vector<cudaEvent_t> pool;
  double stage_ms[FE_STAGE_COUNT] = {0};
  int64_t stage_calls[FE_STAGE_COUNT] = {0};
  mutable int64_t launches = 0;
  double update_flops = 0.0;            // algorithmic flops of the timed update launches
  double update_bf16_flops = 0.0;       // the same for the BF16 superpanel-end launches
  int64_t update_bf16_tiles = 0;        // and their 128 x 128 output tiles

  // batched solve: member DOF ranges, row -> member, per-member scalars
  int64_t *seg_dof = nullptr;
  int32_t *row_seg = nullptr;
  double *bscal = nullptr, *h_bscal = nullptr;
  // batched SpMV schedule (fe_batch.cu): members grouped into size classes
  // by their mean 3x3 blocks per node; each class is a table of row blocks
  // (node ranges of at most kBatchBlockNodes nodes inside one member) and
  // has its own kernel (node-block lanes per node or CSR threads per row),
  // chosen by timing the candidates
  struct SpmvClass {
    int lpn = 16;                  // node-block lanes per node, or -(CSR threads per row)
    int2 *blocks = nullptr;
    int64_t nblocks = 0;
    std::vector<int32_t> members;
  };
  std::vector<SpmvClass> spmv_classes;
  bool spmv_tuned = false;
  // single-mesh SpMV variants (tune_spmv): -1 until the first solve times them
  int spmv_var = -1, res_var = -1;
  double *tune_scal = nullptr;     // scratch scalars and flags of the timing runs

  // adjoint: per-step checkpoints (q_t, v_t, a_t) and reverse-sweep buffers
  std::vector<double *> ckpt;      // each [3n]: q_t, v_t, a_t
  double *qbar = nullptr, *vbar = nullptr, *sbar = nullptr, *ge = nullptr, *kl = nullptr;
};

constexpr int kMaxBlocks = 4096;

// ------------------------------------------------------------ kernel launchers
// (fe_kernels.cu)
void launch_element(const fe_ctx *c, const DeviceState *d, const double *q, bool fp32, cudaStream_t s);
// b = p - f - (alpha M + bh K) v - M w  (w may be NULL); A = (1 + h alpha) M + h (beta + h) K
void launch_assemble(const fe_ctx *c, const DeviceState *d, bool fp32, const double *pext, const double *v,
                     const double *w, double bh, cudaStream_t s);
// Newton iterate of the step: qk = q + h v + h^2 a, vk = v + h a
void launch_newton_state(const fe_ctx *c, const DeviceState *d, const double *a, double *qk, double *vk,
                         cudaStream_t s);
// a += delta; S_NDELTA = ||delta||^2, S_NA = ||a||^2
void launch_newton_update(const fe_ctx *c, const DeviceState *d, const double *delta, double *a, cudaStream_t s);
// y = A x; S_PQ = x.y; S_ALPHA = S_RZ / S_PQ
void launch_spmv_dot(const fe_ctx *c, const DeviceState *d, bool fp32, const void *x, void *y, cudaStream_t s);
// r = b - A x (FP64 accumulation); S_ORR, S_ODONE
void launch_residual(const fe_ctx *c, const DeviceState *d, bool fp32, cudaStream_t s);
// times the SpMV variants of both products once per context (first solve)
int tune_spmv(fe_ctx *c, DeviceState *d);
// x += alpha p; r -= alpha q; S_RR, S_DONE, S_ITERS
void launch_axpy_norm(const fe_ctx *c, const DeviceState *d, bool fp32, void *x, void *r, const void *p,
                      const void *q, cudaStream_t s);
// S_BETA = r.z / S_RZ; S_RZ = r.z
void launch_dot_rz(const fe_ctx *c, const DeviceState *d, bool fp32, const void *r, const void *z, bool first,
                   cudaStream_t s);
// p = z + beta p
void launch_update_p(const fe_ctx *c, const DeviceState *d, bool fp32, const void *z, void *p, bool first,
                     cudaStream_t s);
// x = 0, r = rhs; tolerances (outer: S_BB, S_OTOL2, S_ORR, S_ODONE, S_ITERS = 0)
void launch_init_solve(const fe_ctx *c, const DeviceState *d, bool fp32, void *x, void *r, const double *rhs,
                       double tol, bool outer, cudaStream_t s, bool keep_x = false);
// warm start of the FP64 PCG after the residual r = b - A x: S_RR = S_ORR,
// S_DONE = S_ODONE (or 1 when b = 0)
void launch_warm_fixup(const fe_ctx *c, const DeviceState *d, cudaStream_t s);
void launch_refine_update(const fe_ctx *c, const DeviceState *d, cudaStream_t s);  // x += (double) vd
void launch_integrate(const fe_ctx *c, const DeviceState *d, cudaStream_t s);
// the same, skipped on the device unless the step's solve converged with no
// error flag (the whole-step graph decides without a host read)
void launch_integrate_guarded(const fe_ctx *c, const DeviceState *d, bool fp32, cudaStream_t s);
// sets a graph conditional from the device scalars: mode 0, the inner PCG
// goes on (S_DONE == 0); mode 1, the outer refinement goes on (S_ODONE == 0
// and S_ITERS < max_iters; counts the sweep); mode 2, the same without
// counting; every mode stops on an error flag
void launch_graph_cond(const fe_ctx *c, const DeviceState *d, cudaGraphConditionalHandle h, int mode,
                       cudaStream_t s);
void launch_convert(const void *src, bool src32, void *dst, bool dst32, int64_t n, cudaStream_t s);
void launch_pair_to_double(const float2 *src, double *dst, int64_t n, cudaStream_t s);  // dst = hi + lo

// (fe_batch.cu)
void launch_seg_dot(const fe_ctx *c, const DeviceState *d, bool fp32, const void *x, const void *y, int mode,
                    double tol, cudaStream_t s);
void launch_seg_dot64(const fe_ctx *c, const DeviceState *d, const double *x, const double *y, int mode, double tol,
                      cudaStream_t s);
void launch_seg_init(const fe_ctx *c, const DeviceState *d, bool fp32, void *x, void *r, const double *rhs,
                     bool inner, cudaStream_t s);
void launch_seg_axpy(const fe_ctx *c, const DeviceState *d, bool fp32, void *x, void *r, const void *p,
                     const void *q, cudaStream_t s);
void launch_seg_update_p(const fe_ctx *c, const DeviceState *d, bool fp32, const void *z, void *p, bool first,
                         cudaStream_t s);
// batched node-block SpMV over the row-block schedule: y = A x in the
// vector type, or y = b - A64 x in FP64 when b is given
void launch_batch_spmv(const fe_ctx *c, const DeviceState *d, bool fp32, const void *x, void *y, const double *b,
                       cudaStream_t s);
// builds the batched SpMV schedule (size classes, row blocks) and picks each
// class's lanes per node by timing (CUDA events on the main stream)
int tune_batch_spmv(fe_ctx *c, DeviceState *d);
// graph conditions of the batched solve: mode 0, some member's inner PCG
// goes on; mode 1/2, some member's refinement goes on (1 counts a sweep);
// all stop at max_iters or on an error flag; mode 3 (FP64) / 4 (mixed)
// writes flags[2] = 1 when every member converged with no error flag (the
// guard of the integration)
void launch_seg_cond(const fe_ctx *c, const DeviceState *d, cudaGraphConditionalHandle h, int mode, cudaStream_t s);

// (fe_adjoint.cu)
void launch_adjoint_element(const fe_ctx *c, const DeviceState *d, bool fp32, const double *q, const double *lam,
                            const double *acc, const double *v, double *ge, double *kl, double *sbar,
                            cudaStream_t s);
void launch_adjoint_gather(const fe_ctx *c, const DeviceState *d, const double *ge, const double *kl,
                           const double *lam, double *qbar, double *vbar, double *pbar, cudaStream_t s);
void launch_adjoint_rhs(const fe_ctx *c, const DeviceState *d, const double *qbar, const double *vbar,
                        double *abar, cudaStream_t s);

// stage timing hooks (fe_api.cu); idx < 0 when profiling is off
int stage_begin(fe_ctx *c, int stage, cudaStream_t s);
void stage_end(fe_ctx *c, int idx, cudaStream_t s);

// (fe_factor.cu)
int factor_enqueue(fe_ctx *c, DeviceState *d, int buf, bool fp32, const void *Afac, cudaStream_t s);
// done: optional device flag; every kernel of the application returns at
// once when it is non-zero (PCG iterations replayed past convergence)
// contacts (fe_contact.cu): constraint resolution and motion correction of
// the current step (d->x: a_free in, corrected a out)
int contact_resolve(fe_ctx *c, DeviceState *d, bool fp32);
// forward solves of nrhs right-hand sides in one launch over a subset of
// fronts closed under parents (fe_factor.cu)
void apply_forward_multi_enqueue(const fe_ctx *c, const DeviceState *d, int buf, bool fp32, const void *r, void *yp,
                                 const int32_t *tasks, int64_t ntask, const int *pend_init, int *pend,
                                 int *bdone, int *ctl, void *u, void *part, int *tickets, int nrhs, cudaStream_t s);
void apply_enqueue(const fe_ctx *c, const DeviceState *d, int buf, bool fp32, const void *r, void *z,
                   cudaStream_t s, const double *done = nullptr);
// scratch bytes fe_apply_preconditioner_noalloc needs for this mesh (0
// before the setup), and the size of its file-scope array
int64_t noalloc_scratch_bytes(const fe_ctx *c);
// fe_debug_hold_front: apply a pending hold on the stream (no-op without one)
void launch_pending_hold(const DeviceState *d, cudaStream_t s);
int64_t noalloc_scratch_limit();

}  // namespace fe
