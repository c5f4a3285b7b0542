// Internal definition of the fe_ctx handle shared by the host setup (C++)
// and the CUDA translation units.  Not part of the public ABI.
#pragma once

#include <cstdint>
#include <string>
#include <vector>

#include "../../include/fe_hotpath.h"

namespace fe {

constexpr int kNB = 64;        // panel width of the front factorisation
constexpr int kTile = 64;      // tile edge of the front update kernels
constexpr int kSuper = 512;    // FP32 factor: trailing updates are applied once per kSuper pivots
                               // (512: a synchronous factorisation at 350k DOF takes 23.15 ms,
                               // against 24.05 at 256 and 23.55 at 1024)
constexpr int kSub = 128;      // FP32 factor: inside a superpanel, the updates of its own columns
                               // are applied once per kSub pivots (22.55 ms for the factorisation
                               // above, against 23.15 with an update per 64-pivot panel)
static_assert(kSuper % kSub == 0 && kSub % kNB == 0, "sub-blocks tile a superpanel in whole panels");
constexpr int kBwdCols = 32;   // pivot columns per task of the backward apply
constexpr int kFwdCols = 256;  // pivot columns per task of the forward apply (split over CTAs)
constexpr int kBwdRows = 1024; // rows per task of the backward apply (split over CTAs)
// application tasks per level below which a level's tasks are made narrower
// (forward: fewer pivot columns; backward: fewer rows; down to a quarter):
// about one per resident CTA of the sweeps (four per SM on 152 SMs)
constexpr int kApplyTasksPerLevel = 608;
// rows of Y per 16-byte vector: 8 binary16, 4 FP32, 2 FP64 entries
inline int y_vec(const fe_options &o) { return o.precision == FE_MIXED ? (o.precond_fp16 ? 8 : 4) : 2; }
inline int fwd_rows(const fe_options &o) { return 32 * y_vec(o); }  // 32 threads x one 16-byte vector
// rows per backward task: twice as many for the binary16 Y, so a task moves the
// same bytes (its fixed costs, the dependency wait, staging x and publishing,
// are then spread over as much data as in the FP32 path)
inline int bwd_rows(const fe_options &o) { return o.precision == FE_MIXED && o.precond_fp16 ? 2 * kBwdRows : kBwdRows; }

// Task kinds of the multifrontal factorisation (packed in int4.y >> 24).
enum TaskKind { T_DIAG = 0, T_PANEL = 1, T_XK = 2, T_TRAIL = 3, T_RUPD = 4 };

struct Front {
  int32_t first = 0;      // first pivot, new DOF numbering
  int32_t npiv = 0;       // p: pivots (DOFs) of the front
  int32_t nupd = 0;       // number of update rows (DOFs)
  int32_t parent = -1;
  int32_t level = 0;      // 0 = leaf; children are on lower levels
  int64_t f_off = 0;      // offset of the dense m x m front (column-major, leading dimension ldf)
  int32_t ldf = 0;        // m rounded up to 4: every column starts 16-byte aligned (TMA tiles)
  int64_t y_off = 0;      // offset of the m x p apply operator Y
  int64_t w_off = 0;      // offset of the m-vector work buffer
  int64_t u_off = 0;      // offset of the update vector (nupd)
  int64_t rows_off = 0;   // offset into upd_rows_new / upd_rows_old
  int64_t rmap_off = 0;   // offset of this front's map into its parent's front
  int32_t ldy = 0;        // leading dimension of Y (m rounded up to 4)
  int32_t fcols = kFwdCols;  // pivot columns per forward application task
  int32_t brows = 0;         // rows per backward application task (bwd_rows or a half or quarter of it)
  int32_t m() const { return npiv + nupd; }
};

struct Level {
  std::vector<int32_t> fronts;        // fronts of this level
  int32_t steps = 0;                  // panel steps (max over fronts)
  // factorisation task lists: assembly, then per step {diag, panel+xk, trail+rupd}
  std::vector<int32_t> asm_tasks;     // (front, c0, c1) triples
  std::vector<std::vector<int32_t>> diag, panel, trail;  // int4 per task
  std::vector<double> trail_flops;    // algorithmic flops of each step's update launch
  // superpanel ends in the BF16 kernel (FE_MIXED with update_bf16): the
  // deferred rank-K updates of the rest of the fronts, split off trail
  std::vector<std::vector<int32_t>> tend;
  std::vector<double> tend_flops;
  // apply task lists
  // (front, r0, j0, slot): rows [r0, r0 + fwd_rows) x pivot columns [j0, j0 + kFwdCols)
  std::vector<int32_t> fwd_tasks;
  // (front, c0, i0, slot): pivot columns [c0, c0 + kBwdCols) x rows [i0, i0 + kBwdRows)
  std::vector<int32_t> bwd_tasks;
};

struct DeviceState;  // defined in the CUDA translation unit

}  // namespace fe

struct fe_ctx {
  // ---------------------------------------------------------------- inputs
  int32_t elem_type = 0, npe = 4;
  int64_t n_nodes = 0, n_elems = 0;
  std::vector<double> X;              // [n_nodes * 3]
  std::vector<int32_t> conn;          // [n_elems * npe]
  std::vector<int32_t> fixed_nodes;
  int32_t model = 0;
  double rho = 0;
  std::vector<double> params;         // [n_elems * 3] (expanded)
  double h = 0, alpha = 0, beta = 0;
  fe_options opt{};

  // batched context: members concatenated in the order of seg_member (grouped
  // by material model); member k owns nodes [seg_node[k], seg_node[k+1]) and
  // elements [seg_elem[k], seg_elem[k+1]); model_range[m] = element range of
  // model m (empty when absent).  nseg = 1 for a plain context.
  int32_t nseg = 1;
  std::vector<int64_t> seg_node, seg_elem;
  std::vector<int32_t> seg_member, seg_model;
  int64_t model_range[4][2] = {{0, 0}, {0, 0}, {0, 0}, {0, 0}};

  // ---------------------------------------------------------- setup products
  bool built = false;
  int64_t n = 0, nnz = 0, ntrip = 0;
  std::vector<int8_t> fixed_dof;      // [n]
  std::vector<int32_t> rowptr, colind, C;
  std::vector<int64_t> slot_ptr;      // [nnz + 1]
  std::vector<int32_t> slot_src;      // [slot_ptr[nnz]]
  std::vector<double> mass;           // [nnz]
  std::vector<int32_t> node_ptr, node_src;   // node -> (e * npe + a), ascending
  // 3x3 node-block view of the pattern: node n's blocks [bptr[n], bptr[n+1])
  // with column node bcol, contributing element blocks (e*npe + a)*npe + b in
  // bsrc[bsrc_ptr[k] .. bsrc_ptr[k+1]] (ascending), block mass bmass (M = bmass I3)
  std::vector<int32_t> bptr, bcol, bsrc_ptr, bsrc;
  std::vector<double> bmass;
  std::vector<double> rest;           // element rest data, SoA [ncoef][n_elems]
  int32_t rest_ncoef = 0;

  // nested dissection + multifrontal symbolic analysis
  int64_t n_free = 0;
  std::vector<int32_t> perm;          // new DOF -> original DOF   [n_free]
  std::vector<int32_t> iperm;         // original DOF -> new DOF or -1 [n]
  std::vector<fe::Front> fronts;
  std::vector<int32_t> front_first, front_npiv, front_nupd, front_parent, front_level;
  std::vector<int32_t> upd_rows_new, upd_rows_old;  // per front, update rows
  std::vector<int32_t> rmap;          // per child: positions in its parent's front
  std::vector<int32_t> wsrc_ptr, wsrc; // per front position (w_off + pos): update-vector entries it gathers
  std::vector<int32_t> child_ptr, child_list;       // children of each front, ascending
  std::vector<int64_t> fa_ptr;        // per front, A entries: [fa_ptr[f], fa_ptr[f+1])
  std::vector<int32_t> fa_slot, fa_off;             // CSR slot, offset in the front
  std::vector<int64_t> fa_colptr;     // per front: per local column start into fa_*
  std::vector<fe::Level> levels;
  int64_t f_total = 0, y_total = 0, w_total = 0, u_total = 0;
  // partial-sum slots of the split apply tasks (slot = -1: a block done by one task)
  int64_t fwd_slots = 0, bwd_slots = 0;
  // dataflow application: every level's tasks in one list per direction
  // (level order for the forward solve, reverse level order backward) and
  // the number of tasks of every front in each
  std::vector<int32_t> apply_fwd, apply_bwd;  // int4 per task
  std::vector<int32_t> front_nfwd, front_nbwd;
  double factor_flops = 0;
  int64_t y_nnz = 0;

  // contacts of the following steps (fe_set_contacts): node, normal and
  // plane offset of each constraint n . x >= c
  std::vector<int32_t> contact_node;
  std::vector<double> contact_normal, contact_offset;

  fe::DeviceState *dev = nullptr;
  std::string err;
};

namespace fe {
// host setup (fe_setup.cpp)
int build_pattern_host(fe_ctx *c);
int set_error(const fe_ctx *c, int code, const std::string &msg);
// device side (fe_api.cu)
void destroy_device(fe_ctx *c);
}  // namespace fe
