// C-ABI entry points that use the GPU: device state, one implicit step
// (element kernel -> gather assembly -> [lagged factor on the side stream]
// -> PCG with the level-scheduled LDL^T preconditioner -> backward Euler),
// and the stage-level calls used by the parity tests.
#include <cuda.h>  // CUtensorMap and its enums (the encoder is reached through the runtime)
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <chrono>
#include <cstring>
#include <thread>

#include "fe_device.cuh"

namespace fe {

namespace {

bool mixed(const fe_ctx *c) { return c->opt.precision == FE_MIXED; }
size_t vsz(const fe_ctx *c) { return mixed(c) ? sizeof(float) : sizeof(double); }

}  // namespace

// ------------------------------------------------------ live stage timing
int stage_begin(fe_ctx *c, int stage, cudaStream_t s) {
  DeviceState *d = c->dev;
  if (!c->opt.profile_stages || stage < 0) return -1;
  DeviceState::StageRec r;
  r.stage = stage;
  for (cudaEvent_t *e : {&r.a, &r.b}) {
    if (!d->pool.empty()) {
      *e = d->pool.back();
      d->pool.pop_back();
    } else if (cudaEventCreate(e) != cudaSuccess) {
      return -1;
    }
  }
  cudaEventRecord(r.a, s);
  d->recs.push_back(r);
  return int(d->recs.size() - 1);
}

void stage_end(fe_ctx *c, int idx, cudaStream_t s) {
  if (idx >= 0) cudaEventRecord(c->dev->recs[idx].b, s);
}

namespace {

// Harvest every finished record (both streams must be idle when all = true).
void stage_collect(fe_ctx *c) {
  DeviceState *d = c->dev;
  if (!d) return;
  std::vector<DeviceState::StageRec> keep;
  for (auto &r : d->recs) {
    if (cudaEventQuery(r.b) != cudaSuccess) {
      cudaGetLastError();
      keep.push_back(r);
      continue;
    }
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, r.a, r.b) == cudaSuccess) {
      d->stage_ms[r.stage] += ms;
      d->stage_calls[r.stage] += 1;
    }
    cudaGetLastError();
    d->pool.push_back(r.a);
    d->pool.push_back(r.b);
  }
  d->recs.swap(keep);
}

struct Stage {
  fe_ctx *c;
  cudaStream_t s;
  int idx;
  Stage(fe_ctx *c_, int stage, cudaStream_t s_) : c(c_), s(s_), idx(stage_begin(c_, stage, s_)) {}
  ~Stage() { stage_end(c, idx, s); }
};

template <typename T>
int dalloc(fe_ctx *c, DeviceState *d, T **p, size_t count) {
  *p = nullptr;
  if (count == 0) count = 1;
  cudaError_t e = cudaMalloc(reinterpret_cast<void **>(p), count * sizeof(T));
  if (e != cudaSuccess) {
    cudaGetLastError();
    return set_error(c, FE_ERR_OOM, "cudaMalloc of " + std::to_string(count * sizeof(T)) + " bytes failed");
  }
  d->allocs.push_back(*p);
  d->bytes_total += count * sizeof(T);
  return FE_OK;
}

int dallocv(fe_ctx *c, DeviceState *d, void **p, size_t bytes) {
  return dalloc(c, d, reinterpret_cast<unsigned char **>(p), bytes);
}

template <typename T>
int upload(fe_ctx *c, DeviceState *d, T **p, const std::vector<T> &h) {
  int st = dalloc(c, d, p, h.size());
  if (st) return st;
  if (!h.empty()) FE_CUDA_TRY(cudaMemcpy(*p, h.data(), h.size() * sizeof(T), cudaMemcpyHostToDevice));
  return FE_OK;
}

// v as float pairs (hi = fl32(v), lo = fl32(v - hi)), the layout the
// double-float kernels read
std::vector<float2> float_pairs(const std::vector<double> &v) {
  std::vector<float2> out(v.size());
  for (size_t i = 0; i < v.size(); ++i) {
    const float h = float(v[i]);
    out[i] = make_float2(h, float(v[i] - double(h)));
  }
  return out;
}

// Tensor maps for the TMA loads of the FP32 factor's trailing updates.
// Per front: F as a 2-D array (rows contiguous, leading dimension ldf),
// 128 x 16 boxes (a 128-row tile of 16 columns); Y as a 2-D array (the
// pivot rows of a column contiguous, leading dimension ldy), 4 x 128 boxes
// (4 consecutive pivot rows of 128 columns, which land in shared memory as
// one K group of the MMA operand layout), and Y again with all its rows in
// 128 x 16 boxes (output tiles of the Y updates).  Out-of-range elements
// read as 0.
using EncodeTiledFn = CUresult (*)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                   const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                                   CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

int encode_tensor_maps(fe_ctx *c, DeviceState *d) {
  void *fn = nullptr;
  cudaDriverEntryPointQueryResult q = cudaDriverEntryPointSymbolNotFound;
  if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) != cudaSuccess ||
      q != cudaDriverEntryPointSuccess || !fn) {
    cudaGetLastError();
    return set_error(c, FE_ERR_CUDA, "cuTensorMapEncodeTiled is not available from the driver");
  }
  const EncodeTiledFn encode = reinterpret_cast<EncodeTiledFn>(fn);
  const int64_t nf = int64_t(c->fronts.size());
  std::vector<CUtensorMap> maps(size_t(5 * nf));
  for (int64_t f = 0; f < nf; ++f) {
    const Front &F = c->fronts[f];
    const cuuint32_t es[2] = {1, 1};
    {
      const cuuint64_t dim[2] = {cuuint64_t(F.m()), cuuint64_t(F.m())};
      const cuuint64_t stride[1] = {cuuint64_t(F.ldf) * 4};
      const cuuint32_t box[2] = {128, 16};
      float *base = reinterpret_cast<float *>(d->F) + F.f_off;
      if (encode(&maps[size_t(f)], CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, base, dim, stride, box, es,
                 CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                 CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
        return set_error(c, FE_ERR_CUDA, "tensor map of front " + std::to_string(f) + " (F) rejected");
    }
    for (int b = 0; b < 2; ++b) {
      const cuuint64_t dim[2] = {cuuint64_t(F.npiv), cuuint64_t(F.npiv)};
      const cuuint64_t stride[1] = {cuuint64_t(F.ldy) * 4};
      const cuuint32_t box[2] = {4, 128};
      float *base = reinterpret_cast<float *>(d->Y[b]) + F.y_off;
      if (encode(&maps[size_t((1 + b) * nf + f)], CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, base, dim, stride, box, es,
                 CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                 CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
        return set_error(c, FE_ERR_CUDA, "tensor map of front " + std::to_string(f) + " (Y) rejected");
      const cuuint64_t dimc[2] = {cuuint64_t(F.m()), cuuint64_t(F.npiv)};
      const cuuint32_t boxc[2] = {128, 16};
      if (encode(&maps[size_t((3 + b) * nf + f)], CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, base, dimc, stride, boxc, es,
                 CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                 CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
        return set_error(c, FE_ERR_CUDA, "tensor map of front " + std::to_string(f) + " (Y rows) rejected");
    }
  }
  int st = upload(c, d, reinterpret_cast<CUtensorMap **>(&d->tmaps), maps);
  if (st || !c->opt.update_bf16) return st;
  // update_bf16: the K-major BF16 copies of a superpanel ([rows][kSuper],
  // rows of 2 kSuper bytes) and one map each, 128 rows x 64 columns per box (128 bytes:
  // one 128-byte swizzle span, the MMA operand layout); zeroed once, so that
  // rows a copy never receives read as finite values
  const int64_t rows_wl = std::max<int64_t>(c->w_total, 1), rows_y = std::max<int64_t>(c->n_free, 1);
  st = dallocv(c, d, &d->bt_w, size_t(rows_wl) * kSuper * 2);
  if (!st) st = dallocv(c, d, &d->bt_l, size_t(rows_wl) * kSuper * 2);
  if (!st) st = dallocv(c, d, &d->bt_y, size_t(rows_y) * kSuper * 2);
  if (st) return st;
  FE_CUDA_TRY(cudaMemset(d->bt_w, 0, size_t(rows_wl) * kSuper * 2));
  FE_CUDA_TRY(cudaMemset(d->bt_l, 0, size_t(rows_wl) * kSuper * 2));
  FE_CUDA_TRY(cudaMemset(d->bt_y, 0, size_t(rows_y) * kSuper * 2));
  std::vector<CUtensorMap> bm(3);
  void *bases[3] = {d->bt_w, d->bt_l, d->bt_y};
  const int64_t rows[3] = {rows_wl, rows_wl, rows_y};
  for (int k = 0; k < 3; ++k) {
    const cuuint32_t es[2] = {1, 1};
    const cuuint64_t dim[2] = {cuuint64_t(kSuper), cuuint64_t(rows[k])};
    const cuuint64_t stride[1] = {cuuint64_t(kSuper) * 2};
    const cuuint32_t box[2] = {64, 128};
    if (encode(&bm[size_t(k)], CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, bases[k], dim, stride, box, es,
               CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
      return set_error(c, FE_ERR_CUDA, "tensor map of the BF16 superpanel copies rejected");
  }
  return upload(c, d, reinterpret_cast<CUtensorMap **>(&d->bmaps), bm);
}

#define FE_TRY(x)      \
  do {                 \
    int s_ = (x);      \
    if (s_) return s_; \
  } while (0)

int ensure_device(fe_ctx *c) {
  if (!c->built) return set_error(c, FE_ERR_STATE, "fe_build_pattern has not run");
  if (c->dev) return FE_OK;
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev == 0) {
    cudaGetLastError();
    return set_error(c, FE_ERR_CUDA, "no CUDA device available");
  }
  DeviceState *d = new DeviceState();
  c->dev = d;
  FE_CUDA_TRY(cudaGetDevice(&d->device));
  // The lagged factorisation is background work with R steps of slack: its
  // stream gets the lowest priority, the library's own main stream the
  // highest, so the CTA scheduler serves the PCG first (a caller's stream
  // keeps the priority the caller gave it).
  int prio_low = 0, prio_high = 0;
  FE_CUDA_TRY(cudaDeviceGetStreamPriorityRange(&prio_low, &prio_high));
  if (c->opt.device_ptrs && c->opt.stream) {
    d->stream = reinterpret_cast<cudaStream_t>(c->opt.stream);
  } else {
    FE_CUDA_TRY(cudaStreamCreateWithPriority(&d->stream, cudaStreamNonBlocking, prio_high));
    d->own_stream = true;
  }
  FE_CUDA_TRY(cudaStreamCreateWithPriority(&d->fstream, cudaStreamNonBlocking, prio_low));
  FE_CUDA_TRY(cudaEventCreateWithFlags(&d->ev_assembled, cudaEventDisableTiming));
  FE_CUDA_TRY(cudaEventCreateWithFlags(&d->ev_factored, cudaEventDisableTiming));
  FE_CUDA_TRY(cudaEventCreateWithFlags(&d->ev_apply_done, cudaEventDisableTiming));
  FE_CUDA_TRY(cudaEventCreateWithFlags(&d->ev_main_tail, cudaEventDisableTiming));
  FE_CUDA_TRY(cudaEventCreateWithFlags(&d->ev_noalloc_done, cudaEventDisableTiming));

  const int64_t n = c->n, E = c->n_elems, nf = int64_t(c->fronts.size());
  const int npe = c->npe, ke = 9 * npe * npe;
  const bool fp32 = mixed(c);
  const size_t ts = fp32 ? 4 : 8;
  // mesh / setup products
  FE_TRY(upload(c, d, &d->conn, c->conn));
  FE_TRY(upload(c, d, &d->rest, c->rest));
  {
    std::vector<double> pt(3 * E);
    for (int64_t e = 0; e < E; ++e)
      for (int k = 0; k < 3; ++k) pt[k * E + e] = c->params[3 * e + k];
    FE_TRY(upload(c, d, &d->params, pt));
    if (fp32 && !c->opt.element_fp64) {  // the double-float force's inputs
      FE_TRY(upload(c, d, &d->rest2, float_pairs(c->rest)));
      FE_TRY(upload(c, d, &d->params2, float_pairs(pt)));
      FE_TRY(dalloc(c, d, &d->u2, size_t(n)));
    }
  }
  FE_TRY(upload(c, d, &d->X, c->X));
  FE_TRY(upload(c, d, &d->rowptr, c->rowptr));
  FE_TRY(upload(c, d, &d->colind, c->colind));
  {
    std::vector<int32_t> sp(c->slot_ptr.size());
    for (size_t i = 0; i < sp.size(); ++i) sp[i] = int32_t(c->slot_ptr[i]);
    FE_TRY(upload(c, d, &d->slot_ptr, sp));
  }
  FE_TRY(upload(c, d, &d->slot_src, c->slot_src));
  FE_TRY(upload(c, d, &d->mass, c->mass));
  FE_TRY(upload(c, d, &d->fixed_row, c->fixed_dof));
  FE_TRY(upload(c, d, &d->node_ptr, c->node_ptr));
  FE_TRY(upload(c, d, &d->node_src, c->node_src));
  FE_TRY(upload(c, d, &d->bptr, c->bptr));
  FE_TRY(upload(c, d, &d->bcol, c->bcol));
  FE_TRY(upload(c, d, &d->bsrc_ptr, c->bsrc_ptr));
  FE_TRY(upload(c, d, &d->bsrc, c->bsrc));
  FE_TRY(upload(c, d, &d->bmass, c->bmass));
  {
    std::vector<int64_t> sd(c->nseg + 1);
    std::vector<int32_t> rs(c->n);
    for (int32_t k = 0; k <= c->nseg; ++k) sd[k] = 3 * c->seg_node[k];
    for (int32_t k = 0; k < c->nseg; ++k)
      for (int64_t i = sd[k]; i < sd[k + 1]; ++i) rs[i] = k;
    FE_TRY(upload(c, d, &d->seg_dof, sd));
    FE_TRY(upload(c, d, &d->row_seg, rs));
    FE_TRY(dalloc(c, d, &d->bscal, size_t(c->nseg) * B_COUNT));
    FE_CUDA_TRY(cudaMemset(d->bscal, 0, size_t(c->nseg) * B_COUNT * sizeof(double)));
    FE_CUDA_TRY(cudaMallocHost(&d->h_bscal, size_t(c->nseg) * B_COUNT * sizeof(double)));
  }
  // state
  FE_TRY(upload(c, d, &d->q, c->X));
  FE_TRY(dalloc(c, d, &d->v, n));
  FE_CUDA_TRY(cudaMemset(d->v, 0, n * sizeof(double)));
  FE_TRY(dalloc(c, d, &d->pext, n));
  FE_TRY(dalloc(c, d, &d->acc, n));
  FE_TRY(dalloc(c, d, &d->a_prev, n));
  FE_CUDA_TRY(cudaMemset(d->a_prev, 0, n * sizeof(double)));
  FE_TRY(dalloc(c, d, &d->x, n));
  FE_TRY(dalloc(c, d, &d->r, n));
  FE_TRY(dalloc(c, d, &d->b, n));
  FE_TRY(dalloc(c, d, &d->fe, size_t(E) * 3 * npe));
  FE_TRY(dallocv(c, d, &d->Ke, size_t(E) * ke * (c->opt.element_fp64 ? sizeof(double) : ts)));
  FE_TRY(dallocv(c, d, &d->A, size_t(c->nnz) * ts));
  if (fp32) {
    FE_TRY(dalloc(c, d, &d->A2, size_t(c->nnz)));
    FE_TRY(dalloc(c, d, &d->x2, n));
    FE_CUDA_TRY(cudaMemset(d->x2, 0, n * sizeof(float2)));
    FE_TRY(upload(c, d, &d->bmass2, float_pairs(c->bmass)));
  } else {
    d->A64 = static_cast<double *>(d->A);
  }
  FE_TRY(dallocv(c, d, &d->Afac, size_t(c->nnz) * ts));
  FE_TRY(dallocv(c, d, &d->vz, n * ts));
  FE_TRY(dallocv(c, d, &d->vp, n * ts));
  FE_TRY(dallocv(c, d, &d->vq, n * ts));
  FE_TRY(dallocv(c, d, &d->vr, n * ts));
  FE_TRY(dallocv(c, d, &d->vd, n * ts));
  FE_CUDA_TRY(cudaMemset(d->vz, 0, n * ts));  // fixed DOFs of z stay 0 forever
  FE_TRY(dallocv(c, d, reinterpret_cast<void **>(&d->scal), S_COUNT * sizeof(double) + 4 * sizeof(int)));
  d->flags = reinterpret_cast<int *>(d->scal + S_COUNT);
  FE_CUDA_TRY(cudaMemset(d->scal, 0, S_COUNT * sizeof(double) + 4 * sizeof(int)));
  FE_TRY(dalloc(c, d, &d->partials, kMaxBlocks));
  FE_TRY(dallocv(c, d, reinterpret_cast<void **>(&d->tune_scal), S_COUNT * sizeof(double) + 4 * sizeof(int)));
  FE_TRY(dalloc(c, d, &d->ticket, 4));
  FE_CUDA_TRY(cudaMemset(d->ticket, 0, 4 * sizeof(unsigned int)));
  FE_CUDA_TRY(cudaMallocHost(&d->h_scal, S_COUNT * sizeof(double) + 4 * sizeof(int)));
  d->h_flags = reinterpret_cast<int *>(d->h_scal + S_COUNT);
  FE_CUDA_TRY(cudaMallocHost(&d->stage_in, n * sizeof(double)));
  FE_CUDA_TRY(cudaMallocHost(&d->stage_out, 2 * n * sizeof(double)));

  // multifrontal factor
  std::vector<DFront> df(nf);
  int64_t fac = 0;
  for (int64_t f = 0; f < nf; ++f) {
    const Front &F = c->fronts[f];
    DFront &o = df[f];
    o.first = F.first; o.npiv = F.npiv; o.nupd = F.nupd; o.m = F.m();
    o.child_begin = c->child_ptr[f]; o.child_end = c->child_ptr[f + 1];
    o.f_off = F.f_off; o.y_off = F.y_off; o.w_off = F.w_off; o.u_off = F.u_off;
    o.rows_off = F.rows_off; o.fac_off = fac;
    o.ldy = F.ldy; o.parent = F.parent; o.ldf = F.ldf;
    o.fcols = int16_t(F.fcols); o.brows = int16_t(F.brows);
    o.nfwd = c->front_nfwd[f]; o.nbwd = c->front_nbwd[f];
    fac += F.npiv + 1;
  }
  FE_TRY(upload(c, d, &d->fronts, df));
  FE_TRY(upload(c, d, &d->perm, c->perm));
  FE_TRY(upload(c, d, &d->upd_rows_old, c->upd_rows_old));
  FE_TRY(upload(c, d, &d->rmap, c->rmap));
  FE_TRY(upload(c, d, &d->child_list, c->child_list));
  FE_TRY(upload(c, d, &d->fa_slot, c->fa_slot));
  FE_TRY(upload(c, d, &d->fa_off, c->fa_off));
  FE_TRY(upload(c, d, &d->fa_colptr, c->fa_colptr));
  FE_TRY(upload(c, d, &d->wsrc_ptr, c->wsrc_ptr));
  FE_TRY(upload(c, d, &d->wsrc, c->wsrc));
  // task lists, int4-aligned
  std::vector<int32_t> all;
  std::vector<int32_t> lf;
  auto pad4 = [&]() { while (all.size() % 4) all.push_back(0); };
  d->lt.assign(c->levels.size(), DeviceState::LevelTasks());
  for (size_t lv = 0; lv < c->levels.size(); ++lv) {
    const Level &L = c->levels[lv];
    auto &T = d->lt[lv];
    T.nfronts = int64_t(L.fronts.size());
    T.fronts_off = int64_t(lf.size());
    lf.insert(lf.end(), L.fronts.begin(), L.fronts.end());
    pad4();
    T.asm_off = int64_t(all.size()); T.asm_n = int64_t(L.asm_tasks.size() / 3);
    all.insert(all.end(), L.asm_tasks.begin(), L.asm_tasks.end());
    for (int s = 0; s < L.steps; ++s) {
      pad4();
      T.diag_off.push_back(int64_t(all.size())); T.diag_n.push_back(int64_t(L.diag[s].size() / 4));
      all.insert(all.end(), L.diag[s].begin(), L.diag[s].end());
      T.panel_off.push_back(int64_t(all.size())); T.panel_n.push_back(int64_t(L.panel[s].size() / 4));
      all.insert(all.end(), L.panel[s].begin(), L.panel[s].end());
      T.trail_off.push_back(int64_t(all.size())); T.trail_n.push_back(int64_t(L.trail[s].size() / 4));
      T.trail_flops.push_back(L.trail_flops[s]);
      all.insert(all.end(), L.trail[s].begin(), L.trail[s].end());
      T.tend_off.push_back(int64_t(all.size())); T.tend_n.push_back(int64_t(L.tend[s].size() / 4));
      T.tend_flops.push_back(L.tend_flops[s]);
      all.insert(all.end(), L.tend[s].begin(), L.tend[s].end());
    }
    pad4();
    T.fwd_off = int64_t(all.size()); T.fwd_n = int64_t(L.fwd_tasks.size() / 4);
    all.insert(all.end(), L.fwd_tasks.begin(), L.fwd_tasks.end());
    T.bwd_off = int64_t(all.size()); T.bwd_n = int64_t(L.bwd_tasks.size() / 4);
    all.insert(all.end(), L.bwd_tasks.begin(), L.bwd_tasks.end());
  }
  FE_TRY(upload(c, d, &d->tasks, all));
  FE_TRY(upload(c, d, &d->level_fronts, lf));
  FE_TRY(dallocv(c, d, &d->F, size_t(c->f_total) * ts));
  for (int k = 0; k < 2; ++k) {
    FE_TRY(dallocv(c, d, &d->Y[k], size_t(c->y_total) * ts));
    FE_TRY(dalloc(c, d, &d->D[k], size_t(2 * std::max<int64_t>(c->n_free, 1))));
    if (c->opt.precond_fp16) FE_TRY(dallocv(c, d, &d->Yh[k], size_t(c->y_total) * 2));
  }
  FE_TRY(dallocv(c, d, &d->wbuf, size_t(c->w_total) * ts));
  FE_TRY(dallocv(c, d, &d->ubuf, size_t(std::max<int64_t>(c->u_total, 1)) * ts));
  FE_TRY(dallocv(c, d, &d->yperm, size_t(std::max<int64_t>(c->n_free, 1)) * ts));
  if (c->opt.newton_iters > 1) {
    FE_TRY(dalloc(c, d, &d->na, size_t(c->n)));
    FE_TRY(dalloc(c, d, &d->nq, size_t(c->n)));
    FE_TRY(dalloc(c, d, &d->nv, size_t(c->n)));
  }
  // dataflow application: task lists and counters; the counters start in
  // their reset state (forward: the children's pending forward tasks, kept
  // in df_pend0 for the resets; backward: 0 done) and every application
  // leaves the other direction's counters reset
  FE_TRY(upload(c, d, &d->apply_fwd, c->apply_fwd));
  FE_TRY(upload(c, d, &d->apply_bwd, c->apply_bwd));
  d->n_apply_fwd = int64_t(c->apply_fwd.size() / 4);
  d->n_apply_bwd = int64_t(c->apply_bwd.size() / 4);
  {
    std::vector<int> pend(nf, 0), zero(nf, 0);
    for (int64_t f = 0; f < nf; ++f)
      if (c->fronts[f].parent >= 0) pend[c->fronts[f].parent] += c->front_nfwd[f];
    FE_TRY(upload(c, d, &d->df_pend, pend));
    FE_TRY(upload(c, d, &d->df_pend0, pend));
    FE_TRY(upload(c, d, &d->df_bdone, zero));
    FE_TRY(upload(c, d, &d->df_ctl, std::vector<int>(4, 0)));
  }
  if (mixed(c)) FE_TRY(encode_tensor_maps(c, d));
  const size_t rb = size_t(fwd_rows(c->opt));
  FE_TRY(dallocv(c, d, &d->part_f, size_t(std::max<int64_t>(c->fwd_slots, 1)) * rb * ts));
  FE_TRY(dallocv(c, d, &d->part_b, size_t(std::max<int64_t>(c->bwd_slots, 1)) * kBwdCols * ts));
  FE_TRY(dalloc(c, d, &d->tick_f, size_t(std::max<int64_t>(c->fwd_slots, 1))));
  FE_TRY(dalloc(c, d, &d->tick_b, size_t(std::max<int64_t>(c->bwd_slots, 1))));
  FE_CUDA_TRY(cudaMemset(d->tick_f, 0, size_t(std::max<int64_t>(c->fwd_slots, 1)) * sizeof(int)));
  FE_CUDA_TRY(cudaMemset(d->tick_b, 0, size_t(std::max<int64_t>(c->bwd_slots, 1)) * sizeof(int)));
  FE_CUDA_TRY(cudaDeviceSynchronize());
  return FE_OK;
}

// host or device pointer in -> device buffer (stream-ordered)
int stage_in(fe_ctx *c, double *dst, const double *src, int64_t n) {
  DeviceState *d = c->dev;
  if (c->opt.device_ptrs) {
    FE_CUDA_TRY(cudaMemcpyAsync(dst, src, n * sizeof(double), cudaMemcpyDeviceToDevice, d->stream));
  } else {
    std::memcpy(d->stage_in, src, n * sizeof(double));
    FE_CUDA_TRY(cudaMemcpyAsync(dst, d->stage_in, n * sizeof(double), cudaMemcpyHostToDevice, d->stream));
    FE_CUDA_TRY(cudaStreamSynchronize(d->stream));
  }
  return FE_OK;
}

int stage_out(fe_ctx *c, double *dst, const double *src, int64_t n, int slot) {
  DeviceState *d = c->dev;
  if (c->opt.device_ptrs) {
    FE_CUDA_TRY(cudaMemcpyAsync(dst, src, n * sizeof(double), cudaMemcpyDeviceToDevice, d->stream));
  } else {
    double *h = d->stage_out + slot * c->n;
    FE_CUDA_TRY(cudaMemcpyAsync(h, src, n * sizeof(double), cudaMemcpyDeviceToHost, d->stream));
    FE_CUDA_TRY(cudaStreamSynchronize(d->stream));
    std::memcpy(dst, h, n * sizeof(double));
  }
  return FE_OK;
}

int read_scalars(fe_ctx *c) {
  DeviceState *d = c->dev;
  FE_CUDA_TRY(cudaMemcpyAsync(d->h_scal, d->scal, S_COUNT * sizeof(double) + 4 * sizeof(int),
                              cudaMemcpyDeviceToHost, d->stream));
  FE_CUDA_TRY(cudaStreamSynchronize(d->stream));
  return FE_OK;
}

int flag_status(fe_ctx *c) {
  const int f = c->dev->h_flags[0];
  // a wait that gave up leaves its outputs incomplete, so whatever the later
  // kernels flagged follows from it: timeouts are reported first
  if (f & FLAG_WAIT_TIMEOUT)
    return set_error(c, FE_ERR_TIMEOUT, "a completion wait in the factorisation gave up");
  if (f & FLAG_APPLY_TIMEOUT)
    return set_error(c, FE_ERR_TIMEOUT, "a dependency wait in the preconditioner application gave up");
  if (f & FLAG_INVERTED) return set_error(c, FE_ERR_INVERTED, "an element has det F <= 0");
  if (f & FLAG_PIVOT) return set_error(c, FE_ERR_BREAKDOWN, "LDL^T pivot <= 0");
  if (f & FLAG_BREAKDOWN) return set_error(c, FE_ERR_BREAKDOWN, "CG breakdown (p^T A p <= 0 or r^T z <= 0)");
  if (c->dev->h_flags[1] & FLAG_APPLY_TIMEOUT) {
    // raised by an earlier allocation-free application: reported once
    c->dev->h_flags[1] = 0;
    FE_CUDA_TRY(cudaMemsetAsync(c->dev->flags + 1, 0, sizeof(int), c->dev->stream));
    return set_error(c, FE_ERR_TIMEOUT,
                     "an earlier fe_apply_preconditioner_noalloc gave up on a dependency wait (its z was incomplete)");
  }
  return FE_OK;
}

// Clears the step's own error flags (word 0); word 1, raised by an
// allocation-free application, stays until a flag check reports it.
int clear_flags(fe_ctx *c) {
  FE_CUDA_TRY(cudaMemsetAsync(c->dev->flags, 0, sizeof(int), c->dev->stream));
  return FE_OK;
}

// Wait until the factor launched on the side stream is done: a lagged factor
// with the host deadline factor_timeout_s, a synchronous one (the step's own
// work) with at least 300 s.
int wait_factor(fe_ctx *c, bool lagged) {
  DeviceState *d = c->dev;
  if (d->factor_pending < 0) return FE_OK;
  const double limit = lagged ? c->opt.factor_timeout_s : std::max(c->opt.factor_timeout_s, 300.0);
  auto t0 = std::chrono::steady_clock::now();
  for (;;) {
    cudaError_t e = cudaEventQuery(d->ev_factored);
    if (e == cudaSuccess) break;
    if (e != cudaErrorNotReady) return set_error(c, FE_ERR_CUDA, std::string("factor: ") + cudaGetErrorString(e));
    double el = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    if (el > limit) return set_error(c, FE_ERR_TIMEOUT, "factor not ready before the deadline");
    std::this_thread::sleep_for(std::chrono::microseconds(50));
  }
  FE_CUDA_TRY(cudaStreamWaitEvent(d->stream, d->ev_factored, 0));
  d->cur = d->factor_pending;
  d->cur_step = d->pending_step;
  d->factor_pending = -1;
  d->have_factor = true;
  return FE_OK;
}

// Snapshot A (main stream) and factor it on the side stream into the free buffer.
int launch_factor(fe_ctx *c, int64_t step_tag) {
  DeviceState *d = c->dev;
  const bool fp32 = mixed(c);
  const int buf = d->have_factor ? 1 - d->cur : d->cur;
  FE_CUDA_TRY(cudaMemcpyAsync(d->Afac, d->A, size_t(c->nnz) * vsz(c), cudaMemcpyDeviceToDevice, d->stream));
  FE_CUDA_TRY(cudaEventRecord(d->ev_assembled, d->stream));
  FE_CUDA_TRY(cudaStreamWaitEvent(d->fstream, d->ev_assembled, 0));
  {
    Stage st(c, FE_STAGE_FACTOR, d->fstream);
    factor_enqueue(c, d, buf, fp32, d->Afac, d->fstream);
  }
  FE_CUDA_TRY(cudaGetLastError());
  FE_CUDA_TRY(cudaEventRecord(d->ev_factored, d->fstream));
  d->factor_pending = buf;
  d->pending_step = step_tag;
  return FE_OK;
}

// ------------------------------------------------------- whole-step graph
// use_graph: the solve of a step (the PCG, and in the mixed path the FP64
// refinement around it) and the integration run as one CUDA graph whose
// loops are WHILE conditional nodes; a one-thread kernel at the end of each
// loop body (and one before the loop) sets the loop's condition from the
// device scalars, so the step makes no host read until it is done.

// The graph being captured on s.
static cudaGraph_t capturing_graph(cudaStream_t s) {
  cudaStreamCaptureStatus st;
  cudaGraph_t g = nullptr;
  if (cudaStreamGetCaptureInfo(s, &st, nullptr, &g, nullptr, nullptr, nullptr) != cudaSuccess) return nullptr;
  return g;
}

// Appends a WHILE node on handle h after everything captured so far on s;
// returns its body graph, and the capture on s goes on after the node.
static cudaError_t add_while(cudaStream_t s, cudaGraphConditionalHandle h, cudaGraph_t *body) {
  cudaStreamCaptureStatus st;
  cudaGraph_t g = nullptr;
  const cudaGraphNode_t *deps = nullptr;
  const cudaGraphEdgeData *edges = nullptr;
  size_t nd = 0;
  cudaError_t e = cudaStreamGetCaptureInfo(s, &st, nullptr, &g, &deps, &edges, &nd);
  if (e != cudaSuccess) return e;
  cudaGraphNodeParams p{};
  p.type = cudaGraphNodeTypeConditional;
  p.conditional.handle = h;
  p.conditional.type = cudaGraphCondTypeWhile;
  p.conditional.size = 1;
  cudaGraphNode_t node;
  e = cudaGraphAddNode(&node, g, deps, edges, nd, &p);
  if (e != cudaSuccess) return e;
  *body = p.conditional.phGraph_out[0];
  return cudaStreamUpdateCaptureDependencies(s, &node, nullptr, 1, cudaStreamSetCaptureDependencies);
}

// PCG on (X, R) after init_solve: the prologue (z = P^{-1} r, rz, p = z),
// then WHILE (S_DONE == 0) { q = A p, alpha; x += alpha p, r -= alpha q;
// z = P^{-1} r; beta; p = z + beta p }.  Captured on s; the loop body on s2.
static cudaError_t capture_pcg(fe_ctx *c, bool fp32, void *X, void *R, cudaStream_t s, cudaStream_t s2,
                               DeviceState::StepGraph *sg) {
  DeviceState *d = c->dev;
  const double *done = d->scal + S_DONE;
  int64_t l0 = d->launches;
  apply_enqueue(c, d, d->cur, fp32, R, d->vz, s, done);
  launch_dot_rz(c, d, fp32, R, d->vz, true, s);
  launch_update_p(c, d, fp32, d->vz, d->vp, true, s);
  cudaGraphConditionalHandle h;
  cudaError_t e = cudaGraphConditionalHandleCreate(&h, capturing_graph(s), 0, 0);
  if (e != cudaSuccess) return e;
  launch_graph_cond(c, d, h, 0, s);
  sg->k_pro += d->launches - l0;
  cudaGraph_t body;
  e = add_while(s, h, &body);
  if (e != cudaSuccess) return e;
  e = cudaStreamBeginCaptureToGraph(s2, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal);
  if (e != cudaSuccess) return e;
  l0 = d->launches;
  launch_spmv_dot(c, d, fp32, d->vp, d->vq, s2);
  launch_axpy_norm(c, d, fp32, X, R, d->vp, d->vq, s2);
  apply_enqueue(c, d, d->cur, fp32, R, d->vz, s2, done);
  launch_dot_rz(c, d, fp32, R, d->vz, false, s2);
  launch_update_p(c, d, fp32, d->vz, d->vp, false, s2);
  launch_graph_cond(c, d, h, 0, s2);
  sg->k_inner = d->launches - l0;
  return cudaStreamEndCapture(s2, &body);
}

// Captures the solve and the guarded integration of a step for the current
// factor buffer.  FP64: init (x = 0, r = b), PCG.  Mixed: init; WHILE
// (S_ODONE == 0, S_ITERS < max_iters) { inner init (d = 0, r32 = r); inner
// PCG to inner_tol; x += d; r = b - A x (FP64-accurate: A2, x2 in double-float) }.
static int build_step_graph(fe_ctx *c, DeviceState::StepGraph *sg) {
  DeviceState *d = c->dev;
  const bool fp32 = mixed(c);
  cudaStream_t s = d->stream, s2 = nullptr, s3 = nullptr;
  const int64_t l_save = d->launches;
  *sg = DeviceState::StepGraph{};
  cudaGraph_t g = nullptr;
  cudaError_t e = cudaStreamCreateWithFlags(&s2, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&s3, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal);
  if (e == cudaSuccess) {
    const bool warm = c->opt.warm_start != 0;
    if (warm) e = cudaMemcpyAsync(d->x, d->a_prev, c->n * sizeof(double), cudaMemcpyDeviceToDevice, s);
    if (e == cudaSuccess && !fp32) {
      launch_init_solve(c, d, false, d->x, d->r, d->b, c->opt.tol, true, s, warm);
      sg->k_pro = 1;
      if (warm) {
        launch_residual(c, d, false, s);
        launch_warm_fixup(c, d, s);
        sg->k_pro += 2;
      }
      e = capture_pcg(c, false, d->x, d->r, s, s2, sg);
    } else if (e == cudaSuccess) {
      launch_init_solve(c, d, false, d->x, d->r, d->b, c->opt.tol, true, s, warm);  // x = 0 (or kept), r = b
      if (warm) launch_residual(c, d, true, s);  // r = b - A x
      cudaGraphConditionalHandle ho;
      e = cudaGraphConditionalHandleCreate(&ho, capturing_graph(s), 0, 0);
      if (e == cudaSuccess) {
        launch_graph_cond(c, d, ho, 2, s);
        sg->k_pro = warm ? 3 : 2;
        cudaGraph_t body;
        e = add_while(s, ho, &body);
        if (e == cudaSuccess) e = cudaStreamBeginCaptureToGraph(s2, body, nullptr, nullptr, 0,
                                                                cudaStreamCaptureModeThreadLocal);
        if (e == cudaSuccess) {
          const int64_t l0 = d->launches;
          launch_init_solve(c, d, true, d->vd, d->vr, d->r, c->opt.inner_tol, false, s2);
          DeviceState::StepGraph inner{};
          e = capture_pcg(c, true, d->vd, d->vr, s2, s3, &inner);
          launch_refine_update(c, d, s2);
          launch_residual(c, d, true, s2);
          launch_graph_cond(c, d, ho, 1, s2);
          sg->k_outer = d->launches - l0 - inner.k_inner;
          sg->k_inner = inner.k_inner;
          cudaError_t e2 = cudaStreamEndCapture(s2, &body);
          if (e == cudaSuccess) e = e2;
        }
      }
    }
    launch_integrate_guarded(c, d, fp32, s);
    cudaError_t e2 = cudaStreamEndCapture(s, &g);
    if (e == cudaSuccess) e = e2;
  }
  if (e == cudaSuccess) e = cudaGraphInstantiate(&sg->exec, g, 0);
  if (g) cudaGraphDestroy(g);
  if (s2) cudaStreamDestroy(s2);
  if (s3) cudaStreamDestroy(s3);
  d->launches = l_save;
  if (e != cudaSuccess) {
    cudaGetLastError();
    sg->exec = nullptr;
    return set_error(c, FE_ERR_CUDA, std::string("whole-step graph: ") + cudaGetErrorString(e));
  }
  sg->cur = d->cur;
  return FE_OK;
}

// The batched solve as one graph: the same kernels as pcg_batch and
// solve_batch, with WHILE loops that go on while some member's PCG (or
// refinement) has not converged, none has reached max_iters and no error
// flag is set; a member that converged stops changing (its alpha is 0 and
// its direction frozen).  The integration is guarded by every member
// having converged.
static cudaError_t capture_pcg_batch(fe_ctx *c, bool fp32, void *X, void *R, cudaStream_t s, cudaStream_t s2,
                                     DeviceState::StepGraph *sg) {
  DeviceState *d = c->dev;
  int64_t l0 = d->launches;
  apply_enqueue(c, d, d->cur, fp32, R, d->vz, s);
  launch_seg_dot(c, d, fp32, R, d->vz, SEG_RZ_FIRST, 0.0, s);
  launch_seg_update_p(c, d, fp32, d->vz, d->vp, true, s);
  cudaGraphConditionalHandle h;
  cudaError_t e = cudaGraphConditionalHandleCreate(&h, capturing_graph(s), 0, 0);
  if (e != cudaSuccess) return e;
  launch_seg_cond(c, d, h, 0, s);
  sg->k_pro += d->launches - l0;
  cudaGraph_t body;
  e = add_while(s, h, &body);
  if (e != cudaSuccess) return e;
  e = cudaStreamBeginCaptureToGraph(s2, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal);
  if (e != cudaSuccess) return e;
  l0 = d->launches;
  launch_batch_spmv(c, d, fp32, d->vp, d->vq, nullptr, s2);
  launch_seg_dot(c, d, fp32, d->vp, d->vq, SEG_PQ, 0.0, s2);
  launch_seg_axpy(c, d, fp32, X, R, d->vp, d->vq, s2);
  launch_seg_dot(c, d, fp32, R, R, SEG_RR, 0.0, s2);
  apply_enqueue(c, d, d->cur, fp32, R, d->vz, s2);
  launch_seg_dot(c, d, fp32, R, d->vz, SEG_RZ, 0.0, s2);
  launch_seg_update_p(c, d, fp32, d->vz, d->vp, false, s2);
  launch_seg_cond(c, d, h, 0, s2);
  sg->k_inner = d->launches - l0;
  return cudaStreamEndCapture(s2, &body);
}

static int build_batch_graph(fe_ctx *c, DeviceState::StepGraph *sg) {
  DeviceState *d = c->dev;
  const bool fp32 = mixed(c);
  cudaStream_t s = d->stream, s2 = nullptr, s3 = nullptr;
  const int64_t l_save = d->launches;
  *sg = DeviceState::StepGraph{};
  cudaGraph_t g = nullptr;
  cudaError_t e = cudaStreamCreateWithFlags(&s2, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&s3, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal);
  if (e == cudaSuccess) {
    launch_seg_init(c, d, false, d->x, d->r, d->b, false, s);
    launch_seg_dot64(c, d, d->b, d->b, SEG_INIT_OUTER, c->opt.tol, s);
    sg->k_pro = 2;
    if (!fp32) {
      e = capture_pcg_batch(c, false, d->x, d->r, s, s2, sg);
    } else {
      cudaGraphConditionalHandle ho;
      e = cudaGraphConditionalHandleCreate(&ho, capturing_graph(s), 0, 0);
      if (e == cudaSuccess) {
        launch_seg_cond(c, d, ho, 2, s);
        sg->k_pro += 1;
        cudaGraph_t body;
        e = add_while(s, ho, &body);
        if (e == cudaSuccess)
          e = cudaStreamBeginCaptureToGraph(s2, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal);
        if (e == cudaSuccess) {
          const int64_t l0 = d->launches;
          launch_seg_init(c, d, true, d->vd, d->vr, d->r, true, s2);
          launch_seg_dot(c, d, true, d->vr, d->vr, SEG_INIT_INNER, c->opt.inner_tol, s2);
          DeviceState::StepGraph inner{};
          e = capture_pcg_batch(c, true, d->vd, d->vr, s2, s3, &inner);
          launch_refine_update(c, d, s2);
          launch_batch_spmv(c, d, true, d->x, d->r, d->b, s2);  // r = b - A x (FP64-accurate)
          launch_seg_dot64(c, d, d->r, d->r, SEG_ORR, 0.0, s2);
          launch_seg_cond(c, d, ho, 1, s2);
          sg->k_outer = d->launches - l0 - inner.k_inner;
          sg->k_inner = inner.k_inner;
          cudaError_t e2 = cudaStreamEndCapture(s2, &body);
          if (e == cudaSuccess) e = e2;
        }
      }
    }
    launch_seg_cond(c, d, cudaGraphConditionalHandle{}, fp32 ? 4 : 3, s);
    launch_integrate_guarded(c, d, fp32, s);
    cudaError_t e2 = cudaStreamEndCapture(s, &g);
    if (e == cudaSuccess) e = e2;
  }
  if (e == cudaSuccess) e = cudaGraphInstantiate(&sg->exec, g, 0);
  if (g) cudaGraphDestroy(g);
  if (s2) cudaStreamDestroy(s2);
  if (s3) cudaStreamDestroy(s3);
  d->launches = l_save;
  if (e != cudaSuccess) {
    cudaGetLastError();
    sg->exec = nullptr;
    return set_error(c, FE_ERR_CUDA, std::string("batched whole-step graph: ") + cudaGetErrorString(e));
  }
  sg->cur = d->cur;
  return FE_OK;
}

int read_batch_scalars(fe_ctx *c);
bool all_members(const fe_ctx *c, int slot);
double max_member(const fe_ctx *c, int slot);

// The solve and integration of one step through the cached graph of the
// current factor buffer; one host read at the end.
static int solve_integrate_graph(fe_ctx *c, fe_step_info *info) {
  DeviceState *d = c->dev;
  const bool batch = c->nseg > 1;
  if (batch) FE_TRY(tune_batch_spmv(c, d));
  else FE_TRY(tune_spmv(c, d));
  // the application kernels' grids depend on whether a factorisation is in
  // flight (apply_sm_share): one graph per (factor buffer, in flight)
  const int gi = 2 * d->cur + ((d->factor_pending >= 0 && c->opt.apply_sm_share > 0.0) ? 1 : 0);
  DeviceState::StepGraph &sg = d->step_graph[gi];
  if (!sg.exec || sg.cur != d->cur) FE_TRY(batch ? build_batch_graph(c, &sg) : build_step_graph(c, &sg));
  launch_pending_hold(d, d->stream);
  {
    Stage st(c, FE_STAGE_PCG_GRAPH, d->stream);
    FE_CUDA_TRY(cudaGraphLaunch(sg.exec, d->stream));
  }
  if (batch) {
    FE_TRY(read_batch_scalars(c));
    const double iters = max_member(c, B_ITERS), sweeps = mixed(c) ? d->h_scal[S_SWEEPS] : 1.0;
    d->launches += sg.k_pro + int64_t(iters) * sg.k_inner + int64_t(sweeps) * sg.k_outer + 2;
    FE_TRY(flag_status(c));
    if (!all_members(c, mixed(c) ? B_ODONE : B_DONE))
      return set_error(c, FE_ERR_NOT_CONVERGED, "batched PCG reached max_iters");
    if (info) {
      double worst = 0.0;
      for (int32_t k = 0; k < c->nseg; ++k) {
        const double *b = d->h_bscal + k * B_COUNT;
        const double rr = mixed(c) ? b[B_ORR] : b[B_RR];
        if (b[B_BB] > 0) worst = std::max(worst, std::sqrt(rr / b[B_BB]));
      }
      info->rel_residual = worst;
      info->iters = int32_t(iters);
      info->refinements = int32_t(sweeps);
    }
    return FE_OK;
  }
  FE_TRY(read_scalars(c));
  const double iters = d->h_scal[S_ITERS], sweeps = mixed(c) ? d->h_scal[S_SWEEPS] : 1.0;
  d->launches += sg.k_pro + int64_t(iters) * sg.k_inner + int64_t(sweeps) * sg.k_outer + 1;
  FE_TRY(flag_status(c));
  const bool ok = mixed(c) ? d->h_scal[S_ODONE] == 1.0 : d->h_scal[S_DONE] == 1.0;
  if (!ok) return set_error(c, FE_ERR_NOT_CONVERGED, "PCG reached max_iters");
  if (info) {
    info->iters = int32_t(iters);
    info->refinements = int32_t(sweeps);
    const double rr = mixed(c) ? d->h_scal[S_ORR] : d->h_scal[S_RR];
    info->rel_residual = d->h_scal[S_BB] > 0 ? std::sqrt(rr / d->h_scal[S_BB]) : 0.0;
  }
  return FE_OK;
}

static int pcg_status(fe_ctx *c) {
  if (c->dev->h_scal[S_DONE] == 2.0) return set_error(c, FE_ERR_NOT_CONVERGED, "PCG reached max_iters");
  return FE_OK;
}

// PCG on (X, R) with the current factor; X = 0 and R = rhs were set by
// init_solve.  Iterations accumulate in S_ITERS.  One host read of the
// device scalars per iteration, or per replay of the iteration graph.
int pcg(fe_ctx *c, bool fp32, void *X, void *R) {
  DeviceState *d = c->dev;
  cudaStream_t s = d->stream;
  {
    Stage st(c, FE_STAGE_APPLY, s);
    apply_enqueue(c, d, d->cur, fp32, R, d->vz, s);
  }
  {
    Stage st(c, FE_STAGE_VECTOR, s);
    launch_dot_rz(c, d, fp32, R, d->vz, true, s);
    launch_update_p(c, d, fp32, d->vz, d->vp, true, s);
  }
  for (;;) {
    {
      Stage st(c, FE_STAGE_SPMV, s);
      launch_spmv_dot(c, d, fp32, d->vp, d->vq, s);
    }
    {
      Stage st(c, FE_STAGE_VECTOR, s);
      launch_axpy_norm(c, d, fp32, X, R, d->vp, d->vq, s);
    }
    FE_CUDA_TRY(cudaGetLastError());
    FE_TRY(read_scalars(c));
    FE_TRY(flag_status(c));
    if (d->h_scal[S_DONE] != 0.0) return pcg_status(c);
    {
      Stage st(c, FE_STAGE_APPLY, s);
      apply_enqueue(c, d, d->cur, fp32, R, d->vz, s);
    }
    Stage st(c, FE_STAGE_VECTOR, s);
    launch_dot_rz(c, d, fp32, R, d->vz, false, s);
    launch_update_p(c, d, fp32, d->vz, d->vp, false, s);
  }
}

int read_batch_scalars(fe_ctx *c) {
  DeviceState *d = c->dev;
  FE_CUDA_TRY(cudaMemcpyAsync(d->h_bscal, d->bscal, size_t(c->nseg) * B_COUNT * sizeof(double),
                              cudaMemcpyDeviceToHost, d->stream));
  FE_CUDA_TRY(cudaMemcpyAsync(d->h_scal, d->scal, S_COUNT * sizeof(double) + 4 * sizeof(int),
                              cudaMemcpyDeviceToHost, d->stream));
  FE_CUDA_TRY(cudaStreamSynchronize(d->stream));
  return FE_OK;
}

bool all_members(const fe_ctx *c, int slot) {
  for (int32_t k = 0; k < c->nseg; ++k)
    if (c->dev->h_bscal[k * B_COUNT + slot] == 0.0) return false;
  return true;
}

double max_member(const fe_ctx *c, int slot) {
  double m = 0.0;
  for (int32_t k = 0; k < c->nseg; ++k) m = std::max(m, c->dev->h_bscal[k * B_COUNT + slot]);
  return m;
}

// Batched PCG: per-member alpha, beta, residual and convergence.
int pcg_batch(fe_ctx *c, bool fp32, void *X, void *R) {
  DeviceState *d = c->dev;
  cudaStream_t s = d->stream;
  {
    Stage st(c, FE_STAGE_APPLY, s);
    apply_enqueue(c, d, d->cur, fp32, R, d->vz, s);
  }
  launch_seg_dot(c, d, fp32, R, d->vz, SEG_RZ_FIRST, 0.0, s);
  launch_seg_update_p(c, d, fp32, d->vz, d->vp, true, s);
  for (;;) {
    {
      Stage st(c, FE_STAGE_SPMV, s);
      launch_batch_spmv(c, d, fp32, d->vp, d->vq, nullptr, s);
    }
    {
      Stage st(c, FE_STAGE_VECTOR, s);
      launch_seg_dot(c, d, fp32, d->vp, d->vq, SEG_PQ, 0.0, s);
      launch_seg_axpy(c, d, fp32, X, R, d->vp, d->vq, s);
      launch_seg_dot(c, d, fp32, R, R, SEG_RR, 0.0, s);
    }
    FE_CUDA_TRY(cudaGetLastError());
    FE_TRY(read_batch_scalars(c));
    FE_TRY(flag_status(c));
    if (all_members(c, B_DONE)) break;
    if (max_member(c, B_ITERS) >= c->opt.max_iters)
      return set_error(c, FE_ERR_NOT_CONVERGED, "batched PCG reached max_iters");
    {
      Stage st(c, FE_STAGE_APPLY, s);
      apply_enqueue(c, d, d->cur, fp32, R, d->vz, s);
    }
    Stage st(c, FE_STAGE_VECTOR, s);
    launch_seg_dot(c, d, fp32, R, d->vz, SEG_RZ, 0.0, s);
    launch_seg_update_p(c, d, fp32, d->vz, d->vp, false, s);
  }
  return FE_OK;
}

int solve_batch(fe_ctx *c, fe_step_info *info) {
  DeviceState *d = c->dev;
  cudaStream_t s = d->stream;
  const bool fp32 = mixed(c);
  FE_TRY(tune_batch_spmv(c, d));
  int sweeps = 0;
  launch_seg_init(c, d, false, d->x, d->r, d->b, false, s);
  launch_seg_dot64(c, d, d->b, d->b, SEG_INIT_OUTER, c->opt.tol, s);
  if (!fp32) {
    FE_TRY(read_batch_scalars(c));
    if (!all_members(c, B_DONE)) FE_TRY(pcg_batch(c, false, d->x, d->r));
    sweeps = 1;
  } else {
    for (;;) {
      if (sweeps > 0) {
        Stage st(c, FE_STAGE_RESIDUAL, s);
        launch_batch_spmv(c, d, true, d->x, d->r, d->b, s);  // r = b - A x (FP64-accurate)
        launch_seg_dot64(c, d, d->r, d->r, SEG_ORR, 0.0, s);
      }
      FE_TRY(read_batch_scalars(c));
      FE_TRY(flag_status(c));
      if (all_members(c, B_ODONE)) break;
      if (max_member(c, B_ITERS) >= c->opt.max_iters)
        return set_error(c, FE_ERR_NOT_CONVERGED, "batched refinement reached max_iters");
      launch_seg_init(c, d, true, d->vd, d->vr, d->r, true, s);
      launch_seg_dot(c, d, true, d->vr, d->vr, SEG_INIT_INNER, c->opt.inner_tol, s);
      FE_TRY(pcg_batch(c, true, d->vd, d->vr));
      launch_refine_update(c, d, s);
      ++sweeps;
    }
  }
  if (info) {
    double worst = 0.0;
    for (int32_t k = 0; k < c->nseg; ++k) {
      const double *b = d->h_bscal + k * B_COUNT;
      const double rr = fp32 ? b[B_ORR] : b[B_RR];
      if (b[B_BB] > 0) worst = std::max(worst, std::sqrt(rr / b[B_BB]));
    }
    info->rel_residual = worst;
    info->iters = int32_t(max_member(c, B_ITERS));
    info->refinements = sweeps;
  }
  return FE_OK;
}

// Solve A a = b into d->x (FP64): plain PCG, or FP64 residual refinement
// around an FP32 inner PCG.
int solve(fe_ctx *c, fe_step_info *info, bool warm) {
  DeviceState *d = c->dev;
  if (c->nseg > 1) return solve_batch(c, info);
  FE_TRY(tune_spmv(c, d));
  cudaStream_t s = d->stream;
  const bool fp32 = mixed(c);
  int sweeps = 0;
  if (warm) FE_CUDA_TRY(cudaMemcpyAsync(d->x, d->a_prev, c->n * sizeof(double), cudaMemcpyDeviceToDevice, s));
  if (!fp32) {
    launch_init_solve(c, d, false, d->x, d->r, d->b, c->opt.tol, true, s, warm);
    if (warm) {  // r = b - A x and its norm become the PCG's starting point
      launch_residual(c, d, false, s);
      launch_warm_fixup(c, d, s);
    }
    FE_TRY(read_scalars(c));
    if (d->h_scal[S_DONE] == 0.0) FE_TRY(pcg(c, false, d->x, d->r));
    sweeps = 1;
    if (info) info->rel_residual = d->h_scal[S_BB] > 0 ? std::sqrt(d->h_scal[S_RR] / d->h_scal[S_BB]) : 0.0;
  } else {
    launch_init_solve(c, d, false, d->x, d->r, d->b, c->opt.tol, true, s, warm);  // x = 0 (or kept), r = b
    for (;;) {
      if (sweeps > 0 || warm) {
        Stage st(c, FE_STAGE_RESIDUAL, s);
        launch_residual(c, d, true, s);
      }
      FE_TRY(read_scalars(c));
      FE_TRY(flag_status(c));
      if (d->h_scal[S_ODONE] != 0.0) break;
      if (d->h_scal[S_ITERS] >= c->opt.max_iters)
        return set_error(c, FE_ERR_NOT_CONVERGED, "refinement reached max_iters");
      launch_init_solve(c, d, true, d->vd, d->vr, d->r, c->opt.inner_tol, false, s);
      FE_TRY(pcg(c, true, d->vd, d->vr));
      launch_refine_update(c, d, s);
      ++sweeps;
    }
    if (info) info->rel_residual = d->h_scal[S_BB] > 0 ? std::sqrt(d->h_scal[S_ORR] / d->h_scal[S_BB]) : 0.0;
  }
  if (info) {
    info->iters = int32_t(d->h_scal[S_ITERS]);
    info->refinements = sweeps;
  }
  return FE_OK;
}

}  // namespace

void destroy_device(fe_ctx *c) {
  DeviceState *d = c->dev;
  if (!d) return;
  cudaDeviceSynchronize();
  for (void *p : d->allocs) cudaFree(p);
  for (double *p : d->ckpt) cudaFree(p);
  if (d->h_scal) cudaFreeHost(d->h_scal);
  if (d->h_bscal) cudaFreeHost(d->h_bscal);
  if (d->stage_in) cudaFreeHost(d->stage_in);
  if (d->stage_out) cudaFreeHost(d->stage_out);
  if (d->stage_big) cudaFreeHost(d->stage_big);
  if (d->ev_assembled) cudaEventDestroy(d->ev_assembled);
  if (d->ev_factored) cudaEventDestroy(d->ev_factored);
  if (d->ev_apply_done) cudaEventDestroy(d->ev_apply_done);
  if (d->ev_main_tail) cudaEventDestroy(d->ev_main_tail);
  if (d->ev_noalloc_done) cudaEventDestroy(d->ev_noalloc_done);
  for (auto &r : d->recs) {
    cudaEventDestroy(r.a);
    cudaEventDestroy(r.b);
  }
  for (cudaEvent_t e : d->pool) cudaEventDestroy(e);
  for (auto &g : d->step_graph)
    if (g.exec) cudaGraphExecDestroy(g.exec);
  if (d->fstream) cudaStreamDestroy(d->fstream);
  if (d->own_stream && d->stream) cudaStreamDestroy(d->stream);
  cudaGetLastError();
  delete d;
  c->dev = nullptr;
}

}  // namespace fe

using namespace fe;

extern "C" {

int fe_set_state(fe_ctx *c, const double *q, const double *v) {
  if (!c) return FE_ERR_ARG;
  if (!c->built) return set_error(c, FE_ERR_STATE, "fe_build_pattern has not run");
  if (!c->opt.device_ptrs) {  // host arrays are checked before any device work
    if (q)
      for (int64_t i = 0; i < c->n; ++i)
        if (!std::isfinite(q[i])) return set_error(c, FE_ERR_ARG, "q has a non-finite entry");
    if (v)
      for (int64_t i = 0; i < c->n; ++i) {
        if (!std::isfinite(v[i])) return set_error(c, FE_ERR_ARG, "v has a non-finite entry");
        if (c->fixed_dof[i] && v[i] != 0.0) return set_error(c, FE_ERR_ARG, "v must vanish on fixed DOFs");
      }
  }
  FE_TRY(ensure_device(c));
  if (q) FE_TRY(stage_in(c, c->dev->q, q, c->n));
  if (v) FE_TRY(stage_in(c, c->dev->v, v, c->n));
  // a new state: the next warm start begins from 0 again
  FE_CUDA_TRY(cudaMemsetAsync(c->dev->a_prev, 0, c->n * sizeof(double), c->dev->stream));
  FE_CUDA_TRY(cudaStreamSynchronize(c->dev->stream));
  return FE_OK;
}

int fe_get_state(fe_ctx *c, double *q, double *v) {
  if (!c) return FE_ERR_ARG;
  FE_TRY(ensure_device(c));
  if (q) FE_TRY(stage_out(c, q, c->dev->q, c->n, 0));
  if (v) FE_TRY(stage_out(c, v, c->dev->v, c->n, 1));
  FE_CUDA_TRY(cudaStreamSynchronize(c->dev->stream));
  return FE_OK;
}

int fe_element_eval(fe_ctx *c, const double *q, double *f_e, double *K_e) {
  if (!c) return FE_ERR_ARG;
  FE_TRY(ensure_device(c));
  DeviceState *d = c->dev;
  const double *qd = d->q;
  if (q) {
    FE_TRY(stage_in(c, d->x, q, c->n));
    qd = d->x;
  }
  FE_TRY(clear_flags(c));
  launch_element(c, d, qd, mixed(c), d->stream);
  FE_CUDA_TRY(cudaGetLastError());
  const int64_t nf = c->n_elems * 3 * c->npe, nk = c->n_elems * 9 * c->npe * c->npe;
  double *tmp = nullptr;
  FE_CUDA_TRY(cudaMalloc(&tmp, std::max(nf, nk) * sizeof(double)));
  auto out = [&](double *dst, const void *src, bool src32, int64_t cnt) -> int {
    launch_convert(src, src32, tmp, false, cnt, d->stream);
    FE_CUDA_TRY(cudaMemcpyAsync(dst, tmp, cnt * sizeof(double),
                                c->opt.device_ptrs ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, d->stream));
    FE_CUDA_TRY(cudaStreamSynchronize(d->stream));
    return FE_OK;
  };
  int st = FE_OK;
  if (f_e && d->u2) {  // the double-float force path stores f_e as float pairs
    launch_pair_to_double(reinterpret_cast<const float2 *>(d->fe), tmp, nf, d->stream);
    FE_CUDA_TRY(cudaMemcpyAsync(f_e, tmp, nf * sizeof(double),
                                c->opt.device_ptrs ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, d->stream));
    FE_CUDA_TRY(cudaStreamSynchronize(d->stream));
  } else if (f_e) {
    st = out(f_e, d->fe, false, nf);
  }
  if (!st && K_e) st = out(K_e, d->Ke, mixed(c) && !c->opt.element_fp64, nk);
  cudaFree(tmp);
  if (st) return st;
  FE_TRY(read_scalars(c));
  return flag_status(c);
}

int fe_assemble(fe_ctx *c, const double *p_ext, double *A_vals, double *b) {
  if (!c) return FE_ERR_ARG;
  FE_TRY(ensure_device(c));
  DeviceState *d = c->dev;
  const double *pd = nullptr;
  if (p_ext) {
    FE_TRY(stage_in(c, d->pext, p_ext, c->n));
    pd = d->pext;
  }
  FE_TRY(clear_flags(c));
  launch_element(c, d, d->q, mixed(c), d->stream);
  launch_assemble(c, d, mixed(c), pd, d->v, nullptr, c->beta + c->h, d->stream);
  FE_CUDA_TRY(cudaGetLastError());
  if (A_vals) {
    double *tmp = nullptr;
    FE_CUDA_TRY(cudaMalloc(&tmp, c->nnz * sizeof(double)));
    if (d->A2) launch_pair_to_double(d->A2, tmp, c->nnz, d->stream);  // the float-pair A, as doubles
    else launch_convert(d->A64, false, tmp, false, c->nnz, d->stream);
    cudaError_t e = cudaMemcpyAsync(A_vals, tmp, c->nnz * sizeof(double),
                                    c->opt.device_ptrs ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost,
                                    d->stream);
    cudaStreamSynchronize(d->stream);
    cudaFree(tmp);
    if (e != cudaSuccess) return set_error(c, FE_ERR_CUDA, cudaGetErrorString(e));
  }
  if (b) FE_TRY(stage_out(c, b, d->b, c->n, 0));
  FE_TRY(read_scalars(c));
  return flag_status(c);
}

int fe_factor_now(fe_ctx *c) {
  if (!c) return FE_ERR_ARG;
  FE_TRY(ensure_device(c));
  DeviceState *d = c->dev;
  FE_TRY(clear_flags(c));
  FE_TRY(launch_factor(c, d->step_index));
  FE_TRY(wait_factor(c, false));
  FE_TRY(read_scalars(c));
  return flag_status(c);
}

int fe_apply_preconditioner(fe_ctx *c, const double *r, double *z) {
  if (!c || !r || !z) return FE_ERR_ARG;
  FE_TRY(ensure_device(c));
  DeviceState *d = c->dev;
  if (!d->have_factor) return set_error(c, FE_ERR_STATE, "no factor: call fe_factor_now or fe_step first");
  FE_TRY(stage_in(c, d->r, r, c->n));
  const bool fp32 = mixed(c);
  launch_convert(d->r, false, d->vr, fp32, c->n, d->stream);
  FE_TRY(clear_flags(c));
  apply_enqueue(c, d, d->cur, fp32, d->vr, d->vz, d->stream);
  launch_convert(d->vz, fp32, d->x, false, c->n, d->stream);
  FE_CUDA_TRY(cudaGetLastError());
  FE_TRY(stage_out(c, z, d->x, c->n, 0));
  FE_TRY(read_scalars(c));
  return flag_status(c);
}

int fe_step(fe_ctx *c, const double *p_ext, double *q_out, double *v_out, fe_step_info *info) {
  if (!c) return FE_ERR_ARG;
  FE_TRY(ensure_device(c));
  DeviceState *d = c->dev;
  cudaStream_t s = d->stream;
  const bool fp32 = mixed(c);
  const int64_t step = d->step_index;
  const int R = c->opt.refactor_every;
  const double *pd = nullptr;
  if (p_ext) {
    FE_TRY(stage_in(c, d->pext, p_ext, c->n));
    pd = d->pext;
  }
  FE_TRY(clear_flags(c));
  // S1 element kernel, S3 gather assembly of A and b
  {
    Stage st(c, FE_STAGE_ELEMENT, s);
    launch_element(c, d, d->q, fp32, s);
  }
  {
    Stage st(c, FE_STAGE_ASSEMBLY, s);
    launch_assemble(c, d, fp32, pd, d->v, nullptr, c->beta + c->h, s);
  }
  FE_CUDA_TRY(cudaGetLastError());
  // S4 lagged refactorisation (Eq. "asynchronous preconditioner"): A_s is
  // snapshot at s = 0 mod R and factored on the side stream; its factor
  // replaces the current one at step s + k (k = factor_lag <= R), so it
  // preconditions steps s+k .. s+k+R-1.  Step 0 (and R = 1) factors
  // synchronously.  The schedule depends only on the step index.
  const int lag = c->opt.factor_lag;
  if (d->factor_pending >= 0 && (step >= d->pending_step + lag || step % R == 0))
    FE_TRY(wait_factor(c, true));
  if (step % R == 0) {
    FE_TRY(launch_factor(c, step));
    if (step == 0 || R == 1 || !d->have_factor) FE_TRY(wait_factor(c, false));
  }
  const int age = int(step - d->cur_step);
  // use_graph: S5-S7 PCG, S9 refinement and S8 integration as one graph
  // (no host read inside the step); contacts, Newton iterations and
  // checkpoints take the host-driven path below
  if (c->opt.use_graph && c->contact_node.empty() && d->c_m == 0 && c->opt.newton_iters <= 1 &&
      !c->opt.keep_checkpoints) {
    FE_TRY(solve_integrate_graph(c, info));
    if (q_out) FE_TRY(stage_out(c, q_out, d->q, c->n, 0));
    if (v_out) FE_TRY(stage_out(c, v_out, d->v, c->n, 1));
    if (info) {
      info->factor_age = age;
      info->newton = 1;
      info->newton_correction = 0.0;
    }
    d->step_index = step + 1;
    if (c->opt.profile_stages) stage_collect(c);
    return FE_OK;
  }
  // S5-S7 PCG, S9 refinement
  int st = solve(c, info, c->opt.warm_start && c->nseg == 1);
  if (!st && c->opt.keep_checkpoints) {
    double *ck = nullptr;
    cudaError_t e = cudaMalloc(&ck, 3 * size_t(c->n) * sizeof(double));
    if (e != cudaSuccess) {
      cudaGetLastError();
      return set_error(c, FE_ERR_OOM, "checkpoint allocation failed");
    }
    d->ckpt.push_back(ck);
    FE_CUDA_TRY(cudaMemcpyAsync(ck, d->q, c->n * sizeof(double), cudaMemcpyDeviceToDevice, s));
    FE_CUDA_TRY(cudaMemcpyAsync(ck + c->n, d->v, c->n * sizeof(double), cudaMemcpyDeviceToDevice, s));
    FE_CUDA_TRY(cudaMemcpyAsync(ck + 2 * c->n, d->x, c->n * sizeof(double), cudaMemcpyDeviceToDevice, s));
  }
  if (st) {
    // leave the state untouched; a pending factor still completes on its stream
    return st;
  }
  // Newton iterations beyond the paper's single linearisation: at
  // a_k, q_k = q + h v + h^2 a_k, v_k = v + h a_k; solve
  // A(q_k) delta = p - f(q_k) - (alpha M + beta K(q_k)) v_k - M a_k with the
  // current (lagged) preconditioner, a_{k+1} = a_k + delta.
  int newton = 1;
  double ncorr = 0.0;
  if (c->opt.newton_iters > 1) {
    FE_CUDA_TRY(cudaMemcpyAsync(d->na, d->x, c->n * sizeof(double), cudaMemcpyDeviceToDevice, s));
    fe_step_info sub{};
    for (int k = 1; k < c->opt.newton_iters; ++k) {
      launch_newton_state(c, d, d->na, d->nq, d->nv, s);
      {
        Stage st(c, FE_STAGE_ELEMENT, s);
        launch_element(c, d, d->nq, fp32, s);
      }
      {
        Stage st(c, FE_STAGE_ASSEMBLY, s);
        launch_assemble(c, d, fp32, pd, d->nv, d->na, c->beta, s);
      }
      FE_CUDA_TRY(cudaGetLastError());
      st = solve(c, &sub, false);
      if (st) return st;
      if (info) info->iters += sub.iters;
      launch_newton_update(c, d, d->x, d->na, s);
      FE_TRY(read_scalars(c));
      FE_TRY(flag_status(c));
      ++newton;
      ncorr = d->h_scal[S_NA] > 0 ? std::sqrt(d->h_scal[S_NDELTA] / d->h_scal[S_NA]) : 0.0;
      if (ncorr <= c->opt.newton_tol) break;
    }
    FE_CUDA_TRY(cudaMemcpyAsync(d->x, d->na, c->n * sizeof(double), cudaMemcpyDeviceToDevice, s));
    if (info) info->rel_residual = sub.rel_residual;
  }
  if (info) {
    info->newton = newton;
    info->newton_correction = ncorr;
  }
  // contacts: constraint resolution and motion correction (NEXT-3)
  if (!c->contact_node.empty() || d->c_m > 0) {
    Stage st(c, FE_STAGE_CONTACT, s);
    FE_TRY(contact_resolve(c, d, fp32));
  }
  // S8 backward Euler
  {
    Stage st(c, FE_STAGE_INTEGRATE, s);
    launch_integrate(c, d, s);
  }
  FE_CUDA_TRY(cudaGetLastError());
  if (q_out) FE_TRY(stage_out(c, q_out, d->q, c->n, 0));
  if (v_out) FE_TRY(stage_out(c, v_out, d->v, c->n, 1));
  if (info) info->factor_age = age;
  d->step_index = step + 1;
  if (c->opt.profile_stages) stage_collect(c);
  return FE_OK;
}

int fe_set_params(fe_ctx *c, const double *params) {
  if (!c || !params) return FE_ERR_ARG;
  for (int64_t e = 0; e < c->n_elems; ++e)
    for (int k = 0; k < 3; ++k) c->params[3 * e + k] = params[3 * e + k];
  if (c->dev) {
    const int64_t E = c->n_elems;
    std::vector<double> pt(3 * E);
    for (int64_t e = 0; e < E; ++e)
      for (int k = 0; k < 3; ++k) pt[k * E + e] = c->params[3 * e + k];
    FE_CUDA_TRY(cudaStreamSynchronize(c->dev->stream));
    FE_CUDA_TRY(cudaStreamSynchronize(c->dev->fstream));
    FE_CUDA_TRY(cudaMemcpy(c->dev->params, pt.data(), pt.size() * sizeof(double), cudaMemcpyHostToDevice));
    if (c->dev->params2) {
      const std::vector<float2> p2 = float_pairs(pt);
      FE_CUDA_TRY(cudaMemcpy(c->dev->params2, p2.data(), p2.size() * sizeof(float2), cudaMemcpyHostToDevice));
    }
  }
  return FE_OK;
}

int fe_clear_checkpoints(fe_ctx *c) {
  if (!c) return FE_ERR_ARG;
  if (!c->dev) return FE_OK;
  cudaStreamSynchronize(c->dev->stream);
  for (double *p : c->dev->ckpt) cudaFree(p);
  c->dev->ckpt.clear();
  return FE_OK;
}

int fe_num_checkpoints(fe_ctx *c, int64_t *count) {
  if (!c || !count) return FE_ERR_ARG;
  *count = c->dev ? int64_t(c->dev->ckpt.size()) : 0;
  return FE_OK;
}

int fe_adjoint(fe_ctx *c, const double *dL_dqT, const double *dL_dvT, double *dL_ds, double *dL_dp) {
  if (!c || !dL_dqT) return FE_ERR_ARG;
  if (c->model_range[FE_COROTATIONAL][1] > c->model_range[FE_COROTATIONAL][0])
    return set_error(c, FE_ERR_ARG, "co-rotational elements have no adjoint (no energy, no exact tangent)");
  FE_TRY(ensure_device(c));
  DeviceState *d = c->dev;
  const int64_t T = int64_t(d->ckpt.size());
  if (T == 0) return set_error(c, FE_ERR_STATE, "no checkpoints: run fe_step with keep_checkpoints = 1");
  cudaStream_t s = d->stream;
  const bool fp32 = mixed(c);
  const int64_t n = c->n, E = c->n_elems;
  if (!d->qbar) {
    FE_TRY(dalloc(c, d, &d->qbar, n));
    FE_TRY(dalloc(c, d, &d->vbar, n));
    FE_TRY(dalloc(c, d, &d->sbar, E));
    FE_TRY(dalloc(c, d, &d->ge, size_t(E) * 3 * c->npe));
    FE_TRY(dalloc(c, d, &d->kl, size_t(E) * 3 * c->npe));
  }
  FE_TRY(stage_in(c, d->qbar, dL_dqT, n));
  if (dL_dvT) {
    FE_TRY(stage_in(c, d->vbar, dL_dvT, n));
  } else {
    FE_CUDA_TRY(cudaMemsetAsync(d->vbar, 0, n * sizeof(double), s));
  }
  FE_CUDA_TRY(cudaMemsetAsync(d->sbar, 0, E * sizeof(double), s));
  FE_TRY(clear_flags(c));
  if (d->factor_pending >= 0) FE_TRY(wait_factor(c, false));
  const int R = c->opt.refactor_every;
  double *qsave = d->q, *vsave = d->v;
  int st = FE_OK;
  for (int64_t t = T - 1; t >= 0 && st == FE_OK; --t) {
    double *qt = d->ckpt[t], *vt = d->ckpt[t] + n, *at = d->ckpt[t] + 2 * n;
    // A_t at (q_t, v_t): element kernel + assembly (b is overwritten below)
    d->q = qt;
    d->v = vt;
    launch_element(c, d, qt, fp32, s);
    launch_assemble(c, d, fp32, nullptr, d->v, nullptr, c->beta + c->h, s);
    d->q = qsave;
    d->v = vsave;
    // lagged preconditioner for the reverse sweep: A_{T-1}, then every R steps
    if ((T - 1 - t) % R == 0) {
      st = launch_factor(c, t);
      if (!st) st = wait_factor(c, false);
      if (st) break;
    }
    launch_adjoint_rhs(c, d, d->qbar, d->vbar, d->b, s);
    st = solve(c, nullptr, false);  // lambda in d->x
    if (st) break;
    launch_adjoint_element(c, d, fp32, qt, d->x, at, vt, d->ge, d->kl, d->sbar, s);
    double *pb = nullptr;
    if (dL_dp && c->opt.device_ptrs) pb = dL_dp + t * n;
    launch_adjoint_gather(c, d, d->ge, d->kl, d->x, d->qbar, d->vbar, pb, s);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return set_error(c, FE_ERR_CUDA, cudaGetErrorString(e));
    if (dL_dp && !c->opt.device_ptrs) {
      st = stage_out(c, dL_dp + t * n, d->x, n, 0);
      if (!st)
        for (int64_t i = 0; i < n; ++i)
          if (c->fixed_dof[i]) dL_dp[t * n + i] = 0.0;
    }
  }
  d->q = qsave;
  d->v = vsave;
  if (st) return st;
  FE_TRY(read_scalars(c));
  FE_TRY(flag_status(c));
  FE_CUDA_TRY(cudaStreamSynchronize(s));
  if (dL_ds)
    FE_CUDA_TRY(cudaMemcpy(dL_ds, d->sbar, E * sizeof(double),
                           c->opt.device_ptrs ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost));
  return FE_OK;
}

int fe_get_batch_stats(fe_ctx *c, int32_t *iters, double *rel_residual) {
  if (!c) return FE_ERR_ARG;
  DeviceState *d = c->dev;
  for (int32_t k = 0; k < c->nseg; ++k) {
    const double *b = d ? d->h_bscal + k * B_COUNT : nullptr;
    if (iters) iters[k] = b ? int32_t(b[B_ITERS]) : 0;
    if (rel_residual) {
      const double rr = b ? (mixed(c) ? b[B_ORR] : b[B_RR]) : 0.0;
      rel_residual[k] = (b && b[B_BB] > 0) ? std::sqrt(rr / b[B_BB]) : 0.0;
    }
  }
  return FE_OK;
}

int fe_get_info(fe_ctx *c, fe_info *info) {
  if (!c || !info) return FE_ERR_ARG;
  if (!c->built) return set_error(c, FE_ERR_STATE, "fe_build_pattern has not run");
  info->n = c->n;
  info->nnz = c->nnz;
  info->ntrip = c->ntrip;
  info->n_free = c->n_free;
  info->n_fronts = int64_t(c->fronts.size());
  info->n_levels = int64_t(c->levels.size());
  info->y_nnz = c->y_nnz;
  info->factor_flops = c->factor_flops;
  info->device_bytes = c->dev ? int64_t(c->dev->bytes_total) : 0;
  info->noalloc_bytes = noalloc_scratch_bytes(c);
  info->ntrip_kept = c->slot_ptr.empty() ? 0 : c->slot_ptr.back();
  info->n_blocks = int64_t(c->bcol.size());
  return FE_OK;
}

int fe_debug_hold_front(fe_ctx *c, int64_t front, int32_t extra) {
  if (!c) return FE_ERR_ARG;
  if (!c->built) return set_error(c, FE_ERR_STATE, "fe_build_pattern has not run");
  if (front < 0 || front >= int64_t(c->fronts.size()) || extra <= 0)
    return set_error(c, FE_ERR_ARG, "front out of range or extra <= 0");
  FE_TRY(ensure_device(c));
  c->dev->df_hold = int(front);
  c->dev->df_hold_extra = extra;
  return FE_OK;
}

int fe_get_stage_times(fe_ctx *c, double *ms, int64_t *calls, int64_t *kernel_launches) {
  if (!c) return FE_ERR_ARG;
  DeviceState *d = c->dev;
  if (d) {
    cudaStreamSynchronize(d->stream);
    cudaStreamSynchronize(d->fstream);
    stage_collect(c);
  }
  for (int k = 0; k < FE_STAGE_COUNT; ++k) {
    if (ms) ms[k] = d ? d->stage_ms[k] : 0.0;
    if (calls) calls[k] = d ? d->stage_calls[k] : 0;
  }
  if (kernel_launches) *kernel_launches = d ? d->launches : 0;
  return FE_OK;
}

int fe_get_update_flops(fe_ctx *c, double *flops) {
  if (!c || !flops) return FE_ERR_ARG;
  *flops = c->dev ? c->dev->update_flops : 0.0;
  return FE_OK;
}

int fe_get_update_bf16_flops(fe_ctx *c, double *flops) {
  if (!c || !flops) return FE_ERR_ARG;
  *flops = c->dev ? c->dev->update_bf16_flops : 0.0;
  return FE_OK;
}

int fe_get_update_bf16_tiles(fe_ctx *c, int64_t *tiles) {
  if (!c || !tiles) return FE_ERR_ARG;
  *tiles = c->dev ? c->dev->update_bf16_tiles : 0;
  return FE_OK;
}

int fe_reset_stage_times(fe_ctx *c) {
  if (!c) return FE_ERR_ARG;
  DeviceState *d = c->dev;
  if (!d) return FE_OK;
  cudaStreamSynchronize(d->stream);
  cudaStreamSynchronize(d->fstream);
  stage_collect(c);
  for (int k = 0; k < FE_STAGE_COUNT; ++k) {
    d->stage_ms[k] = 0.0;
    d->stage_calls[k] = 0;
  }
  d->launches = 0;
  d->update_flops = 0.0;
  d->update_bf16_flops = 0.0;
  d->update_bf16_tiles = 0;
  return FE_OK;
}

}  // extern "C"
