// C-ABI entry points that need no GPU: context creation, setup, getters.
#include <cmath>
#include <cstring>
#include <new>

#include "fe_ctx.h"

using fe::set_error;

extern "C" {

int fe_options_default(fe_options *o) {
  if (!o) return FE_ERR_ARG;
  std::memset(o, 0, sizeof(*o));
  o->precision = FE_FP64;
  o->tol = 1e-8;
  o->max_iters = 1000;
  o->refactor_every = 1;
  o->device_ptrs = 0;
  o->stream = nullptr;
  o->keep_checkpoints = 0;
  o->nd_leaf_nodes = 64;
  o->inner_tol = 1e-4;
  o->factor_timeout_s = 30.0;
  o->use_graph = 0;
  o->newton_iters = 1;
  o->newton_tol = 0.0;
  o->factor_tf32 = 0;
  o->precond_fp16 = 0;
  o->contact_sweeps = 200;
  o->contact_tol = 1e-12;
  o->factor_lag = 1;
  o->dep_wait_s = 1.0;
  o->element_fp64 = 0;
  o->warm_start = 0;
  o->spmv_variant = -1;
  o->apply_sm_share = 0.0;
  o->update_bf16 = 1;
  return FE_OK;
}

int fe_create(const fe_mesh *mesh, const fe_material *mat, double h, double alpha, double beta,
              const fe_options *opt, fe_ctx **out) {
  if (!out) return FE_ERR_ARG;
  *out = nullptr;
  if (!mesh || !mat || !mesh->rest_xyz || !mesh->conn || mesh->n_nodes <= 0 || mesh->n_elems <= 0)
    return FE_ERR_ARG;
  if (mesh->elem_type != FE_TET4 && mesh->elem_type != FE_HEX8) return FE_ERR_ARG;
  if (mat->model < FE_SVK || mat->model > FE_COROTATIONAL || !mat->params) return FE_ERR_ARG;
  if (!(h > 0) || !std::isfinite(h) || !(mat->rho > 0) || !std::isfinite(mat->rho) || mesh->n_fixed < 0 ||
      (mesh->n_fixed > 0 && !mesh->fixed_nodes))
    return FE_ERR_ARG;
  if (!(alpha >= 0) || !std::isfinite(alpha) || !(beta >= 0) || !std::isfinite(beta)) return FE_ERR_ARG;
  if (mesh->n_nodes > (int64_t(1) << 29)) return FE_ERR_ARG;
  fe_ctx *c = new (std::nothrow) fe_ctx();
  if (!c) return FE_ERR_OOM;
  try {
    c->elem_type = mesh->elem_type;
    c->npe = mesh->elem_type == FE_TET4 ? 4 : 8;
    c->n_nodes = mesh->n_nodes;
    c->n_elems = mesh->n_elems;
    c->X.assign(mesh->rest_xyz, mesh->rest_xyz + 3 * mesh->n_nodes);
    for (double x : c->X)
      if (!std::isfinite(x)) { delete c; return FE_ERR_ARG; }
    c->conn.assign(mesh->conn, mesh->conn + c->npe * mesh->n_elems);
    for (int32_t v : c->conn)
      if (v < 0 || v >= mesh->n_nodes) { delete c; return FE_ERR_ARG; }
    if (mesh->n_fixed > 0) c->fixed_nodes.assign(mesh->fixed_nodes, mesh->fixed_nodes + mesh->n_fixed);
    for (int32_t v : c->fixed_nodes)
      if (v < 0 || v >= mesh->n_nodes) { delete c; return FE_ERR_ARG; }
    c->model = mat->model;
    c->rho = mat->rho;
    c->params.resize(3 * mesh->n_elems);
    for (int64_t e = 0; e < mesh->n_elems; ++e)
      for (int k = 0; k < 3; ++k) c->params[3 * e + k] = mat->per_element ? mat->params[3 * e + k] : mat->params[k];
    for (double p : c->params)
      if (!std::isfinite(p)) { delete c; return FE_ERR_ARG; }
    c->h = h;
    c->alpha = alpha;
    c->beta = beta;
    if (opt) c->opt = *opt; else fe_options_default(&c->opt);
    if (c->opt.max_iters <= 0) c->opt.max_iters = 1000;
    if (c->opt.refactor_every <= 0) c->opt.refactor_every = 1;
    if (!(c->opt.tol > 0)) c->opt.tol = 1e-8;
    if (!(c->opt.inner_tol > 0)) c->opt.inner_tol = 1e-4;
    if (!(c->opt.factor_timeout_s > 0)) c->opt.factor_timeout_s = 30.0;
    if (c->opt.nd_leaf_nodes <= 0) c->opt.nd_leaf_nodes = 64;
    if (c->opt.newton_iters <= 0) c->opt.newton_iters = 1;
    if (c->opt.precision != FE_MIXED) c->opt.precond_fp16 = 0;
    if (c->opt.contact_sweeps <= 0) c->opt.contact_sweeps = 200;
    if (!(c->opt.contact_tol > 0)) c->opt.contact_tol = 1e-12;
    c->opt.precond_fp16 = c->opt.precond_fp16 ? 1 : 0;
    if (c->opt.factor_lag <= 0) c->opt.factor_lag = 1;
    if (c->opt.refactor_every == 1) c->opt.factor_lag = 1;
    if (c->opt.factor_lag > c->opt.refactor_every) {
      delete c;
      return FE_ERR_ARG;  // two factor buffers: the next snapshot must come after the swap
    }
    if (!(c->opt.dep_wait_s > 0) || !std::isfinite(c->opt.dep_wait_s)) c->opt.dep_wait_s = 1.0;
    c->opt.element_fp64 = (c->opt.precision == FE_MIXED && c->opt.element_fp64) ? 1 : 0;
    c->opt.warm_start = c->opt.warm_start ? 1 : 0;
    c->opt.update_bf16 = (c->opt.precision == FE_MIXED && c->opt.update_bf16) ? 1 : 0;
    if (!(c->opt.apply_sm_share >= 0.0 && c->opt.apply_sm_share <= 0.9)) {
      delete c;
      return FE_ERR_ARG;
    }
    if (c->opt.spmv_variant < -1 || c->opt.spmv_variant > 5) {
      delete c;
      return FE_ERR_ARG;
    }
    if (c->opt.newton_iters > 1 && c->opt.keep_checkpoints) {
      delete c;
      return FE_ERR_ARG;  // the adjoint differentiates the single-linearisation step
    }
    if (c->model == FE_COROTATIONAL && c->opt.keep_checkpoints) {
      delete c;
      return FE_ERR_ARG;  // no energy, no exact tangent: no adjoint
    }
    c->nseg = 1;
    c->seg_node = {0, c->n_nodes};
    c->seg_elem = {0, c->n_elems};
    c->seg_member = {0};
    c->seg_model = {c->model};
    for (int k = 0; k < 4; ++k) c->model_range[k][0] = c->model_range[k][1] = 0;
    c->model_range[c->model][1] = c->n_elems;
  } catch (const std::bad_alloc &) {
    delete c;
    return FE_ERR_OOM;
  }
  *out = c;
  return FE_OK;
}

int fe_create_batch(int32_t nb, const fe_mesh *meshes, const fe_material *mats, double h, double alpha,
                    double beta, const fe_options *opt, fe_ctx **out) {
  if (!out) return FE_ERR_ARG;
  *out = nullptr;
  if (nb <= 0 || !meshes || !mats) return FE_ERR_ARG;
  for (int32_t k = 0; k < nb; ++k) {
    const fe_mesh &m = meshes[k];
    if (!m.rest_xyz || !m.conn || m.n_nodes <= 0 || m.n_elems <= 0 || m.elem_type != meshes[0].elem_type ||
        (m.n_fixed > 0 && !m.fixed_nodes) || mats[k].model < FE_SVK || mats[k].model > FE_COROTATIONAL ||
        !mats[k].params || !(mats[k].rho > 0) || mats[k].rho != mats[0].rho)
      return FE_ERR_ARG;
  }
  // members grouped by material model (stable), so each model is one element range
  std::vector<int32_t> order;
  for (int md = FE_SVK; md <= FE_COROTATIONAL; ++md)
    for (int32_t k = 0; k < nb; ++k)
      if (mats[k].model == md) order.push_back(k);
  const int npe = meshes[0].elem_type == FE_TET4 ? 4 : 8;
  int64_t NN = 0, NE = 0, NF = 0;
  for (int32_t k = 0; k < nb; ++k) {
    NN += meshes[k].n_nodes;
    NE += meshes[k].n_elems;
    NF += meshes[k].n_fixed;
  }
  try {
    std::vector<double> X(3 * NN), P(3 * NE);
    std::vector<int32_t> conn(npe * NE), fixed;
    fixed.reserve(NF);
    std::vector<int64_t> seg_node(nb + 1, 0), seg_elem(nb + 1, 0);
    std::vector<int32_t> seg_model(nb);
    for (int32_t s = 0; s < nb; ++s) {
      const int32_t k = order[s];
      const fe_mesh &m = meshes[k];
      const int64_t n0 = seg_node[s], e0 = seg_elem[s];
      if (n0 + m.n_nodes > (int64_t(1) << 29)) return FE_ERR_ARG;
      for (int64_t i = 0; i < 3 * m.n_nodes; ++i) X[3 * n0 + i] = m.rest_xyz[i];
      for (int64_t i = 0; i < npe * m.n_elems; ++i) {
        if (m.conn[i] < 0 || m.conn[i] >= m.n_nodes) return FE_ERR_ARG;
        conn[npe * e0 + i] = int32_t(m.conn[i] + n0);
      }
      for (int64_t i = 0; i < m.n_fixed; ++i) {
        if (m.fixed_nodes[i] < 0 || m.fixed_nodes[i] >= m.n_nodes) return FE_ERR_ARG;
        fixed.push_back(int32_t(m.fixed_nodes[i] + n0));
      }
      for (int64_t e = 0; e < m.n_elems; ++e)
        for (int q = 0; q < 3; ++q)
          P[3 * (e0 + e) + q] = mats[k].per_element ? mats[k].params[3 * e + q] : mats[k].params[q];
      seg_node[s + 1] = n0 + m.n_nodes;
      seg_elem[s + 1] = e0 + m.n_elems;
      seg_model[s] = mats[k].model;
    }
    fe_mesh all{meshes[0].elem_type, NN, NE, X.data(), conn.data(), int64_t(fixed.size()), fixed.data()};
    fe_material mat{mats[order[0]].model, mats[0].rho, P.data(), 1};
    int st = fe_create(&all, &mat, h, alpha, beta, opt, out);
    if (st) return st;
    fe_ctx *c = *out;
    c->nseg = nb;
    c->seg_node = seg_node;
    c->seg_elem = seg_elem;
    c->seg_member = order;
    c->seg_model = seg_model;
    for (int md = 0; md < 4; ++md) c->model_range[md][0] = c->model_range[md][1] = 0;
    for (int32_t s = 0; s < nb; ++s) {
      const int md = seg_model[s];
      if (c->model_range[md][1] == 0) c->model_range[md][0] = seg_elem[s];
      c->model_range[md][1] = seg_elem[s + 1];
    }
  } catch (const std::bad_alloc &) {
    return FE_ERR_OOM;
  }
  return FE_OK;
}

int fe_get_batch_layout(fe_ctx *c, int32_t *nb, const int32_t **member, const int64_t **node_off,
                        const int64_t **elem_off) {
  if (!c) return FE_ERR_ARG;
  if (nb) *nb = c->nseg;
  if (member) *member = c->seg_member.data();
  if (node_off) *node_off = c->seg_node.data();
  if (elem_off) *elem_off = c->seg_elem.data();
  return FE_OK;
}

int fe_build_pattern(fe_ctx *c) {
  if (!c) return FE_ERR_ARG;
  if (c->built) return set_error(c, FE_ERR_STATE, "pattern already built");
  try {
    return fe::build_pattern_host(c);
  } catch (const std::bad_alloc &) {
    return set_error(c, FE_ERR_OOM, "host allocation failed in fe_build_pattern");
  }
}

int fe_get_pattern(fe_ctx *c, int64_t *n, int64_t *nnz, const int32_t **rowptr, const int32_t **colind,
                   int64_t *ntrip, const int32_t **scatter) {
  if (!c) return FE_ERR_ARG;
  if (!c->built) return set_error(c, FE_ERR_STATE, "fe_build_pattern has not run");
  if (n) *n = c->n;
  if (nnz) *nnz = c->nnz;
  if (rowptr) *rowptr = c->rowptr.data();
  if (colind) *colind = c->colind.data();
  if (ntrip) *ntrip = c->ntrip;
  if (scatter) *scatter = c->C.data();
  return FE_OK;
}

int fe_get_inverse_map(fe_ctx *c, const int64_t **slot_ptr, const int32_t **slot_src) {
  if (!c) return FE_ERR_ARG;
  if (!c->built) return set_error(c, FE_ERR_STATE, "fe_build_pattern has not run");
  if (slot_ptr) *slot_ptr = c->slot_ptr.data();
  if (slot_src) *slot_src = c->slot_src.data();
  return FE_OK;
}

int fe_get_mass(fe_ctx *c, const double **mass_vals) {
  if (!c || !mass_vals) return FE_ERR_ARG;
  if (!c->built) return set_error(c, FE_ERR_STATE, "fe_build_pattern has not run");
  *mass_vals = c->mass.data();
  return FE_OK;
}

int fe_get_ordering(fe_ctx *c, int64_t *n_free, const int32_t **perm, int64_t *n_fronts,
                    const int32_t **first, const int32_t **npiv, const int32_t **nupd,
                    const int32_t **parent, const int32_t **level) {
  if (!c) return FE_ERR_ARG;
  if (!c->built) return set_error(c, FE_ERR_STATE, "fe_build_pattern has not run");
  if (n_free) *n_free = c->n_free;
  if (perm) *perm = c->perm.data();
  if (n_fronts) *n_fronts = int64_t(c->fronts.size());
  if (first) *first = c->front_first.data();
  if (npiv) *npiv = c->front_npiv.data();
  if (nupd) *nupd = c->front_nupd.data();
  if (parent) *parent = c->front_parent.data();
  if (level) *level = c->front_level.data();
  return FE_OK;
}

int fe_get_front_rows(fe_ctx *c, int64_t f, int64_t *n_upd, const int32_t **rows) {
  if (!c) return FE_ERR_ARG;
  if (!c->built) return set_error(c, FE_ERR_STATE, "fe_build_pattern has not run");
  if (f < 0 || f >= int64_t(c->fronts.size())) return set_error(c, FE_ERR_ARG, "front id out of range");
  if (n_upd) *n_upd = c->fronts[f].nupd;
  if (rows) *rows = c->upd_rows_old.data() + c->fronts[f].rows_off;
  return FE_OK;
}

const char *fe_last_error(const fe_ctx *c) { return c ? c->err.c_str() : "null context"; }

void fe_destroy(fe_ctx *c) {
  if (!c) return;
  fe::destroy_device(c);
  delete c;
}

}  // extern "C"
