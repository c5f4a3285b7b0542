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
  return FE_OK;
}

int fe_create(const fe_mesh *mesh, const fe_material *mat, double h, double alpha, double beta,
              const fe_options *opt, fe_ctx **out) {
  if (!out) return FE_ERR_ARG;
  *out = nullptr;
  if (!mesh || !mat || !mesh->rest_xyz || !mesh->conn || mesh->n_nodes <= 0 || mesh->n_elems <= 0)
    return FE_ERR_ARG;
  if (mesh->elem_type != FE_TET4 && mesh->elem_type != FE_HEX8) return FE_ERR_ARG;
  if (mat->model < FE_SVK || mat->model > FE_MOONEY_RIVLIN || !mat->params) return FE_ERR_ARG;
  if (!(h > 0) || !(mat->rho > 0) || mesh->n_fixed < 0 || (mesh->n_fixed > 0 && !mesh->fixed_nodes))
    return FE_ERR_ARG;
  if (mesh->n_nodes > (int64_t(1) << 29)) return FE_ERR_ARG;
  fe_ctx *c = new (std::nothrow) fe_ctx();
  if (!c) return FE_ERR_OOM;
  try {
    c->elem_type = mesh->elem_type;
    c->npe = mesh->elem_type == FE_TET4 ? 4 : 8;
    c->n_nodes = mesh->n_nodes;
    c->n_elems = mesh->n_elems;
    c->X.assign(mesh->rest_xyz, mesh->rest_xyz + 3 * mesh->n_nodes);
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
  } catch (const std::bad_alloc &) {
    delete c;
    return FE_ERR_OOM;
  }
  *out = c;
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
