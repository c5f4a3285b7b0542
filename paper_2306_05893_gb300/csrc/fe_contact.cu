// Frictionless contact against rigid planes by Lagrange multipliers
// (Section "Lagrangian multipliers", Eq. "KKT"): after the free motion
// A a_free = b of a step, the compliance W = H P^{-1} H^T is built with the
// step's preconditioner P = L D L^T, the LCP lambda >= 0,
// w = W lambda - (delta - H a_free) >= 0, lambda . w = 0 is solved by
// projected Gauss-Seidel, and the motion is corrected,
// a = a_free + P^{-1} H^T lambda.  Since P^{-1} = L^{-T} D^{-1} L^{-1},
// W = G^T D G with G = D^{-1} L^{-1} H^T: one forward solve per constraint
// (the pivot output of the forward sweep) instead of a full application,
// and a single full application for the correction.  Constraint i:
// n_i . x >= c_i for node i's end-of-step position x = q + h v + h^2 a,
// i.e. on the unknown a: n_i . a_node >= delta_i = (c_i - n_i . (q + h v)_node) / h^2.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <string>
#include <vector>

#include "../../include/fe_hotpath.h"
#include "fe_device.cuh"

namespace fe {

namespace {

constexpr int kMaxContacts = 4096;  // multipliers kept in shared memory by the solver (32 KB)
constexpr int kRhsPerLaunch = 64;   // right-hand sides per forward launch (the front id's high byte)

// RHS of constraint i in the preconditioner's precision: n_i on node i's DOFs
// (the vector is cleared before)
template <typename T>
__global__ void contact_column_kernel(T *r, const int32_t *__restrict__ node, const double *__restrict__ normal,
                                      int i) {
  if (threadIdx.x < 3) r[3 * int64_t(node[i]) + threadIdx.x] = T(normal[3 * i + threadIdx.x]);
}

// The right-hand sides H^T e_i of constraints i = i0 + k, k < nrhs (and
// i < m), into the vectors r + k n (cleared before)
template <typename T>
__global__ void contact_group_kernel(T *r, int64_t n, const int32_t *__restrict__ node,
                                     const double *__restrict__ normal, int i0, int m, int nrhs) {
  const int k = threadIdx.x;
  const int i = i0 + k;
  if (k >= nrhs || i >= m) return;
  for (int j = 0; j < 3; ++j) r[int64_t(k) * n + 3 * int64_t(node[i]) + j] = T(normal[3 * i + j]);
}

// W[i m + j] = W[j m + i] = sum_k G_i[k] d_k G_j[k] (block (i, j), j >= i;
// per-thread partial sums in a fixed order, then a fixed-shape tree: the
// result does not depend on scheduling, and W is exactly symmetric)
template <typename T>
__global__ void __launch_bounds__(256) contact_w_kernel(const T *__restrict__ G, const double *__restrict__ Dk,
                                                        int64_t nf, int m, double *__restrict__ W) {
  const int i = blockIdx.x, j = blockIdx.y;
  if (j < i) return;
  const T *gi = G + int64_t(i) * nf, *gj = G + int64_t(j) * nf;
  double acc = 0.0;
  for (int64_t k = threadIdx.x; k < nf; k += 256) acc += double(gi[k]) * Dk[k] * double(gj[k]);
  __shared__ double red[256];
  red[threadIdx.x] = acc;
  __syncthreads();
  for (int w = 128; w > 0; w >>= 1) {
    if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    W[int64_t(i) * m + j] = red[0];
    W[int64_t(j) * m + i] = red[0];
  }
}

// rhs_i = delta_i - n_i . a_free(node i)
__global__ void contact_rhs_kernel(const int32_t *__restrict__ node, const double *__restrict__ normal,
                                   const double *__restrict__ off, const double *__restrict__ q,
                                   const double *__restrict__ v, const double *__restrict__ a, double h, int m,
                                   double *__restrict__ rhs) {
  const int64_t t = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (t < m) {
    const int i = int(t);
    const int64_t base = 3 * int64_t(node[i]);
    double nx = 0.0, na = 0.0;
    for (int k = 0; k < 3; ++k) {
      nx += normal[3 * i + k] * (q[base + k] + h * v[base + k]);
      na += normal[3 * i + k] * a[base + k];
    }
    rhs[i] = (off[i] - nx) / (h * h) - na;
  }
}

// Projected Gauss-Seidel on one warp: constraints in index order, each set
// to the non-negative value that zeroes its own residual given the others
// (the row's dot product over the warp, reduced by lane 0's butterfly and
// broadcast, so every lane takes the same decision); stops when a sweep
// changes no multiplier by more than tol * max |lambda|.  W_ii <= 0 (a node
// that cannot move) keeps lambda_i = 0.
__global__ void __launch_bounds__(32) pgs_kernel(const double *__restrict__ W, const double *__restrict__ r,
                                                 double *__restrict__ lam, int m, int sweeps, double tol) {
  __shared__ double sl[kMaxContacts];
  const int lane = threadIdx.x;
  for (int i = lane; i < m; i += 32) sl[i] = 0.0;
  __syncwarp();
  for (int sw = 0; sw < sweeps; ++sw) {
    double dmax = 0.0;
    for (int i = 0; i < m; ++i) {
      const double *Wi = W + int64_t(i) * m;
      double acc = 0.0;
      for (int j = lane; j < m; j += 32) acc += Wi[j] * sl[j];
      for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
      acc = __shfl_sync(0xffffffffu, acc, 0);
      const double wii = Wi[i];
      if (wii > 0.0) {
        const double old = sl[i];
        const double nw = fmax(0.0, old + (r[i] - acc) / wii);
        dmax = fmax(dmax, fabs(nw - old));
        __syncwarp();
        if (lane == 0) sl[i] = nw;
      }
      __syncwarp();
    }
    double lmax = 0.0;
    for (int i = lane; i < m; i += 32) lmax = fmax(lmax, fabs(sl[i]));
    for (int o = 16; o > 0; o >>= 1) lmax = fmax(lmax, __shfl_xor_sync(0xffffffffu, lmax, o));
    if (dmax <= tol * fmax(1e-300, lmax)) break;
  }
  for (int i = lane; i < m; i += 32) lam[i] = sl[i];
}

// r = H^T lambda in the solve's precision (the vector is cleared before;
// one thread, constraints in order: several on one node add up
// deterministically)
template <typename T>
__global__ void contact_force_kernel(T *r, const int32_t *__restrict__ node, const double *__restrict__ normal,
                                     const double *__restrict__ lam, int m) {
  if (threadIdx.x != 0) return;
  for (int i = 0; i < m; ++i)
    for (int k = 0; k < 3; ++k) r[3 * int64_t(node[i]) + k] += T(lam[i] * normal[3 * i + k]);
}

// a += z (z in the solve's precision)
template <typename T>
__global__ void add_vector_kernel(double *__restrict__ a, const T *__restrict__ z, int64_t n) {
  const int64_t r = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (r < n) a[r] += double(z[r]);
}

// (re)allocate a contact buffer, keeping the context's allocation list exact
int regrow(fe_ctx *c, DeviceState *d, void **p, size_t bytes) {
  if (*p) {
    d->allocs.erase(std::remove(d->allocs.begin(), d->allocs.end(), *p), d->allocs.end());
    cudaFree(*p);
    *p = nullptr;
  }
  cudaError_t e = cudaMalloc(p, std::max<size_t>(bytes, 8));
  if (e != cudaSuccess) {
    cudaGetLastError();
    *p = nullptr;
    return set_error(c, FE_ERR_OOM, "cudaMalloc of " + std::to_string(bytes) + " bytes for contacts failed");
  }
  d->allocs.push_back(*p);
  return FE_OK;
}

// grow a buffer to at least `bytes` (kept when large enough: a contact set
// that changes every step does not reallocate)
int grow(fe_ctx *c, DeviceState *d, void **p, size_t &cap, size_t bytes) {
  if (*p && bytes <= cap) return FE_OK;
  const int st = regrow(c, d, p, bytes);
  cap = st ? 0 : std::max<size_t>(bytes, 8);
  return st;
}

}  // namespace

// Upload the constraint set (host copy in the context) to the device buffers.
static int contact_upload(fe_ctx *c, DeviceState *d) {
  const int64_t m = int64_t(c->contact_node.size());
  if (m > d->c_cap) {
    const int64_t cap = std::max<int64_t>(m, 2 * d->c_cap);
    int st = regrow(c, d, reinterpret_cast<void **>(&d->c_node), size_t(cap) * sizeof(int32_t));
    if (!st) st = regrow(c, d, reinterpret_cast<void **>(&d->c_normal), size_t(3 * cap) * sizeof(double));
    if (!st) st = regrow(c, d, reinterpret_cast<void **>(&d->c_off), size_t(cap) * sizeof(double));
    if (!st) st = regrow(c, d, reinterpret_cast<void **>(&d->c_W), size_t(cap) * size_t(cap) * sizeof(double));
    if (!st) st = regrow(c, d, reinterpret_cast<void **>(&d->c_rhs), size_t(cap) * sizeof(double));
    if (!st) st = regrow(c, d, reinterpret_cast<void **>(&d->c_lam), size_t(cap) * sizeof(double));
    if (!st && !d->c_pend)
      st = regrow(c, d, reinterpret_cast<void **>(&d->c_pend), std::max<size_t>(c->fronts.size(), 1) * sizeof(int));
    if (st) {
      d->c_cap = 0;
      return st;
    }
    d->c_cap = cap;
  }
  if (m > 0) {
    FE_CUDA_TRY(cudaMemcpy(d->c_node, c->contact_node.data(), size_t(m) * sizeof(int32_t), cudaMemcpyHostToDevice));
    FE_CUDA_TRY(cudaMemcpy(d->c_normal, c->contact_normal.data(), size_t(3 * m) * sizeof(double),
                           cudaMemcpyHostToDevice));
    FE_CUDA_TRY(cudaMemcpy(d->c_off, c->contact_offset.data(), size_t(m) * sizeof(double), cudaMemcpyHostToDevice));
    FE_CUDA_TRY(cudaMemset(d->c_lam, 0, size_t(m) * sizeof(double)));
  }
  // the fronts on the constraints' paths to the root (a right-hand side
  // H^T e_i is zero outside them, so their forward solve stays there), their
  // tasks in the forward list's (topological) order and their numbers of
  // children on the paths
  if (m > 0) {
    const int64_t nf = int64_t(c->fronts.size());
    std::vector<int32_t> piv_front(size_t(std::max<int64_t>(c->n_free, 1)), -1);
    for (int64_t f = 0; f < nf; ++f)
      for (int32_t k = 0; k < c->fronts[f].npiv; ++k) piv_front[size_t(c->fronts[f].first + k)] = int32_t(f);
    std::vector<char> on(size_t(nf), 0);
    for (int64_t i = 0; i < m; ++i)
      for (int k = 0; k < 3; ++k) {
        const int32_t piv = c->iperm[3 * int64_t(c->contact_node[i]) + k];
        for (int32_t f = piv >= 0 ? piv_front[piv] : -1; f >= 0 && !on[f]; f = c->fronts[f].parent) on[f] = 1;
      }
    std::vector<int32_t> sub;
    for (size_t t = 0; t + 3 < c->apply_fwd.size(); t += 4)
      if (on[c->apply_fwd[t]]) sub.insert(sub.end(), c->apply_fwd.begin() + t, c->apply_fwd.begin() + t + 4);
    // each front's pending count: its children's forward tasks in the subset
    std::vector<int> pend(size_t(nf), 0);
    for (int64_t f = 0; f < nf; ++f)
      if (on[f] && c->fronts[f].parent >= 0) pend[c->fronts[f].parent] += c->front_nfwd[f];
    // the right-hand sides of one launch (at most kRhsPerLaunch; the task's
    // right-hand side rides in the front id's high byte), each subset task
    // repeated for them in order (the list stays topological)
    const int nr = int(std::min<int64_t>(m, kRhsPerLaunch));
    std::vector<int32_t> multi;
    multi.reserve(sub.size() * size_t(nr));
    for (size_t t = 0; t + 3 < sub.size(); t += 4)
      for (int k = 0; k < nr; ++k) {
        multi.push_back(sub[t] | (k << 24));
        multi.insert(multi.end(), sub.begin() + t + 1, sub.begin() + t + 4);
      }
    const size_t ts = c->opt.precision == FE_MIXED ? sizeof(float) : sizeof(double);
    const int64_t groups = (m + nr - 1) / nr;
    const size_t slots = size_t(std::max<int64_t>(c->fwd_slots, 1));
    size_t *cb = d->c_bytes;
    int st = grow(c, d, reinterpret_cast<void **>(&d->c_tasks), cb[0],
                  std::max<size_t>(multi.size(), 4) * sizeof(int32_t));
    if (!st) st = grow(c, d, &d->c_G, cb[1], size_t(groups * nr) * size_t(std::max<int64_t>(c->n_free, 1)) * ts);
    if (!st) st = grow(c, d, &d->c_r, cb[2], size_t(nr) * size_t(c->n) * ts);
    if (!st) st = grow(c, d, &d->c_u, cb[3], size_t(nr) * size_t(std::max<int64_t>(c->u_total, 1)) * ts);
    if (!st) st = grow(c, d, &d->c_part, cb[4], size_t(nr) * slots * size_t(fwd_rows(c->opt)) * ts);
    if (!st) st = grow(c, d, reinterpret_cast<void **>(&d->c_tick), cb[5], size_t(nr) * slots * sizeof(int));
    if (!st) st = grow(c, d, reinterpret_cast<void **>(&d->c_pendm), cb[6], size_t(nr) * size_t(nf) * sizeof(int));
    if (!st) st = grow(c, d, reinterpret_cast<void **>(&d->c_bdm), cb[7], size_t(nf) * sizeof(int));
    if (!st) st = grow(c, d, reinterpret_cast<void **>(&d->c_ctl), cb[8], 4 * sizeof(int));
    if (st) return st;
    if (!multi.empty())
      FE_CUDA_TRY(cudaMemcpy(d->c_tasks, multi.data(), multi.size() * sizeof(int32_t), cudaMemcpyHostToDevice));
    FE_CUDA_TRY(cudaMemcpy(d->c_pend, pend.data(), pend.size() * sizeof(int), cudaMemcpyHostToDevice));
    FE_CUDA_TRY(cudaMemset(d->c_tick, 0, size_t(nr) * slots * sizeof(int)));
    d->c_ntask = int64_t(multi.size() / 4);
    d->c_nrhs = nr;
  }
  d->c_m = m;
  d->c_dirty = false;
  return FE_OK;
}

// Constraint resolution and motion correction of the current step: d->x
// holds a_free on entry and the corrected a on return (all on d->stream).
int contact_resolve(fe_ctx *c, DeviceState *d, bool fp32) {
  cudaStream_t s = d->stream;
  if (d->c_dirty) {
    FE_CUDA_TRY(cudaStreamSynchronize(s));
    const int st = contact_upload(c, d);
    if (st) return st;
  }
  const int m = int(d->c_m);
  if (m == 0) return FE_OK;
  const int64_t n = c->n, nf = c->n_free;
  const size_t ts = fp32 ? sizeof(float) : sizeof(double);
  // G_i = D^{-1} L^{-1} H^T e_i: the forward solves of up to kRhsPerLaunch
  // constraints per launch, over the fronts on the constraints' paths only
  // (G and the update vectors outside them stay at the zeros written here)
  const int nr = int(d->c_nrhs);
  const int64_t groups = (m + nr - 1) / nr;
  FE_CUDA_TRY(cudaMemsetAsync(d->c_G, 0, size_t(groups * nr) * size_t(nf) * ts, s));
  for (int64_t gi = 0; gi < groups; ++gi) {
    FE_CUDA_TRY(cudaMemsetAsync(d->c_r, 0, size_t(nr) * size_t(n) * ts, s));
    FE_CUDA_TRY(cudaMemsetAsync(d->c_u, 0, size_t(nr) * size_t(std::max<int64_t>(c->u_total, 1)) * ts, s));
    if (fp32)
      contact_group_kernel<float><<<1, kRhsPerLaunch, 0, s>>>(static_cast<float *>(d->c_r), n, d->c_node,
                                                             d->c_normal, int(gi * nr), m, nr);
    else
      contact_group_kernel<double><<<1, kRhsPerLaunch, 0, s>>>(static_cast<double *>(d->c_r), n, d->c_node,
                                                              d->c_normal, int(gi * nr), m, nr);
    apply_forward_multi_enqueue(c, d, d->cur, fp32, d->c_r,
                                static_cast<unsigned char *>(d->c_G) + size_t(gi * nr) * size_t(nf) * ts, d->c_tasks,
                                d->c_ntask, d->c_pend, d->c_pendm, d->c_bdm, d->c_ctl, d->c_u, d->c_part,
                                d->c_tick, nr, s);
    d->launches += 1;
  }
  // W = G^T D G, the PGS right-hand side, the multipliers
  const dim3 wg = dim3(unsigned(m), unsigned(m), 1u);
  if (fp32)
    contact_w_kernel<float><<<wg, 256, 0, s>>>(static_cast<const float *>(d->c_G), d->D[d->cur], nf, m, d->c_W);
  else
    contact_w_kernel<double><<<wg, 256, 0, s>>>(static_cast<const double *>(d->c_G), d->D[d->cur], nf, m, d->c_W);
  contact_rhs_kernel<<<unsigned((m + 255) / 256), 256, 0, s>>>(d->c_node, d->c_normal, d->c_off, d->q, d->v, d->x,
                                                               c->h, m, d->c_rhs);
  pgs_kernel<<<1, 32, 0, s>>>(d->c_W, d->c_rhs, d->c_lam, m, c->opt.contact_sweeps, c->opt.contact_tol);
  // motion correction: a += P^{-1} H^T lambda (one full application)
  FE_CUDA_TRY(cudaMemsetAsync(d->vr, 0, size_t(n) * ts, s));
  if (fp32)
    contact_force_kernel<float><<<1, 32, 0, s>>>(static_cast<float *>(d->vr), d->c_node, d->c_normal, d->c_lam, m);
  else
    contact_force_kernel<double><<<1, 32, 0, s>>>(static_cast<double *>(d->vr), d->c_node, d->c_normal, d->c_lam, m);
  apply_enqueue(c, d, d->cur, fp32, d->vr, d->vz, s);
  if (fp32)
    add_vector_kernel<float><<<unsigned((n + 255) / 256), 256, 0, s>>>(d->x, static_cast<const float *>(d->vz), n);
  else
    add_vector_kernel<double><<<unsigned((n + 255) / 256), 256, 0, s>>>(d->x, static_cast<const double *>(d->vz), n);
  d->launches += 5;  // W, right-hand side, PGS, H^T lambda, a += z (the applications count their own)
  FE_CUDA_TRY(cudaGetLastError());
  return FE_OK;
}

}  // namespace fe

extern "C" int fe_set_contacts(fe_ctx *c, int32_t m, const int32_t *nodes, const double *normals,
                               const double *offsets) {
  using namespace fe;
  if (!c || m < 0 || m > kMaxContacts || (m > 0 && (!nodes || !normals || !offsets))) return FE_ERR_ARG;
  if (m > 0 && (c->opt.keep_checkpoints || c->opt.newton_iters > 1))
    return set_error(c, FE_ERR_STATE, "contacts need keep_checkpoints = 0 and newton_iters = 1");
  for (int32_t i = 0; i < m; ++i) {
    if (nodes[i] < 0 || nodes[i] >= c->n_nodes)
      return set_error(c, FE_ERR_ARG, "contact " + std::to_string(i) + ": node out of range");
    const double nn = normals[3 * i] * normals[3 * i] + normals[3 * i + 1] * normals[3 * i + 1] +
                      normals[3 * i + 2] * normals[3 * i + 2];
    if (!(nn > 0) || !std::isfinite(offsets[i]))
      return set_error(c, FE_ERR_ARG, "contact " + std::to_string(i) + ": zero normal or non-finite offset");
  }
  c->contact_node.assign(nodes, nodes + m);
  c->contact_normal.assign(normals, normals + 3 * int64_t(m));
  c->contact_offset.assign(offsets, offsets + m);
  if (c->dev) c->dev->c_dirty = true;
  return FE_OK;
}

extern "C" int fe_get_contact_forces(fe_ctx *c, double *lambda) {
  using namespace fe;
  if (!c || !lambda) return FE_ERR_ARG;
  const int64_t m = int64_t(c->contact_node.size());
  if (m == 0) return FE_OK;
  DeviceState *d = c->dev;
  if (!d || d->c_m != m || !d->c_lam) return set_error(c, FE_ERR_STATE, "no step with these contacts yet");
  FE_CUDA_TRY(cudaStreamSynchronize(d->stream));
  FE_CUDA_TRY(cudaMemcpy(lambda, d->c_lam, size_t(m) * sizeof(double), cudaMemcpyDeviceToHost));
  return FE_OK;
}
