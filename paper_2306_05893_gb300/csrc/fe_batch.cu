// Batched stepping of independent meshes in one block-diagonal system: the
// element, assembly, SpMV, factor and apply stages run once over all
// members; the CG scalars are per member (segmented reductions), so each
// member converges on its own test ||r_k|| <= tol ||b_k|| and stops
// changing once it has.  One CTA per member reduces that member's DOF range
// in a fixed order (deterministic) and updates its scalars.
#include <cuda_runtime.h>

#include "fe_device.cuh"

namespace fe {

namespace {

template <int BLOCK>
__device__ __forceinline__ double cta_sum(double v, double *sh) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = v;
  __syncthreads();
  if (threadIdx.x < 32) {
    v = (threadIdx.x < BLOCK / 32) ? sh[threadIdx.x] : 0.0;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  }
  __syncthreads();
  return v;
}

// x . y over member blockIdx.x's DOFs, then the member's scalar update.
template <typename TV>
__global__ void __launch_bounds__(256) seg_dot_kernel(const TV *__restrict__ x, const TV *__restrict__ y,
                                                      const int64_t *__restrict__ seg_dof, int mode, double tol,
                                                      double *__restrict__ bs, int *flags) {
  __shared__ double sh[8];
  const int b = blockIdx.x;
  double *s = bs + int64_t(b) * B_COUNT;
  const int64_t d0 = seg_dof[b], d1 = seg_dof[b + 1];
  double acc = 0.0;
  for (int64_t i = d0 + threadIdx.x; i < d1; i += 256) acc += double(x[i]) * double(y[i]);
  const double tot = cta_sum<256>(acc, sh);
  if (threadIdx.x != 0) return;
  switch (mode) {
    case SEG_PQ:
      if (s[B_DONE] != 0.0) {
        s[B_ALPHA] = 0.0;
      } else if (!(tot > 0.0)) {
        atomicOr(flags, FLAG_BREAKDOWN);
        s[B_DONE] = 1.0;
        s[B_ALPHA] = 0.0;
      } else {
        s[B_ALPHA] = s[B_RZ] / tot;
      }
      break;
    case SEG_RR:
      s[B_RR] = tot;
      if (s[B_DONE] == 0.0) {
        s[B_ITERS] += 1.0;
        if (tot <= s[B_TOL2]) s[B_DONE] = 1.0;
      }
      break;
    case SEG_RZ_FIRST:
    case SEG_RZ:
      if (s[B_DONE] == 0.0 && !(tot > 0.0) && s[B_RR] > 0.0) {
        atomicOr(flags, FLAG_BREAKDOWN);
        s[B_DONE] = 1.0;
      }
      s[B_BETA] = (mode == SEG_RZ_FIRST || s[B_DONE] != 0.0) ? 0.0 : tot / s[B_RZ];
      s[B_RZ] = tot;
      break;
    case SEG_INIT_OUTER:  // rhs . rhs of the step: outer and inner tolerances
      s[B_BB] = tot;
      s[B_OTOL2] = tol * tol * tot;
      s[B_ORR] = tot;
      s[B_ODONE] = (tot == 0.0) ? 1.0 : 0.0;
      s[B_ITERS] = 0.0;
      s[B_TOL2] = tol * tol * tot;
      s[B_RR] = tot;
      s[B_DONE] = s[B_ODONE];
      break;
    case SEG_INIT_INNER:  // inner solve of a refinement sweep on the residual
      s[B_TOL2] = tol * tol * tot;
      s[B_RR] = tot;
      s[B_DONE] = (s[B_ODONE] != 0.0 || tot == 0.0) ? 1.0 : 0.0;
      break;
    case SEG_ORR:  // FP64 residual of the sweep
      s[B_ORR] = tot;
      if (tot <= s[B_OTOL2]) s[B_ODONE] = 1.0;
      break;
  }
}

// x = 0, r = rhs (cast); members already converged keep r = 0 so they stay put
template <typename TV>
__global__ void seg_init_kernel(int64_t n, TV *__restrict__ x, TV *__restrict__ r, const double *__restrict__ rhs,
                                const int32_t *__restrict__ row_seg, const double *__restrict__ bs, int inner) {
  for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x) {
    x[i] = TV(0);
    const bool frozen = inner && bs[int64_t(row_seg[i]) * B_COUNT + B_ODONE] != 0.0;
    r[i] = frozen ? TV(0) : TV(rhs[i]);
  }
}

template <typename TV>
__global__ void seg_axpy_kernel(int64_t n, TV *__restrict__ x, TV *__restrict__ r, const TV *__restrict__ p,
                                const TV *__restrict__ q, const int32_t *__restrict__ row_seg,
                                const double *__restrict__ bs) {
  for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x) {
    const TV al = TV(bs[int64_t(row_seg[i]) * B_COUNT + B_ALPHA]);
    x[i] += al * p[i];
    r[i] -= al * q[i];
  }
}

template <typename TV>
__global__ void seg_update_p_kernel(int64_t n, const TV *__restrict__ z, TV *__restrict__ p,
                                    const int32_t *__restrict__ row_seg, const double *__restrict__ bs, int first) {
  for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x) {
    const double *s = bs + int64_t(row_seg[i]) * B_COUNT;
    if (first) {
      p[i] = z[i];  // whatever p held (converged members' p is never used: their alpha is 0)
    } else if (s[B_DONE] == 0.0) {
      p[i] = z[i] + TV(s[B_BETA]) * p[i];
    }
  }
}

// y = A x, TPR threads per row (warp-uniform loop bound)
template <typename TA, typename TV, typename TACC, int TPR>
__global__ void __launch_bounds__(256) spmv_kernel(int64_t n, const int32_t *__restrict__ rowptr,
                                                   const int32_t *__restrict__ colind, const TA *__restrict__ A,
                                                   const TV *__restrict__ x, const double *__restrict__ b,
                                                   TACC *__restrict__ y) {
  const int sub = threadIdx.x % TPR;
  const int64_t groups = int64_t(gridDim.x) * (256 / TPR);
  const int64_t warp_row0 = int64_t(blockIdx.x) * (256 / TPR) + (threadIdx.x / 32) * (32 / TPR);
  for (int64_t r0 = warp_row0; r0 < n; r0 += groups) {
    const int64_t row = r0 + (threadIdx.x % 32) / TPR;
    TACC acc = TACC(0);
    if (row < n) {
      const int32_t k1 = rowptr[row + 1];
      for (int32_t k = rowptr[row] + sub; k < k1; k += TPR) acc += TACC(A[k]) * TACC(x[colind[k]]);
    }
#pragma unroll
    for (int o = TPR / 2; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o, TPR);
    if (sub == 0 && row < n) y[row] = b ? TACC(b[row]) - acc : acc;
  }
}

unsigned grid_for(int64_t n) { return unsigned(std::max<int64_t>(1, std::min<int64_t>((n + 255) / 256, 152 * 16))); }

}  // namespace

void launch_seg_dot(const fe_ctx *c, const DeviceState *d, bool fp32, const void *x, const void *y, int mode,
                    double tol, cudaStream_t s) {
  d->launches++;
  if (fp32)
    seg_dot_kernel<float><<<unsigned(c->nseg), 256, 0, s>>>((const float *)x, (const float *)y, d->seg_dof, mode, tol,
                                                            d->bscal, d->flags);
  else
    seg_dot_kernel<double><<<unsigned(c->nseg), 256, 0, s>>>((const double *)x, (const double *)y, d->seg_dof, mode,
                                                             tol, d->bscal, d->flags);
}

void launch_seg_dot64(const fe_ctx *c, const DeviceState *d, const double *x, const double *y, int mode, double tol,
                      cudaStream_t s) {
  d->launches++;
  seg_dot_kernel<double><<<unsigned(c->nseg), 256, 0, s>>>(x, y, d->seg_dof, mode, tol, d->bscal, d->flags);
}

void launch_seg_init(const fe_ctx *c, const DeviceState *d, bool fp32, void *x, void *r, const double *rhs,
                     bool inner, cudaStream_t s) {
  d->launches++;
  if (fp32)
    seg_init_kernel<float><<<grid_for(c->n), 256, 0, s>>>(c->n, (float *)x, (float *)r, rhs, d->row_seg, d->bscal,
                                                          inner);
  else
    seg_init_kernel<double><<<grid_for(c->n), 256, 0, s>>>(c->n, (double *)x, (double *)r, rhs, d->row_seg,
                                                           d->bscal, inner);
}

void launch_seg_axpy(const fe_ctx *c, const DeviceState *d, bool fp32, void *x, void *r, const void *p,
                     const void *q, cudaStream_t s) {
  d->launches++;
  if (fp32)
    seg_axpy_kernel<float><<<grid_for(c->n), 256, 0, s>>>(c->n, (float *)x, (float *)r, (const float *)p,
                                                          (const float *)q, d->row_seg, d->bscal);
  else
    seg_axpy_kernel<double><<<grid_for(c->n), 256, 0, s>>>(c->n, (double *)x, (double *)r, (const double *)p,
                                                           (const double *)q, d->row_seg, d->bscal);
}

void launch_seg_update_p(const fe_ctx *c, const DeviceState *d, bool fp32, const void *z, void *p, bool first,
                         cudaStream_t s) {
  d->launches++;
  if (fp32)
    seg_update_p_kernel<float><<<grid_for(c->n), 256, 0, s>>>(c->n, (const float *)z, (float *)p, d->row_seg,
                                                              d->bscal, first);
  else
    seg_update_p_kernel<double><<<grid_for(c->n), 256, 0, s>>>(c->n, (const double *)z, (double *)p, d->row_seg,
                                                               d->bscal, first);
}

// y = A x (matrix/vector type), or y = b - A x in FP64 when b is given.
template <int TPR>
static void spmv_t(const fe_ctx *c, const DeviceState *d, bool fp32, const void *x, void *y, const double *b,
                   cudaStream_t s) {
  const unsigned g = unsigned(std::max<int64_t>(1, std::min<int64_t>((c->n * TPR + 255) / 256, 152 * 8)));
  if (b) {
    if (fp32)
      spmv_kernel<float, double, double, TPR><<<g, 256, 0, s>>>(c->n, d->rowptr, d->colind, (const float *)d->A,
                                                                (const double *)x, b, (double *)y);
    else
      spmv_kernel<double, double, double, TPR><<<g, 256, 0, s>>>(c->n, d->rowptr, d->colind, (const double *)d->A,
                                                                 (const double *)x, b, (double *)y);
  } else {
    if (fp32)
      spmv_kernel<float, float, float, TPR><<<g, 256, 0, s>>>(c->n, d->rowptr, d->colind, (const float *)d->A,
                                                              (const float *)x, nullptr, (float *)y);
    else
      spmv_kernel<double, double, double, TPR><<<g, 256, 0, s>>>(c->n, d->rowptr, d->colind, (const double *)d->A,
                                                                 (const double *)x, nullptr, (double *)y);
  }
}

void launch_spmv_plain(const fe_ctx *c, const DeviceState *d, bool fp32, const void *x, void *y, const double *b,
                       int tpr, cudaStream_t s) {
  d->launches++;
  switch (tpr) {
    case 4: spmv_t<4>(c, d, fp32, x, y, b, s); break;
    case 16: spmv_t<16>(c, d, fp32, x, y, b, s); break;
    case 32: spmv_t<32>(c, d, fp32, x, y, b, s); break;
    default: spmv_t<8>(c, d, fp32, x, y, b, s);
  }
}

}  // namespace fe
