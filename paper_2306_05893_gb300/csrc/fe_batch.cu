// Batched stepping of independent meshes in one block-diagonal system: the
// element, assembly, SpMV, factor and apply stages run once over all
// members; the CG scalars are per member (segmented reductions), so each
// member converges on its own test ||r_k|| <= tol ||b_k|| and stops
// changing once it has.  One CTA per member reduces that member's DOF range
// in a fixed order (deterministic) and updates its scalars.
#include <cuda_runtime.h>

#include <algorithm>
#include <string>
#include <utility>
#include <vector>

#include "fe_device.cuh"
#include "fe_df.cuh"

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
  DotAcc<TV> acc;
  for (int64_t i = d0 + threadIdx.x; i < d1; i += 256) acc.add(x[i], y[i]);
  const double tot = cta_sum<256>(acc.value(), sh);
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
                                const int32_t *__restrict__ row_seg, const double *__restrict__ bs, int inner,
                                float2 *__restrict__ x2) {
  for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x) {
    x[i] = TV(0);
    if (x2) x2[i] = make_float2(0.f, 0.f);  // the outer x's float-pair mirror (mixed path)
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

unsigned grid_for(int64_t n) { return unsigned(std::max<int64_t>(1, std::min<int64_t>((n + 255) / 256, 152 * 16))); }

constexpr int kBatchBlockNodes = 64;  // nodes per row block of the batched SpMV

// Node-block SpMV over a table of row blocks (one CTA per block: a node
// range inside one member).  Every free node's three rows share one column
// structure of 3x3 blocks, so a block's column index is read once for its 9
// values; LPN lanes per node, the three row sums reduced across them; fixed
// nodes keep their lone diagonal.  MODE 0: y = A x in TV; MODE 1: y = b - A x
// in FP64 (TA = double, the FP64 copy of A).
template <typename TA, typename TV, int LPN, int MODE>
__global__ void __launch_bounds__(256) batch_bspmv_kernel(const int2 *__restrict__ blocks,
                                                          const int32_t *__restrict__ rowptr,
                                                          const int32_t *__restrict__ bptr,
                                                          const int32_t *__restrict__ bcol,
                                                          const int8_t *__restrict__ fixed_row,
                                                          const TA *__restrict__ A, const TV *__restrict__ x,
                                                          const double *__restrict__ b, TV *__restrict__ y) {
  const int2 blk = blocks[blockIdx.x];
  const int sub = threadIdx.x % LPN;
  for (int64_t n0 = blk.x + int64_t(threadIdx.x / 32) * (32 / LPN); n0 < blk.y; n0 += 256 / LPN) {
    const int64_t nd = n0 + (threadIdx.x % 32) / LPN;  // the loop bound is warp-uniform
    TV a0 = TV(0), a1 = TV(0), a2 = TV(0);
    bool fixed = true;
    if (nd < blk.y) {
      fixed = fixed_row[3 * nd] != 0;
      if (!fixed) {
        const int32_t k0 = bptr[nd], k1 = bptr[nd + 1];
        const int32_t r0 = rowptr[3 * nd], r1 = rowptr[3 * nd + 1], r2 = rowptr[3 * nd + 2];
        for (int32_t k = k0 + sub; k < k1; k += LPN) {
          const int64_t cc = 3 * int64_t(bcol[k]);
          const TV x0 = x[cc], x1 = x[cc + 1], x2 = x[cc + 2];
          const int32_t o = 3 * (k - k0);
          a0 += TV(A[r0 + o]) * x0 + TV(A[r0 + o + 1]) * x1 + TV(A[r0 + o + 2]) * x2;
          a1 += TV(A[r1 + o]) * x0 + TV(A[r1 + o + 1]) * x1 + TV(A[r1 + o + 2]) * x2;
          a2 += TV(A[r2 + o]) * x0 + TV(A[r2 + o + 1]) * x1 + TV(A[r2 + o + 2]) * x2;
        }
      }
    }
#pragma unroll
    for (int o = LPN / 2; o > 0; o >>= 1) {
      a0 += __shfl_xor_sync(0xffffffffu, a0, o, LPN);
      a1 += __shfl_xor_sync(0xffffffffu, a1, o, LPN);
      a2 += __shfl_xor_sync(0xffffffffu, a2, o, LPN);
    }
    if (sub == 0 && nd < blk.y) {
      const TV acc[3] = {a0, a1, a2};
#pragma unroll
      for (int i = 0; i < 3; ++i) {
        const int64_t r = 3 * nd + i;
        const TV yi = fixed ? TV(A[rowptr[r]]) * x[r] : acc[i];
        y[r] = MODE == 0 ? yi : TV(b[r] - double(yi));
      }
    }
  }
}

// CSR SpMV over the same row blocks: the rows [3 n0, 3 n1) of each node
// range, TPR threads per row (warp-uniform loop bound).
template <typename TA, typename TV, int TPR, int MODE>
__global__ void __launch_bounds__(256) batch_csr_kernel(const int2 *__restrict__ blocks,
                                                        const int32_t *__restrict__ rowptr,
                                                        const int32_t *__restrict__ colind, const TA *__restrict__ A,
                                                        const TV *__restrict__ x, const double *__restrict__ b,
                                                        TV *__restrict__ y) {
  const int2 blk = blocks[blockIdx.x];
  const int64_t rb = 3 * int64_t(blk.x), re = 3 * int64_t(blk.y);
  const int sub = threadIdx.x % TPR;
  for (int64_t r0 = rb + int64_t(threadIdx.x / 32) * (32 / TPR); r0 < re; r0 += 256 / TPR) {
    const int64_t row = r0 + (threadIdx.x % 32) / TPR;
    TV acc = TV(0);
    if (row < re) {
      const int32_t k1 = rowptr[row + 1];
      for (int32_t k = rowptr[row] + sub; k < k1; k += TPR) acc += TV(A[k]) * x[colind[k]];
    }
#pragma unroll
    for (int o = TPR / 2; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o, TPR);
    if (sub == 0 && row < re) y[row] = MODE == 0 ? acc : TV(b[row] - double(acc));
  }
}

// y = b - A x in the mixed path (A2 and x2 as float pairs, double-float
// products and sums, y in FP64): the node-block and CSR forms of the two
// kernels above.
template <int LPN>
__global__ void __launch_bounds__(256) batch_bres_df_kernel(const int2 *__restrict__ blocks,
                                                            const int32_t *__restrict__ rowptr,
                                                            const int32_t *__restrict__ bptr,
                                                            const int32_t *__restrict__ bcol,
                                                            const int8_t *__restrict__ fixed_row,
                                                            const float2 *__restrict__ A, const float2 *__restrict__ x,
                                                            const double *__restrict__ b, double *__restrict__ y) {
  const int2 blk = blocks[blockIdx.x];
  const int sub = threadIdx.x % LPN;
  for (int64_t n0 = blk.x + int64_t(threadIdx.x / 32) * (32 / LPN); n0 < blk.y; n0 += 256 / LPN) {
    const int64_t nd = n0 + (threadIdx.x % 32) / LPN;  // the loop bound is warp-uniform
    float h0 = 0.f, l0 = 0.f, h1 = 0.f, l1 = 0.f, h2 = 0.f, l2 = 0.f;
    bool fixed = true;
    if (nd < blk.y) {
      fixed = fixed_row[3 * nd] != 0;
      if (!fixed) {
        const int32_t k0 = bptr[nd], k1 = bptr[nd + 1];
        const int32_t r0 = rowptr[3 * nd], r1 = rowptr[3 * nd + 1], r2 = rowptr[3 * nd + 2];
        for (int32_t k = k0 + sub; k < k1; k += LPN) {
          const int64_t cc = 3 * int64_t(bcol[k]);
          const float2 x0 = x[cc], x1 = x[cc + 1], x2 = x[cc + 2];
          const int32_t o = 3 * (k - k0);
          df_fma_to(h0, l0, A[r0 + o], x0);
          df_fma_to(h0, l0, A[r0 + o + 1], x1);
          df_fma_to(h0, l0, A[r0 + o + 2], x2);
          df_fma_to(h1, l1, A[r1 + o], x0);
          df_fma_to(h1, l1, A[r1 + o + 1], x1);
          df_fma_to(h1, l1, A[r1 + o + 2], x2);
          df_fma_to(h2, l2, A[r2 + o], x0);
          df_fma_to(h2, l2, A[r2 + o + 1], x1);
          df_fma_to(h2, l2, A[r2 + o + 2], x2);
        }
      }
    }
#pragma unroll
    for (int o = LPN / 2; o > 0; o >>= 1) {
      df_shfl_add<LPN>(h0, l0, o);
      df_shfl_add<LPN>(h1, l1, o);
      df_shfl_add<LPN>(h2, l2, o);
    }
    if (sub < 3 && nd < blk.y) {
      const int64_t rw = 3 * nd + sub;
      float hi = sub == 0 ? h0 : (sub == 1 ? h1 : h2), lo = sub == 0 ? l0 : (sub == 1 ? l1 : l2);
      if (fixed) {
        hi = lo = 0.f;
        df_fma_to(hi, lo, A[rowptr[rw]], x[rw]);
      }
      y[rw] = b[rw] - df_value(hi, lo);
    }
  }
}

template <int TPR>
__global__ void __launch_bounds__(256) batch_csr_res_df_kernel(const int2 *__restrict__ blocks,
                                                               const int32_t *__restrict__ rowptr,
                                                               const int32_t *__restrict__ colind,
                                                               const float2 *__restrict__ A,
                                                               const float2 *__restrict__ x,
                                                               const double *__restrict__ b, double *__restrict__ y) {
  const int2 blk = blocks[blockIdx.x];
  const int64_t rb = 3 * int64_t(blk.x), re = 3 * int64_t(blk.y);
  const int sub = threadIdx.x % TPR;
  for (int64_t r0 = rb + int64_t(threadIdx.x / 32) * (32 / TPR); r0 < re; r0 += 256 / TPR) {
    const int64_t row = r0 + (threadIdx.x % 32) / TPR;
    float hi = 0.f, lo = 0.f;
    if (row < re) {
      const int32_t k1 = rowptr[row + 1];
      for (int32_t k = rowptr[row] + sub; k < k1; k += TPR) df_fma_to(hi, lo, A[k], x[colind[k]]);
    }
#pragma unroll
    for (int o = TPR / 2; o > 0; o >>= 1) df_shfl_add<TPR>(hi, lo, o);
    if (sub == 0 && row < re) y[row] = b[row] - df_value(hi, lo);
  }
}

void launch_class_res_df(const DeviceState::SpmvClass &k, const DeviceState *d, const double *b, double *y,
                         cudaStream_t s) {
  if (!k.nblocks) return;
  const unsigned g = unsigned(k.nblocks);
  if (k.lpn < 0) {  // CSR, -lpn threads per row
    if (k.lpn == -16)
      batch_csr_res_df_kernel<16><<<g, 256, 0, s>>>(k.blocks, d->rowptr, d->colind, d->A2, d->x2, b, y);
    else
      batch_csr_res_df_kernel<8><<<g, 256, 0, s>>>(k.blocks, d->rowptr, d->colind, d->A2, d->x2, b, y);
    return;
  }
  switch (k.lpn) {
    case 4:
      batch_bres_df_kernel<4><<<g, 256, 0, s>>>(k.blocks, d->rowptr, d->bptr, d->bcol, d->fixed_row, d->A2, d->x2, b, y);
      break;
    case 8:
      batch_bres_df_kernel<8><<<g, 256, 0, s>>>(k.blocks, d->rowptr, d->bptr, d->bcol, d->fixed_row, d->A2, d->x2, b, y);
      break;
    case 32:
      batch_bres_df_kernel<32><<<g, 256, 0, s>>>(k.blocks, d->rowptr, d->bptr, d->bcol, d->fixed_row, d->A2, d->x2, b, y);
      break;
    default:
      batch_bres_df_kernel<16><<<g, 256, 0, s>>>(k.blocks, d->rowptr, d->bptr, d->bcol, d->fixed_row, d->A2, d->x2, b, y);
  }
}

template <typename TA, typename TV, int MODE>
void launch_class(const DeviceState::SpmvClass &k, const DeviceState *d, const TA *A, const TV *x, const double *b,
                  TV *y, cudaStream_t s) {
  if (!k.nblocks) return;
  const unsigned g = unsigned(k.nblocks);
  if (k.lpn < 0) {  // CSR, -lpn threads per row
    if (k.lpn == -16)
      batch_csr_kernel<TA, TV, 16, MODE><<<g, 256, 0, s>>>(k.blocks, d->rowptr, d->colind, A, x, b, y);
    else
      batch_csr_kernel<TA, TV, 8, MODE><<<g, 256, 0, s>>>(k.blocks, d->rowptr, d->colind, A, x, b, y);
    return;
  }
  switch (k.lpn) {
    case 4:
      batch_bspmv_kernel<TA, TV, 4, MODE><<<g, 256, 0, s>>>(k.blocks, d->rowptr, d->bptr, d->bcol, d->fixed_row, A, x, b, y);
      break;
    case 8:
      batch_bspmv_kernel<TA, TV, 8, MODE><<<g, 256, 0, s>>>(k.blocks, d->rowptr, d->bptr, d->bcol, d->fixed_row, A, x, b, y);
      break;
    case 32:
      batch_bspmv_kernel<TA, TV, 32, MODE><<<g, 256, 0, s>>>(k.blocks, d->rowptr, d->bptr, d->bcol, d->fixed_row, A, x, b, y);
      break;
    default:
      batch_bspmv_kernel<TA, TV, 16, MODE><<<g, 256, 0, s>>>(k.blocks, d->rowptr, d->bptr, d->bcol, d->fixed_row, A, x, b, y);
  }
}

void run_class(const fe_ctx *c, const DeviceState *d, const DeviceState::SpmvClass &k, bool fp32, const void *x,
               void *y, const double *b, cudaStream_t s) {
  if (b && d->A2)  // the mixed path's residual: A2 and the mirror x2 of x (= d->x)
    launch_class_res_df(k, d, b, static_cast<double *>(y), s);
  else if (b)
    launch_class<double, double, 1>(k, d, d->A64, static_cast<const double *>(x), b, static_cast<double *>(y), s);
  else if (fp32)
    launch_class<float, float, 0>(k, d, static_cast<const float *>(d->A), static_cast<const float *>(x), nullptr,
                                  static_cast<float *>(y), s);
  else
    launch_class<double, double, 0>(k, d, static_cast<const double *>(d->A), static_cast<const double *>(x), nullptr,
                                    static_cast<double *>(y), s);
}

// graph conditions of the batched solve (one CTA over the members)
__global__ void __launch_bounds__(256) seg_cond_kernel(cudaGraphConditionalHandle h, double *bs, double *scal,
                                                       int nseg, int mode, double max_iters, int *flags) {
  __shared__ int s_open;
  __shared__ double s_iters;
  if (threadIdx.x == 0) {
    s_open = 0;
    s_iters = 0.0;
  }
  __syncthreads();
  const int slot = (mode == 0 || mode == 3) ? B_DONE : B_ODONE;
  int open = 0;
  double it = 0.0;
  for (int k = threadIdx.x; k < nseg; k += 256) {
    open |= bs[int64_t(k) * B_COUNT + slot] == 0.0;
    it = fmax(it, bs[int64_t(k) * B_COUNT + B_ITERS]);
  }
  if (open) atomicOr(&s_open, 1);
  // non-negative doubles order like their bit patterns
  if (it > 0.0) atomicMax(reinterpret_cast<unsigned long long *>(&s_iters), __double_as_longlong(it));
  __syncthreads();
  if (threadIdx.x != 0) return;
  if (mode >= 3) {
    flags[2] = (!s_open && flags[0] == 0) ? 1 : 0;
    return;
  }
  if (mode == 2) scal[S_SWEEPS] = 0.0;
  if (mode == 1) scal[S_SWEEPS] += 1.0;
  const bool go = s_open && s_iters < max_iters && flags[0] == 0;
  cudaGraphSetConditional(h, go ? 1u : 0u);
}

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
                                                          inner, nullptr);
  else
    seg_init_kernel<double><<<grid_for(c->n), 256, 0, s>>>(c->n, (double *)x, (double *)r, rhs, d->row_seg,
                                                           d->bscal, inner, x == d->x ? d->x2 : nullptr);
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

}  // namespace fe

namespace fe {

void launch_batch_spmv(const fe_ctx *c, const DeviceState *d, bool fp32, const void *x, void *y, const double *b,
                       cudaStream_t s) {
  d->launches += int64_t(d->spmv_classes.size());
  for (const auto &k : d->spmv_classes) run_class(c, d, k, fp32, x, y, b, s);
}

void launch_seg_cond(const fe_ctx *c, const DeviceState *d, cudaGraphConditionalHandle h, int mode,
                     cudaStream_t s) {
  d->launches++;
  seg_cond_kernel<<<1, 256, 0, s>>>(h, d->bscal, d->scal, c->nseg, mode, double(c->opt.max_iters), d->flags);
}

// Size classes and row blocks of the batched SpMV, then each class's kernel
// by timing its own row blocks on the assembled matrix (CUDA events, one
// untimed run then the median of five): the node-block kernel with 4, 8, 16
// or 32 lanes per node, or CSR with 8 or 16 threads per row.  Members are ordered by
// their mean blocks per free node and cut into at most three classes of
// about equal node counts: longer rows want more lanes per node.
int tune_batch_spmv(fe_ctx *c, DeviceState *d) {
  if (d->spmv_tuned) return FE_OK;
  const int32_t nb = c->nseg;
  std::vector<std::pair<double, int32_t>> mean(nb);
  int64_t total_nodes = 0;
  for (int32_t k = 0; k < nb; ++k) {
    int64_t blocks = 0, freen = 0;
    for (int64_t n = c->seg_node[k]; n < c->seg_node[k + 1]; ++n) {
      if (c->fixed_dof[3 * n]) continue;
      blocks += c->bptr[n + 1] - c->bptr[n];
      ++freen;
    }
    mean[k] = {freen ? double(blocks) / double(freen) : 0.0, k};
    total_nodes += c->seg_node[k + 1] - c->seg_node[k];
  }
  std::stable_sort(mean.begin(), mean.end());
  const int ncls = nb >= 3 ? 3 : nb;
  d->spmv_classes.assign(ncls, DeviceState::SpmvClass());
  int64_t acc = 0;
  for (const auto &m : mean) {
    const int32_t k = m.second;
    const int cls = std::min<int>(ncls - 1, int(acc * ncls / std::max<int64_t>(total_nodes, 1)));
    d->spmv_classes[cls].members.push_back(k);
    acc += c->seg_node[k + 1] - c->seg_node[k];
  }
  for (auto &cl : d->spmv_classes) {
    std::vector<int2> blk;
    std::sort(cl.members.begin(), cl.members.end());
    for (int32_t k : cl.members)
      for (int64_t n0 = c->seg_node[k]; n0 < c->seg_node[k + 1]; n0 += kBatchBlockNodes)
        blk.push_back(make_int2(int(n0), int(std::min<int64_t>(n0 + kBatchBlockNodes, c->seg_node[k + 1]))));
    cl.nblocks = int64_t(blk.size());
    if (!blk.empty()) {
      cudaError_t e = cudaMalloc(&cl.blocks, blk.size() * sizeof(int2));
      if (e != cudaSuccess) {
        cudaGetLastError();
        return set_error(c, FE_ERR_OOM, "batched SpMV schedule allocation failed");
      }
      d->allocs.push_back(cl.blocks);
      FE_CUDA_TRY(cudaMemcpy(cl.blocks, blk.data(), blk.size() * sizeof(int2), cudaMemcpyHostToDevice));
    }
  }
  const bool fp32 = c->opt.precision == FE_MIXED;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  FE_CUDA_TRY(cudaEventCreate(&e0));
  cudaError_t er = cudaEventCreate(&e1);
  const int fixed = c->opt.spmv_variant;
  for (auto &cl : d->spmv_classes) {
    if (fixed >= 0) {  // fixed by the caller: no timing
      cl.lpn = fixed <= 3 ? (4 << fixed) : (fixed == 4 ? -8 : -16);
      continue;
    }
    if (er != cudaSuccess || !cl.nblocks) continue;
    float best = 1e30f;
    int best_lpn = 16;
    for (int lpn : {4, 8, 16, 32, -8, -16}) {  // node-block lanes per node, or CSR threads per row
      cl.lpn = lpn;
      float t[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
      for (int rep = 0; rep < 6 && er == cudaSuccess; ++rep) {  // one untimed run, five timed
        er = cudaEventRecord(e0, d->stream);
        if (er == cudaSuccess) run_class(c, d, cl, fp32, d->vp, d->vq, nullptr, d->stream);
        if (er == cudaSuccess) er = cudaGetLastError();
        if (er == cudaSuccess) er = cudaEventRecord(e1, d->stream);
        if (er == cudaSuccess) er = cudaEventSynchronize(e1);
        if (er == cudaSuccess) er = cudaEventElapsedTime(&t[rep], e0, e1);
      }
      std::sort(t + 1, t + 6);
      if (er == cudaSuccess && t[3] < best) {
        best = t[3];
        best_lpn = lpn;
      }
    }
    cl.lpn = best_lpn;
  }
  cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (er != cudaSuccess) {
    cudaGetLastError();
    return set_error(c, FE_ERR_CUDA, std::string("batched SpMV autotuner: ") + cudaGetErrorString(er));
  }
  d->spmv_tuned = true;
  return FE_OK;
}

}  // namespace fe
