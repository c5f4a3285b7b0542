// Numeric LDL^T of A on the nested-dissection fronts (Section 3.3, Eq.
// "asynchronous preconditioner"; Section 6.1, Eq. "regional problem") and its
// level-scheduled application z = (L D L^T)^{-1} r.
//
// Every front f holds pivots P (a separator or a leaf sub-domain) and update
// rows U (ancestor DOFs coupled to its subtree).  The dense front
// F = [A_PP A_PU; A_UP A_UU] + extend-add of the children's Schur complements
// is factored right-looking in panels of kNB pivots.  Alongside L and D the
// same eliminations build the front's apply operator
//     Y = [L_PP 0; L_UP I]^{-1} [I; 0] = [L_PP^{-1}; -L_UP L_PP^{-1}],
// so that, level by level,
//     forward :  y_P = Y_P w_P,            u = w_U + Y_U w_P
//     backward:  z_P = Y^T [D^{-1} y_P; z_U]
// are dense GEMVs over Y, parallel across all rows/columns of all fronts of
// a level: the only serial dependency left is the level order
// (leaves up for L, root down for L^T), as in the paper's level schedule.
#include <cuda_runtime.h>

#include "fe_device.cuh"

namespace fe {

// -------------------------------------------------------------- assembly
// Task (front, c0, c1): zero the lower part of columns [c0, c1) of F and of
// the pivot columns of Y, scatter the A entries of those columns, then add
// every child's update block (children in fixed order: deterministic).
template <typename TF>
__global__ void __launch_bounds__(256) front_assemble_kernel(
    const int32_t *__restrict__ tasks, const DFront *__restrict__ fronts,
    const int32_t *__restrict__ child_list, const int32_t *__restrict__ rmap,
    const int64_t *__restrict__ fa_colptr, const int32_t *__restrict__ fa_slot,
    const int32_t *__restrict__ fa_off, const TF *__restrict__ A, TF *__restrict__ F, TF *__restrict__ Y) {
  const int32_t f = tasks[3 * blockIdx.x], c0 = tasks[3 * blockIdx.x + 1], c1 = tasks[3 * blockIdx.x + 2];
  const DFront fr = fronts[f];
  const int32_t m = fr.m, p = fr.npiv;
  TF *Ff = F + fr.f_off;
  for (int32_t col = c0; col < c1; ++col) {
    TF *cp = Ff + int64_t(col) * m;
    for (int32_t r = col + threadIdx.x; r < m; r += blockDim.x) cp[r] = TF(0);
    if (col < p) {
      TF *yp = Y + fr.y_off + int64_t(col) * m;
      for (int32_t r = threadIdx.x; r < m; r += blockDim.x) yp[r] = TF(0);
    }
  }
  __syncthreads();
  const int32_t ce = c1 < p ? c1 : p;
  for (int32_t col = c0; col < ce; ++col) {
    const int64_t e0 = fa_colptr[fr.fac_off + col], e1 = fa_colptr[fr.fac_off + col + 1];
    for (int64_t e = e0 + threadIdx.x; e < e1; e += blockDim.x) Ff[fa_off[e]] = A[fa_slot[e]];
  }
  __syncthreads();
  for (int32_t ci = fr.child_begin; ci < fr.child_end; ++ci) {
    const DFront ch = fronts[child_list[ci]];
    const int32_t *rm = rmap + ch.rows_off;
    const int32_t nu = ch.nupd, pc = ch.npiv, mc = ch.m;
    // child columns mapping into [c0, c1): contiguous since rm is increasing
    int32_t lo = 0, hi = nu;
    while (lo < hi) { int32_t mid = (lo + hi) >> 1; if (rm[mid] < c0) lo = mid + 1; else hi = mid; }
    const int32_t jlo = lo;
    hi = nu;
    while (lo < hi) { int32_t mid = (lo + hi) >> 1; if (rm[mid] < c1) lo = mid + 1; else hi = mid; }
    const int32_t jhi = lo;
    const TF *Fc = F + ch.f_off;
    for (int32_t j = jlo; j < jhi; ++j) {
      const TF *src = Fc + int64_t(pc + j) * mc + pc;
      TF *dst = Ff + int64_t(rm[j]) * m;
      for (int32_t i = j + threadIdx.x; i < nu; i += blockDim.x) dst[rm[i]] += src[i];
    }
    __syncthreads();
  }
}

// ---------------------------------------------------------------- diagonal
// Task (front, k0, kb): LDL^T of the kb x kb diagonal block in FP64, pivots
// to D (and 1/D), L back into F, L^{-1} of the block into Y[K, K].
template <typename TF>
__global__ void __launch_bounds__(256) front_diag_kernel(const int32_t *__restrict__ tasks,
                                                         const DFront *__restrict__ fronts, TF *__restrict__ F,
                                                         TF *__restrict__ Y, double *__restrict__ D,
                                                         double *__restrict__ Dinv, int *flags) {
  extern __shared__ double dsm[];
  double *L = dsm;                 // [64][65]
  double *Xi = dsm + 64 * 65;      // [64][65]
  const int4 t = reinterpret_cast<const int4 *>(tasks)[blockIdx.x];
  const DFront fr = fronts[t.x];
  const int32_t k0 = t.y & 0xffffff, kb = t.z, m = fr.m;
  TF *Ff = F + fr.f_off;
  for (int idx = threadIdx.x; idx < kb * kb; idx += blockDim.x) {
    const int i = idx % kb, j = idx / kb;
    L[i * 65 + j] = (i >= j) ? double(Ff[(k0 + i) + int64_t(k0 + j) * m]) : 0.0;
  }
  __syncthreads();
  for (int j = 0; j < kb; ++j) {
    double d = L[j * 65 + j];
    if (!(d > 0.0)) {
      if (threadIdx.x == 0) atomicOr(flags, FLAG_PIVOT);
      d = 1.0;
    }
    const double invd = 1.0 / d;
    const int T = kb - j - 1;
    for (int idx = threadIdx.x; idx < T * T; idx += blockDim.x) {
      const int ii = idx / T, kk = idx % T;
      if (kk <= ii) {
        const int i = j + 1 + ii, k = j + 1 + kk;
        L[i * 65 + k] -= L[i * 65 + j] * L[k * 65 + j] * invd;
      }
    }
    __syncthreads();
    for (int i = j + 1 + threadIdx.x; i < kb; i += blockDim.x) L[i * 65 + j] *= invd;
    if (threadIdx.x == 0) {
      L[j * 65 + j] = d;
      D[fr.first + k0 + j] = d;
      Dinv[fr.first + k0 + j] = invd;
    }
    __syncthreads();
  }
  // L^{-1} of the unit lower block, one column per thread
  if (threadIdx.x < kb) {
    const int c = threadIdx.x;
    for (int i = 0; i < kb; ++i) Xi[i * 65 + c] = (i == c) ? 1.0 : 0.0;
    for (int i = c + 1; i < kb; ++i) {
      double s = 0.0;
      for (int j = c; j < i; ++j) s += L[i * 65 + j] * Xi[j * 65 + c];
      Xi[i * 65 + c] = -s;
    }
  }
  __syncthreads();
  TF *Yf = Y + fr.y_off;
  for (int idx = threadIdx.x; idx < kb * kb; idx += blockDim.x) {
    const int i = idx % kb, j = idx / kb;
    if (i > j) Ff[(k0 + i) + int64_t(k0 + j) * m] = TF(L[i * 65 + j]);
    Yf[(k0 + i) + int64_t(k0 + j) * m] = TF(Xi[i * 65 + j]);
  }
}

// ------------------------------------------------------- panel and X_K
// PANEL (front, k0, r0): rows [r0, r0+64) of the panel: L = F L_KK^{-T} D^{-1}.
// XK    (front, k0, c0): Y[K, c0:c0+64] <- L_KK^{-1} Y[K, c0:c0+64].
template <typename TF>
__global__ void __launch_bounds__(256) front_panel_kernel(const int32_t *__restrict__ tasks,
                                                          const DFront *__restrict__ fronts,
                                                          TF *__restrict__ F, TF *__restrict__ Y,
                                                          const double *__restrict__ Dinv) {
  extern __shared__ unsigned char psm[];
  TF(*Ls)[65] = reinterpret_cast<TF(*)[65]>(psm);
  TF(*Bs)[65] = reinterpret_cast<TF(*)[65]>(psm + 64 * 65 * sizeof(TF));
  const int4 t = reinterpret_cast<const int4 *>(tasks)[blockIdx.x];
  const DFront fr = fronts[t.x];
  const int kind = t.y >> 24;
  const int32_t k0 = t.y & 0xffffff, a0 = t.z, m = fr.m;
  const int32_t kb = (fr.npiv - k0) < 64 ? (fr.npiv - k0) : 64;
  TF *Ff = F + fr.f_off;
  TF *Yf = Y + fr.y_off;
  for (int idx = threadIdx.x; idx < 64 * 64; idx += blockDim.x) {
    const int i = idx % 64, j = idx / 64;
    Ls[i][j] = (i < kb && j < kb && i >= j) ? Yf[(k0 + i) + int64_t(k0 + j) * m] : TF(0);
  }
  const int tr = threadIdx.x / 16, tc = threadIdx.x % 16;
  if (kind == T_PANEL) {
    for (int idx = threadIdx.x; idx < 64 * 64; idx += blockDim.x) {
      const int i = idx % 64, j = idx / 64;
      const int32_t r = a0 + i;
      Bs[i][j] = (r < m && j < kb) ? Ff[r + int64_t(k0 + j) * m] : TF(0);
    }
    __syncthreads();
    TF acc[4][4] = {};
    for (int j = 0; j < kb; ++j) {
      TF av[4], bv[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) av[u] = Bs[tr * 4 + u][j];
#pragma unroll
      for (int s = 0; s < 4; ++s) bv[s] = Ls[tc + 16 * s][j];  // (L^{-T})[j][c] = Linv[c][j]
#pragma unroll
      for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int s = 0; s < 4; ++s) acc[u][s] += av[u] * bv[s];
    }
#pragma unroll
    for (int s = 0; s < 4; ++s) {
      const int c = tc + 16 * s;
      if (c >= kb) continue;
      const TF di = TF(Dinv[fr.first + k0 + c]);
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int32_t r = a0 + tr * 4 + u;
        if (r < m) Ff[r + int64_t(k0 + c) * m] = acc[u][s] * di;
      }
    }
  } else {  // T_XK
    for (int idx = threadIdx.x; idx < 64 * 64; idx += blockDim.x) {
      const int j = idx % 64, c = idx / 64;
      Bs[j][c] = (j < kb && a0 + c < k0) ? Yf[(k0 + j) + int64_t(a0 + c) * m] : TF(0);
    }
    __syncthreads();
    TF acc[4][4] = {};
    for (int j = 0; j < kb; ++j) {
      TF av[4], bv[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) av[u] = Ls[tr * 4 + u][j];
#pragma unroll
      for (int s = 0; s < 4; ++s) bv[s] = Bs[j][tc + 16 * s];
#pragma unroll
      for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int s = 0; s < 4; ++s) acc[u][s] += av[u] * bv[s];
    }
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int i = tr * 4 + u;
      if (i >= kb) continue;
#pragma unroll
      for (int s = 0; s < 4; ++s) {
        const int32_t c = a0 + tc + 16 * s;
        if (c < k0) Yf[(k0 + i) + int64_t(c) * m] = acc[u][s];
      }
    }
  }
}

// ------------------------------------------------------ trailing updates
// TRAIL (front, k0, i0, j0): F[I, J] -= L[I, K] D_K L[J, K]^T (lower part).
// RUPD  (front, k0, i0, c0): Y[I, C] -= L[I, K] Y[K, C]  (Y[K, :] = X_K).
template <typename TF>
__global__ void __launch_bounds__(256) front_update_kernel(const int32_t *__restrict__ tasks,
                                                           const DFront *__restrict__ fronts,
                                                           TF *__restrict__ F, TF *__restrict__ Y,
                                                           const double *__restrict__ D) {
  extern __shared__ unsigned char usm[];
  TF(*As)[65] = reinterpret_cast<TF(*)[65]>(usm);
  TF(*Bs)[65] = reinterpret_cast<TF(*)[65]>(usm + 64 * 65 * sizeof(TF));
  const int4 t = reinterpret_cast<const int4 *>(tasks)[blockIdx.x];
  const DFront fr = fronts[t.x];
  const int kind = t.y >> 24;
  const int32_t k0 = t.y & 0xffffff, i0 = t.z, j0 = t.w, m = fr.m;
  const int32_t kb = (fr.npiv - k0) < 64 ? (fr.npiv - k0) : 64;
  TF *Ff = F + fr.f_off;
  TF *Yf = Y + fr.y_off;
  for (int idx = threadIdx.x; idx < 64 * 64; idx += blockDim.x) {
    const int i = idx % 64, l = idx / 64;
    const int32_t r = i0 + i;
    As[i][l] = (r < m && l < kb) ? Ff[r + int64_t(k0 + l) * m] : TF(0);
  }
  if (kind == T_TRAIL) {
    for (int idx = threadIdx.x; idx < 64 * 64; idx += blockDim.x) {
      const int j = idx % 64, l = idx / 64;
      const int32_t r = j0 + j;
      Bs[j][l] = (r < m && l < kb) ? Ff[r + int64_t(k0 + l) * m] * TF(D[fr.first + k0 + l]) : TF(0);
    }
  } else {
    for (int idx = threadIdx.x; idx < 64 * 64; idx += blockDim.x) {
      const int l = idx % 64, j = idx / 64;
      const int32_t c = j0 + j;
      Bs[j][l] = (l < kb && c < k0 + kb) ? Yf[(k0 + l) + int64_t(c) * m] : TF(0);
    }
  }
  __syncthreads();
  const int tr = threadIdx.x / 16, tc = threadIdx.x % 16;
  TF acc[4][4] = {};
  for (int l = 0; l < kb; ++l) {
    TF av[4], bv[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) av[u] = As[tr + 16 * u][l];
#pragma unroll
    for (int s = 0; s < 4; ++s) bv[s] = Bs[tc + 16 * s][l];
#pragma unroll
    for (int u = 0; u < 4; ++u)
#pragma unroll
      for (int s = 0; s < 4; ++s) acc[u][s] += av[u] * bv[s];
  }
  if (kind == T_TRAIL) {
#pragma unroll
    for (int s = 0; s < 4; ++s) {
      const int32_t c = j0 + tc + 16 * s;
      if (c >= m) continue;
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int32_t r = i0 + tr + 16 * u;
        if (r < m && r >= c) Ff[r + int64_t(c) * m] -= acc[u][s];
      }
    }
  } else {
#pragma unroll
    for (int s = 0; s < 4; ++s) {
      const int32_t c = j0 + tc + 16 * s;
      if (c >= k0 + kb) continue;
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int32_t r = i0 + tr + 16 * u;
        if (r < m) Yf[r + int64_t(c) * m] -= acc[u][s];
      }
    }
  }
}

// ------------------------------------------------------------------ apply
// Forward, part 1 (one block per front of the level): w = [r_P; 0] plus the
// children's update vectors extend-added in fixed order.
template <typename TV>
__global__ void __launch_bounds__(256) fwd_gather_kernel(const int32_t *__restrict__ level_fronts,
                                                         const DFront *__restrict__ fronts,
                                                         const int32_t *__restrict__ child_list,
                                                         const int32_t *__restrict__ rmap,
                                                         const int32_t *__restrict__ perm,
                                                         const TV *__restrict__ r, TV *__restrict__ wbuf,
                                                         const TV *__restrict__ ubuf) {
  const DFront fr = fronts[level_fronts[blockIdx.x]];
  TV *w = wbuf + fr.w_off;
  for (int32_t i = threadIdx.x; i < fr.m; i += blockDim.x) w[i] = (i < fr.npiv) ? r[perm[fr.first + i]] : TV(0);
  __syncthreads();
  for (int32_t ci = fr.child_begin; ci < fr.child_end; ++ci) {
    const DFront ch = fronts[child_list[ci]];
    const int32_t *rm = rmap + ch.rows_off;
    const TV *u = ubuf + ch.u_off;
    for (int32_t j = threadIdx.x; j < ch.nupd; j += blockDim.x) w[rm[j]] += u[j];
    __syncthreads();
  }
}

// Forward, part 2, task (front, r0): rows [r0, r0+64) of Y w_P;
// y_P (times D^{-1}) to yperm, U rows to the update vector.
template <typename TF, typename TV>
__global__ void __launch_bounds__(256) fwd_gemv_kernel(const int32_t *__restrict__ tasks,
                                                       const DFront *__restrict__ fronts,
                                                       const TF *__restrict__ Y,
                                                       const double *__restrict__ Dinv,
                                                       const TV *__restrict__ wbuf, TV *__restrict__ ubuf,
                                                       TV *__restrict__ yperm) {
  extern __shared__ unsigned char sraw[];
  TV *wp = reinterpret_cast<TV *>(sraw);
  __shared__ TV part[4][64];
  const DFront fr = fronts[tasks[2 * blockIdx.x]];
  const int32_t r0 = tasks[2 * blockIdx.x + 1];
  const int32_t p = fr.npiv, m = fr.m;
  const TV *w = wbuf + fr.w_off;
  const int32_t rend = (r0 + 64 < m) ? r0 + 64 : m;
  const int32_t jmax = (rend < p) ? rend : p;
  for (int32_t j = threadIdx.x; j < jmax; j += blockDim.x) wp[j] = w[j];
  __syncthreads();
  const int lr = threadIdx.x & 63, g = threadIdx.x >> 6;
  const int32_t row = r0 + lr;
  TV acc = TV(0);
  if (row < m) {
    const int32_t je = (row < p) ? row + 1 : p;
    const TF *yc = Y + fr.y_off + row;
    for (int32_t j = g; j < je; j += 4) acc += TV(yc[int64_t(j) * m]) * wp[j];
  }
  part[g][lr] = acc;
  __syncthreads();
  if (g == 0 && row < m) {
    const TV s = part[0][lr] + part[1][lr] + part[2][lr] + part[3][lr];
    if (row < p)
      yperm[fr.first + row] = TV(double(s) * Dinv[fr.first + row]);
    else
      ubuf[fr.u_off + row - p] = w[row] + s;
  }
}

// Backward, task (front, c0): one warp per pivot column j in [c0, c0+8):
// z_j = sum_i Y[i, j] x_i, x = [D^{-1} y_P; z_U].
template <typename TF, typename TV>
__global__ void __launch_bounds__(256) bwd_kernel(const int32_t *__restrict__ tasks,
                                                  const DFront *__restrict__ fronts, const TF *__restrict__ Y,
                                                  const int32_t *__restrict__ perm,
                                                  const int32_t *__restrict__ upd_rows_old,
                                                  const TV *__restrict__ yperm, TV *__restrict__ z) {
  const DFront fr = fronts[tasks[2 * blockIdx.x]];
  const int32_t j = tasks[2 * blockIdx.x + 1] + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  if (j >= fr.npiv) return;
  const int32_t p = fr.npiv, m = fr.m;
  const TF *yc = Y + fr.y_off + int64_t(j) * m;
  const int32_t *urows = upd_rows_old + fr.rows_off;
  TV acc = TV(0);
  for (int32_t i = j + lane; i < m; i += 32) {
    const TV xi = (i < p) ? yperm[fr.first + i] : z[urows[i - p]];
    acc += TV(yc[i]) * xi;
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if (lane == 0) z[perm[fr.first + j]] = acc;
}

// ------------------------------------------------------------ host drivers

template <typename TF>
static void factor_levels(const fe_ctx *c, DeviceState *d, int buf, const TF *Afac, cudaStream_t s) {
  TF *F = reinterpret_cast<TF *>(d->F);
  TF *Y = reinterpret_cast<TF *>(d->Y[buf]);
  const size_t dsm = 2 * 64 * 65 * sizeof(double);
  const size_t tsm = 2 * 64 * 65 * sizeof(TF);
  cudaFuncSetAttribute(front_diag_kernel<TF>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(dsm));
  cudaFuncSetAttribute(front_panel_kernel<TF>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(tsm));
  cudaFuncSetAttribute(front_update_kernel<TF>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(tsm));
  for (size_t lv = 0; lv < d->lt.size(); ++lv) {
    const auto &L = d->lt[lv];
    if (L.asm_n) d->launches++;
    if (L.asm_n)
      front_assemble_kernel<TF><<<unsigned(L.asm_n), 256, 0, s>>>(d->tasks + L.asm_off, d->fronts, d->child_list,
                                                                  d->rmap, d->fa_colptr, d->fa_slot, d->fa_off,
                                                                  Afac, F, Y);
    for (size_t st = 0; st < L.diag_n.size(); ++st) {
      d->launches += (L.diag_n[st] > 0) + (L.panel_n[st] > 0) + (L.trail_n[st] > 0);
      if (L.diag_n[st])
        front_diag_kernel<TF><<<unsigned(L.diag_n[st]), 256, dsm, s>>>(d->tasks + L.diag_off[st], d->fronts, F, Y,
                                                                       d->D[buf], d->D[buf] + c->n_free, d->flags);
      if (L.panel_n[st])
        front_panel_kernel<TF><<<unsigned(L.panel_n[st]), 256, tsm, s>>>(d->tasks + L.panel_off[st], d->fronts, F, Y,
                                                                       d->D[buf] + c->n_free);
      if (L.trail_n[st])
        front_update_kernel<TF><<<unsigned(L.trail_n[st]), 256, tsm, s>>>(d->tasks + L.trail_off[st], d->fronts, F, Y,
                                                                        d->D[buf]);
    }
  }
}

int factor_enqueue(fe_ctx *c, DeviceState *d, int buf, bool fp32, const void *Afac, cudaStream_t s) {
  if (fp32)
    factor_levels<float>(c, d, buf, reinterpret_cast<const float *>(Afac), s);
  else
    factor_levels<double>(c, d, buf, reinterpret_cast<const double *>(Afac), s);
  return FE_OK;
}

template <typename TF, typename TV>
static void apply_levels(const fe_ctx *c, const DeviceState *d, int buf, const TV *r, TV *z, cudaStream_t s) {
  const TF *Y = reinterpret_cast<const TF *>(d->Y[buf]);
  const double *Dinv = d->D[buf] + c->n_free;
  TV *w = reinterpret_cast<TV *>(d->wbuf);
  TV *u = reinterpret_cast<TV *>(d->ubuf);
  TV *yp = reinterpret_cast<TV *>(d->yperm);
  int32_t pmax = 0;
  for (const auto &f : c->fronts) pmax = std::max(pmax, f.npiv);
  const size_t sm = size_t(pmax) * sizeof(TV);
  cudaFuncSetAttribute(fwd_gemv_kernel<TF, TV>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(sm));
  d->launches += 3 * int64_t(d->lt.size());
  for (size_t lv = 0; lv < d->lt.size(); ++lv) {
    const auto &L = d->lt[lv];
    fwd_gather_kernel<TV><<<unsigned(L.nfronts), 256, 0, s>>>(d->level_fronts + L.fronts_off, d->fronts,
                                                              d->child_list, d->rmap, d->perm, r, w, u);
    fwd_gemv_kernel<TF, TV><<<unsigned(L.fwd_n), 256, sm, s>>>(d->tasks + L.fwd_off, d->fronts, Y, Dinv, w, u, yp);
  }
  for (size_t lv = d->lt.size(); lv-- > 0;) {
    const auto &L = d->lt[lv];
    bwd_kernel<TF, TV><<<unsigned(L.bwd_n), 256, 0, s>>>(d->tasks + L.bwd_off, d->fronts, Y, d->perm,
                                                         d->upd_rows_old, yp, z);
  }
}

void apply_enqueue(const fe_ctx *c, const DeviceState *d, int buf, bool fp32, const void *r, void *z,
                   cudaStream_t s) {
  if (fp32)
    apply_levels<float, float>(c, d, buf, reinterpret_cast<const float *>(r), reinterpret_cast<float *>(z), s);
  else
    apply_levels<double, double>(c, d, buf, reinterpret_cast<const double *>(r), reinterpret_cast<double *>(z), s);
}

}  // namespace fe
