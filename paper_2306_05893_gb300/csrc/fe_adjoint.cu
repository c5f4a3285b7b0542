// Discrete adjoint of the implicit rollout: per-element kernels that give,
// in one forward-mode (dual-number) pass over the element tangent,
//   ge_e  = dK_e[lambda_e] u_e + K_e lambda_e,   u = c_K a + (beta + h) v,
//   kl_e  = K_e lambda_e,
//   s_bar_e -= lambda_e . (K_e u_e + f_e)        (energy scale of element e),
// and a per-node gather that updates (q_bar, v_bar):
//   q_bar <- q_bar - sum_e ge_e,
//   v_bar <- v_bar + h q_bar - (alpha M + (beta + h) K) lambda.
// K_e u_e is never formed as a matrix: K_e u_e = int grad N_a . (CC : grad u),
// the linearised stress of the nodal field u, so one contraction of the
// 3x3 tangent blocks with grad u (dual) and grad lambda (real) suffices.
#include <cuda_runtime.h>

#include "fe_device.cuh"
#include "fe_material.cuh"

namespace fe {

template <typename T>
struct Dual {
  T re, du;
  __device__ Dual() : re(T(0)), du(T(0)) {}
  __device__ Dual(double r) : re(T(r)), du(T(0)) {}  // NOLINT: constants of the laws
  __device__ Dual(T r, T d) : re(r), du(d) {}
  __device__ Dual &operator+=(const Dual &o) { re += o.re; du += o.du; return *this; }
  __device__ Dual &operator-=(const Dual &o) { re -= o.re; du -= o.du; return *this; }
  __device__ Dual &operator*=(const Dual &o) { du = du * o.re + re * o.du; re *= o.re; return *this; }
};
template <typename T>
__device__ __forceinline__ Dual<T> operator+(Dual<T> a, const Dual<T> &b) { return a += b; }
template <typename T>
__device__ __forceinline__ Dual<T> operator-(Dual<T> a, const Dual<T> &b) { return a -= b; }
template <typename T>
__device__ __forceinline__ Dual<T> operator-(const Dual<T> &a) { return Dual<T>(-a.re, -a.du); }
template <typename T>
__device__ __forceinline__ Dual<T> operator*(const Dual<T> &a, const Dual<T> &b) {
  return Dual<T>(a.re * b.re, a.du * b.re + a.re * b.du);
}
template <typename T>
__device__ __forceinline__ Dual<T> operator/(const Dual<T> &a, const Dual<T> &b) {
  const T inv = T(1) / b.re;
  return Dual<T>(a.re * inv, (a.du - a.re * inv * b.du) * inv);
}
template <>
__device__ __forceinline__ Dual<double> mlog1p<Dual<double>>(Dual<double> x) {
  return Dual<double>(log1p(x.re), x.du / (1.0 + x.re));
}
template <>
__device__ __forceinline__ Dual<float> mlog1p<Dual<float>>(Dual<float> x) {
  return Dual<float>(log1pf(x.re), x.du / (1.0f + x.re));
}
template <>
__device__ __forceinline__ Dual<double> mexp<Dual<double>>(Dual<double> x) {
  const double e = exp(x.re);
  return Dual<double>(e, e * x.du);
}
template <>
__device__ __forceinline__ Dual<float> mexp<Dual<float>>(Dual<float> x) {
  const float e = expf(x.re);
  return Dual<float>(e, e * x.du);
}

// One quadrature point: adds w * (grad N_a . dP) contributions for every node.
template <int MODEL, typename T, int NPE>
__device__ __forceinline__ void adjoint_point(const T (&g)[NPE][3], T w, const T (&H)[3][3], const T (&Hl)[3][3],
                                              const T (&Gu)[3][3], T p0, T p1, T p2, T (&ge)[NPE][3],
                                              T (&kl)[NPE][3], T (&ku)[NPE][3], T (&fa)[NPE][3], int *flags) {
  using D = Dual<T>;
  D Hd[3][3];
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int J = 0; J < 3; ++J) Hd[i][J] = D(H[i][J], Hl[i][J]);
  Kin<D> kin;
  kin.init(Hd);
  if (!(kin.J.re > T(0))) atomicOr(flags, FLAG_INVERTED);
  Law<MODEL, D> law;
  D P[3][3];
  law.init(kin, Hd, D(p0, T(0)), D(p1, T(0)), D(p2, T(0)), P);
  D dPu[3][3];
  T dPl[3][3];
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int J = 0; J < 3; ++J) {
      dPu[i][J] = D(T(0), T(0));
      dPl[i][J] = T(0);
    }
#pragma unroll 1
  for (int i = 0; i < 3; ++i)
#pragma unroll 1
    for (int k = 0; k < 3; ++k) {
      D C[3][3];
      law.block(i, k, C);
#pragma unroll
      for (int J = 0; J < 3; ++J)
#pragma unroll
        for (int L = 0; L < 3; ++L) {
          dPu[i][J] += C[J][L] * D(Gu[k][L], T(0));
          dPl[i][J] += C[J][L].re * Hl[k][L];
        }
    }
#pragma unroll
  for (int a = 0; a < NPE; ++a)
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      D su(T(0), T(0));
      T sl = T(0), sf = T(0);
#pragma unroll
      for (int J = 0; J < 3; ++J) {
        su += D(g[a][J], T(0)) * dPu[i][J];
        sl += g[a][J] * dPl[i][J];
        sf += g[a][J] * P[i][J].re;
      }
      ge[a][i] += w * (su.du + sl);
      kl[a][i] += w * sl;
      ku[a][i] += w * su.re;
      fa[a][i] += w * sf;
    }
}

// One thread per element (tets: 1 point; hexes: 8 Gauss points).
template <int MODEL, typename T, int NPE>
__global__ void __launch_bounds__(128) adjoint_element_kernel(
    int64_t E, int64_t e_begin, int64_t e_end, const int32_t *__restrict__ conn, const double *__restrict__ rest,
    const double *__restrict__ params, const double *__restrict__ X, const double *__restrict__ q,
    const double *__restrict__ lam, const double *__restrict__ acc, const double *__restrict__ v, double cK,
    double bh, double *__restrict__ ge_out, double *__restrict__ kl_out, double *__restrict__ sbar, int *flags) {
  const int64_t e = e_begin + int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (e >= e_end) return;
  int nd[NPE];
#pragma unroll
  for (int a = 0; a < NPE; ++a) nd[a] = conn[e * NPE + a];
  T du[NPE][3], dl[NPE][3], uu[NPE][3];
#pragma unroll
  for (int a = 0; a < NPE; ++a)
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      const int64_t dof = 3 * int64_t(nd[a]) + i;
      du[a][i] = T(q[dof] - X[dof]);
      dl[a][i] = T(lam[dof]);
      uu[a][i] = T(cK * acc[dof] + bh * v[dof]);
    }
  const T p0 = T(params[e]), p1 = T(params[E + e]), p2 = T(params[2 * E + e]);
  T ge[NPE][3], kl[NPE][3], ku[NPE][3], fa[NPE][3];
#pragma unroll
  for (int a = 0; a < NPE; ++a)
#pragma unroll
    for (int i = 0; i < 3; ++i) ge[a][i] = kl[a][i] = ku[a][i] = fa[a][i] = T(0);
  constexpr int NQ = NPE == 4 ? 1 : 8;
#pragma unroll 1
  for (int gp = 0; gp < NQ; ++gp) {
    T g[NPE][3];
    T w;
    if (NPE == 4) {
#pragma unroll
      for (int a = 1; a < 4; ++a)
#pragma unroll
        for (int J = 0; J < 3; ++J) g[a][J] = T(rest[(3 * (a - 1) + J) * E + e]);
#pragma unroll
      for (int J = 0; J < 3; ++J) g[0][J] = -(g[1][J] + g[2][J] + g[3][J]);
      w = T(rest[9 * E + e]);
    } else {
#pragma unroll
      for (int a = 0; a < NPE; ++a)
#pragma unroll
        for (int J = 0; J < 3; ++J) g[a][J] = T(rest[(gp * 25 + 3 * a + J) * E + e]);
      w = T(rest[(gp * 25 + 24) * E + e]);
    }
    T H[3][3], Hl[3][3], Gu[3][3];
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
      for (int J = 0; J < 3; ++J) {
        T a0 = T(0), a1 = T(0), a2 = T(0);
#pragma unroll
        for (int a = 0; a < NPE; ++a) {
          a0 += du[a][i] * g[a][J];
          a1 += dl[a][i] * g[a][J];
          a2 += uu[a][i] * g[a][J];
        }
        H[i][J] = a0;
        Hl[i][J] = a1;
        Gu[i][J] = a2;
      }
    adjoint_point<MODEL, T, NPE>(g, w, H, Hl, Gu, p0, p1, p2, ge, kl, ku, fa, flags);
  }
  double sb = 0.0;
#pragma unroll
  for (int a = 0; a < NPE; ++a)
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      ge_out[(e * NPE + a) * 3 + i] = double(ge[a][i]);
      kl_out[(e * NPE + a) * 3 + i] = double(kl[a][i]);
      sb += double(dl[a][i]) * (double(ku[a][i]) + double(fa[a][i]));
    }
  sbar[e] -= sb;
}

// Per node: gather ge, kl over the node's elements and M lambda over its
// blocks; update q_bar, v_bar (zero on fixed nodes); p_bar = lambda.
__global__ void adjoint_gather_kernel(int64_t n_nodes, const int32_t *__restrict__ node_ptr,
                                      const int32_t *__restrict__ node_src, const int32_t *__restrict__ bptr,
                                      const int32_t *__restrict__ bcol, const double *__restrict__ bmass,
                                      const int8_t *__restrict__ fixed_row, const double *__restrict__ ge,
                                      const double *__restrict__ kl, const double *__restrict__ lam, double h,
                                      double al, double bh, double *__restrict__ qbar, double *__restrict__ vbar,
                                      double *__restrict__ pbar) {
  const int64_t nd = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (nd >= n_nodes) return;
  const int64_t r0 = 3 * nd;
  if (fixed_row[r0]) {
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      qbar[r0 + i] = 0.0;
      vbar[r0 + i] = 0.0;
      if (pbar) pbar[r0 + i] = 0.0;
    }
    return;
  }
  double gq[3] = {0, 0, 0}, kv[3] = {0, 0, 0}, mv[3] = {0, 0, 0};
  for (int32_t j = node_ptr[nd]; j < node_ptr[nd + 1]; ++j) {
    const int64_t s = int64_t(node_src[j]) * 3;
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      gq[i] += ge[s + i];
      kv[i] += kl[s + i];
    }
  }
  for (int32_t k = bptr[nd]; k < bptr[nd + 1]; ++k) {
    const int64_t cn = 3 * int64_t(bcol[k]);
#pragma unroll
    for (int i = 0; i < 3; ++i) mv[i] += bmass[k] * lam[cn + i];
  }
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    const double qb = qbar[r0 + i];
    qbar[r0 + i] = qb - gq[i];
    vbar[r0 + i] = vbar[r0 + i] + h * qb - (al * mv[i] + bh * kv[i]);
    if (pbar) pbar[r0 + i] = lam[r0 + i];
  }
}

// a_bar = h v_bar + h^2 q_bar, zero on fixed DOFs.
__global__ void adjoint_rhs_kernel(int64_t n, double h, const int8_t *__restrict__ fixed_row,
                                   const double *__restrict__ qbar, const double *__restrict__ vbar,
                                   double *__restrict__ abar) {
  const int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i < n) abar[i] = fixed_row[i] ? 0.0 : h * vbar[i] + h * h * qbar[i];
}

template <int MODEL, typename T>
static void launch_adj_t(const fe_ctx *c, const DeviceState *d, const double *q, const double *lam,
                         const double *acc, const double *v, double *ge, double *kl, double *sbar,
                         cudaStream_t s) {
  const double h = c->h, cK = h * (c->beta + h), bh = c->beta + h;
  const int64_t E = c->n_elems;
  const int64_t eb = c->model_range[MODEL][0], ee = c->model_range[MODEL][1];
  if (ee <= eb) return;
  const unsigned g = unsigned((ee - eb + 127) / 128);
  if (c->elem_type == FE_TET4)
    adjoint_element_kernel<MODEL, T, 4><<<g, 128, 0, s>>>(E, eb, ee, d->conn, d->rest, d->params, d->X, q, lam, acc,
                                                          v, cK, bh, ge, kl, sbar, d->flags);
  else
    adjoint_element_kernel<MODEL, T, 8><<<g, 128, 0, s>>>(E, eb, ee, d->conn, d->rest, d->params, d->X, q, lam, acc,
                                                          v, cK, bh, ge, kl, sbar, d->flags);
}

void launch_adjoint_element(const fe_ctx *c, const DeviceState *d, bool fp32, const double *q, const double *lam,
                            const double *acc, const double *v, double *ge, double *kl, double *sbar,
                            cudaStream_t s) {
  for (int md = FE_SVK; md <= FE_MOONEY_RIVLIN; ++md) {
    if (c->model_range[md][1] <= c->model_range[md][0]) continue;
    d->launches++;
    if (md == FE_SVK)
      fp32 ? launch_adj_t<FE_SVK, float>(c, d, q, lam, acc, v, ge, kl, sbar, s)
           : launch_adj_t<FE_SVK, double>(c, d, q, lam, acc, v, ge, kl, sbar, s);
    else if (md == FE_NEOHOOKE)
      fp32 ? launch_adj_t<FE_NEOHOOKE, float>(c, d, q, lam, acc, v, ge, kl, sbar, s)
           : launch_adj_t<FE_NEOHOOKE, double>(c, d, q, lam, acc, v, ge, kl, sbar, s);
    else
      fp32 ? launch_adj_t<FE_MOONEY_RIVLIN, float>(c, d, q, lam, acc, v, ge, kl, sbar, s)
           : launch_adj_t<FE_MOONEY_RIVLIN, double>(c, d, q, lam, acc, v, ge, kl, sbar, s);
  }
}

void launch_adjoint_gather(const fe_ctx *c, const DeviceState *d, const double *ge, const double *kl,
                           const double *lam, double *qbar, double *vbar, double *pbar, cudaStream_t s) {
  d->launches++;
  const int64_t nn = c->n_nodes;
  adjoint_gather_kernel<<<unsigned((nn + 127) / 128), 128, 0, s>>>(
      nn, d->node_ptr, d->node_src, d->bptr, d->bcol, d->bmass, d->fixed_row, ge, kl, lam, c->h, c->alpha,
      c->beta + c->h, qbar, vbar, pbar);
}

void launch_adjoint_rhs(const fe_ctx *c, const DeviceState *d, const double *qbar, const double *vbar,
                        double *abar, cudaStream_t s) {
  d->launches++;
  adjoint_rhs_kernel<<<unsigned((c->n + 255) / 256), 256, 0, s>>>(c->n, c->h, d->fixed_row, qbar, vbar, abar);
}

}  // namespace fe
