// Hot-path kernels of one implicit step: element force/tangent (Section 3.1),
// gather assembly of A and b through the inverse of the map C (Section 4.2,
// Eq. "dynamic equation2"), CSR SpMV and the fused CG vector operations
// (Section 6.2, Fig. "DataTransfer"), backward-Euler integration
// (Eq. "implicit integration").  Every reduction is deterministic: per-block
// partials in a fixed order, summed in a fixed order by the last block.
#include <cuda_runtime.h>

#include <algorithm>
#include <string>
#include <type_traits>

#include "fe_device.cuh"
#include "fe_df.cuh"
#include "fe_material.cuh"

namespace fe {

// ------------------------------------------------------------- reductions

template <int BLOCK>
__device__ __forceinline__ double block_sum(double v, double *sh) {
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
  return v;  // valid in thread 0
}

// Grid-wide deterministic sum; returns true in the last block to finish, whose
// thread 0 then holds the total in *out.
template <int BLOCK>
__device__ __forceinline__ bool grid_sum(double v, double *partials, unsigned int *ticket,
                                         double *out) {
  __shared__ double sh[BLOCK / 32];
  __shared__ bool last;
  double s = block_sum<BLOCK>(v, sh);
  if (threadIdx.x == 0) {
    partials[blockIdx.x] = s;
    __threadfence();
    unsigned int t = atomicAdd(ticket, 1u);
    last = (t == gridDim.x - 1);
  }
  __syncthreads();
  if (!last) return false;
  __threadfence();
  double acc = 0.0;
  for (int i = threadIdx.x; i < (int)gridDim.x; i += BLOCK) acc += ((volatile double *)partials)[i];
  double tot = block_sum<BLOCK>(acc, sh);
  if (threadIdx.x == 0) {
    *out = tot;
    *ticket = 0u;
  }
  return true;
}

__device__ __forceinline__ bool solve_done(const double *scal) { return scal[S_DONE] != 0.0; }

// ---------------------------------------------------------- element kernels

// An element kernel's inputs in its force type TF.  FP64: read from the
// stored doubles.  Double-float (the mixed path with FP32 tangents): read
// from float-pair copies (rest data and parameters made once, the
// displacement q - X per launch by disp_pairs_kernel), so the force path
// issues no FP64 conversion; f_e is stored as float pairs.
template <typename TF>
struct ElemSrc {
  const double *rest, *params, *X, *q;
  using fout = double;
  __device__ __forceinline__ TF rest_at(int64_t i) const { return TF(__ldg(rest + i)); }
  __device__ __forceinline__ TF param_at(int64_t i) const { return TF(__ldg(params + i)); }
  __device__ __forceinline__ TF disp(int64_t dof) const { return TF(__ldg(q + dof) - __ldg(X + dof)); }
  __device__ __forceinline__ static double out(TF v) { return double(v); }
};
template <>
struct ElemSrc<dfloat> {
  const float2 *rest, *params, *u;
  using fout = float2;
  __device__ __forceinline__ dfloat rest_at(int64_t i) const { return dfloat(__ldg(rest + i)); }
  __device__ __forceinline__ dfloat param_at(int64_t i) const { return dfloat(__ldg(params + i)); }
  __device__ __forceinline__ dfloat disp(int64_t dof) const { return dfloat(__ldg(u + dof)); }
  __device__ __forceinline__ static float2 out(dfloat v) { return v.pair(); }
};

// u = q - X as float pairs (the double-float force's displacement)
__global__ void disp_pairs_kernel(int64_t n, const double *__restrict__ q, const double *__restrict__ X,
                                  float2 *__restrict__ u) {
  for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x)
    u[i] = df_split(q[i] - X[i]);
}

// The tangent part of a tet: 144 entries of K_e = V grad N^T CC grad N in
// fill order ((a*4 + b)*9 + 3i + k), into one shared-memory row.
template <typename T, typename L>
__device__ __forceinline__ void tet_tangent(const L &law, const T g[4][3], T V, T *row) {
#pragma unroll 1
  for (int i = 0; i < 3; ++i) {
#pragma unroll 1
    for (int k = i; k < 3; ++k) {
      T C[3][3];
      law.block(i, k, C);
      T hb[4][3];
#pragma unroll
      for (int b = 0; b < 4; ++b)
#pragma unroll
        for (int J = 0; J < 3; ++J) hb[b][J] = C[J][0] * g[b][0] + C[J][1] * g[b][1] + C[J][2] * g[b][2];
#pragma unroll
      for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) {
          const T val = V * (g[a][0] * hb[b][0] + g[a][1] * hb[b][1] + g[a][2] * hb[b][2]);
          row[(a * 4 + b) * 9 + 3 * i + k] = val;
          if (i != k) row[(b * 4 + a) * 9 + 3 * k + i] = val;  // major symmetry of CC
        }
    }
  }
}

// One thread per tet.  Rest data SoA [10][E]: rows of Dm^{-1} (= grad N_1..3),
// volume.  Outputs f_e [E][4][3] (force type TF: FP64, or float pairs) and
// K_e [E][144] (tangent type T) in fill order, K_e staged through shared
// memory for coalesced stores.  With TF = dfloat and T = float (the mixed
// path) the kinematics, stress and force are evaluated in double-float
// (about 2^-46 per operation, on the FP32 pipe: GB300's FP64 pipe bound the
// FP64 version) and the tangent in FP32 from the same displacement gradient.
template <int MODEL, typename T, typename TF, int BLOCK>
__global__ void __launch_bounds__(BLOCK) tet_kernel(int64_t E, int64_t e_begin, int64_t e_end,
                                                    const int32_t *__restrict__ conn, ElemSrc<TF> src,
                                                    typename ElemSrc<TF>::fout *__restrict__ f_out,
                                                    T *__restrict__ K_out, int *flags) {
  extern __shared__ unsigned char smem_raw[];
  T *sk = reinterpret_cast<T *>(smem_raw);
  constexpr int LD = 145;
  const int64_t e0 = e_begin + int64_t(blockIdx.x) * BLOCK;
  const int64_t e = e0 + threadIdx.x;
  if (e < e_end) {
    const int4 cn = reinterpret_cast<const int4 *>(conn)[e];
    const int nd[4] = {cn.x, cn.y, cn.z, cn.w};
    TF g[4][3];
#pragma unroll
    for (int a = 1; a < 4; ++a)
#pragma unroll
      for (int J = 0; J < 3; ++J) g[a][J] = src.rest_at((3 * (a - 1) + J) * E + e);
#pragma unroll
    for (int J = 0; J < 3; ++J) g[0][J] = -(g[1][J] + g[2][J] + g[3][J]);
    const TF V = src.rest_at(9 * E + e);
    const TF p0 = src.param_at(e), p1 = src.param_at(E + e), p2 = src.param_at(2 * E + e);
    TF H[3][3];
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
      for (int J = 0; J < 3; ++J) H[i][J] = TF(0);
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
      for (int i = 0; i < 3; ++i) {
        // displacement in FP64 (or its float pair), then the working type
        const TF u = src.disp(3 * nd[a] + i);
#pragma unroll
        for (int J = 0; J < 3; ++J) H[i][J] += u * g[a][J];
      }
    T *row = sk + threadIdx.x * LD;
    {
      Kin<TF> kin;
      kin.init(H);
      if (!(kin.J > TF(0))) atomicOr(flags, FLAG_INVERTED);
      Law<MODEL, TF> law;
      if constexpr (MODEL == FE_COROTATIONAL) law.set_frame(H);
      TF P[3][3];
      law.init(kin, H, p0, p1, p2, P);
#pragma unroll
      for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int i = 0; i < 3; ++i) {
          TF s = TF(0);
#pragma unroll
          for (int J = 0; J < 3; ++J) s += P[i][J] * g[a][J];
          f_out[e * 12 + 3 * a + i] = ElemSrc<TF>::out(V * s);
        }
      if constexpr (sizeof(T) == sizeof(TF)) tet_tangent<T>(law, g, V, row);
    }
    if constexpr (sizeof(T) != sizeof(TF)) {
      // the tangent in its own (narrower) type from the same H
      T gt[4][3], Ht[3][3], Pt[3][3];
#pragma unroll
      for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int J = 0; J < 3; ++J) gt[a][J] = T(g[a][J]);
#pragma unroll
      for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int J = 0; J < 3; ++J) Ht[i][J] = T(H[i][J]);
      Kin<T> kt;
      kt.init(Ht);
      Law<MODEL, T> lt;
      if constexpr (MODEL == FE_COROTATIONAL) lt.set_frame(Ht);
      lt.init(kt, Ht, T(p0), T(p1), T(p2), Pt);
      tet_tangent<T>(lt, gt, T(V), row);
    }
  }
  __syncthreads();
  const int64_t nvalid = (e_end - e0) < BLOCK ? (e_end - e0) : BLOCK;
  T *dst = K_out + e0 * 144;
  for (int64_t idx = threadIdx.x; idx < nvalid * 144; idx += BLOCK)
    dst[idx] = sk[(idx / 144) * LD + idx % 144];
}

// One thread per (hex, local node a); 8 Gauss points.  Rest data SoA
// [8 * 25][E]: per Gauss point grad N (8 x 3) and w det J0.  Thread a owns
// the block row a of K_e (72 values, tangent type T) and f_a (force type TF;
// with TF = dfloat and T = float the stress and force are evaluated in
// double-float and the tangent in FP32 from the same displacement gradient).
template <int MODEL, typename T, typename TF, int BLOCK>
__global__ void __launch_bounds__(BLOCK) hex_kernel(int64_t E, int64_t e_begin, int64_t e_end,
                                                    const int32_t *__restrict__ conn, ElemSrc<TF> src,
                                                    typename ElemSrc<TF>::fout *__restrict__ f_out,
                                                    T *__restrict__ K_out, int *flags) {
  extern __shared__ unsigned char smem_raw[];
  T *sk = reinterpret_cast<T *>(smem_raw);
  constexpr int EPB = BLOCK / 8;  // elements per block
  constexpr int LD = 577;
  constexpr bool SPLIT = sizeof(T) != sizeof(TF);
  const int64_t e0 = e_begin + int64_t(blockIdx.x) * EPB;
  const int el = threadIdx.x >> 3, a = threadIdx.x & 7;
  const int64_t e = e0 + el;
  if (e < e_end) {
    TF u[8][3];
#pragma unroll
    for (int b = 0; b < 8; ++b) {
      const int nb = __ldg(conn + e * 8 + b);
#pragma unroll
      for (int i = 0; i < 3; ++i) u[b][i] = src.disp(3 * nb + i);
    }
    const TF p0 = src.param_at(e), p1 = src.param_at(E + e), p2 = src.param_at(2 * E + e);
    Law<MODEL, TF> law;
    Law<MODEL, T> lt;
    if constexpr (MODEL == FE_COROTATIONAL) {
      // the element frame from the volume-averaged displacement gradient
      TF Hb[3][3], vol = TF(0);
#pragma unroll
      for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int J = 0; J < 3; ++J) Hb[i][J] = TF(0);
#pragma unroll 1
      for (int gp = 0; gp < 8; ++gp) {
        const TF w = src.rest_at((gp * 25 + 24) * E + e);
        vol += w;
#pragma unroll
        for (int b = 0; b < 8; ++b) {
          TF gb[3];
#pragma unroll
          for (int J = 0; J < 3; ++J) gb[J] = w * src.rest_at((gp * 25 + 3 * b + J) * E + e);
#pragma unroll
          for (int i = 0; i < 3; ++i)
#pragma unroll
            for (int J = 0; J < 3; ++J) Hb[i][J] += u[b][i] * gb[J];
        }
      }
#pragma unroll
      for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int J = 0; J < 3; ++J) Hb[i][J] /= vol;
      law.set_frame(Hb);
      if constexpr (SPLIT) {
        T Hbt[3][3];
#pragma unroll
        for (int i = 0; i < 3; ++i)
#pragma unroll
          for (int J = 0; J < 3; ++J) Hbt[i][J] = T(Hb[i][J]);
        lt.set_frame(Hbt);
      }
    }
    T acc[8][9];
#pragma unroll
    for (int b = 0; b < 8; ++b)
#pragma unroll
      for (int c = 0; c < 9; ++c) acc[b][c] = T(0);
    TF fa[3] = {TF(0), TF(0), TF(0)};
#pragma unroll 1
    for (int gp = 0; gp < 8; ++gp) {
      TF g[8][3];
#pragma unroll
      for (int b = 0; b < 8; ++b)
#pragma unroll
        for (int J = 0; J < 3; ++J) g[b][J] = src.rest_at((gp * 25 + 3 * b + J) * E + e);
      const TF w = src.rest_at((gp * 25 + 24) * E + e);
      TF H[3][3];
#pragma unroll
      for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int J = 0; J < 3; ++J) {
          TF s = TF(0);
#pragma unroll
          for (int b = 0; b < 8; ++b) s += u[b][i] * g[b][J];
          H[i][J] = s;
        }
      Kin<TF> kin;
      kin.init(H);
      if (!(kin.J > TF(0)) && a == 0) atomicOr(flags, FLAG_INVERTED);
      TF P[3][3];
      law.init(kin, H, p0, p1, p2, P);
#pragma unroll
      for (int i = 0; i < 3; ++i) fa[i] += w * (P[i][0] * g[a][0] + P[i][1] * g[a][1] + P[i][2] * g[a][2]);
      // the tangent in type T: the same law object, or one in T from the same H
      T gt[8][3];
#pragma unroll
      for (int b = 0; b < 8; ++b)
#pragma unroll
        for (int J = 0; J < 3; ++J) gt[b][J] = T(g[b][J]);
      const T wt = T(w);
      if constexpr (SPLIT) {
        T Ht[3][3], Pt[3][3];
#pragma unroll
        for (int i = 0; i < 3; ++i)
#pragma unroll
          for (int J = 0; J < 3; ++J) Ht[i][J] = T(H[i][J]);
        Kin<T> kt;
        kt.init(Ht);
        lt.init(kt, Ht, T(p0), T(p1), T(p2), Pt);
      }
      const auto &lk = [&]() -> const Law<MODEL, T> & {
        if constexpr (SPLIT) return lt; else return law;
      }();
#pragma unroll 1
      for (int i = 0; i < 3; ++i)
#pragma unroll 1
        for (int k = 0; k < 3; ++k) {
          T C[3][3];
          lk.block(i, k, C);
          T vL[3];
#pragma unroll
          for (int L = 0; L < 3; ++L) vL[L] = wt * (gt[a][0] * C[0][L] + gt[a][1] * C[1][L] + gt[a][2] * C[2][L]);
#pragma unroll
          for (int b = 0; b < 8; ++b) acc[b][3 * i + k] += vL[0] * gt[b][0] + vL[1] * gt[b][1] + vL[2] * gt[b][2];
        }
    }
#pragma unroll
    for (int i = 0; i < 3; ++i) f_out[e * 24 + 3 * a + i] = ElemSrc<TF>::out(fa[i]);
    T *row = sk + el * LD + a * 72;
#pragma unroll
    for (int b = 0; b < 8; ++b)
#pragma unroll
      for (int c = 0; c < 9; ++c) row[b * 9 + c] = acc[b][c];
  }
  __syncthreads();
  const int64_t nvalid = (e_end - e0) < EPB ? (e_end - e0) : EPB;
  T *dst = K_out + e0 * 576;
  for (int64_t idx = threadIdx.x; idx < nvalid * 576; idx += BLOCK)
    dst[idx] = sk[(idx / 576) * LD + idx % 576];
}

// T = float (FP32 tangents): the force in double-float from the float-pair
// inputs; T = double: FP64 throughout.
template <int MODEL, typename T>
static void launch_element_t(const fe_ctx *c, const DeviceState *d, const double *q, cudaStream_t s) {
  using TF = std::conditional_t<sizeof(T) == 4, dfloat, double>;
  const int64_t E = c->n_elems;
  const int64_t eb = c->model_range[MODEL][0], ee = c->model_range[MODEL][1];
  if (ee <= eb) return;
  const int64_t EN = ee - eb;
  ElemSrc<TF> src;
  if constexpr (sizeof(T) == 4)
    src = ElemSrc<TF>{d->rest2, d->params2, d->u2};
  else
    src = ElemSrc<TF>{d->rest, d->params, d->X, q};
  auto *fo = reinterpret_cast<typename ElemSrc<TF>::fout *>(d->fe);
  T *Ko = reinterpret_cast<T *>(d->Ke);
  if (c->elem_type == FE_TET4) {
    constexpr int B = sizeof(T) == 8 ? 64 : 128;
    const size_t sm = size_t(B) * 145 * sizeof(T);
    cudaFuncSetAttribute(tet_kernel<MODEL, T, TF, B>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(sm));
    tet_kernel<MODEL, T, TF, B><<<unsigned((EN + B - 1) / B), B, sm, s>>>(E, eb, ee, d->conn, src, fo, Ko, d->flags);
  } else {
    constexpr int B = 128, EPB = B / 8;
    const size_t sm = size_t(EPB) * 577 * sizeof(T);
    cudaFuncSetAttribute(hex_kernel<MODEL, T, TF, B>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(sm));
    hex_kernel<MODEL, T, TF, B><<<unsigned((EN + EPB - 1) / EPB), B, sm, s>>>(E, eb, ee, d->conn, src, fo, Ko,
                                                                             d->flags);
  }
}

// Element forces in FP64, or in double-float (float pairs) with the FP32
// tangents of the mixed path (unless element_fp64, which keeps both in FP64).
void launch_element(const fe_ctx *c, const DeviceState *d, const double *q, bool fp32, cudaStream_t s) {
  const bool k32 = fp32 && !c->opt.element_fp64;
  if (k32) {  // the displacement as float pairs, once for every law's launch
    d->launches++;
    disp_pairs_kernel<<<unsigned(std::max<int64_t>(1, std::min<int64_t>((c->n + 255) / 256, 152 * 16))), 256, 0, s>>>(
        c->n, q, d->X, d->u2);
  }
  // one launch per material model present (a batch groups its members by model)
  for (int md = FE_SVK; md <= FE_COROTATIONAL; ++md) {
    if (c->model_range[md][1] <= c->model_range[md][0]) continue;
    d->launches++;
    if (md == FE_SVK)
      k32 ? launch_element_t<FE_SVK, float>(c, d, q, s) : launch_element_t<FE_SVK, double>(c, d, q, s);
    else if (md == FE_NEOHOOKE)
      k32 ? launch_element_t<FE_NEOHOOKE, float>(c, d, q, s) : launch_element_t<FE_NEOHOOKE, double>(c, d, q, s);
    else if (md == FE_MOONEY_RIVLIN)
      k32 ? launch_element_t<FE_MOONEY_RIVLIN, float>(c, d, q, s)
          : launch_element_t<FE_MOONEY_RIVLIN, double>(c, d, q, s);
    else
      k32 ? launch_element_t<FE_COROTATIONAL, float>(c, d, q, s)
          : launch_element_t<FE_COROTATIONAL, double>(c, d, q, s);
  }
}

// ------------------------------------------------------ gather assembly
// One warp per node over its 3x3 node blocks (lanes = blocks).  A block sums
// its element blocks' 9 contiguous values in ascending order (the order of
// the inverse of C, so every slot equals the per-slot sum), writes its 9
// slots (rows 3n+i, position 3*bp + k in the row) and its share of
// (alpha M + (beta+h) K) v; the node's element forces (FP64) come from its
// incidence list.  Fixed nodes keep the lone unit diagonal and b = 0.
//
// FP64 path: every sum in FP64.  Mixed path (FP32 tangents): GB300's FP64
// pipe issues at a small fraction of the FP32 rate, so the kernel keeps FP64
// work out of the per-block code: the block sums are double-float pairs
// (hi + lo, Knuth's TwoSum: the exact sum of the FP32 values to about
// 2^-46), A = cM M + cK K is formed in double-float (Dekker's product through
// FMA for cK K and cM M, the block mass read as a float pair), and A is
// written rounded to FP32 (the inner solve and the factor) and as the pair
// itself (A2, the FP64-accurate copy the refinement residual reads in
// double-float).  The damping part of b is summed in FP32 per lane (its
// terms carry the FP32 tangent's rounding already); with the element forces
// (double-float pairs in this path) the lanes' sums are reduced across the
// warp in double-float, the three rows in one transposed reduction
// (warp_sum3) instead of three.
__device__ __forceinline__ void two_sum_acc(float &hi, float &lo, float x) {
  const float s = hi + x;
  const float bb = s - hi;
  lo += (hi - (s - bb)) + (x - bb);
  hi = s;
}

// Warp sum of three values at once: after exchanging halves (lane ^ 16:
// lanes below 16 keep v0, v1, the others v2 and a zero) and quarters (lane ^
// 8), each lane sums one value over its group of eight.  Lane l ends with the
// total of v[(l >> 3) & 3] (v[3] = 0): lanes 0, 8 and 16 hold v0, v1, v2.
// Six additions instead of fifteen; a fixed order, so deterministic.
template <typename T>
__device__ __forceinline__ T shfl_xor_any(T v, int o) { return __shfl_xor_sync(0xffffffffu, v, o); }
template <>
__device__ __forceinline__ dfloat shfl_xor_any<dfloat>(dfloat v, int o) {
  return dfloat(__shfl_xor_sync(0xffffffffu, v.hi, o), __shfl_xor_sync(0xffffffffu, v.lo, o));
}

template <typename T>
__device__ __forceinline__ T warp_sum3(T v0, T v1, T v2) {
  const int lane = threadIdx.x & 31;
  const bool up = (lane & 16) != 0;
  T k0 = up ? v2 : v0, k1 = up ? T(0) : v1;
  const T s0 = up ? v0 : v2, s1 = up ? v1 : T(0);
  k0 += shfl_xor_any(s0, 16);
  k1 += shfl_xor_any(s1, 16);
  const bool hi8 = (lane & 8) != 0;
  T k = hi8 ? k1 : k0;
  k += shfl_xor_any(hi8 ? k0 : k1, 8);
#pragma unroll
  for (int o = 4; o > 0; o >>= 1) k += shfl_xor_any(k, o);
  return k;
}

template <typename TK, typename TA>
__global__ void __launch_bounds__(256) assemble_block_kernel(
    int64_t n_nodes, const int32_t *__restrict__ rowptr, const int32_t *__restrict__ bptr,
    const int32_t *__restrict__ bcol, const int32_t *__restrict__ bsrc_ptr, const int32_t *__restrict__ bsrc,
    const double *__restrict__ bmass, const float2 *__restrict__ bmass2, const TK *__restrict__ Ke,
    const void *__restrict__ fe, const int32_t *__restrict__ node_ptr, const int32_t *__restrict__ node_src,
    const int8_t *__restrict__ fixed_row, const double *__restrict__ v, const double *__restrict__ w,
    const double *__restrict__ p, double cM, double cK, double al, double bh, TA *__restrict__ A,
    float2 *__restrict__ A2, double *__restrict__ b) {
  constexpr bool DF = sizeof(TK) == 4;  // FP32 tangents: double-float sums
  const int lane = threadIdx.x & 31;
  const int64_t warps = int64_t(gridDim.x) * (blockDim.x >> 5);
  // cK and cM as float pairs (c = ch + cl to 2^-48)
  const float ckh = float(cK), ckl = float(cK - double(ckh));
  const float cmh = float(cM), cml = float(cM - double(cmh));
  const float alf = float(al), bhf = float(bh);
  for (int64_t nd = int64_t(blockIdx.x) * (blockDim.x >> 5) + (threadIdx.x >> 5); nd < n_nodes; nd += warps) {
    const int64_t r0 = 3 * nd;
    if (fixed_row[r0]) {
      if (lane < 3) {
        A[rowptr[r0 + lane]] = TA(1);
        if (A2) A2[rowptr[r0 + lane]] = make_float2(1.f, 0.f);
        b[r0 + lane] = 0.0;
      }
      continue;
    }
    const int32_t rps[3] = {rowptr[r0], rowptr[r0 + 1], rowptr[r0 + 2]};
    double acc[3] = {0.0, 0.0, 0.0};
    float accf[3] = {0.f, 0.f, 0.f};
    for (int32_t k = bptr[nd] + lane; k < bptr[nd + 1]; k += 32) {
      const int32_t j1 = bsrc_ptr[k + 1];
      const int32_t bp = 3 * (k - bptr[nd]);
      const int64_t cn = 3 * int64_t(bcol[k]);
      if constexpr (DF) {
        float hi[9], lo[9];
#pragma unroll
        for (int q = 0; q < 9; ++q) hi[q] = lo[q] = 0.f;
        for (int32_t j = bsrc_ptr[k]; j < j1; ++j) {
          const TK *src = Ke + int64_t(bsrc[j]) * 9;
#pragma unroll
          for (int q = 0; q < 9; ++q) two_sum_acc(hi[q], lo[q], float(src[q]));
        }
        // cM mb in double-float: (cmh + cml)(mb.x + mb.y), the cml mb.y term
        // (~2^-48 of the product) dropped
        const float2 mb = bmass2[k];
        const float mh = mb.x * cmh;
        const float ml = fmaf(mb.x, cmh, -mh) + fmaf(mb.y, cmh, mb.x * cml);
        const float alm = alf * mb.x;
        const float vv[3] = {float(v[cn]), float(v[cn + 1]), float(v[cn + 2])};
#pragma unroll
        for (int i = 0; i < 3; ++i) {
#pragma unroll
          for (int kk = 0; kk < 3; ++kk) {
            const int q = 3 * i + kk;
            // cK (hi + lo) in double-float, then + cM mb on the diagonal
            float ph = ckh * hi[q];
            float pl = fmaf(ckh, hi[q], -ph) + (ckh * lo[q] + ckl * hi[q]);
            if (i == kk) {
              const float s = ph + mh, bb = s - ph;
              pl += ((ph - (s - bb)) + (mh - bb)) + ml;
              ph = s;
            }
            const float sh = ph + pl;  // renormalise: sh = fl(ph + pl)
            const float sl = pl - (sh - ph);
            A[rps[i] + bp + kk] = TA(sh);
            A2[rps[i] + bp + kk] = make_float2(sh, sl);
            accf[i] += ((i == kk ? alm : 0.f) + bhf * hi[q]) * vv[kk];
          }
          if (w) acc[i] += bmass[k] * w[cn + i];  // the M w term of a Newton correction
        }
      } else {
        const double mb = bmass[k];
        double blk[9];
#pragma unroll
        for (int q = 0; q < 9; ++q) blk[q] = 0.0;
        for (int32_t j = bsrc_ptr[k]; j < j1; ++j) {
          const TK *src = Ke + int64_t(bsrc[j]) * 9;
#pragma unroll
          for (int q = 0; q < 9; ++q) blk[q] += double(src[q]);
        }
        const double vv[3] = {v[cn], v[cn + 1], v[cn + 2]};
#pragma unroll
        for (int i = 0; i < 3; ++i) {
#pragma unroll
          for (int kk = 0; kk < 3; ++kk) {
            const double Ms = (i == kk) ? mb : 0.0;
            const double Ks = blk[3 * i + kk];
            const double a = cM * Ms + cK * Ks;
            A[rps[i] + bp + kk] = TA(a);
            if (A2) A2[rps[i] + bp + kk] = df_split(a);
            acc[i] += (al * Ms + bh * Ks) * vv[kk];
          }
          if (w) acc[i] += mb * w[cn + i];  // the M w term of a Newton correction
        }
      }
    }
    double tot;
    if constexpr (DF) {
      // the element forces as float pairs, summed in double-float with each
      // lane's FP32 damping part; the M w term (Newton corrections) in FP64
      dfloat fs[3] = {dfloat(accf[0], 0.f), dfloat(accf[1], 0.f), dfloat(accf[2], 0.f)};
      const float2 *fe2 = static_cast<const float2 *>(fe);
      for (int32_t j = node_ptr[nd] + lane; j < node_ptr[nd + 1]; j += 32) {
        const float2 *f = fe2 + int64_t(node_src[j]) * 3;
        fs[0] += dfloat(f[0]);
        fs[1] += dfloat(f[1]);
        fs[2] += dfloat(f[2]);
      }
      tot = double(warp_sum3<dfloat>(fs[0], fs[1], fs[2]));
      if (w) tot += warp_sum3<double>(acc[0], acc[1], acc[2]);
    } else {
      double fs[3] = {acc[0], acc[1], acc[2]};
      const double *fe64 = static_cast<const double *>(fe);
      for (int32_t j = node_ptr[nd] + lane; j < node_ptr[nd + 1]; j += 32) {
        const double *f = fe64 + int64_t(node_src[j]) * 3;
        fs[0] += f[0];
        fs[1] += f[1];
        fs[2] += f[2];
      }
      tot = warp_sum3<double>(fs[0], fs[1], fs[2]);
    }
    if ((lane & 7) == 0 && lane < 24) {
      const int i = lane >> 3;
      b[r0 + i] = (p ? p[r0 + i] : 0.0) - tot;
    }
  }
}

void launch_assemble(const fe_ctx *c, const DeviceState *d, bool fp32, const double *pext, const double *v,
                     const double *w, double bh, cudaStream_t s) {
  d->launches++;
  const double h = c->h, al = c->alpha, be = c->beta;
  const double cM = 1.0 + h * al, cK = h * (be + h);
  const int64_t nn = c->n_nodes;
  const unsigned grid = unsigned(std::min<int64_t>((nn + 7) / 8, 152 * 64));
  if (fp32 && !c->opt.element_fp64)
    assemble_block_kernel<float, float><<<grid, 256, 0, s>>>(
        nn, d->rowptr, d->bptr, d->bcol, d->bsrc_ptr, d->bsrc, d->bmass, d->bmass2, (const float *)d->Ke, d->fe,
        d->node_ptr, d->node_src, d->fixed_row, v, w, pext, cM, cK, al, bh, (float *)d->A, d->A2, d->b);
  else if (fp32)
    assemble_block_kernel<double, float><<<grid, 256, 0, s>>>(
        nn, d->rowptr, d->bptr, d->bcol, d->bsrc_ptr, d->bsrc, d->bmass, d->bmass2, (const double *)d->Ke, d->fe,
        d->node_ptr, d->node_src, d->fixed_row, v, w, pext, cM, cK, al, bh, (float *)d->A, d->A2, d->b);
  else
    assemble_block_kernel<double, double><<<grid, 256, 0, s>>>(
        nn, d->rowptr, d->bptr, d->bcol, d->bsrc_ptr, d->bsrc, d->bmass, nullptr, (const double *)d->Ke, d->fe,
        d->node_ptr, d->node_src, d->fixed_row, v, w, pext, cM, cK, al, bh, (double *)d->A, nullptr, d->b);
}

// ------------------------------------------------------------------ SpMV
constexpr int kRedBlock = 256;

// four blocks per SM: the grid-wide sum's tail (the last block adding the
// partials) stays short; at 350k DOF this measured 0.8 % more steps/s than
// eight per SM, and two per SM 0.8 % fewer
static unsigned red_grid(int64_t n) {
  int64_t g = (n + kRedBlock - 1) / kRedBlock;
  return unsigned(std::max<int64_t>(1, std::min<int64_t>(g, 152 * 4)));
}
// the sparse products keep eight blocks per SM: their rows wait on dependent
// loads (row pointer, column, x), so more of them in flight pays (47 against
// 57 us per product at 350k DOF with four)
static unsigned spmv_grid(int64_t n) {
  int64_t g = (n + kRedBlock - 1) / kRedBlock;
  return unsigned(std::max<int64_t>(1, std::min<int64_t>(g, 152 * 8)));
}

// y = A x (TPR threads per row) fused with x.y; the last block sets
// alpha = rz / (x.y) and flags a breakdown when x.y <= 0.
template <typename TA, typename TV, int TPR>
__global__ void __launch_bounds__(kRedBlock) spmv_dot_kernel(
    int64_t n, const int32_t *__restrict__ rowptr, const int32_t *__restrict__ colind,
    const TA *__restrict__ A, const TV *__restrict__ x, TV *__restrict__ y, double *scal,
    double *partials, unsigned int *ticket, int *flags) {
  if (solve_done(scal)) return;
  const int sub = threadIdx.x % TPR;
  const int64_t groups = int64_t(gridDim.x) * (kRedBlock / TPR);
  // the loop bound is warp-uniform so every lane reaches every shuffle
  const int64_t warp_row0 = int64_t(blockIdx.x) * (kRedBlock / TPR) + (threadIdx.x / 32) * (32 / TPR);
  DotAcc<TV> dot;
  for (int64_t r0 = warp_row0; r0 < n; r0 += groups) {
    const int64_t row = r0 + (threadIdx.x % 32) / TPR;
    TV acc = TV(0);
    if (row < n) {
      const int32_t k1 = rowptr[row + 1];
      for (int32_t k = rowptr[row] + sub; k < k1; k += TPR) acc += TV(A[k]) * x[colind[k]];
    }
#pragma unroll
    for (int o = TPR / 2; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o, TPR);
    if (sub == 0 && row < n) {
      y[row] = acc;
      dot.add(x[row], acc);
    }
  }
  double tot;
  if (grid_sum<kRedBlock>(dot.value(), partials, ticket, &tot) && threadIdx.x == 0) {
    scal[S_PQ] = tot;
    if (!(tot > 0.0)) {
      atomicOr(flags, FLAG_BREAKDOWN);
      scal[S_DONE] = 1.0;
      scal[S_ALPHA] = 0.0;
    } else {
      scal[S_ALPHA] = scal[S_RZ] / tot;
    }
  }
}

// Node-block SpMV.  Every free node's three rows share one column structure
// (3x3 blocks: columns 3 bcol[k] + kk, the values of row i at rowptr[3 nd + i]
// + 3 (k - bptr[nd]) + kk, the order the gather assembly writes), so a
// block's column index is read once for its 9 values instead of once per
// value.  LPN lanes per node, each lane one block at a time (its three x
// entries loaded once for the three rows), the three row sums reduced across
// the node's lanes; fixed nodes keep their lone diagonal entry.
// MODE 0: y = A x fused with x.y (then alpha = S_RZ / x.y, breakdown when
// x.y <= 0), in the vector type; MODE 1: r = b - A x and ||r||^2 -> S_ORR,
// S_ODONE, in FP64 (the refinement residual on the FP64 copy of A).
template <typename TA, typename TV, int LPN, int MODE>
__global__ void __launch_bounds__(kRedBlock) bspmv_kernel(
    int64_t n_nodes, const int32_t *__restrict__ rowptr, const int32_t *__restrict__ bptr,
    const int32_t *__restrict__ bcol, const int8_t *__restrict__ fixed_row, const TA *__restrict__ A,
    const TV *__restrict__ x, TV *__restrict__ y, const double *__restrict__ b, double *scal, double *partials,
    unsigned int *ticket, int *flags) {
  if (MODE == 0 && solve_done(scal)) return;
  constexpr int GPW = 32 / LPN;  // nodes per warp
  const int sub = threadIdx.x % LPN;
  const int64_t groups = int64_t(gridDim.x) * (kRedBlock / LPN);
  // the loop bound is warp-uniform so every lane reaches every shuffle
  const int64_t warp_node0 = int64_t(blockIdx.x) * (kRedBlock / LPN) + (threadIdx.x / 32) * GPW;
  DotAcc<TV> red;  // MODE 0: x.y; MODE 1: ||r||^2 (FP64)
  for (int64_t n0 = warp_node0; n0 < n_nodes; n0 += groups) {
    const int64_t nd = n0 + (threadIdx.x % 32) / LPN;
    TV a0 = TV(0), a1 = TV(0), a2 = TV(0);
    bool fixed = true;
    if (nd < n_nodes) {
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
    // every lane of the group holds the three sums: lane i < 3 finishes row 3 nd + i
    if (sub < 3 && nd < n_nodes) {
      const int64_t r = 3 * nd + sub;
      const TV yi = fixed ? TV(A[rowptr[r]]) * x[r] : (sub == 0 ? a0 : (sub == 1 ? a1 : a2));
      if constexpr (MODE == 0) {
        y[r] = yi;
        red.add(x[r], yi);
      } else {
        const double ri = b[r] - double(yi);
        y[r] = TV(ri);
        red.s += ri * ri;
      }
    }
  }
  double tot;
  if (grid_sum<kRedBlock>(red.value(), partials, ticket, &tot) && threadIdx.x == 0) {
    if constexpr (MODE == 0) {
      scal[S_PQ] = tot;
      if (!(tot > 0.0)) {
        atomicOr(flags, FLAG_BREAKDOWN);
        scal[S_DONE] = 1.0;
        scal[S_ALPHA] = 0.0;
      } else {
        scal[S_ALPHA] = scal[S_RZ] / tot;
      }
    } else {
      scal[S_ORR] = tot;
      scal[S_ODONE] = (tot <= scal[S_OTOL2]) ? 1.0 : 0.0;
    }
  }
}

// r = b - A x in FP64 (A in its storage type); ||r||^2 -> S_ORR, S_ODONE.
template <typename TA, int TPR>
__global__ void __launch_bounds__(kRedBlock) residual_kernel(
    int64_t n, const int32_t *__restrict__ rowptr, const int32_t *__restrict__ colind,
    const TA *__restrict__ A, const double *__restrict__ x, const double *__restrict__ b,
    double *__restrict__ r, double *scal, double *partials, unsigned int *ticket) {
  const int sub = threadIdx.x % TPR;
  const int64_t groups = int64_t(gridDim.x) * (kRedBlock / TPR);
  const int64_t warp_row0 = int64_t(blockIdx.x) * (kRedBlock / TPR) + (threadIdx.x / 32) * (32 / TPR);
  double rr = 0.0;
  for (int64_t r0 = warp_row0; r0 < n; r0 += groups) {
    const int64_t row = r0 + (threadIdx.x % 32) / TPR;
    double acc = 0.0;
    if (row < n) {
      const int32_t k1 = rowptr[row + 1];
      for (int32_t k = rowptr[row] + sub; k < k1; k += TPR) acc += double(A[k]) * x[colind[k]];
    }
#pragma unroll
    for (int o = TPR / 2; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o, TPR);
    if (sub == 0 && row < n) {
      const double ri = b[row] - acc;
      r[row] = ri;
      rr += ri * ri;
    }
  }
  double tot;
  if (grid_sum<kRedBlock>(rr, partials, ticket, &tot) && threadIdx.x == 0) {
    scal[S_ORR] = tot;
    scal[S_ODONE] = (tot <= scal[S_OTOL2]) ? 1.0 : 0.0;
  }
}

// r = b - A x in the mixed path: A and x as float pairs (A2, the assembly's
// FP64-accurate copy of A, and x2, the refinement iterate's mirror), every
// product and sum in double-float on the FP32 pipe; r and ||r||^2 in FP64
// (one conversion per row) -> S_ORR, S_ODONE.  The same 8 bytes per value as
// the FP64 kernels, about a dozen FP32 instructions per product instead of
// one FP64 multiply-add (fe_df.cuh).  Node-block form as bspmv_kernel (LPN
// lanes per node); after the group's reduction every lane holds the three
// row sums and lane i < 3 finishes row 3 nd + i.
template <int LPN>
__global__ void __launch_bounds__(kRedBlock) bres_df_kernel(
    int64_t n_nodes, const int32_t *__restrict__ rowptr, const int32_t *__restrict__ bptr,
    const int32_t *__restrict__ bcol, const int8_t *__restrict__ fixed_row, const float2 *__restrict__ A,
    const float2 *__restrict__ x, double *__restrict__ r, const double *__restrict__ b, double *scal,
    double *partials, unsigned int *ticket) {
  constexpr int GPW = 32 / LPN;  // nodes per warp
  const int sub = threadIdx.x % LPN;
  const int64_t groups = int64_t(gridDim.x) * (kRedBlock / LPN);
  // the loop bound is warp-uniform so every lane reaches every shuffle
  const int64_t warp_node0 = int64_t(blockIdx.x) * (kRedBlock / LPN) + (threadIdx.x / 32) * GPW;
  double red = 0.0;
  for (int64_t n0 = warp_node0; n0 < n_nodes; n0 += groups) {
    const int64_t nd = n0 + (threadIdx.x % 32) / LPN;
    float h0 = 0.f, l0 = 0.f, h1 = 0.f, l1 = 0.f, h2 = 0.f, l2 = 0.f;
    bool fixed = true;
    if (nd < n_nodes) {
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
    if (sub < 3 && nd < n_nodes) {
      const int64_t rw = 3 * nd + sub;
      float hi = sub == 0 ? h0 : (sub == 1 ? h1 : h2), lo = sub == 0 ? l0 : (sub == 1 ? l1 : l2);
      if (fixed) {  // the lone diagonal entry
        hi = lo = 0.f;
        df_fma_to(hi, lo, A[rowptr[rw]], x[rw]);
      }
      const double ri = b[rw] - df_value(hi, lo);
      r[rw] = ri;
      red += ri * ri;
    }
  }
  double tot;
  if (grid_sum<kRedBlock>(red, partials, ticket, &tot) && threadIdx.x == 0) {
    scal[S_ORR] = tot;
    scal[S_ODONE] = (tot <= scal[S_OTOL2]) ? 1.0 : 0.0;
  }
}

// The CSR form of bres_df_kernel (TPR threads per row).
template <int TPR>
__global__ void __launch_bounds__(kRedBlock) residual_df_kernel(
    int64_t n, const int32_t *__restrict__ rowptr, const int32_t *__restrict__ colind, const float2 *__restrict__ A,
    const float2 *__restrict__ x, const double *__restrict__ b, double *__restrict__ r, double *scal,
    double *partials, unsigned int *ticket) {
  const int sub = threadIdx.x % TPR;
  const int64_t groups = int64_t(gridDim.x) * (kRedBlock / TPR);
  const int64_t warp_row0 = int64_t(blockIdx.x) * (kRedBlock / TPR) + (threadIdx.x / 32) * (32 / TPR);
  double rr = 0.0;
  for (int64_t r0 = warp_row0; r0 < n; r0 += groups) {
    const int64_t row = r0 + (threadIdx.x % 32) / TPR;
    float hi = 0.f, lo = 0.f;
    if (row < n) {
      const int32_t k1 = rowptr[row + 1];
      for (int32_t k = rowptr[row] + sub; k < k1; k += TPR) df_fma_to(hi, lo, A[k], x[colind[k]]);
    }
#pragma unroll
    for (int o = TPR / 2; o > 0; o >>= 1) df_shfl_add<TPR>(hi, lo, o);
    if (sub == 0 && row < n) {
      const double ri = b[row] - df_value(hi, lo);
      r[row] = ri;
      rr += ri * ri;
    }
  }
  double tot;
  if (grid_sum<kRedBlock>(rr, partials, ticket, &tot) && threadIdx.x == 0) {
    scal[S_ORR] = tot;
    scal[S_ODONE] = (tot <= scal[S_OTOL2]) ? 1.0 : 0.0;
  }
}

// x += alpha p; r -= alpha q; ||r||^2 -> S_RR; S_DONE when below S_TOL2.
template <typename TV>
__global__ void __launch_bounds__(kRedBlock) axpy_norm_kernel(int64_t n, TV *__restrict__ x,
                                                              TV *__restrict__ r,
                                                              const TV *__restrict__ p,
                                                              const TV *__restrict__ q, double *scal,
                                                              double *partials, unsigned int *ticket,
                                                              double max_iters) {
  if (solve_done(scal)) return;
  const TV al = TV(scal[S_ALPHA]);
  DotAcc<TV> rr;
  for (int64_t i = int64_t(blockIdx.x) * kRedBlock + threadIdx.x; i < n; i += int64_t(gridDim.x) * kRedBlock) {
    x[i] += al * p[i];
    const TV ri = r[i] - al * q[i];
    r[i] = ri;
    rr.add(ri, ri);
  }
  double tot;
  if (grid_sum<kRedBlock>(rr.value(), partials, ticket, &tot) && threadIdx.x == 0) {
    scal[S_RR] = tot;
    scal[S_ITERS] += 1.0;
    if (tot <= scal[S_TOL2])
      scal[S_DONE] = 1.0;
    else if (scal[S_ITERS] >= max_iters)
      scal[S_DONE] = 2.0;  // iteration cap: stops the solve, reported as not converged
  }
}

// rz_new = r.z; first: S_RZ = rz_new; else beta = rz_new / S_RZ, S_RZ = rz_new.
template <typename TV>
__global__ void __launch_bounds__(kRedBlock) dot_rz_kernel(int64_t n, const TV *__restrict__ r,
                                                           const TV *__restrict__ z, int first,
                                                           double *scal, double *partials,
                                                           unsigned int *ticket, int *flags) {
  if (solve_done(scal)) return;
  DotAcc<TV> s;
  for (int64_t i = int64_t(blockIdx.x) * kRedBlock + threadIdx.x; i < n; i += int64_t(gridDim.x) * kRedBlock)
    s.add(r[i], z[i]);
  double tot;
  if (grid_sum<kRedBlock>(s.value(), partials, ticket, &tot) && threadIdx.x == 0) {
    if (!(tot > 0.0) && scal[S_RR] > 0.0) {  // P^{-1} lost definiteness
      atomicOr(flags, FLAG_BREAKDOWN);
      scal[S_DONE] = 1.0;
    }
    if (first) {
      scal[S_BETA] = 0.0;
    } else {
      scal[S_BETA] = tot / scal[S_RZ];
    }
    scal[S_RZ] = tot;
  }
}

template <typename TV>
__global__ void update_p_kernel(int64_t n, const TV *__restrict__ z, TV *__restrict__ p, int first,
                                const double *scal) {
  if (solve_done(scal)) return;
  const TV be = TV(scal[S_BETA]);
  for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x)
    p[i] = first ? z[i] : z[i] + be * p[i];  // first: p = z, whatever p held
}

// Start of a (sub)solve: x = 0, r = rhs (cast), ||rhs||^2 -> tolerance.
// outer = 1: S_BB, S_OTOL2 = tol^2 * bb, S_ORR, S_ODONE.  outer = 0: inner
// solve with S_TOL2 = tol^2 * ||rhs||^2, S_DONE.
// x2 (mixed path's outer solve, else null): x as float pairs, for the residual.
template <typename TV>
__global__ void __launch_bounds__(kRedBlock) init_solve_kernel(int64_t n, TV *__restrict__ x,
                                                               TV *__restrict__ r,
                                                               const double *__restrict__ rhs,
                                                               double tol, int outer, double *scal,
                                                               double *partials, unsigned int *ticket,
                                                               int keep_x, float2 *__restrict__ x2) {
  double s = 0.0;
  for (int64_t i = int64_t(blockIdx.x) * kRedBlock + threadIdx.x; i < n; i += int64_t(gridDim.x) * kRedBlock) {
    const double v = rhs[i];
    if (!keep_x) x[i] = TV(0);  // a warm start keeps x (its residual follows)
    if (x2) x2[i] = keep_x ? df_split(double(x[i])) : make_float2(0.f, 0.f);
    r[i] = TV(v);
    s += v * v;
  }
  double tot;
  if (grid_sum<kRedBlock>(s, partials, ticket, &tot) && threadIdx.x == 0) {
    if (outer) {
      scal[S_BB] = tot;
      scal[S_OTOL2] = tol * tol * tot;
      scal[S_ORR] = tot;
      scal[S_ODONE] = (tot == 0.0) ? 1.0 : 0.0;
      scal[S_ITERS] = 0.0;
      scal[S_SWEEPS] = 0.0;
    }
    scal[S_TOL2] = tol * tol * tot;
    scal[S_RR] = tot;
    scal[S_DONE] = (tot == 0.0) ? 1.0 : 0.0;
  }
}

// x += d, and its float-pair mirror x2 (read by the double-float residual)
__global__ void refine_update_kernel(int64_t n, double *__restrict__ x, const float *__restrict__ d,
                                     float2 *__restrict__ x2) {
  for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x) {
    const double xi = x[i] + double(d[i]);
    x[i] = xi;
    if (x2) x2[i] = df_split(xi);
  }
}

__global__ void integrate_kernel(int64_t n, double h, const double *__restrict__ a, double *__restrict__ v,
                                 double *__restrict__ q, double *__restrict__ a_prev) {
  for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x) {
    const double ai = a[i];
    const double vn = v[i] + h * ai;
    v[i] = vn;
    q[i] += h * vn;
    a_prev[i] = ai;  // the next step's warm start
  }
}

// mode 0: FP64 solve (S_DONE == 1), 1: refined mixed solve (S_ODONE == 1),
// 2: batched solve (flags[2] == 1, set when every member converged)
__global__ void integrate_guard_kernel(int64_t n, double h, const double *__restrict__ a, double *__restrict__ v,
                                       double *__restrict__ q, double *__restrict__ a_prev, const double *scal,
                                       const int *flags, int mode) {
  const bool ok = flags[0] == 0 && (mode == 2 ? flags[2] == 1 : mode == 1 ? scal[S_ODONE] == 1.0 : scal[S_DONE] == 1.0);
  if (!ok) return;
  for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x) {
    const double ai = a[i];
    const double vn = v[i] + h * ai;
    v[i] = vn;
    q[i] += h * vn;
    a_prev[i] = ai;  // the next step's warm start
  }
}

__global__ void graph_cond_kernel(cudaGraphConditionalHandle hnd, double *scal, const int *flags, int mode,
                                  double max_iters) {
  bool go;
  if (mode == 0) {
    go = scal[S_DONE] == 0.0;
  } else {
    go = scal[S_ODONE] == 0.0 && scal[S_ITERS] < max_iters;
    if (mode == 1) scal[S_SWEEPS] += 1.0;
  }
  cudaGraphSetConditional(hnd, (go && flags[0] == 0) ? 1u : 0u);
}

__global__ void newton_state_kernel(int64_t n, double h, const double *__restrict__ q, const double *__restrict__ v,
                                    const double *__restrict__ a, double *__restrict__ qk,
                                    double *__restrict__ vk) {
  for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x) {
    const double vn = v[i] + h * a[i];
    vk[i] = vn;
    qk[i] = q[i] + h * vn;
  }
}

// a += delta with ||delta||^2 and ||a||^2 (two deterministic grid sums)
__global__ void __launch_bounds__(kRedBlock) newton_update_kernel(int64_t n, const double *__restrict__ delta,
                                                                  double *__restrict__ a, double *scal,
                                                                  double *partials, unsigned int *ticket) {
  double dd = 0.0, aa = 0.0;
  for (int64_t i = int64_t(blockIdx.x) * kRedBlock + threadIdx.x; i < n; i += int64_t(gridDim.x) * kRedBlock) {
    const double di = delta[i], ai = a[i] + di;
    a[i] = ai;
    dd += di * di;
    aa += ai * ai;
  }
  double tot;
  if (grid_sum<kRedBlock>(dd, partials, ticket, &tot) && threadIdx.x == 0) scal[S_NDELTA] = tot;
  if (grid_sum<kRedBlock>(aa, partials + gridDim.x, ticket + 1, &tot) && threadIdx.x == 0) scal[S_NA] = tot;
}

template <typename S, typename D>
__global__ void convert_kernel(const S *__restrict__ src, D *__restrict__ dst, int64_t n) {
  for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x)
    dst[i] = D(src[i]);
}

static unsigned ew_grid(int64_t n) {
  return unsigned(std::max<int64_t>(1, std::min<int64_t>((n + 255) / 256, 152 * 16)));
}

// SpMV variants: 0-3 the node-block kernel with 4, 8, 16 or 32 lanes per
// node, 4-5 the CSR kernel with 8 or 16 threads per row.  The first solve
// of a context times them (tune_spmv) and keeps the fastest for each of the
// two products: y = A x with x.y in the inner solve's type, and the
// refinement residual r = b - A x (FP64, or double-float on float pairs).
constexpr int kSpmvVariants = 6;

template <typename TA, typename TV, int MODE>
static void launch_spmv_variant(const fe_ctx *c, const DeviceState *d, int var, const TA *A, const TV *x, TV *y,
                                const double *b, double *scal, int *flags, cudaStream_t s) {
  const int64_t nn = c->n_nodes, n = c->n;
  switch (var) {
#define FE_BSPMV(V, L)                                                                                            \
  case V:                                                                                                         \
    bspmv_kernel<TA, TV, L, MODE><<<spmv_grid(nn * L), kRedBlock, 0, s>>>(nn, d->rowptr, d->bptr, d->bcol,          \
                                                                       d->fixed_row, A, x, y, b, scal,           \
                                                                       d->partials, d->ticket, flags);           \
    break;
    FE_BSPMV(0, 4)
    FE_BSPMV(1, 8)
    FE_BSPMV(2, 16)
    FE_BSPMV(3, 32)
#undef FE_BSPMV
    default: {
      const bool t16 = var == 5;
      const unsigned g = spmv_grid(n * (t16 ? 16 : 8) / 4);
      if constexpr (MODE == 0) {
        if (t16)
          spmv_dot_kernel<TA, TV, 16><<<g, kRedBlock, 0, s>>>(n, d->rowptr, d->colind, A, x, y, scal, d->partials,
                                                              d->ticket, flags);
        else
          spmv_dot_kernel<TA, TV, 8><<<g, kRedBlock, 0, s>>>(n, d->rowptr, d->colind, A, x, y, scal, d->partials,
                                                             d->ticket, flags);
      } else {
        if (t16)
          residual_kernel<TA, 16><<<g, kRedBlock, 0, s>>>(n, d->rowptr, d->colind, A, x, b, y, scal, d->partials,
                                                          d->ticket);
        else
          residual_kernel<TA, 8><<<g, kRedBlock, 0, s>>>(n, d->rowptr, d->colind, A, x, b, y, scal, d->partials,
                                                         d->ticket);
      }
    }
  }
}

static void spmv_dot_var(const fe_ctx *c, const DeviceState *d, int var, bool fp32, const void *x, void *y,
                         double *scal, int *flags, cudaStream_t s) {
  if (fp32)
    launch_spmv_variant<float, float, 0>(c, d, var, (const float *)d->A, (const float *)x, (float *)y, nullptr, scal,
                                         flags, s);
  else
    launch_spmv_variant<double, double, 0>(c, d, var, (const double *)d->A, (const double *)x, (double *)y, nullptr,
                                           scal, flags, s);
}

void launch_spmv_dot(const fe_ctx *c, const DeviceState *d, bool fp32, const void *x, void *y,
                     cudaStream_t s) {
  d->launches++;
  spmv_dot_var(c, d, d->spmv_var, fp32, x, y, d->scal, d->flags, s);
}

// r = b - A x for the refinement: A itself in the FP64 path; in the mixed
// path A2 and x2 (float pairs) in double-float, the variant numbering as
// launch_spmv_variant's.
static void res_var_launch(const fe_ctx *c, const DeviceState *d, int var, double *scal, int *flags,
                           cudaStream_t s) {
  if (!d->A2) {
    launch_spmv_variant<double, double, 1>(c, d, var, d->A64, d->x, d->r, d->b, scal, flags, s);
    return;
  }
  const int64_t nn = c->n_nodes, n = c->n;
  switch (var) {
#define FE_BRES(V, L)                                                                                         \
  case V:                                                                                                     \
    bres_df_kernel<L><<<spmv_grid(nn * L), kRedBlock, 0, s>>>(nn, d->rowptr, d->bptr, d->bcol, d->fixed_row,   \
                                                             d->A2, d->x2, d->r, d->b, scal, d->partials,    \
                                                             d->ticket);                                     \
    break;
    FE_BRES(0, 4)
    FE_BRES(1, 8)
    FE_BRES(2, 16)
    FE_BRES(3, 32)
#undef FE_BRES
    default: {
      const bool t16 = var == 5;
      const unsigned g = spmv_grid(n * (t16 ? 16 : 8) / 4);
      if (t16)
        residual_df_kernel<16><<<g, kRedBlock, 0, s>>>(n, d->rowptr, d->colind, d->A2, d->x2, d->b, d->r, scal,
                                                       d->partials, d->ticket);
      else
        residual_df_kernel<8><<<g, kRedBlock, 0, s>>>(n, d->rowptr, d->colind, d->A2, d->x2, d->b, d->r, scal,
                                                      d->partials, d->ticket);
    }
  }
}

void launch_residual(const fe_ctx *c, const DeviceState *d, bool, cudaStream_t s) {
  d->launches++;
  res_var_launch(c, d, d->res_var, d->scal, d->flags, s);
}

// Times every variant of both products (CUDA events on the main stream, one
// untimed run then the median of five) on the assembled matrix; the timing
// runs write their scalars and flags to scratch words, not the solve's.
int tune_spmv(fe_ctx *c, DeviceState *d) {
  if (d->spmv_var >= 0) return FE_OK;
  if (c->opt.spmv_variant >= 0) {  // fixed by the caller
    d->spmv_var = d->res_var = c->opt.spmv_variant;
    return FE_OK;
  }
  const bool fp32 = c->opt.precision == FE_MIXED;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  FE_CUDA_TRY(cudaEventCreate(&e0));
  cudaError_t er = cudaEventCreate(&e1);
  double *ts = d->tune_scal;
  int *tf = reinterpret_cast<int *>(d->tune_scal + S_COUNT);
  int best[2] = {2, 2};
  for (int prod = 0; prod < 2 && er == cudaSuccess; ++prod) {
    float bt = 1e30f;
    for (int var = 0; var < kSpmvVariants && er == cudaSuccess; ++var) {
      // one untimed run (caches, first-launch costs), then five timed ones
      float t[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
      for (int rep = 0; rep < 6 && er == cudaSuccess; ++rep) {
        er = cudaMemsetAsync(ts, 0, S_COUNT * sizeof(double) + 4 * sizeof(int), d->stream);
        if (er == cudaSuccess) er = cudaEventRecord(e0, d->stream);
        if (er == cudaSuccess) {
          if (prod == 0)
            spmv_dot_var(c, d, var, fp32, d->vp, d->vq, ts, tf, d->stream);
          else
            res_var_launch(c, d, var, ts, tf, d->stream);
          er = cudaGetLastError();
        }
        if (er == cudaSuccess) er = cudaEventRecord(e1, d->stream);
        if (er == cudaSuccess) er = cudaEventSynchronize(e1);
        if (er == cudaSuccess) er = cudaEventElapsedTime(&t[rep], e0, e1);
      }
      std::sort(t + 1, t + 6);
      if (er == cudaSuccess && t[3] < bt) {  // the median of the timed runs
        bt = t[3];
        best[prod] = var;
      }
    }
  }
  cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (er != cudaSuccess) {
    cudaGetLastError();
    return set_error(c, FE_ERR_CUDA, std::string("SpMV autotuner: ") + cudaGetErrorString(er));
  }
  d->spmv_var = best[0];
  d->res_var = best[1];
  return FE_OK;
}

void launch_axpy_norm(const fe_ctx *c, const DeviceState *d, bool fp32, void *x, void *r, const void *p,
                      const void *q, cudaStream_t s) {
  d->launches++;
  const int64_t n = c->n;
  if (fp32)
    axpy_norm_kernel<float><<<red_grid(n), kRedBlock, 0, s>>>(n, (float *)x, (float *)r, (const float *)p,
                                                              (const float *)q, d->scal, d->partials, d->ticket,
                                                              double(c->opt.max_iters));
  else
    axpy_norm_kernel<double><<<red_grid(n), kRedBlock, 0, s>>>(n, (double *)x, (double *)r,
                                                               (const double *)p, (const double *)q, d->scal,
                                                               d->partials, d->ticket, double(c->opt.max_iters));
}

void launch_dot_rz(const fe_ctx *c, const DeviceState *d, bool fp32, const void *r, const void *z, bool first,
                   cudaStream_t s) {
  d->launches++;
  const int64_t n = c->n;
  if (fp32)
    dot_rz_kernel<float><<<red_grid(n), kRedBlock, 0, s>>>(n, (const float *)r, (const float *)z, first,
                                                           d->scal, d->partials, d->ticket, d->flags);
  else
    dot_rz_kernel<double><<<red_grid(n), kRedBlock, 0, s>>>(n, (const double *)r, (const double *)z, first,
                                                            d->scal, d->partials, d->ticket, d->flags);
}

void launch_update_p(const fe_ctx *c, const DeviceState *d, bool fp32, const void *z, void *p, bool first,
                     cudaStream_t s) {
  d->launches++;
  const int64_t n = c->n;
  if (fp32)
    update_p_kernel<float><<<ew_grid(n), 256, 0, s>>>(n, (const float *)z, (float *)p, first, d->scal);
  else
    update_p_kernel<double><<<ew_grid(n), 256, 0, s>>>(n, (const double *)z, (double *)p, first, d->scal);
}

void launch_init_solve(const fe_ctx *c, const DeviceState *d, bool fp32, void *x, void *r, const double *rhs,
                       double tol, bool outer, cudaStream_t s, bool keep_x) {
  d->launches++;
  const int64_t n = c->n;
  if (fp32)
    init_solve_kernel<float><<<red_grid(n), kRedBlock, 0, s>>>(n, (float *)x, (float *)r, rhs, tol, outer,
                                                               d->scal, d->partials, d->ticket, keep_x ? 1 : 0,
                                                               nullptr);
  else  // the outer solve's x: its float-pair mirror too (mixed path)
    init_solve_kernel<double><<<red_grid(n), kRedBlock, 0, s>>>(n, (double *)x, (double *)r, rhs, tol, outer,
                                                                d->scal, d->partials, d->ticket, keep_x ? 1 : 0,
                                                                x == d->x ? d->x2 : nullptr);
}

__global__ void warm_fixup_kernel(double *scal) {
  scal[S_RR] = scal[S_ORR];
  scal[S_DONE] = (scal[S_BB] == 0.0 || scal[S_ODONE] != 0.0) ? 1.0 : 0.0;
}

void launch_warm_fixup(const fe_ctx *c, const DeviceState *d, cudaStream_t s) {
  d->launches++;
  warm_fixup_kernel<<<1, 1, 0, s>>>(d->scal);
}

void launch_refine_update(const fe_ctx *c, const DeviceState *d, cudaStream_t s) {
  d->launches++;
  refine_update_kernel<<<ew_grid(c->n), 256, 0, s>>>(c->n, d->x, (const float *)d->vd, d->x2);
}

void launch_integrate(const fe_ctx *c, const DeviceState *d, cudaStream_t s) {
  d->launches++;
  integrate_kernel<<<ew_grid(c->n), 256, 0, s>>>(c->n, c->h, d->x, d->v, d->q, d->a_prev);
}

void launch_integrate_guarded(const fe_ctx *c, const DeviceState *d, bool fp32, cudaStream_t s) {
  d->launches++;
  integrate_guard_kernel<<<ew_grid(c->n), 256, 0, s>>>(c->n, c->h, d->x, d->v, d->q, d->a_prev, d->scal, d->flags,
                                                        c->nseg > 1 ? 2 : (fp32 ? 1 : 0));
}

void launch_graph_cond(const fe_ctx *c, const DeviceState *d, cudaGraphConditionalHandle h, int mode,
                       cudaStream_t s) {
  d->launches++;
  graph_cond_kernel<<<1, 1, 0, s>>>(h, d->scal, d->flags, mode, double(c->opt.max_iters));
}

void launch_newton_state(const fe_ctx *c, const DeviceState *d, const double *a, double *qk, double *vk,
                         cudaStream_t s) {
  d->launches++;
  newton_state_kernel<<<ew_grid(c->n), 256, 0, s>>>(c->n, c->h, d->q, d->v, a, qk, vk);
}

void launch_newton_update(const fe_ctx *c, const DeviceState *d, const double *delta, double *a, cudaStream_t s) {
  d->launches++;
  newton_update_kernel<<<red_grid(c->n), kRedBlock, 0, s>>>(c->n, delta, a, d->scal, d->partials, d->ticket);
}

void launch_convert(const void *src, bool src32, void *dst, bool dst32, int64_t n, cudaStream_t s) {
  const unsigned g = ew_grid(n);
  if (src32 && dst32)
    convert_kernel<float, float><<<g, 256, 0, s>>>((const float *)src, (float *)dst, n);
  else if (src32)
    convert_kernel<float, double><<<g, 256, 0, s>>>((const float *)src, (double *)dst, n);
  else if (dst32)
    convert_kernel<double, float><<<g, 256, 0, s>>>((const double *)src, (float *)dst, n);
  else
    convert_kernel<double, double><<<g, 256, 0, s>>>((const double *)src, (double *)dst, n);
}

__global__ void pair_to_double_kernel(const float2 *__restrict__ src, double *__restrict__ dst, int64_t n) {
  for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x)
    dst[i] = df_value(src[i]);
}

void launch_pair_to_double(const float2 *src, double *dst, int64_t n, cudaStream_t s) {
  pair_to_double_kernel<<<ew_grid(n), 256, 0, s>>>(src, dst, n);
}

}  // namespace fe
