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
#include <cuda.h>  // CUtensorMap
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include <mutex>

#include "fe_device.cuh"

namespace fe {

// Programmatic dependent launch: the next kernel in the stream may start
// once every CTA of this one has signalled, and waits for this kernel's
// completion (and memory) before touching what it produced.  Both are no-ops
// for a kernel launched without the attribute.
__device__ __forceinline__ void pdl_launch_dependents() {
  asm volatile("griddepcontrol.launch_dependents;\n" ::: "memory");
}
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;\n" ::: "memory"); }

template <typename... KArgs, typename... Args>
static void launch_pdl(void (*kern)(KArgs...), unsigned grid, unsigned block, size_t smem, cudaStream_t s,
                       Args... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(grid);
  cfg.blockDim = dim3(block);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  cudaLaunchKernelEx(&cfg, kern, static_cast<KArgs>(args)...);
}

// 16-byte vectors along the rows of Y (its leading dimension is a multiple of 8).
template <typename T>
struct Vec16;
template <>
struct Vec16<__half> {
  using type = uint4;
  static constexpr int n = 8;
};
template <>
struct Vec16<float> {
  using type = float4;
  static constexpr int n = 4;
};
template <>
struct Vec16<double> {
  using type = double2;
  static constexpr int n = 2;
};
// element q of a 16-byte vector held in registers (q is a compile-time
// constant after unrolling, so no address is taken)
__device__ __forceinline__ float vget(const float4 &v, int q) {
  return q == 0 ? v.x : q == 1 ? v.y : q == 2 ? v.z : v.w;
}
__device__ __forceinline__ double vget(const double2 &v, int q) { return q == 0 ? v.x : v.y; }
__device__ __forceinline__ float vget(const uint4 &v, int q) {
  const uint32_t w = q < 2 ? v.x : q < 4 ? v.y : q < 6 ? v.z : v.w;
  return __half2float(__ushort_as_half(static_cast<unsigned short>((q & 1) ? (w >> 16) : (w & 0xffffu))));
}

// Binary16 copy of Y for the application (precond_fp16): round to nearest,
// clamped to the largest finite binary16 so that no entry becomes infinite.
// 8 entries per thread (y_total is a multiple of 8).
__global__ void __launch_bounds__(256) y_to_half_kernel(const float4 *__restrict__ Y, uint4 *__restrict__ Yh,
                                                        int64_t n8) {
  for (int64_t i = int64_t(blockIdx.x) * 256 + threadIdx.x; i < n8; i += int64_t(gridDim.x) * 256) {
    const float4 a = Y[2 * i], b = Y[2 * i + 1];
    auto h2 = [](float x, float y) {
      const float lim = 65504.f;
      const __half2 h = __floats2half2_rn(fminf(fmaxf(x, -lim), lim), fminf(fmaxf(y, -lim), lim));
      return *reinterpret_cast<const uint32_t *>(&h);
    };
    Yh[i] = make_uint4(h2(a.x, a.y), h2(a.z, a.w), h2(b.x, b.y), h2(b.z, b.w));
  }
}

// -------------------------------------------------------------- assembly
// Task (front, c0, c1): zero the lower part of columns [c0, c1) of F and of
// the pivot columns of Y, scatter the A entries of those columns, then add
// every child's update block (children in fixed order: deterministic).
//
// Extend-add of one child: its update rows map to parent rows through the
// increasing map rm, so the child columns landing in [c0, c1) are the
// contiguous range [jlo, jhi) with jlo = #{rm < c0}, jhi = #{rm < c1}.  One
// pass over rm stages it in shared memory and counts both (no dependent
// binary-search loads); then warp w takes the columns jlo + w, jlo + w + 8,
// ... in 32-row chunks, eight chunks' loads in flight per lane before their
// stores.  Distinct (column, row) pairs of one child hit distinct parent
// entries (rm is injective), so the warps never collide; children follow one
// another behind a barrier (two children can share parent entries).
constexpr int kRmCap = 4096;  // row maps longer than this are read from global memory

template <typename TF>
__global__ void __launch_bounds__(256) front_assemble_kernel(
    const int32_t *__restrict__ tasks, const DFront *__restrict__ fronts,
    const int32_t *__restrict__ child_list, const int32_t *__restrict__ rmap,
    const int64_t *__restrict__ fa_colptr, const int32_t *__restrict__ fa_slot,
    const int32_t *__restrict__ fa_off, const TF *__restrict__ A, TF *__restrict__ F, TF *__restrict__ Y) {
  __shared__ int32_t rms[kRmCap];
  __shared__ int s_cnt[2][2];  // (jlo, jhi) counts, double-buffered by child parity
  pdl_launch_dependents();
  const int32_t f = tasks[3 * blockIdx.x], c0 = tasks[3 * blockIdx.x + 1], c1 = tasks[3 * blockIdx.x + 2];
  const DFront fr = fronts[f];
  const int32_t m = fr.m, p = fr.npiv;
  TF *Ff = F + fr.f_off;
  if (threadIdx.x < 4) s_cnt[threadIdx.x >> 1][threadIdx.x & 1] = 0;
  pdl_wait();
  for (int32_t col = c0; col < c1; ++col) {
    TF *cp = Ff + int64_t(col) * fr.ldf;
    for (int32_t r = col + threadIdx.x; r < m; r += blockDim.x) cp[r] = TF(0);
    if (col < p) {
      TF *yp = Y + fr.y_off + int64_t(col) * fr.ldy;
      for (int32_t r = threadIdx.x; r < fr.ldy; r += blockDim.x) yp[r] = TF(0);
    }
  }
  __syncthreads();
  const int32_t ce = c1 < p ? c1 : p;
  if (ce > c0) {  // the entries of columns [c0, ce) are contiguous in the fa lists
    const int64_t e0 = fa_colptr[fr.fac_off + c0], e1 = fa_colptr[fr.fac_off + ce];
    for (int64_t e = e0 + threadIdx.x; e < e1; e += 4 * 256) {
      int32_t off[4];
      TF v[4];
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        const int64_t ee = e + 256 * k;
        off[k] = ee < e1 ? fa_off[ee] : -1;
        v[k] = ee < e1 ? A[fa_slot[ee]] : TF(0);
      }
#pragma unroll
      for (int k = 0; k < 4; ++k)
        if (off[k] >= 0) Ff[off[k]] = v[k];
    }
  }
  __syncthreads();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarp = blockDim.x >> 5;
  for (int32_t ci = fr.child_begin; ci < fr.child_end; ++ci) {
    const int b = (ci - fr.child_begin) & 1;
    const DFront ch = fronts[child_list[ci]];
    const int32_t *rm = rmap + ch.rows_off;
    const int32_t nu = ch.nupd, pc = ch.npiv;
    const bool staged = nu <= kRmCap;
    int n0 = 0, n1 = 0;
    for (int32_t i = threadIdx.x; i < nu; i += blockDim.x) {
      const int32_t v = rm[i];
      if (staged) rms[i] = v;
      n0 += v < c0;
      n1 += v < c1;
    }
    n0 = __reduce_add_sync(0xffffffffu, n0);
    n1 = __reduce_add_sync(0xffffffffu, n1);
    if (lane == 0 && n1 > 0) {
      atomicAdd(&s_cnt[b][0], n0);
      atomicAdd(&s_cnt[b][1], n1);
    }
    __syncthreads();
    const int32_t jlo = s_cnt[b][0], jhi = s_cnt[b][1];
    // the other buffer was last read before the previous child's closing
    // barrier; the next child accumulates into it after this child's
    if (threadIdx.x < 2) s_cnt[b ^ 1][threadIdx.x] = 0;
    const int32_t *rp = staged ? rms : rm;
    const TF *Fc = F + ch.f_off + pc;
    int32_t j = jlo + warp, r = j;  // this warp's current column and chunk start (warp-uniform)
    while (j < jhi) {
      TF sv[8], dv[8];
      TF *dp[8];
#pragma unroll
      for (int k = 0; k < 8; ++k) {
        sv[k] = TF(0);
        dv[k] = TF(0);
        dp[k] = nullptr;
        if (j < jhi) {
          const int32_t i = r + lane;
          if (i < nu) {
            sv[k] = Fc[int64_t(pc + j) * ch.ldf + i];
            dp[k] = Ff + int64_t(rp[j]) * fr.ldf + rp[i];
            dv[k] = *dp[k];
          }
          r += 32;
          if (r >= nu) {
            j += nwarp;
            r = j;
          }
        }
      }
#pragma unroll
      for (int k = 0; k < 8; ++k)
        if (dp[k]) *dp[k] = dv[k] + sv[k];
    }
    __syncthreads();
  }
}

// ---------------------------------------------------------------- diagonal
// Pivots of the FP32 factor are accumulated in double-float: a value is an
// unevaluated sum hi + lo of two floats (~48-bit significand), updated with
// the error-free transformations of Knuth (TwoSum) and Dekker (TwoProduct,
// here through FMA).  GB300's FP64 pipe issues a warp instruction every ~64
// cycles per SM sub-partition, so a pivot step's FP64 chain, which sits on
// the block's serial path, cost more than the whole FP32 elimination step;
// double-float keeps FP64-level pivots at FP32 latency.
struct DF {
  float hi, lo;
};
__device__ __forceinline__ DF df_two_sum(float a, float b) {
  const float s = a + b, bb = s - a;
  return {s, (a - (s - bb)) + (b - bb)};
}
__device__ __forceinline__ DF df_quick(float a, float b) {  // |a| >= |b|
  const float s = a + b;
  return {s, b - (s - a)};
}
__device__ __forceinline__ DF df_two_prod(float a, float b) {
  const float p = a * b;
  return {p, fmaf(a, b, -p)};
}
__device__ __forceinline__ DF df_mul(DF x, DF y) {
  DF p = df_two_prod(x.hi, y.hi);
  p.lo = fmaf(x.hi, y.lo, fmaf(x.lo, y.hi, p.lo));
  return df_quick(p.hi, p.lo);
}
__device__ __forceinline__ DF df_sub(DF x, DF y) {
  DF s = df_two_sum(x.hi, -y.hi);
  s.lo += x.lo - y.lo;
  return df_quick(s.hi, s.lo);
}
// 1/d: the hardware reciprocal estimate (within 2 ulp) refined by one Newton
// step x + x (1 - d x) with the residual formed in double-float, which
// squares its relative error (~2^-44).  Branch-free: a non-positive pivot is
// replaced by 1 so the factorisation finishes without NaNs, and the caller
// flags it.
__device__ __forceinline__ DF df_pivot_inverse(DF d) {
  const bool ok = d.hi > 0.f;
  d.hi = ok ? d.hi : 1.f;
  d.lo = ok ? d.lo : 0.f;
  const float x = __fdividef(1.f, d.hi);
  const DF dx = df_mul(d, {x, 0.f});
  const float r = (1.f - dx.hi) - dx.lo;
  const DF q = df_two_prod(x, r);
  DF out = df_quick(x, q.hi);
  out.lo += q.lo;
  return out;
}
__device__ __forceinline__ double pivot_inverse(double d, int *flags, bool report) {
  if (!(d > 0.0)) {
    if (report) atomicOr(flags, FLAG_PIVOT);
    d = 1.0;
  }
  return 1.0 / d;
}

// Task (front, k0, kb): LDL^T of the kb x kb diagonal block (kb <= 64),
// blocked in 16-pivot sub-blocks so that the serial chain of a sub-block runs
// inside one warp and the eight elimination warps meet at three barriers per
// sub-block instead of one per pivot.  For sub-block b (columns
// B = [16b, 16b + 16)):
//  A. one warp factors the 16 x 16 diagonal sub-block (lane l keeps row 16b + l
//     in registers; each pivot and column reaches the lanes by shuffles);
//  B. one thread per row below solves the sub-block's columns,
//     W[i, B] = S[i, B] L_BB^{-T} (forward substitution);
//  C. all eight warps apply the rank-16 update S[I, J] -= L[I, B] W[J, B]^T
//     to the sub-blocks below and right of b (thread (tr, tc): rows
//     tr + 16a, columns tc + 16c).
// The eliminations run in TF with the pivots of the running Schur complement
// in TF; S ends holding the final unscaled columns W = L d and Lsc the
// scaled L.  The pivots D are accumulated beside them from the final columns
// by a ninth warp that follows the sub-blocks as they are published (thread 0
// releases a progress word after the barrier that ends step B, the warp
// acquires it; lane l keeps rows l and l + 32).  FP32 factor: in
// double-float, d_i = a_ii - sum_j W_ij L_ij, each term the exact product of
// the elimination's final W and L entries, so no pivot waits for an earlier
// one and the 64 inverses are taken at once at the end; the sum of the
// squares of W over the pivot warp's own pivots (a serial recurrence of 64
// double-float reciprocals) made this warp the block's critical path, and it
// is no more accurate, since W and L carry the FP32 elimination's rounding
// either way.  FP64 factor: d_i = a_ii - sum_j W_ij^2 / d_j in FP64, 16 steps
// per sub-block each taking a pivot's inverse and folding its column into
// every later row at once.  The FP32 elimination takes the fast reciprocal of
// its own pivots; the stored L is W times the inverses of the pivot warp's
// pivots.  L_KK^{-1} (written into
// Y[K, K]) is formed after the elimination by blocked inversion of the unit
// lower L: the diagonal
// 16 x 16 inverses by one warp each, then, one block diagonal at a time,
// X_ij = -X_ii sum_{k=j}^{i-1} L_ik X_kj.  GB300's FP64 pipe issues a warp
// instruction only every ~64 cycles per SM sub-partition, so no FP64 or
// double-float work sits on the elimination's chain.
constexpr int kDiagThreads = 288;
constexpr int kDP = 65;  // row pitch of the 64 x 64 shared arrays (conflict-free columns)

// S, Lsc, X (64 x kDP each), T (3 x 16 x 17), the TF pivot inverses (64),
// then the FP64 / double-float pivots and their inverses (64 doubles each)
template <typename TF>
constexpr size_t diag_smem() {
  return size_t(3 * 64 * kDP + 3 * 16 * 17 + 64) * sizeof(TF) + 2 * 64 * sizeof(double);
}
static_assert((3 * 64 * kDP + 3 * 16 * 17 + 64) % 2 == 0, "the pivot arrays stay 8-byte aligned");

// block-scope acquire / release on a shared word (the pivot warp follows the
// elimination's progress without joining its barriers)
__device__ __forceinline__ int ld_acquire_cta_shared(const int *p) {
  int v;
  asm volatile("ld.acquire.cta.shared::cta.b32 %0, [%1];\n"
               : "=r"(v)
               : "r"(static_cast<uint32_t>(__cvta_generic_to_shared(p)))
               : "memory");
  return v;
}
__device__ __forceinline__ void st_release_cta_shared(int *p, int v) {
  asm volatile("st.release.cta.shared::cta.b32 [%0], %1;\n" ::"r"(static_cast<uint32_t>(__cvta_generic_to_shared(p))),
               "r"(v)
               : "memory");
}
__device__ __forceinline__ void elim_barrier() { asm volatile("bar.sync 1, 256;\n" ::: "memory"); }

template <typename TF>
__global__ void __launch_bounds__(kDiagThreads) front_diag_kernel(const int32_t *__restrict__ tasks,
                                                                  const DFront *__restrict__ fronts,
                                                                  TF *__restrict__ F, TF *__restrict__ Y,
                                                                  double *__restrict__ D,
                                                                  double *__restrict__ Dinv, int *flags,
                                                                  __nv_bfloat16 *__restrict__ by) {
  constexpr bool kDF = sizeof(TF) == 4;
  constexpr unsigned kAll = 0xffffffffu;
  extern __shared__ __align__(16) unsigned char dsm_raw[];
  TF(*S)[kDP] = reinterpret_cast<TF(*)[kDP]>(dsm_raw);  // input, then W (lower) and the TF pivots
  TF(*Lsc)[kDP] = S + 64;                               // L = W / d (TF pivots), strictly lower
  TF(*X)[kDP] = S + 128;                                // L^{-1}, lower blocks
  TF(*T)[16][17] = reinterpret_cast<TF(*)[16][17]>(S + 192);
  TF *pinv = reinterpret_cast<TF *>(T + 3);
  double *dg = reinterpret_cast<double *>(pinv + 64);  // [64] FP64 pivots, or DF pivots
  double *s_inv = dg + 64;                             // [64] FP64 inverses, or DF inverses
  DF *dgf = reinterpret_cast<DF *>(dg);
  DF *s_invf = reinterpret_cast<DF *>(s_inv);
  __shared__ int s_done;  // columns [0, s_done) of S hold their final values
  pdl_launch_dependents();
  const int4 t = reinterpret_cast<const int4 *>(tasks)[blockIdx.x];
  const DFront fr = fronts[t.x];
  const int32_t k0 = t.y & 0xffffff, kb = t.z;
  const int nsb = (kb + 15) >> 4, n16 = 16 * nsb;
  TF *Ff = F + fr.f_off;
  pdl_wait();
  {  // all of a thread's loads of the block in flight before its stores
    constexpr int kPer = (64 * 64 + kDiagThreads - 1) / kDiagThreads;
    TF v[kPer];
#pragma unroll
    for (int k = 0; k < kPer; ++k) {
      const int idx = threadIdx.x + k * kDiagThreads, i = idx % 64, j = idx / 64;
      v[k] = (idx < 64 * 64 && i < kb && j < kb && i >= j) ? Ff[(k0 + i) + int64_t(k0 + j) * fr.ldf] : TF(0);
    }
#pragma unroll
    for (int k = 0; k < kPer; ++k) {
      const int idx = threadIdx.x + k * kDiagThreads;
      if (idx < 64 * 64) S[idx % 64][idx / 64] = v[k];
      if (idx < 64 * 64 && idx % 64 == idx / 64) dg[idx % 64] = double(v[k]);  // the pivot warp's start
    }
  }
  if (threadIdx.x == 0) s_done = 0;
  __syncthreads();
  // the elimination's own pivots (the stored D comes from the pivot warp):
  // the fast reciprocal for FP32
  auto safe_inv = [](TF d) {
    if constexpr (sizeof(TF) == 4)
      return d > TF(0) ? __fdividef(1.f, d) : TF(1);
    else
      return d > TF(0) ? TF(1) / d : TF(1);
  };
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  // the pivot warp is warp 1, so that it shares no SM sub-partition with
  // warp 0, which runs the elimination's serial step A
  if (warp == 1) {
    // ------------------------------------------------------- pivot warp
    // lane l keeps rows l and l + 32 in double-float (FP32 factor) or FP64
    DF p0 = {1.f, 0.f}, p1 = {1.f, 0.f};
    double q0 = 1.0, q1 = 1.0;
    // (from the copy of the input diagonal: the elimination overwrites S's)
    if constexpr (kDF) {
      if (lane < kb) p0 = {float(dg[lane]), 0.f};
      if (lane + 32 < kb) p1 = {float(dg[lane + 32]), 0.f};
    } else {
      if (lane < kb) q0 = dg[lane];
      if (lane + 32 < kb) q1 = dg[lane + 32];
    }
    for (int sb = 0; sb < nsb; ++sb) {
      const int b0 = 16 * sb, b1 = b0 + 16;
      int late = 0;
      if (lane == 0) {
        for (int spins = 0; ld_acquire_cta_shared(&s_done) < b1; ++spins)
          if (spins > (1 << 24)) {
            atomicOr(flags, FLAG_WAIT_TIMEOUT);
            late = 1;
            break;
          }
      }
      __syncwarp();
      if (__shfl_sync(kAll, late, 0)) break;
      const int i0 = lane, i1 = lane + 32;
      if constexpr (kDF) {
        // the sub-block's final columns folded into every later row as exact
        // products W_ij L_ij with the elimination's own scaled column L (no
        // pivot waits for an earlier pivot's inverse: only each row's sum is
        // a chain, and the two rows of a lane interleave)
#pragma unroll
        for (int jj = 0; jj < 16; ++jj) {
          const int j = b0 + jj;
          if (j < kb) {  // (warp-uniform)
            const DF n0 = df_sub(p0, df_two_prod(float(S[i0][j]), float(Lsc[i0][j])));
            const DF n1 = df_sub(p1, df_two_prod(float(S[i1][j]), float(Lsc[i1][j])));
            p0 = (i0 > j && i0 < kb) ? n0 : p0;
            p1 = (i1 > j && i1 < kb) ? n1 : p1;
          }
        }
      } else {
        double sq0[16], sq1[16];
#pragma unroll
        for (int jj = 0; jj < 16; ++jj) {
          const double w0 = double(S[i0][b0 + jj]), w1 = double(S[i1][b0 + jj]);
          sq0[jj] = w0 * w0;
          sq1[jj] = w1 * w1;
        }
#pragma unroll
        for (int jj = 0; jj < 16; ++jj) {
          const int j = b0 + jj;
          if (j >= kb) break;
          const double dj = __shfl_sync(kAll, j < 32 ? q0 : q1, j & 31);
          const double inv = pivot_inverse(dj, flags, lane == 0);
          if (lane == 0) s_inv[j] = inv;
          if (i0 > j && i0 < kb) q0 -= sq0[jj] * inv;
          if (i1 > j && i1 < kb) q1 -= sq1[jj] * inv;
        }
      }
    }
    if constexpr (kDF) {
      // the pivots are final: their inverses, all at once (a bad pivot is
      // flagged once; the inverse of a non-positive one is taken of 1)
      const bool bad = (lane < kb && !(p0.hi > 0.f)) || (lane + 32 < kb && !(p1.hi > 0.f));
      if (__any_sync(kAll, bad) && lane == 0) atomicOr(flags, FLAG_PIVOT);
      if (lane < kb) s_invf[lane] = df_pivot_inverse(p0);
      if (lane + 32 < kb) s_invf[lane + 32] = df_pivot_inverse(p1);
      dgf[lane] = p0;
      dgf[lane + 32] = p1;
    } else {
      dg[lane] = q0;
      dg[lane + 32] = q1;
    }
  } else {
    // ------------------------------------------------ elimination warps
    const int ew = warp == 0 ? 0 : warp - 1;  // 0-7
    const int tid = 32 * ew + lane;
    for (int sb = 0; sb < nsb; ++sb) {
      const int b0 = 16 * sb, b1 = b0 + 16;
      if (ew == 0) {
        // A: the 16 x 16 diagonal sub-block (lanes 16-31 mirror 0-15)
        const int l = lane & 15, row = b0 + l;
        const bool own = lane < 16;
        TF r[16];
#pragma unroll
        for (int c = 0; c < 16; ++c) r[c] = S[row][b0 + c];
#pragma unroll
        for (int j = 0; j < 16; ++j) {
          // column j reaches the lanes first (its entries are final), then
          // the pivot's reciprocal, the row's L entry and the updates
          TF wc[16];
#pragma unroll
          for (int c = 1; c < 16; ++c)  // (constant bounds: r stays in registers)
            if (c > j) wc[c] = __shfl_sync(kAll, r[j], c);  // W[b0 + c, b0 + j]
          const TF inv = safe_inv(__shfl_sync(kAll, r[j], j));
          const TF lj = r[j] * inv;  // row's L entry (its W entry r[j] is final)
#pragma unroll
          for (int c = 1; c < 16; ++c)
            if (c > j && l >= c) r[c] -= lj * wc[c];
          if (own && l > j) {
            S[row][b0 + j] = r[j];
            Lsc[row][b0 + j] = lj;
          }
          if (own && l == j) {
            S[row][row] = r[j];
            pinv[row] = inv;
          }
        }
      }
      elim_barrier();
      // B: the rows below, one thread per row
      if (tid < n16 - b1) {
        const int i = b1 + tid;
        TF s[16];
#pragma unroll
        for (int c = 0; c < 16; ++c) s[c] = S[i][b0 + c];
#pragma unroll
        for (int c = 0; c < 16; ++c)
#pragma unroll
          for (int c2 = 1; c2 < 16; ++c2)
            if (c2 > c) s[c2] -= s[c] * Lsc[b0 + c2][b0 + c];
#pragma unroll
        for (int c = 0; c < 16; ++c) {
          S[i][b0 + c] = s[c];
          Lsc[i][b0 + c] = s[c] * pinv[b0 + c];
        }
      }
      elim_barrier();
      if (tid == 0) st_release_cta_shared(&s_done, b1);  // columns < b1 are final in S
      // C: rank-16 update of the sub-blocks below and right of sb
      if (b1 < n16) {
        const int tr = tid >> 4, tc = tid & 15;
        TF acc[4][4];
#pragma unroll
        for (int a = 0; a < 4; ++a)
#pragma unroll
          for (int c = 0; c < 4; ++c)
            acc[a][c] = (c > sb && a >= c && a < nsb) ? S[tr + 16 * a][tc + 16 * c] : TF(0);
#pragma unroll
        for (int j = 0; j < 16; ++j) {
          TF li[4], wc[4];
#pragma unroll
          for (int a = 0; a < 4; ++a) {
            li[a] = (a > sb && a < nsb) ? Lsc[tr + 16 * a][b0 + j] : TF(0);
            wc[a] = (a > sb && a < nsb) ? S[tc + 16 * a][b0 + j] : TF(0);
          }
#pragma unroll
          for (int a = 0; a < 4; ++a)
#pragma unroll
            for (int c = 0; c < 4; ++c)
              if (c <= a) acc[a][c] -= li[a] * wc[c];
        }
#pragma unroll
        for (int a = 0; a < 4; ++a)
#pragma unroll
          for (int c = 0; c < 4; ++c)
            if (c > sb && a >= c && a < nsb) S[tr + 16 * a][tc + 16 * c] = acc[a][c];
      }
      elim_barrier();
    }
    // L^{-1}: the diagonal 16 x 16 inverses (warp w: block w, lane c: column c)
    if (ew < nsb) {
      const int w0 = 16 * ew, c = lane & 15;
      TF x[16];
#pragma unroll
      for (int i = 0; i < 16; ++i) {
        TF acc = i == c ? TF(1) : TF(0);
#pragma unroll
        for (int k = 0; k < 15; ++k)
          if (k < i) acc -= Lsc[w0 + i][w0 + k] * x[k];
        x[i] = acc;
      }
      if (lane < 16) {
#pragma unroll
        for (int i = 0; i < 16; ++i) X[w0 + i][w0 + c] = x[i];
      }
    }
    elim_barrier();
    // then the blocks below the diagonal, one block diagonal o at a time
    const int r = tid >> 4, c = tid & 15;
    for (int o = 1; o < nsb; ++o) {
      for (int bj = 0; bj + o < nsb; ++bj) {
        const int bi = bj + o;
        TF acc = TF(0);
        for (int k = bj; k < bi; ++k)
#pragma unroll
          for (int m = 0; m < 16; ++m) acc += Lsc[16 * bi + r][16 * k + m] * X[16 * k + m][16 * bj + c];
        T[bj][r][c] = acc;
      }
      elim_barrier();
      for (int bj = 0; bj + o < nsb; ++bj) {
        const int bi = bj + o;
        TF acc = TF(0);
#pragma unroll
        for (int m = 0; m < 16; ++m) acc += X[16 * bi + r][16 * bi + m] * T[bj][m][c];
        X[16 * bi + r][16 * bj + c] = -acc;
      }
      elim_barrier();
    }
  }
  __syncthreads();
  if (threadIdx.x < kb) {
    double d, dinv;
    if constexpr (kDF) {
      d = double(dgf[threadIdx.x].hi) + double(dgf[threadIdx.x].lo);
      dinv = double(s_invf[threadIdx.x].hi) + double(s_invf[threadIdx.x].lo);
    } else {
      d = dg[threadIdx.x];
      dinv = s_inv[threadIdx.x];
    }
    if (!(d > 0.0)) d = 1.0;
    D[fr.first + k0 + threadIdx.x] = d;
    Dinv[fr.first + k0 + threadIdx.x] = dinv;
  }
  TF *Yf = Y + fr.y_off;
  if (by) {
    // the BF16 copy's chunk of this panel is zero in the columns of the
    // superpanel's later panels (Y's upper triangle there): the copy is
    // reused by every superpanel and factorisation, and those positions may
    // hold another superpanel's values.  Then the panel's own columns,
    // L_KK^{-1} column j with all 64 rows of the chunk (zeros past kb); both
    // as 16-byte stores of eight BF16.
    const int32_t s1 = min((k0 / kSuper + 1) * kSuper, fr.npiv);
    const int ncol = s1 - (k0 + kb);
    for (int idx = threadIdx.x; idx < 8 * ncol; idx += blockDim.x)
      *reinterpret_cast<uint4 *>(by + (int64_t(fr.first) + k0 + kb + idx / 8) * kSuper + (k0 % kSuper) +
                                 8 * (idx & 7)) = make_uint4(0u, 0u, 0u, 0u);
    for (int idx = threadIdx.x; idx < 8 * kb; idx += blockDim.x) {
      const int j = idx >> 3, ib = 8 * (idx & 7);
      __align__(16) __nv_bfloat16 v[8];
#pragma unroll
      for (int e = 0; e < 8; ++e) {
        const int i = ib + e;
        v[e] = __float2bfloat16_rn(i >= kb ? 0.f : float(i > j ? X[i][j] : (i == j ? TF(1) : TF(0))));
      }
      *reinterpret_cast<uint4 *>(by + (int64_t(fr.first) + k0 + j) * kSuper + (k0 % kSuper) + ib) =
          *reinterpret_cast<const uint4 *>(v);
    }
  }
  for (int idx = threadIdx.x; idx < 64 * 64; idx += blockDim.x) {
    const int i = idx & 63, j = idx >> 6;
    if (i >= kb || j >= kb) continue;
    TF sc;
    if constexpr (kDF)
      sc = s_invf[j].hi;
    else
      sc = TF(s_inv[j]);
    if (i > j) Ff[(k0 + i) + int64_t(k0 + j) * fr.ldf] = S[i][j] * sc;
    Yf[(k0 + i) + int64_t(k0 + j) * fr.ldy] = i > j ? X[i][j] : (i == j ? TF(1) : TF(0));
  }
}

// ------------------------------------------------------- panel and X_K
// row pitch (BF16 entries) of the staged copy tiles: 144-byte rows keep the
// 16-byte row chunks aligned and spread a warp's scalar stores over banks
constexpr int kPanelStage = 72;
// PANEL (front, k0, r0): rows [r0, r0+64) of the panel: L = F L_KK^{-T} D^{-1}.
// XK    (front, k0, c0): Y[K, c0:c0+64] <- L_KK^{-1} Y[K, c0:c0+64].
// With the BF16 superpanel ends (bw non-null), both also write their results
// into the K-major BF16 copies of the superpanel, at column k0 - s0 of the
// kSuper: PANEL the rows of W = F L_KK^{-T} (bw) and of L (bl), XK the pivot rows
// of Y as row first + c of by; the 64 columns of a panel's chunk are written
// whole (zeros past the panel's kb pivots), so the last, partial chunk of a
// superpanel adds nothing.
template <typename TF>
__global__ void __launch_bounds__(256) front_panel_kernel(const int32_t *__restrict__ tasks,
                                                          const DFront *__restrict__ fronts,
                                                          TF *__restrict__ F, TF *__restrict__ Y,
                                                          const double *__restrict__ Dinv,
                                                          __nv_bfloat16 *__restrict__ bw,
                                                          __nv_bfloat16 *__restrict__ bl,
                                                          __nv_bfloat16 *__restrict__ by) {
  extern __shared__ __align__(16) unsigned char psm[];
  TF(*Ls)[65] = reinterpret_cast<TF(*)[65]>(psm);
  TF(*Bs)[65] = reinterpret_cast<TF(*)[65]>(psm + 64 * 65 * sizeof(TF));
  pdl_launch_dependents();
  const int4 t = reinterpret_cast<const int4 *>(tasks)[blockIdx.x];
  const DFront fr = fronts[t.x];
  const int kind = t.y >> 24;
  const int32_t k0 = t.y & 0xffffff, a0 = t.z, m = fr.m;
  const int32_t kb = (fr.npiv - k0) < 64 ? (fr.npiv - k0) : 64;
  TF *Ff = F + fr.f_off;
  TF *Yf = Y + fr.y_off;
  pdl_wait();
  for (int idx = threadIdx.x; idx < 64 * 64; idx += blockDim.x) {
    const int i = idx % 64, j = idx / 64;
    Ls[i][j] = (i < kb && j < kb && i >= j) ? Yf[(k0 + i) + int64_t(k0 + j) * fr.ldy] : TF(0);
  }
  const int tr = threadIdx.x / 16, tc = threadIdx.x % 16;
  if (kind == T_PANEL) {
    for (int idx = threadIdx.x; idx < 64 * 64; idx += blockDim.x) {
      const int i = idx % 64, j = idx / 64;
      const int32_t r = a0 + i;
      Bs[i][j] = (r < m && j < kb) ? Ff[r + int64_t(k0 + j) * fr.ldf] : TF(0);
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
    TF di[4];
#pragma unroll
    for (int s = 0; s < 4; ++s) {
      const int c = tc + 16 * s;
      di[s] = c < kb ? TF(Dinv[fr.first + k0 + c]) : TF(0);
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int32_t r = a0 + tr * 4 + u;
        if (r < m && c < kb) Ff[r + int64_t(k0 + c) * fr.ldf] = acc[u][s] * di[s];
      }
    }
    if (bw) {
      // the rows of the BF16 copies, staged so that each row's 64 columns
      // (128 bytes) leave as eight 16-byte stores
      __syncthreads();
      __nv_bfloat16(*tw)[kPanelStage] = reinterpret_cast<__nv_bfloat16(*)[kPanelStage]>(psm);
      __nv_bfloat16(*tl)[kPanelStage] = tw + 64;
#pragma unroll
      for (int s = 0; s < 4; ++s)
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          tw[tr * 4 + u][tc + 16 * s] = __float2bfloat16_rn(float(acc[u][s]));
          tl[tr * 4 + u][tc + 16 * s] = __float2bfloat16_rn(float(acc[u][s] * di[s]));
        }
      __syncthreads();
      for (int idx = threadIdx.x; idx < 2 * 64 * 8; idx += blockDim.x) {
        const int h = idx >> 9, row = (idx >> 3) & 63, ch = idx & 7;
        const int32_t r = a0 + row;
        if (r >= m) continue;
        const uint4 v = *reinterpret_cast<const uint4 *>((h ? tl : tw)[row] + 8 * ch);
        __nv_bfloat16 *dst = (h ? bl : bw) + (fr.w_off + r) * int64_t(kSuper) + (k0 % kSuper) + 8 * ch;
        *reinterpret_cast<uint4 *>(dst) = v;
      }
    }
  } else {  // T_XK
    for (int idx = threadIdx.x; idx < 64 * 64; idx += blockDim.x) {
      const int j = idx % 64, c = idx / 64;
      Bs[j][c] = (j < kb && a0 + c < k0) ? Yf[(k0 + j) + int64_t(a0 + c) * fr.ldy] : TF(0);
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
#pragma unroll
      for (int s = 0; s < 4; ++s) {
        const int32_t c = a0 + tc + 16 * s;
        if (c < k0 && i < kb) Yf[(k0 + i) + int64_t(c) * fr.ldy] = acc[u][s];
      }
    }
    if (by) {
      // the pivot rows of Y in the BF16 copy: per column c its 64 entries
      // (128 bytes), staged and written as eight 16-byte stores
      __syncthreads();
      __nv_bfloat16(*ty)[kPanelStage] = reinterpret_cast<__nv_bfloat16(*)[kPanelStage]>(psm);
#pragma unroll
      for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int s = 0; s < 4; ++s) ty[tc + 16 * s][tr * 4 + u] = __float2bfloat16_rn(float(acc[u][s]));
      __syncthreads();
      for (int idx = threadIdx.x; idx < 64 * 8; idx += blockDim.x) {
        const int col = idx >> 3, ch = idx & 7;
        const int32_t c = a0 + col;
        if (c >= k0) continue;
        const uint4 v = *reinterpret_cast<const uint4 *>(ty[col] + 8 * ch);
        *reinterpret_cast<uint4 *>(by + (int64_t(fr.first) + c) * kSuper + (k0 % kSuper) + 8 * ch) = v;
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
  pdl_launch_dependents();
  const int4 t = reinterpret_cast<const int4 *>(tasks)[blockIdx.x];
  const DFront fr = fronts[t.x];
  const int kind = t.y >> 24;
  const int32_t k0 = t.y & 0xffffff, i0 = t.z, j0 = t.w, m = fr.m;
  const int32_t kb = (fr.npiv - k0) < 64 ? (fr.npiv - k0) : 64;
  TF *Ff = F + fr.f_off;
  TF *Yf = Y + fr.y_off;
  pdl_wait();
  for (int idx = threadIdx.x; idx < 64 * 64; idx += blockDim.x) {
    const int i = idx % 64, l = idx / 64;
    const int32_t r = i0 + i;
    As[i][l] = (r < m && l < kb) ? Ff[r + int64_t(k0 + l) * fr.ldf] : TF(0);
  }
  if (kind == T_TRAIL) {
    for (int idx = threadIdx.x; idx < 64 * 64; idx += blockDim.x) {
      const int j = idx % 64, l = idx / 64;
      const int32_t r = j0 + j;
      Bs[j][l] = (r < m && l < kb) ? Ff[r + int64_t(k0 + l) * fr.ldf] * TF(D[fr.first + k0 + l]) : TF(0);
    }
  } else {
    for (int idx = threadIdx.x; idx < 64 * 64; idx += blockDim.x) {
      const int l = idx % 64, j = idx / 64;
      const int32_t c = j0 + j;
      Bs[j][l] = (l < kb && c < k0 + kb) ? Yf[(k0 + l) + int64_t(c) * fr.ldy] : TF(0);
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
        if (r < m && r >= c) Ff[r + int64_t(c) * fr.ldf] -= acc[u][s];
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
        if (r < m) Yf[r + int64_t(c) * fr.ldy] -= acc[u][s];
      }
    }
  }
}

// FP32 trailing updates on the tensor cores.  Task (front, kind | chunks, i0,
// j0) updates a 128 x 128 tile with the rank-K product of the factor columns
// [k0, k0 + K), K = 64 x chunks <= kSuper:
//   TRAIL  F[i, j] -= sum_l L[i, l] d_l L[j, l]    (lower part, r >= c)
//   RUPD   Y[i, c] -= sum_l L[i, l] Y[l, c]         (c < k0 + K)
// A task whose K range ends before the end of its superpanel (kSuper
// columns) is an eager one: it updates only the columns (TRAIL) or rows
// (RUPD) that are still inside the superpanel, and only those inside its
// sub-block (kSub columns) when its K range also ends before the
// sub-block's end.  A sub-block's last panel step applies the sub-block
// (K = kSub) to the rest of the superpanel, and the superpanel's last panel
// step applies the whole superpanel at once (K up to kSuper) to the rest of
// the front, so the trailing matrix is read and written once per kSuper
// pivots instead of once per 64, and the superpanel's own columns once per
// kSub.
//
// Blackwell tensor cores (tcgen05, kind::tf32) with a 3xTF32 split
// (a = a_hi + a_lo, a b ~ a_hi b_hi + a_hi b_lo + a_lo b_hi) so products keep
// ~FP32 accuracy, fed by the TMA unit, with warp-specialised roles (320
// threads):
//  * warp 9, producer: keeps a ring of 5-6 raw K chunks (16 columns each)
//    in flight: per chunk one tensor-map load of the 128 x 16 A tile (F rows
//    i0.., columns k..k + 16, rows contiguous) and either the 128 x 16 B
//    tile of F (TRAIL) or four 4 x 128 boxes of Y (RUPD: pivot rows k.. of
//    columns j0.., which land directly in the operand layout), plus the
//    chunk's d_l (loaded one chunk ahead), completing on the stage's full
//    mbarrier; a stage is refilled once the eight converter warps have
//    arrived on its empty mbarrier;
//  * warps 0-3, A converters: each thread owns one row (the warp's lane
//    quarter of tensor memory), reads its 16 raw values (consecutive rows
//    across a warp: no bank conflicts), scales them by d_l (TRAIL), splits
//    them into TF32 high and low parts and writes both into tensor memory
//    with two tcgen05.st (columns 128 + 32 stage);
//  * warps 4-7, B converters: the same split for B (columns at or past the
//    task's K end zeroed), stored as 16-byte vectors into one of two
//    shared-memory operand stages in the K-major, no-swizzle core-matrix
//    layout (8 rows x 16 bytes per core matrix; 128 B between 8-row groups,
//    2048 B between 4-column K groups), so the conversion of chunk q
//    overlaps the MMAs of chunk q - 1;
//  * warp 8, MMA issuer: once all eight converter warps have arrived on a
//    stage's ready mbarrier, one lane issues the chunk's MMAs (A from tensor
//    memory, B from shared memory, M = N = 128, K = 8 each) into a 128 x 128
//    FP32 accumulator in tensor memory and commits them to the operand
//    stage's mbarrier.
// Epilogue: once the last MMAs have completed, warps 0-7 read the
// accumulator with tcgen05.ld (warp w: lanes 32 (w % 4) .., columns
// 64 (w / 4) ..) and stage its negative (0 outside the task's range) in the
// freed shared memory, and one thread adds the staged 128 x 128 tile to F
// or Y with eight TMA reduce-add boxes (each entry receives exactly one
// addition per launch: deterministic).  Every mbarrier wait is bounded in
// time and gives up at once when another thread of the CTA has given up (a
// shared abort word); the CTA then raises FLAG_WAIT_TIMEOUT, waits (bounded)
// for the copies and MMAs it has in flight, frees its tensor memory and
// returns.
constexpr int kT128 = 128;
constexpr int kUK = 16;                              // K columns per chunk
constexpr int kUOpBytes = kT128 * kUK * 4;           // one operand of one chunk: 8 KB
constexpr int kUThreads = 320;  // 8 converter/epilogue warps, 1 MMA-issuer warp, 1 TMA-producer warp
constexpr int kUmmaLbo = 2048;                       // K-direction core-matrix stride
constexpr int kUmmaSbo = 128;                        // M/N-direction (8-row group) stride
// raw ring (A and B per stage) + two operand stages (hi and lo parts of A
// and B, or the TF32 parts alone) + d_l per raw stage + mbarriers/TMEM slot:
// 112.3 KB for 3xTF32, so that two CTAs fit on an SM (228 KB, 1 KB reserved
// per CTA).  The staged output tile of the epilogue (64 KB) reuses the front.
template <int NMMA>
__host__ __device__ constexpr int update_nop() { return NMMA == 3 ? 2 : 1; }  // B operands in shared memory
// operand stages (the A parts of a stage live in tensor memory) and raw
// stages (the TMA ring): with A out of shared memory the space goes to raw
// chunks in flight, which hide the TMA latency under load (≈ 2-3 µs)
template <int NMMA>
__host__ __device__ constexpr int update_nops() { return 2; }
template <int NMMA>
__host__ __device__ constexpr int update_nrs() { return NMMA == 3 ? 5 : 6; }
constexpr int kUTmemCols = 256;  // accumulator [0, 128) + A of 4 stages (hi, lo: 16 columns each)
constexpr int kUDqOff(int nrs, int nop, int nops) { return nrs * 2 * kUOpBytes + nops * nop * kUOpBytes; }
template <int NMMA>
constexpr size_t update_smem() {
  return size_t(kUDqOff(update_nrs<NMMA>(), update_nop<NMMA>(), update_nops<NMMA>())) + update_nrs<NMMA>() * kUK * 4 +
         256;
}
static_assert(5 * 2 * kUOpBytes >= kT128 * kT128 * 4, "the output tile fits the raw ring");
constexpr uint64_t kWaitLimitNs = 1000000000ull;     // give up an mbarrier wait after 1 s

// tcgen05 instruction descriptor, kind::tf32: D F32 (bits 4-5 = 1), A and B
// TF32 (bits 7-9, 10-12 = 2), both K-major, N >> 3 at bit 17, M >> 4 at bit 24.
constexpr uint32_t kIdescTf32 = (1u << 4) | (2u << 7) | (2u << 10) | (uint32_t(kT128 >> 3) << 17) |
                                (uint32_t(kT128 >> 4) << 24);

__device__ __forceinline__ uint64_t umma_desc(uint32_t saddr) {
  // start address >> 4 (bits 0-13), LBO >> 4 (16-29), SBO >> 4 (32-45),
  // fixed 0b001 at bits 46-48, no swizzle (bits 61-63 = 0)
  return uint64_t((saddr & 0x3FFFFu) >> 4) | (uint64_t(kUmmaLbo >> 4) << 16) | (uint64_t(kUmmaSbo >> 4) << 32) |
         (uint64_t(1) << 46);
}

// TF32 parts by integer arithmetic on the FP32 bit pattern (full-rate ALU
// instead of conversions): the high part rounds the 10-bit mantissa to
// nearest (ties away from zero: add half a unit of the 13 dropped bits,
// then clear them; a carry into the exponent is the correct rounding), the
// low part x - hi is exact in FP32 and is truncated to TF32 (error at most
// 2^-10 of it, i.e. ~2^-21 of x).
__device__ __forceinline__ uint32_t tf32_hi(float x) { return (__float_as_uint(x) + 0x1000u) & 0xffffe000u; }
__device__ __forceinline__ uint32_t tf32_lo(float x, uint32_t hi) {
  return __float_as_uint(x - __uint_as_float(hi)) & 0xffffe000u;
}

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ uint64_t global_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %globaltimer;\n" : "=l"(t));
  return t;
}

// Bounded wait on the mbarrier phase with the given parity; false if the
// limit ran out or (when given) the abort word is set.
__device__ __forceinline__ bool mbar_try(uint32_t bar, uint32_t parity) {
  uint32_t done;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(done)
      : "r"(bar), "r"(parity)
      : "memory");
  return done != 0;
}
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity, const volatile int *abort_word = nullptr) {
  if (mbar_try(bar, parity)) return true;  // (the timer is read only when the phase is still open)
  const uint64_t t0 = global_ns();
  for (;;) {
    if (mbar_try(bar, parity)) return true;
    if ((abort_word && *abort_word) || global_ns() - t0 > kWaitLimitNs) return false;
  }
}

// 2-D tensor-map load into shared memory, completing on an mbarrier
__device__ __forceinline__ void tma_load_2d(uint32_t dst, const void *map, int32_t x, int32_t y, uint32_t bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];\n" ::"r"(
          dst),
      "l"(map), "r"(x), "r"(y), "r"(bar)
      : "memory");
}

// 2-D tensor-map reduce-add of one box from shared memory into global
// memory (FP32 additions performed in L2; bulk async group)
__device__ __forceinline__ void tma_reduce_add_2d(const void *map, int32_t x, int32_t y, uint32_t src) {
  asm volatile("cp.reduce.async.bulk.tensor.2d.global.shared::cta.add.tile.bulk_group [%0, {%1, %2}], [%3];\n" ::"l"(
                   map),
               "r"(x), "r"(y), "r"(src)
               : "memory");
}

// 16 consecutive 32-bit tensor-memory columns of the calling thread's lane
// (warp w writes lanes 32 (w % 4) ..), from registers
__device__ __forceinline__ void tmem_st16(uint32_t taddr, const uint32_t (&v)[16]) {
  asm volatile(
      "tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16};\n" ::"r"(
          taddr),
      "r"(v[0]), "r"(v[1]), "r"(v[2]), "r"(v[3]), "r"(v[4]), "r"(v[5]), "r"(v[6]), "r"(v[7]), "r"(v[8]), "r"(v[9]),
      "r"(v[10]), "r"(v[11]), "r"(v[12]), "r"(v[13]), "r"(v[14]), "r"(v[15])
      : "memory");
}

// NMMA = 3: the 3xTF32 split (FP32-accurate products); NMMA = 1: one TF32
// MMA per product (operands rounded to TF32, ~1e-3 relative; the factor is
// only a preconditioner and the solve is refined in FP64).
template <int NMMA>
__global__ void __launch_bounds__(kUThreads, 2) front_update_tc_kernel(
    const int32_t *__restrict__ tasks, const DFront *__restrict__ fronts, float *__restrict__ F,
    float *__restrict__ Y, const double *__restrict__ D, const CUtensorMap *__restrict__ fmaps,
    const CUtensorMap *__restrict__ ymaps, const CUtensorMap *__restrict__ ycmaps, int *flags) {
  static_assert(NMMA == 1 || NMMA == 3, "3xTF32 or TF32");
  constexpr int NOP = update_nop<NMMA>();
  constexpr int NOS = update_nops<NMMA>();  // operand stages
  constexpr int OPF = kUOpBytes / 4;  // floats per operand chunk
  extern __shared__ __align__(1024) unsigned char usm[];
  constexpr int NRS = update_nrs<NMMA>();  // raw stages
  unsigned char *raw = usm;                                            // NRS x (A, B)
  unsigned char *opnd = usm + NRS * 2 * kUOpBytes;                     // NOS x NOP operands
  float *Dq = reinterpret_cast<float *>(usm + kUDqOff(NRS, NOP, NOS));  // d_l of each raw stage
  uint64_t *bars = reinterpret_cast<uint64_t *>(Dq + NRS * kUK);  // full[NRS], empty[NRS], ready[NOS], mma[NOS]
  uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(bars + 2 * NRS + 2 * NOS);
  int &s_abort = *reinterpret_cast<int *>(tmem_slot + 1);  // (dynamic: no static shared memory)
  const volatile int *abort_word = &s_abort;
  pdl_launch_dependents();
  const int4 t = reinterpret_cast<const int4 *>(tasks)[blockIdx.x];
  const DFront fr = fronts[t.x];
  const int kind = (t.y >> 24) & 7;
  const int chunks = ((t.y >> 27) & 7) + 1;
  const int32_t k0 = t.y & 0xffffff, i0 = t.z, j0 = t.w, m = fr.m, p = fr.npiv;
  const int32_t kend = min(k0 + 64 * chunks, p);
  const int32_t kw = kend - k0;
  const int32_t s_end = min((k0 / kSuper + 1) * kSuper, p);
  const int32_t b_end = min((k0 / kSub + 1) * kSub, s_end);
  const bool eager = kend < s_end;
  const int32_t e_end = kend < b_end ? b_end : s_end;  // an eager task's column (row) bound
  // TRAIL writes the lower part of columns < cmax (the sub-block's or the
  // superpanel's end for an eager task), RUPD rows < rmax of columns < kend;
  // a delayed task's tile may start below the superpanel's end (its origin is
  // rounded down to a multiple of 4), and those rows and columns are not
  // touched
  const int32_t cmax = kind == T_TRAIL ? (eager ? e_end : m) : kend;
  const int32_t rmax = (kind != T_TRAIL && eager) ? e_end : m;
  const int32_t lo = eager ? 0 : s_end;
  const bool trail = kind == T_TRAIL;
  const CUtensorMap *mapA = fmaps + t.x;
  const CUtensorMap *mapB = trail ? fmaps + t.x : ymaps + t.x;
  const CUtensorMap *mapC = trail ? fmaps + t.x : ycmaps + t.x;  // the output tile (F or all rows of Y)
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int nq = (kw + kUK - 1) / kUK;
  const uint32_t bar_full = smem_u32(bars), bar_empty = bar_full + 8 * NRS, bar_ready = bar_empty + 8 * NRS;
  const uint32_t bar_mma = bar_ready + 8 * NOS;
  const uint32_t raw_u = smem_u32(raw), op_u = smem_u32(opnd);
  pdl_wait();
  if (threadIdx.x == 0) {
    s_abort = 0;
    for (int b = 0; b < NRS; ++b) {
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(bar_full + 8 * b) : "memory");
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 8;\n" ::"r"(bar_empty + 8 * b) : "memory");  // 8 warps
    }
    for (int b = 0; b < NOS; ++b) {
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 8;\n" ::"r"(bar_ready + 8 * b) : "memory");  // 8 warps
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(bar_mma + 8 * b) : "memory");
    }
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(smem_u32(tmem_slot)),
                 "r"(kUTmemCols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
  const uint32_t tmem = *tmem_slot;
  bool ok = true;
  int issued = 0, mma_issued = 0;  // warp 9 (copies issued) and warp 8 (MMA chunks issued)

  if (warp == 9) {
    // ------------------------------------------------------------ producer
    // raw chunk q into stage q % NRS once the converters have released the
    // stage (its previous chunk): d_l (lanes 0-15, loaded one chunk ahead),
    // then the expected bytes and the TMA loads (lane 0); the stage's
    // mbarrier completes once the loads have landed and lane 0 has arrived
    auto load_d = [&](int q) {
      const int32_t kq = k0 + kUK * q;
      return (q < nq && lane < kUK && trail && kq + lane < kend) ? float(D[fr.first + kq + lane]) : 0.f;
    };
    float dv_next = load_d(0);
    for (int q = 0; q < nq && ok; ++q) {
      const int s = q % NRS;
      const int32_t kq = k0 + kUK * q;
      const uint32_t bar = bar_full + 8 * s;
      if (q >= NRS) {
        if (lane == 0) ok = mbar_wait(bar_empty + 8 * s, uint32_t((q - NRS) / NRS) & 1u, abort_word);
        ok = __shfl_sync(0xffffffffu, ok ? 1 : 0, 0) != 0;
        if (!ok) break;
      }
      const float dv = dv_next;
      dv_next = load_d(q + 1);
      if (lane == 0) {
        asm volatile("mbarrier.expect_tx.relaxed.cta.shared::cta.b64 [%0], %1;\n" ::"r"(bar), "r"(2 * kUOpBytes)
                     : "memory");
        const uint32_t dA = raw_u + uint32_t(s) * 2 * kUOpBytes, dB = dA + kUOpBytes;
        tma_load_2d(dA, mapA, i0, kq, bar);
        if (trail) {
          tma_load_2d(dB, mapB, j0, kq, bar);
        } else {
#pragma unroll
          for (int g = 0; g < 4; ++g) tma_load_2d(dB + uint32_t(g) * (kUOpBytes / 4), mapB, kq + 4 * g, j0, bar);
        }
      }
      if (lane < kUK) Dq[s * kUK + lane] = dv;
      __syncwarp();
      if (lane == 0) asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];\n" ::"r"(bar) : "memory");
      issued = q + 1;
    }
  } else if (warp == 8) {
    // ---------------------------------------------------------- MMA issuer
    for (int q = 0; q < nq && ok; ++q) {
      const int o = q % NOS;
      if (lane == 0) ok = mbar_wait(bar_ready + 8 * o, uint32_t(q / NOS) & 1u, abort_word);
      ok = __shfl_sync(0xffffffffu, ok ? 1 : 0, 0) != 0;
      if (!ok) break;
      if (lane == 0) {
        asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
        // A (hi, lo) in tensor memory, columns 128 + 32 o (+ 16 for lo);
        // B (hi, lo) in shared memory
        const uint32_t ah = tmem + 128u + 32u * uint32_t(o), al = ah + 16u;
        const uint32_t bh = op_u + uint32_t(o) * NOP * kUOpBytes, bl = bh + kUOpBytes;
#pragma unroll
        for (int s = 0; s < kUK / 8; ++s) {
          const uint32_t ko = uint32_t(s) * 2 * kUmmaLbo;  // two K groups of 4 per MMA
          const uint32_t ka = uint32_t(s) * 8u;             // 8 K columns of A per MMA
          const uint32_t acc0 = (q > 0 || s > 0) ? 1u : 0u;
          if constexpr (NMMA == 3) {
            asm volatile(
                "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
                " tcgen05.mma.cta_group::1.kind::tf32 [%0], [%1], %2, %3, p;\n}\n" ::"r"(tmem),
                "r"(al + ka), "l"(umma_desc(bh + ko)), "r"(kIdescTf32), "r"(acc0)
                : "memory");
            asm volatile("tcgen05.mma.cta_group::1.kind::tf32 [%0], [%1], %2, %3, 1;\n" ::"r"(tmem), "r"(ah + ka),
                         "l"(umma_desc(bl + ko)), "r"(kIdescTf32)
                         : "memory");
            asm volatile("tcgen05.mma.cta_group::1.kind::tf32 [%0], [%1], %2, %3, 1;\n" ::"r"(tmem), "r"(ah + ka),
                         "l"(umma_desc(bh + ko)), "r"(kIdescTf32)
                         : "memory");
          } else {
            asm volatile(
                "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
                " tcgen05.mma.cta_group::1.kind::tf32 [%0], [%1], %2, %3, p;\n}\n" ::"r"(tmem),
                "r"(ah + ka), "l"(umma_desc(bh + ko)), "r"(kIdescTf32), "r"(acc0)
                : "memory");
            (void)al;
            (void)bl;
          }
        }
        asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(
                         bar_mma + 8 * o)
                     : "memory");
      }
      mma_issued = q + 1;
    }
  } else {
    // ------------------------------------------------------- converters
    // warps 0-3: A of rows 32 w + lane into tensor memory (the warp's own
    // lane quarter); warps 4-7: B of rows 32 (w - 4) + lane into shared memory
    const bool a_side = warp < 4;
    const int row = 32 * (warp & 3) + lane;
    for (int q = 0; q < nq && ok; ++q) {
      const int s = q % NRS, o = q % NOS;
      ok = mbar_wait(bar_full + 8 * s, uint32_t(q / NRS) & 1u, abort_word);
      // the MMAs of chunk q - NOS have read operand stage o
      if (ok && q >= NOS) ok = mbar_wait(bar_mma + 8 * o, uint32_t((q - NOS) / NOS) & 1u, abort_word);
      if (!ok) break;
      const float *rA = reinterpret_cast<const float *>(raw + s * 2 * kUOpBytes);
      const float *rB = rA + OPF;
      const int kl0 = kUK * q;  // local column of the chunk's first entry
      const float *dq = Dq + s * kUK;
      if (a_side) {
        // A carries the d_l scaling of TRAIL (C -= (A D) B^T): the A side has
        // the lighter conversion (its parts go to tensor memory in two stores)
        float a[kUK];
#pragma unroll
        for (int k = 0; k < kUK; ++k) a[k] = rA[k * kT128 + row];  // raw A: [k][row]
#pragma unroll
        for (int k = 0; k < kUK; ++k) a[k] = kl0 + k < kw ? (trail ? a[k] * dq[k] : a[k]) : 0.f;
        uint32_t h[kUK];
#pragma unroll
        for (int k = 0; k < kUK; ++k) h[k] = tf32_hi(a[k]);
        const uint32_t ta = tmem + (uint32_t(32 * warp) << 16) + 128u + 32u * uint32_t(o);
        tmem_st16(ta, h);
        if constexpr (NMMA == 3) {
          uint32_t l[kUK];
#pragma unroll
          for (int k = 0; k < kUK; ++k) l[k] = tf32_lo(a[k], h[k]);
          tmem_st16(ta + 16u, l);
        }
        asm volatile("tcgen05.wait::st.sync.aligned;\n" ::: "memory");
        asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
      } else {
        float *ob = reinterpret_cast<float *>(opnd + o * NOP * kUOpBytes);
        // all 16 loads of the row before any store (the raw and operand
        // buffers could alias as far as the compiler knows)
        float b[kUK];
        if (trail) {
#pragma unroll
          for (int k = 0; k < kUK; ++k) b[k] = rB[k * kT128 + row];  // raw B: [k][row]
        } else {  // raw B: [g][row][4], already the operand layout
#pragma unroll
          for (int g = 0; g < 4; ++g) {
            const float4 v = *reinterpret_cast<const float4 *>(rB + g * (OPF / 4) + 4 * row);
            b[4 * g] = v.x; b[4 * g + 1] = v.y; b[4 * g + 2] = v.z; b[4 * g + 3] = v.w;
          }
        }
#pragma unroll
        for (int g = 0; g < 4; ++g) {
          uint32_t bh[4];
#pragma unroll
          for (int i = 0; i < 4; ++i) {
            if (kl0 + 4 * g + i >= kw) b[4 * g + i] = 0.f;
            bh[i] = tf32_hi(b[4 * g + i]);
          }
          const int off = g * (OPF / 4) + 4 * row;  // K group g, row: 16-byte slot
          *reinterpret_cast<uint4 *>(ob + off) = make_uint4(bh[0], bh[1], bh[2], bh[3]);
          if constexpr (NMMA == 3) {
            uint32_t bl[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) bl[i] = tf32_lo(b[4 * g + i], bh[i]);
            *reinterpret_cast<uint4 *>(ob + OPF + off) = make_uint4(bl[0], bl[1], bl[2], bl[3]);
          }
        }
        asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");  // generic-proxy stores -> tensor core
      }
      __syncwarp();
      if (lane == 0) {
        asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];\n" ::"r"(bar_ready + 8 * o) : "memory");
        asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];\n" ::"r"(bar_empty + 8 * s) : "memory");
      }
    }
    // the accumulator is complete (and every operand read: the shared
    // memory is free for the staged tile)
    if (ok && nq > 0) ok = mbar_wait(bar_mma + 8 * ((nq - 1) % NOS), uint32_t((nq - 1) / NOS) & 1u, abort_word);
    asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
    if (ok) {
      const int g = warp & 3, h = warp >> 2;
      const int rl = 32 * g + lane;
      const int32_t r = i0 + rl;
      float *ct = reinterpret_cast<float *>(raw);  // staged tile: [column][row], the TMA box layout
      // this row's columns in range, as tile-local bounds [clo, chi)
      const bool rin = r < rmax && r >= lo;
      const int32_t chi_g = trail ? min(cmax, r + 1) : cmax;
      const int clo = trail ? max(0, lo - j0) : 0;
      const int chi = rin ? max(0, min(kT128, chi_g - j0)) : 0;
      // the warp's 64 accumulator columns in four loads and one wait (each
      // tensor-memory access queues behind MMAs of the SM's other CTA)
      uint32_t v[4][16];
#pragma unroll
      for (int x = 0; x < 4; ++x) {
        const uint32_t ta = tmem + (uint32_t(32 * g) << 16) + uint32_t(64 * h + 16 * x);
        asm volatile(
            "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, "
            "[%16];\n"
            : "=r"(v[x][0]), "=r"(v[x][1]), "=r"(v[x][2]), "=r"(v[x][3]), "=r"(v[x][4]), "=r"(v[x][5]),
              "=r"(v[x][6]), "=r"(v[x][7]), "=r"(v[x][8]), "=r"(v[x][9]), "=r"(v[x][10]), "=r"(v[x][11]),
              "=r"(v[x][12]), "=r"(v[x][13]), "=r"(v[x][14]), "=r"(v[x][15])
            : "r"(ta));
      }
      asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
#pragma unroll
      for (int x = 0; x < 4; ++x) {
#pragma unroll
        for (int e = 0; e < 16; ++e) {
          const int cl = 64 * h + 16 * x + e;
          ct[cl * kT128 + rl] = (cl >= clo && cl < chi) ? -__uint_as_float(v[x][e]) : 0.f;
        }
      }
      asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");  // generic-proxy stores -> TMA
    }
  }
  if (!ok) s_abort = 1;
  ok = __syncthreads_and(ok) != 0;
  if (ok && threadIdx.x == 0) {
    // F (or Y) += the staged tile: TMA reduce-add boxes of 16 columns,
    // clipped to the front (entries outside the task's range add 0); a box
    // whose columns are all outside the range of every row of the tile
    // (TRAIL: at or beyond min(cmax, the tile's last row + 1); RUPD: beyond
    // kend; both: below lo for TRAIL) is left out
    const int32_t c_hi = trail ? min(cmax, min(i0 + kT128, rmax)) : cmax;
    const int32_t c_lo = trail ? lo : 0;
    for (int b = 0; b < 8; ++b) {
      const int32_t cb = j0 + 16 * b;
      if (cb < c_hi && cb + 16 > c_lo) tma_reduce_add_2d(mapC, i0, cb, raw_u + uint32_t(b) * kT128 * 16 * 4);
    }
    asm volatile("cp.async.bulk.commit_group;\n" ::: "memory");
    asm volatile("cp.async.bulk.wait_group 0;\n" ::: "memory");
  }
  // on a timeout: let the copies (warp 9) and MMAs (warp 8) still in flight
  // finish before the shared and tensor memory are given up (each wait bounded)
  if (!ok && warp == 9 && lane == 0) {
    atomicOr(flags, FLAG_WAIT_TIMEOUT);
    for (int q = max(0, issued - NRS); q < issued; ++q)
      mbar_wait(bar_full + 8 * (q % NRS), uint32_t(q / NRS) & 1u);
  }
  if (!ok && warp == 8 && lane == 0) {
    if (mma_issued > 0) mbar_wait(bar_mma + 8 * ((mma_issued - 1) % NOS), uint32_t((mma_issued - 1) / NOS) & 1u);
  }
  asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
  __syncthreads();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem), "r"(kUTmemCols) : "memory");
}

// ------------------------------------------ superpanel ends in BF16
// update_bf16: the deferred update of a superpanel (columns [s0, s1),
// K = s1 - s0 <= kSuper) applied to the rest of the front, task
// (front, kind | chunks, i0, j0) as for front_update_tc_kernel:
//   TRAIL  F[i, j] -= sum_l W[i, l] L[j, l]   (i >= j >= s1, lower part)
//   RUPD   Y[i, c] -= sum_l L[i, l] Y[l, c]   (i >= s1, c < s1)
// with W = L D.  The operands are the K-major BF16 copies of the superpanel
// that the panel and diagonal kernels wrote (Wt, Lt: row w_off + r of the
// front; Yk: row first + c; kSuper BF16 per row), loaded by TMA as 128-row x
// 64-column boxes in the 128-byte-swizzled layout that tcgen05.mma reads
// directly, so no thread touches an operand:
//  * warp 0 (one lane): streams the K chunks (A and B box of 16 KB each)
//    through a two-stage ring, a stage refilled once the MMAs that read it
//    have completed;
//  * warp 1: allocates the tensor memory; one lane issues four
//    tcgen05.mma.kind::f16 (BF16 x BF16, M = N = 128, K = 16) per chunk into
//    a 128 x 128 FP32 accumulator and commits each chunk to its stage's
//    empty mbarrier and the last to the accumulator's;
//  * warps 2-5: read the accumulator (warp w: lanes 32 (w % 4) ..), stage
//    its negative in the freed ring (0 outside the task's rows and columns:
//    rows below s1 or past the front, columns past the superpanel for RUPD,
//    the upper part for TRAIL) and one lane adds it to F or Y with eight TMA
//    reduce-add boxes (each entry receives exactly one addition per launch:
//    deterministic).
// The two stages (64 KB) hold the staged FP32 tile afterwards, so three CTAs
// fit an SM.  Every mbarrier wait is bounded as in front_update_tc_kernel.
constexpr int kBfThreads = 192;
constexpr int kBfBox = 128 * 64 * 2;  // bytes of one operand box
constexpr int kBfStages = 2;
constexpr size_t bf16_update_smem() { return size_t(kBfStages) * 2 * kBfBox + 1024; }  // + alignment slack
static_assert(kBfStages * 2 * kBfBox == 128 * 128 * 4, "the staged output tile fills the ring");

// tcgen05 instruction descriptor, kind::f16: D F32 (bits 4-5 = 1), A and B
// BF16 (bits 7-9, 10-12 = 1), both K-major, N >> 3 at bit 17, M >> 4 at bit 24.
constexpr uint32_t kIdescBf16 = (1u << 4) | (1u << 7) | (1u << 10) | (uint32_t(kT128 >> 3) << 17) |
                                (uint32_t(kT128 >> 4) << 24);

// shared-memory descriptor of a K-major operand in the 128-byte swizzle
// layout (8-row groups of 128-byte rows, 1024 bytes apart): start address
// >> 4 (bits 0-13), leading offset unused (1), stride 1024 >> 4 (bits
// 32-45), fixed 0b001 at bits 46-48, swizzle mode 2 (128 bytes) at bits
// 61-63.  The box is 1024-byte aligned; a K step of 16 BF16 (32 bytes)
// inside the 128-byte row advances the start address by 2.
__device__ __forceinline__ uint64_t umma_desc_sw128(uint32_t saddr) {
  return uint64_t((saddr & 0x3FFFFu) >> 4) | (uint64_t(1) << 16) | (uint64_t(1024 >> 4) << 32) |
         (uint64_t(1) << 46) | (uint64_t(2) << 61);
}

__global__ void __launch_bounds__(kBfThreads) front_update_bf16_kernel(
    const int32_t *__restrict__ tasks, const DFront *__restrict__ fronts, const CUtensorMap *__restrict__ bmaps,
    const CUtensorMap *__restrict__ fmaps, const CUtensorMap *__restrict__ ycmaps, int *flags) {
  extern __shared__ __align__(1024) unsigned char bsm_raw[];
  __shared__ __align__(8) uint64_t bars[2 * kBfStages + 1];  // full[2], empty[2], accumulator
  __shared__ uint32_t tmem_slot;
  __shared__ int s_abort;
  const volatile int *abort_word = &s_abort;
  pdl_launch_dependents();
  const int4 t = reinterpret_cast<const int4 *>(tasks)[blockIdx.x];
  const DFront fr = fronts[t.x];
  const int kind = (t.y >> 24) & 7;
  const int32_t s0 = t.y & 0xffffff, i0 = t.z, j0 = t.w, m = fr.m, p = fr.npiv;
  const int32_t s1 = min(s0 + kSuper, p);
  const int nq = (s1 - s0 + 63) / 64;  // 64-column chunks (a partial last one reads zeros)
  const bool trail = kind == T_TRAIL;
  const CUtensorMap *mapA = trail ? bmaps : bmaps + 1;      // Wt or Lt
  const CUtensorMap *mapB = trail ? bmaps + 1 : bmaps + 2;  // Lt or Yk
  const CUtensorMap *mapC = trail ? fmaps + t.x : ycmaps + t.x;
  const int32_t rowA = int32_t(fr.w_off) + i0;
  const int32_t rowB = trail ? int32_t(fr.w_off) + j0 : fr.first + j0;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const uint32_t ring = (smem_u32(bsm_raw) + 1023u) & ~1023u;  // 1024-byte aligned stages
  float *ring_f = reinterpret_cast<float *>(bsm_raw + (ring - smem_u32(bsm_raw)));
  const uint32_t bar_full = smem_u32(bars), bar_empty = bar_full + 8 * kBfStages, bar_acc = bar_empty + 8 * kBfStages;
  // the copies and F / Y come from the preceding launches; waiting for them
  // before the tensor-memory allocation also keeps a CTA from holding tensor
  // memory while an earlier update launch still needs some
  pdl_wait();
  if (threadIdx.x == 0) {
    s_abort = 0;
    for (int b = 0; b < kBfStages; ++b) {
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(bar_full + 8 * b) : "memory");
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(bar_empty + 8 * b) : "memory");
    }
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(bar_acc) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(smem_u32(&tmem_slot)),
                 "r"(128)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
  const uint32_t tmem = tmem_slot;
  bool ok = true;
  int issued = 0, mma_chunks = 0;
  if (warp == 0) {
    if (lane == 0) {
      for (int q = 0; q < nq && ok; ++q) {
        const int s = q % kBfStages;
        if (q >= kBfStages) ok = mbar_wait(bar_empty + 8 * s, uint32_t((q - kBfStages) / kBfStages) & 1u, abort_word);
        if (!ok) break;
        const uint32_t bar = bar_full + 8 * s, dA = ring + uint32_t(s) * 2 * kBfBox, dB = dA + kBfBox;
        asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(bar), "r"(2 * kBfBox)
                     : "memory");
        tma_load_2d(dA, mapA, 64 * q, rowA, bar);
        tma_load_2d(dB, mapB, 64 * q, rowB, bar);
        issued = q + 1;
      }
    }
    __syncwarp();
  } else if (warp == 1) {
    if (lane == 0) {
      for (int q = 0; q < nq && ok; ++q) {
        const int s = q % kBfStages;
        ok = mbar_wait(bar_full + 8 * s, uint32_t(q / kBfStages) & 1u, abort_word);
        if (!ok) break;
        asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
        const uint32_t a = ring + uint32_t(s) * 2 * kBfBox, b = a + kBfBox;
#pragma unroll
        for (int kk = 0; kk < 4; ++kk) {
          const uint64_t da = umma_desc_sw128(a) + uint64_t(2 * kk), db = umma_desc_sw128(b) + uint64_t(2 * kk);
          const uint32_t acc = (q > 0 || kk > 0) ? 1u : 0u;
          asm volatile(
              "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
              " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem),
              "l"(da), "l"(db), "r"(kIdescBf16), "r"(acc)
              : "memory");
        }
        asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(
                         bar_empty + 8 * s)
                     : "memory");
        mma_chunks = q + 1;
      }
      if (ok)
        asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(bar_acc)
                     : "memory");
    }
    __syncwarp();
  } else {
    // epilogue warps 2-5: TMEM lane quarter g = warp % 4
    const int g = warp & 3;
    if (lane == 0) ok = mbar_wait(bar_acc, 0u, abort_word);
    ok = __shfl_sync(0xffffffffu, ok ? 1 : 0, 0) != 0;
    asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
    if (ok) {
      const int rl = 32 * g + lane;
      const int32_t r = i0 + rl;
      const bool rin = r >= s1 && r < m;
      const int32_t chi_g = trail ? min(m, r + 1) : s1;
      const int clo = trail ? max(0, s1 - j0) : 0;
      const int chi = rin ? max(0, min(kT128, chi_g - j0)) : 0;
#pragma unroll
      for (int h = 0; h < 2; ++h) {  // 64 columns per round
        uint32_t v[4][16];
#pragma unroll
        for (int x = 0; x < 4; ++x) {
          const uint32_t ta = tmem + (uint32_t(32 * g) << 16) + uint32_t(64 * h + 16 * x);
          asm volatile(
              "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, "
              "[%16];\n"
              : "=r"(v[x][0]), "=r"(v[x][1]), "=r"(v[x][2]), "=r"(v[x][3]), "=r"(v[x][4]), "=r"(v[x][5]),
                "=r"(v[x][6]), "=r"(v[x][7]), "=r"(v[x][8]), "=r"(v[x][9]), "=r"(v[x][10]), "=r"(v[x][11]),
                "=r"(v[x][12]), "=r"(v[x][13]), "=r"(v[x][14]), "=r"(v[x][15])
              : "r"(ta));
        }
        asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
#pragma unroll
        for (int x = 0; x < 4; ++x)
#pragma unroll
          for (int e = 0; e < 16; ++e) {
            const int cl = 64 * h + 16 * x + e;
            ring_f[cl * kT128 + rl] = (cl >= clo && cl < chi) ? -__uint_as_float(v[x][e]) : 0.f;
          }
      }
      asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");  // generic-proxy stores -> TMA
    }
  }
  if (!ok) s_abort = 1;
  ok = __syncthreads_and(ok) != 0;
  if (ok && threadIdx.x == 64) {
    for (int b = 0; b < 8; ++b) tma_reduce_add_2d(mapC, i0, j0 + 16 * b, ring + uint32_t(b) * kT128 * 16 * 4);
    asm volatile("cp.async.bulk.commit_group;\n" ::: "memory");
    asm volatile("cp.async.bulk.wait_group 0;\n" ::: "memory");
  }
  // on a timeout: the loads (warp 0) and MMAs (warp 1) still in flight finish
  // before the shared and tensor memory are given up (each wait bounded)
  if (!ok && warp == 0 && lane == 0) {
    atomicOr(flags, FLAG_WAIT_TIMEOUT);
    for (int q = max(0, issued - kBfStages); q < issued; ++q)
      mbar_wait(bar_full + 8 * (q % kBfStages), uint32_t(q / kBfStages) & 1u);
  }
  if (!ok && warp == 1 && lane == 0 && mma_chunks > 0) {
    const int q = mma_chunks - 1;
    mbar_wait(bar_empty + 8 * (q % kBfStages), uint32_t(q / kBfStages) & 1u);
  }
  asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
  __syncthreads();
  if (warp == 1)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem), "r"(128) : "memory");
}

// ------------------------------------------------------------------ apply

// Deterministic combination of a block split over several CTAs: each CTA
// stores its partial sums, and the last of the block's CTAs to arrive (a
// ticket per block) adds the partials in chunk order, so the result does not
// depend on which CTA finishes last.  Returns true in that last CTA, whose
// ticket is reset for the next application.
// The ordering is thread 0's alone, after a CTA barrier: the barrier orders
// every thread's partial-sum stores before thread 0's GPU-scope
// acquire-release increment of the ticket, and release is cumulative in the
// PTX memory model, so the increment releases the whole CTA's stores and, in
// the last CTA, acquires the other CTAs' (the pattern of a grid-wide
// barrier), with one ordered atomic instead of a fence per thread.
__device__ __forceinline__ int atom_add_acq_rel(int *p, int v) {
  int old;
  asm volatile("atom.acq_rel.gpu.add.s32 %0, [%1], %2;\n" : "=r"(old) : "l"(p), "r"(v) : "memory");
  return old;
}
__device__ __forceinline__ void red_add_release(int *p, int v) {
  asm volatile("red.release.gpu.add.s32 [%0], %1;\n" ::"l"(p), "r"(v) : "memory");
}

__device__ __forceinline__ bool last_of_block(int *ticket, int nch) {
  __shared__ int s_last;
  __syncthreads();
  if (threadIdx.x == 0) {
    const int t = atom_add_acq_rel(ticket, 1);
    s_last = (t == nch - 1);
    if (s_last) *ticket = 0;
  }
  __syncthreads();
  return s_last;
}

// The preconditioner application as a dataflow over the front tree: one
// persistent launch per direction.  CTAs take tasks from a queue in the
// lists' order (forward: every level's tasks, leaves first; backward: root
// first), which is a topological order of the dependencies, and a task waits
// only for tasks fetched before it (held by running CTAs), so the waits
// always end; they are bounded in time anyway (FLAG_WAIT_TIMEOUT, then every
// later wait gives up at once through the abort word).  Dependencies:
// forward, a front's tasks wait until all its children are done (counter
// of pending children, decremented by each child's last task); backward,
// until all tasks of the parent are done.  Vectors written by other tasks
// of the same launch are read through L2 (ld.cg), never a stale L1 line.
// Control words df_ctl: [0] forward queue, [1] backward queue, [2] forward
// abort, [3] backward abort; each launch resets the other direction's words.
// dependency waits of the application kernels give up after wait_ns
// (fe_options.dep_wait_s), raising FLAG_APPLY_TIMEOUT and the launch's abort word

__device__ __forceinline__ int ld_acquire(const int *p) {
  int v;
  asm volatile("ld.acquire.gpu.global.b32 %0, [%1];\n" : "=r"(v) : "l"(p) : "memory");
  return v;
}

// thread 0: wait until *p == target (or abort / timeout); true when satisfied
__device__ __forceinline__ bool dep_wait(const int *p, int target, int *abort_word, int *flags, uint64_t wait_ns) {
  const uint64_t t0 = global_ns();
  for (;;) {
    if (ld_acquire(p) == target) return true;
    if (ld_acquire(abort_word) != 0) return false;
    if (global_ns() - t0 > wait_ns) {
      atomicOr(flags, FLAG_APPLY_TIMEOUT);
      atomicExch(abort_word, 1);
      return false;
    }
    __nanosleep(64);
  }
}

// Forward task (front, r0, j0, slot): rows [r0, r0 + 32*VW) of Y w_P over the
// pivot columns [j0, j0 + fcols) (the front's task width: kFwdCols, or a half
// or a quarter of it on the tree's sparsely populated last levels), where
// w = [r_P; 0] + the children's
// update vectors (gathered through the position lists, children in fixed
// order).  256 threads: 32 row lanes of VW consecutive rows (one 16-byte
// load per column) x 8 column groups, the next 4 columns' loads in flight
// while the current ones are used.  Static data (descriptors, gather
// indices, the first Y vectors) is loaded before the dependency wait.  Rows
// < p give y_P (times D^{-1}) into yperm, rows >= p the update vector.  Row
// blocks with more than fcols columns are split over tasks (slot >= 0) and
// combined in chunk order by the last one (deterministic).
constexpr int kPre = 4;  // gather sources prefetched per position

// Asynchronous 4- or 8-byte copy global -> shared (cp.async): a task starts
// the copies of the inputs that no task of its launch writes before its
// dependency wait, and waits for them (cp_async_wait_all, the issuing
// thread's own copies) after it, so their latency overlaps the wait without
// holding registers.
template <int BYTES>
__device__ __forceinline__ void cp_async_small(void *smem, const void *gmem) {
  static_assert(BYTES == 4 || BYTES == 8, "4- or 8-byte copies");
  asm volatile("cp.async.ca.shared.global [%0], [%1], %2;\n" ::"r"(smem_u32(smem)), "l"(gmem), "n"(BYTES)
               : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;\n" ::: "memory"); }

// One task of look-ahead in the persistent apply kernels: a CTA takes the
// index of its next task while it starts the current one, and lanes 0-5 of
// warp 0 load that task's descriptor (its int4 and the 96-byte DFront of its
// front) while the current task finishes, so the next task starts from
// shared memory instead of three dependent global round trips.  (Taking a
// task early cannot deadlock: tasks are handed out in topological order, so
// the lowest unfinished task is always a CTA's current task, and its
// dependencies are finished.)
static_assert(sizeof(DFront) == 96, "the descriptor is copied as six 16-byte pieces");

// Element strides between the right-hand sides of a multi-right-hand-side
// forward solve (all zero for a single one): input vector, update vectors,
// pivot output, partial sums, tickets, per-front counters.
struct RhsStrides {
  int64_t r, u, y, p, t, f;
};
struct NextDesc {
  int4 t, f;
};
__device__ __forceinline__ NextDesc load_desc(const int4 *__restrict__ tasks, const DFront *__restrict__ fronts,
                                              int64_t tn, int64_t ntask, int lane) {
  NextDesc d{};
  if (tn < ntask && lane < 6) {
    d.t = tasks[tn];
    d.f = reinterpret_cast<const int4 *>(fronts + (d.t.x & 0xffffff))[lane];
  }
  return d;
}
__device__ __forceinline__ void store_desc(const NextDesc &d, int4 &s_t, DFront &s_fr, int lane) {
  if (lane < 6) reinterpret_cast<int4 *>(&s_fr)[lane] = d.f;
  if (lane == 0) s_t = d.t;
}
constexpr int kFwdU = 8;  // columns per thread per load round

template <typename TF, typename TV>
__global__ void __launch_bounds__(256, 4) fwd_kernel(const int4 *__restrict__ tasks, int64_t ntask,
                                                  const DFront *__restrict__ fronts, const TF *__restrict__ Y,
                                                  const double *__restrict__ Dinv,
                                                  const int32_t *__restrict__ perm,
                                                  const int32_t *__restrict__ wsrc_ptr,
                                                  const int32_t *__restrict__ wsrc, const TV *__restrict__ r,
                                                  TV *__restrict__ ubuf, TV *__restrict__ yperm,
                                                  TV *__restrict__ part, int *__restrict__ tickets,
                                                  int *pend, int *bdone, int *ctl, int nfronts,
                                                  int *flags, uint64_t wait_ns, const double *__restrict__ done,
                                                  RhsStrides rs = RhsStrides{}) {
  static_assert(kFwdCols == 256, "one gathered column per thread");
  using V = typename Vec16<TF>::type;
  constexpr int VW = Vec16<TF>::n;
  constexpr int RB = 32 * VW;
  __shared__ TV gpart[8 * RB];
  __shared__ TV wp[kFwdCols];
  __shared__ double s_dinv[RB];
  __shared__ int s_task, s_next, s_ok;
  __shared__ int4 s_t;
  __shared__ __align__(16) DFront s_fr;
  if (done && *done != 0.0) return;
  // leave the backward counters reset for the backward launch that follows
  for (int i = blockIdx.x * 256 + threadIdx.x; i < nfronts; i += gridDim.x * 256) bdone[i] = 0;
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    ctl[1] = 0;
    ctl[3] = 0;
  }
  if (threadIdx.x == 0) s_task = atomicAdd(ctl + 0, 1);
  __syncthreads();
  if (threadIdx.x < 32) store_desc(load_desc(tasks, fronts, s_task, ntask, threadIdx.x), s_t, s_fr, threadIdx.x);
  for (;;) {
    __syncthreads();  // this task's index and descriptor
    const int64_t ti = s_task;
    if (ti >= ntask) break;
    const int4 t = s_t;
    const DFront fr = s_fr;
    if (threadIdx.x == 0) s_next = atomicAdd(ctl + 0, 1);  // the next task, one ahead
    const int32_t r0 = t.y, j0 = t.z, slot = t.w;
    // a multi-right-hand-side list carries the right-hand side in the front
    // id's high byte: its vectors, partial sums and counters are offset
    const int32_t fid = t.x & 0xffffff;
    const int64_t rk = t.x >> 24;
    const TV *const rv = r + rk * rs.r;
    TV *const uv = ubuf + rk * rs.u;
    TV *const yv = yperm + rk * rs.y;
    TV *const pv = part + rk * rs.p;
    int *const tv = tickets + rk * rs.t;
    int *const pendv = pend + rk * rs.f;
    const int32_t p = fr.npiv, m = fr.m;
    const int32_t jmax = (r0 + RB < p) ? r0 + RB : p;
    const int32_t fc = fr.fcols;  // this front's columns per task (at most kFwdCols)
    const int32_t j1 = (j0 + fc < jmax) ? j0 + fc : jmax;
    // static gather indices: column j0 + tid of w, and row r0 + tid's child sum
    const int32_t jg = j0 + int32_t(threadIdx.x);
    int32_t gq0 = 0, gq1 = 0, gperm = 0, gsrc[kPre];
    if (jg < j1) {
      gq0 = wsrc_ptr[fr.w_off + jg];
      gq1 = wsrc_ptr[fr.w_off + jg + 1];
      gperm = perm[fr.first + jg];
    }
#pragma unroll
    for (int k = 0; k < kPre; ++k) gsrc[k] = gq0 + k < gq1 ? wsrc[gq0 + k] : -1;
    // inputs that no task of this launch writes are copied to shared memory
    // asynchronously before the wait: this column's entry of r, and D^{-1}
    // of this block's pivot rows
    if (jg < j1) cp_async_small<sizeof(TV)>(wp + (jg - j0), rv + gperm);
#pragma unroll
    for (int k = 0; k < (RB + 255) / 256; ++k) {
      const int32_t tt = int32_t(threadIdx.x) + 256 * k, i = r0 + tt;
      if (tt < RB && i < p && i < m) cp_async_small<8>(s_dinv + tt, Dinv + fr.first + i);
    }
    const int32_t ie = r0 + int32_t(threadIdx.x);
    int32_t eq0 = 0, eq1 = 0, esrc[kPre];
    if (threadIdx.x < RB && ie >= p && ie < m) {
      eq0 = wsrc_ptr[fr.w_off + ie];
      eq1 = wsrc_ptr[fr.w_off + ie + 1];
    }
#pragma unroll
    for (int k = 0; k < kPre; ++k) esrc[k] = eq0 + k < eq1 ? wsrc[eq0 + k] : -1;
    const int rl = threadIdx.x & 31, g = threadIdx.x >> 5;
    const int32_t row = r0 + VW * rl;
    const TF *yc = Y + fr.y_off + row;
    // warp g owns columns j0 + g + 8u; each round issues the loads of kFwdU
    // columns before using any (kFwdU 16-byte loads in flight per thread;
    // the first round's go out before the dependency wait)
    int32_t jq = j0 + g;
    const bool live = row < m;
    V cv[kFwdU];
#pragma unroll
    for (int u = 0; u < kFwdU; ++u)
      cv[u] = (live && jq + 8 * u < j1) ? *reinterpret_cast<const V *>(yc + int64_t(jq + 8 * u) * fr.ldy) : V{};
    // the children's update vectors must be complete
    if (threadIdx.x == 0) s_ok = dep_wait(pendv + fid, 0, ctl + 2, flags, wait_ns);
    cp_async_wait_all();
    __syncthreads();
    bool wnz = false;
    if (s_ok) {
      if (jg < j1) {
        TV w = wp[jg - j0];
#pragma unroll
        for (int k = 0; k < kPre; ++k)
          if (gsrc[k] >= 0) w += __ldcg(uv + gsrc[k]);
        for (int32_t q = gq0 + kPre; q < gq1; ++q) w += __ldcg(uv + wsrc[q]);
        wp[jg - j0] = w;
        wnz = w != TV(0);
      }
    }
    TV csum = TV(0);
    if (s_ok) {
#pragma unroll
      for (int k = 0; k < kPre; ++k)
        if (esrc[k] >= 0) csum += __ldcg(uv + esrc[k]);
      for (int32_t q = eq0 + kPre; q < eq1; ++q) csum += __ldcg(uv + wsrc[q]);
    }
    // a block whose gathered w is all zero contributes exactly nothing (a
    // sparse right-hand side, such as a contact's column, leaves most fronts
    // at zero): Y is not streamed then
    const bool wany = __syncthreads_or(wnz) != 0;
    TV acc[VW];
#pragma unroll
    for (int e = 0; e < VW; ++e) acc[e] = TV(0);
    if (s_ok && live && wany) {
      for (;;) {
        TV wv[kFwdU];
#pragma unroll
        for (int u = 0; u < kFwdU; ++u) wv[u] = jq + 8 * u < j1 ? wp[jq + 8 * u - j0] : TV(0);
        // each column's registers are reloaded with the next round's column
        // as soon as they are used, so the thread's loads stay in flight
        // while it computes
        const int32_t jn = jq + 8 * kFwdU;
#pragma unroll
        for (int u = 0; u < kFwdU; ++u) {
#pragma unroll
          for (int e = 0; e < VW; ++e) acc[e] += TV(vget(cv[u], e)) * wv[u];
          cv[u] = jn + 8 * u < j1 ? *reinterpret_cast<const V *>(yc + int64_t(jn + 8 * u) * fr.ldy) : V{};
        }
        jq = jn;
        if (jq >= j1) break;
      }
    }
    NextDesc nd{};
    if (threadIdx.x < 32) nd = load_desc(tasks, fronts, s_next, ntask, threadIdx.x);
#pragma unroll
    for (int e = 0; e < VW; ++e) gpart[g * RB + VW * rl + e] = acc[e];
    __syncthreads();
    TV sums[(RB + 255) / 256];
#pragma unroll
    for (int k = 0; k < (RB + 255) / 256; ++k) {
      const int tt = threadIdx.x + 256 * k;
      TV sm = TV(0);
      if (tt < RB) {
#pragma unroll
        for (int gg = 0; gg < 8; ++gg) sm += gpart[gg * RB + tt];
      }
      sums[k] = sm;
    }
    bool final = true;
    if (slot >= 0) {
      const int nch = (jmax + fc - 1) / fc;
#pragma unroll
      for (int k = 0; k < (RB + 255) / 256; ++k) {
        const int tt = threadIdx.x + 256 * k;
        if (tt < RB) pv[int64_t(slot + j0 / fc) * RB + tt] = sums[k];
      }
      final = last_of_block(tv + slot, nch);
      if (final) {
#pragma unroll
        for (int k = 0; k < (RB + 255) / 256; ++k) {
          const int tt = threadIdx.x + 256 * k;
          TV sm = TV(0);
          if (tt < RB) {
            // in chunk order; unrolled so that the loads overlap
#pragma unroll 8
            for (int ch = 0; ch < nch; ++ch) sm += __ldcg(pv + int64_t(slot + ch) * RB + tt);
          }
          sums[k] = sm;
        }
      }
    }
    if (final) {
#pragma unroll
      for (int k = 0; k < (RB + 255) / 256; ++k) {
        const int tt = threadIdx.x + 256 * k;
        const int32_t i = r0 + tt;
        if (tt >= RB || i >= m) continue;
        if (i < p)
          yv[fr.first + i] = TV(double(sums[k]) * s_dinv[tt]);
        else
          uv[fr.u_off + i - p] = csum + sums[k];
      }
    }
    // completion: the parent's counter holds its children's pending tasks,
    // so every task releases its share without waiting for an answer (a
    // release reduction by thread 0 after the barrier, cumulative over the
    // CTA's stores as in last_of_block)
    __syncthreads();
    if (threadIdx.x == 0) {
      if (fr.parent >= 0) red_add_release(pendv + fr.parent, -1);
      s_task = s_next;
    }
    if (threadIdx.x < 32) store_desc(nd, s_t, s_fr, threadIdx.x);
  }
}

// VW consecutive entries of the staged x (16-byte aligned) as vector loads
template <int VW>
__device__ __forceinline__ void xs_vec(const float *p, float (&x)[VW]) {
#pragma unroll
  for (int h = 0; h < VW / 4; ++h) {
    const float4 t = reinterpret_cast<const float4 *>(p)[h];
    x[4 * h] = t.x; x[4 * h + 1] = t.y; x[4 * h + 2] = t.z; x[4 * h + 3] = t.w;
  }
}
template <int VW>
__device__ __forceinline__ void xs_vec(const double *p, double (&x)[VW]) {
#pragma unroll
  for (int h = 0; h < VW / 2; ++h) {
    const double2 t = reinterpret_cast<const double2 *>(p)[h];
    x[2 * h] = t.x; x[2 * h + 1] = t.y;
  }
}

// Backward task (front, c0, i0, slot): pivot columns [c0, c0 + 32) over the
// rows [i0, i0 + brows) (the front's task height: BR = kBwdRows, twice that
// for the binary16 Y, or a half or a quarter of BR on the tree's sparsely
// populated last levels); warp w
// owns columns c0 + w + 8k (k < 4) and streams them together, eight 16-byte
// loads per lane in flight.
// x = [D^{-1} y_P; z_U] is staged in shared memory from the VW-aligned row at
// or below c0 (rows above a column are zeros of L^{-1}, so reading from the
// aligned row is exact); z_U was written by the parent's tasks.  Columns
// longer than brows rows are split over tasks (slot >= 0) and combined in
// row-chunk order.  Also resets the forward counters for the next
// application.
template <typename TF, typename TV>
__global__ void __launch_bounds__(256, 4) bwd_kernel(const int4 *__restrict__ tasks, int64_t ntask,
                                                  const DFront *__restrict__ fronts, const TF *__restrict__ Y,
                                                  const int32_t *__restrict__ perm,
                                                  const int32_t *__restrict__ upd_rows_old,
                                                  const TV *__restrict__ yperm, TV *__restrict__ z,
                                                  TV *__restrict__ part, int *__restrict__ tickets,
                                                  int *pend, const int *__restrict__ pend0, int *bdone, int *ctl,
                                                  int nfronts, int *flags, uint64_t wait_ns,
                                                  const double *__restrict__ done) {
  using V = typename Vec16<TF>::type;
  constexpr int VW = Vec16<TF>::n;
  constexpr int BR = sizeof(TF) == 2 ? 2 * kBwdRows : kBwdRows;  // rows per task
  constexpr int XS = BR / 256;                                   // staged rows per thread
  __shared__ __align__(16) TV xs[BR];
  __shared__ int s_zpos[kBwdCols];
  __shared__ int s_task, s_next, s_ok;
  __shared__ int4 s_t;
  __shared__ __align__(16) DFront s_fr;
  if (done && *done != 0.0) return;
  // the forward counters for the next application: each front's children's
  // forward tasks
  for (int i = blockIdx.x * 256 + threadIdx.x; i < nfronts; i += gridDim.x * 256) pend[i] = pend0[i];
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    ctl[0] = 0;
    ctl[2] = 0;
  }
  if (threadIdx.x == 0) s_task = atomicAdd(ctl + 1, 1);
  __syncthreads();
  if (threadIdx.x < 32) store_desc(load_desc(tasks, fronts, s_task, ntask, threadIdx.x), s_t, s_fr, threadIdx.x);
  for (;;) {
    __syncthreads();  // this task's index and descriptor
    const int64_t ti = s_task;
    if (ti >= ntask) break;
    const int4 t = s_t;
    const DFront fr = s_fr;
    if (threadIdx.x == 0) s_next = atomicAdd(ctl + 1, 1);  // the next task, one ahead
    const int32_t c0 = t.y, ilo0 = t.z, slot = t.w;
    const int32_t p = fr.npiv, m = fr.m;
    const int32_t a0 = c0 & ~(VW - 1);
    const int32_t xa = a0 > ilo0 ? a0 : ilo0;                                 // first row of this task
    const int32_t br = fr.brows;  // this front's rows per task (at most BR)
    const int32_t xb = (ilo0 + br < fr.ldy) ? ilo0 + br : fr.ldy;  // end row
    // static: where each staged row comes from (-1: zero, >= 0: yperm index,
    // <= -2: z index -2 - idx)
    const int32_t *urows = upd_rows_old + fr.rows_off;
    int32_t xsrc[XS];
#pragma unroll
    for (int k = 0; k < XS; ++k) {
      const int32_t tt = int32_t(threadIdx.x) + 256 * k;
      const int32_t i = xa + tt;
      xsrc[k] = -1;
      if (tt < xb - xa && i >= c0 && i < m) xsrc[k] = i < p ? fr.first + i : -2 - urows[i - p];
    }
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    // the four columns are all read from the task's first row (rows above a
    // column's diagonal hold zeros of L^{-1}), so one vector load of the
    // staged x per row block serves all of them, without bank conflicts
    int32_t jc[4];
    const TF *yc[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      jc[k] = c0 + w + 8 * k;
      const int32_t j = jc[k] < p ? jc[k] : c0;  // out-of-range columns read a valid one, result dropped
      yc[k] = Y + fr.y_off + int64_t(j) * fr.ldy;
    }
    // each round loads two row blocks of the four columns (eight 16-byte
    // loads in flight per thread) before using any; the first round's go
    // out before the dependency wait
    const int32_t ist = xa + VW * lane;
    V cv[2][4];
#pragma unroll
    for (int h = 0; h < 2; ++h) {
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        const int32_t i = ist + 32 * VW * h;
        cv[h][k] = i < xb ? *reinterpret_cast<const V *>(yc[k] + i) : V{};
      }
    }
    // copied to shared memory asynchronously before the wait: the pivot
    // rows of x, which the forward launch wrote, and the output positions of
    // the task's columns; the update rows of x come from the parent's tasks
#pragma unroll
    for (int k = 0; k < XS; ++k) {
      const int32_t tt = int32_t(threadIdx.x) + 256 * k;
      if (tt < xb - xa && xsrc[k] >= 0) cp_async_small<sizeof(TV)>(xs + tt, yperm + xsrc[k]);
    }
    if (threadIdx.x < kBwdCols) {
      if (c0 + int32_t(threadIdx.x) < p)
        cp_async_small<4>(s_zpos + threadIdx.x, perm + fr.first + c0 + int32_t(threadIdx.x));
      else
        s_zpos[threadIdx.x] = -1;
    }
    // the parent's solution entries must be complete
    if (threadIdx.x == 0)
      s_ok = fr.parent < 0 ? 1 : dep_wait(bdone + fr.parent, fronts[fr.parent].nbwd, ctl + 3, flags, wait_ns);
    cp_async_wait_all();
    __syncthreads();
    bool xnz = false;
#pragma unroll
    for (int k = 0; k < XS; ++k) {
      const int32_t tt = int32_t(threadIdx.x) + 256 * k;
      if (tt < xb - xa) {
        const TV xv = (xsrc[k] == -1 || !s_ok) ? TV(0) : (xsrc[k] >= 0 ? xs[tt] : __ldcg(z + (-2 - xsrc[k])));
        xs[tt] = xv;
        xnz = xnz || xv != TV(0);
      }
    }
    // an all-zero x contributes exactly nothing: Y is not streamed then
    const bool xany = __syncthreads_or(xnz) != 0;
    TV acc[4] = {TV(0), TV(0), TV(0), TV(0)};
    for (int32_t off = 0; xany;) {
      // each row block's registers are reloaded with the next round's rows
      // as soon as they are used (the thread's loads stay in flight)
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const int32_t i = ist + off + 32 * VW * h, inext = i + 64 * VW;
        if (i < xb) {
          TV xv[VW];
          xs_vec<VW>(xs + (i - xa), xv);
#pragma unroll
          for (int k = 0; k < 4; ++k) {
#pragma unroll
            for (int q = 0; q < VW; ++q) acc[k] += TV(vget(cv[h][k], q)) * xv[q];
          }
        }
#pragma unroll
        for (int k = 0; k < 4; ++k) cv[h][k] = inext < xb ? *reinterpret_cast<const V *>(yc[k] + inext) : V{};
      }
      off += 64 * VW;
      if (xa + off >= xb) break;
    }
    NextDesc nd{};
    if (threadIdx.x < 32) nd = load_desc(tasks, fronts, s_next, ntask, threadIdx.x);
#pragma unroll
    for (int k = 0; k < 4; ++k) {
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) acc[k] += __shfl_xor_sync(0xffffffffu, acc[k], o);
    }
    if (slot < 0) {
      if (lane == 0) {
#pragma unroll
        for (int k = 0; k < 4; ++k) {
          const int32_t zp = s_zpos[w + 8 * k];
          if (zp >= 0) z[zp] = acc[k];
        }
      }
    } else {
      const int32_t k_first = a0 / br;
      const int nch = (fr.ldy - 1) / br - k_first + 1;
      if (lane == 0) {
#pragma unroll
        for (int k = 0; k < 4; ++k)
          part[int64_t(slot + ilo0 / br - k_first) * kBwdCols + w + 8 * k] = acc[k];
      }
      if (last_of_block(tickets + slot, nch) && threadIdx.x < kBwdCols) {
        TV sm = TV(0);
        // in chunk order; unrolled so that the loads overlap
#pragma unroll 8
        for (int ch = 0; ch < nch; ++ch) sm += __ldcg(part + int64_t(slot + ch) * kBwdCols + threadIdx.x);
        const int32_t zp = s_zpos[threadIdx.x];
        if (zp >= 0) z[zp] = sm;
      }
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      red_add_release(bdone + t.x, 1);
      s_task = s_next;
    }
    if (threadIdx.x < 32) store_desc(nd, s_t, s_fr, threadIdx.x);
  }
}

// ------------------------------------------------------------ host drivers

template <typename TF>
static void factor_levels(fe_ctx *c, DeviceState *d, int buf, const TF *Afac, cudaStream_t s) {
  TF *F = reinterpret_cast<TF *>(d->F);
  TF *Y = reinterpret_cast<TF *>(d->Y[buf]);
  const int64_t nf = int64_t(c->fronts.size());
  const CUtensorMap *fmaps = reinterpret_cast<const CUtensorMap *>(d->tmaps);
  const CUtensorMap *ymaps = fmaps ? fmaps + (1 + buf) * nf : nullptr;
  const CUtensorMap *ycmaps = fmaps ? fmaps + (3 + buf) * nf : nullptr;
  const size_t tsm = 2 * 64 * 65 * sizeof(TF);
  const size_t dsm = diag_smem<TF>();
  cudaFuncSetAttribute(front_diag_kernel<TF>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(dsm));
  cudaFuncSetAttribute(front_panel_kernel<TF>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(tsm));
  cudaFuncSetAttribute(front_update_kernel<TF>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(tsm));
  cudaFuncSetAttribute(front_update_tc_kernel<3>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(update_smem<3>()));
  cudaFuncSetAttribute(front_update_tc_kernel<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(update_smem<1>()));
  cudaFuncSetAttribute(front_update_bf16_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, int(bf16_update_smem()));
  // BF16 copies of the superpanels (FP32 factor with update_bf16)
  __nv_bfloat16 *bw = nullptr, *bl = nullptr, *by = nullptr;
  if constexpr (sizeof(TF) == 4) {
    if (c->opt.update_bf16 && d->bt_w) {
      bw = reinterpret_cast<__nv_bfloat16 *>(d->bt_w);
      bl = reinterpret_cast<__nv_bfloat16 *>(d->bt_l);
      by = reinterpret_cast<__nv_bfloat16 *>(d->bt_y);
    }
  }
  const CUtensorMap *bmaps = reinterpret_cast<const CUtensorMap *>(d->bmaps);
  for (size_t lv = 0; lv < d->lt.size(); ++lv) {
    const auto &L = d->lt[lv];
    if (L.asm_n) d->launches++;
    if (L.asm_n)
      launch_pdl(front_assemble_kernel<TF>, unsigned(L.asm_n), 256, 0, s, d->tasks + L.asm_off, d->fronts,
                 d->child_list, d->rmap, d->fa_colptr, d->fa_slot, d->fa_off, Afac, F, Y);
    for (size_t st = 0; st < L.diag_n.size(); ++st) {
      d->launches += (L.diag_n[st] > 0) + (L.panel_n[st] > 0) + (L.trail_n[st] > 0);
      if (L.diag_n[st])
        launch_pdl(front_diag_kernel<TF>, unsigned(L.diag_n[st]), kDiagThreads, dsm, s, d->tasks + L.diag_off[st],
                   d->fronts, F, Y, d->D[buf], d->D[buf] + c->n_free, d->flags, by);
      if (L.panel_n[st])
        launch_pdl(front_panel_kernel<TF>, unsigned(L.panel_n[st]), 256, tsm, s, d->tasks + L.panel_off[st],
                   d->fronts, F, Y, d->D[buf] + c->n_free, bw, bl, by);
      if (L.trail_n[st]) {
        const int ev = stage_begin(c, FE_STAGE_FACTOR_UPDATE, s);
        if (ev >= 0) d->update_flops += L.trail_flops[st];
        if constexpr (sizeof(TF) == 4)
          if (c->opt.factor_tf32)
            launch_pdl(front_update_tc_kernel<1>, unsigned(L.trail_n[st]), kUThreads, update_smem<1>(), s,
                       d->tasks + L.trail_off[st], d->fronts, F, Y, d->D[buf], fmaps, ymaps, ycmaps, d->flags);
          else
            launch_pdl(front_update_tc_kernel<3>, unsigned(L.trail_n[st]), kUThreads, update_smem<3>(), s,
                       d->tasks + L.trail_off[st], d->fronts, F, Y, d->D[buf], fmaps, ymaps, ycmaps, d->flags);
        else
          launch_pdl(front_update_kernel<TF>, unsigned(L.trail_n[st]), 256, tsm, s, d->tasks + L.trail_off[st],
                     d->fronts, F, Y, d->D[buf]);
        stage_end(c, ev, s);
      }
      if (L.tend_n[st] && bw) {
        d->launches++;
        const int ev = stage_begin(c, FE_STAGE_FACTOR_UPDATE_BF16, s);
        if (ev >= 0) {
          d->update_bf16_flops += L.tend_flops[st];
          d->update_bf16_tiles += L.tend_n[st];
        }
        launch_pdl(front_update_bf16_kernel, unsigned(L.tend_n[st]), kBfThreads, bf16_update_smem(), s,
                   d->tasks + L.tend_off[st], d->fronts, bmaps, fmaps, ycmaps, d->flags);
        stage_end(c, ev, s);
      }
    }
  }
  if constexpr (sizeof(TF) == 4) {
    if (c->opt.precond_fp16) {
      const int64_t n8 = c->y_total / 8;
      d->launches++;
      y_to_half_kernel<<<unsigned(std::max<int64_t>(1, std::min<int64_t>((n8 + 255) / 256, 152 * 16))), 256, 0,
                         s>>>(reinterpret_cast<const float4 *>(Y), reinterpret_cast<uint4 *>(d->Yh[buf]), n8);
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

// The per-right-hand-side forward counters of a multi-right-hand-side
// launch set to the subset's own dependencies, and its control words cleared
// (see apply_forward_multi_enqueue).
__global__ void multi_reset_kernel(const int *__restrict__ pend_init, int *pend, int *ctl, int nfronts,
                                   int64_t total) {
  for (int64_t i = int64_t(blockIdx.x) * 256 + threadIdx.x; i < total; i += int64_t(gridDim.x) * 256)
    pend[i] = pend_init[i % nfronts];
  if (blockIdx.x == 0 && threadIdx.x < 4) ctl[threadIdx.x] = 0;
}

static uint64_t wait_ns_of(const fe_ctx *c) { return uint64_t(c->opt.dep_wait_s * 1e9); }

// fe_debug_hold_front: more pending child tasks on a front for one
// application, so its forward tasks wait on a count that nothing reaches
// (the backward launch resets every counter afterwards)
__global__ void hold_front_kernel(int *pend, int front, int extra) { pend[front] += extra; }

void launch_pending_hold(const DeviceState *d, cudaStream_t s) {
  if (d->df_hold < 0) return;
  hold_front_kernel<<<1, 1, 0, s>>>(d->df_pend, d->df_hold, d->df_hold_extra);
  d->df_hold = -1;
}

template <typename TF, typename TV>
static void apply_levels_with(const fe_ctx *c, const DeviceState *d, int buf, const TV *r, TV *z, TV *u, TV *yp,
                              TV *part_f, TV *part_b, int *tick_f, int *tick_b, int *flags, cudaStream_t s,
                              const double *done = nullptr) {
  const TF *Y = reinterpret_cast<const TF *>(sizeof(TF) == 2 ? d->Yh[buf] : d->Y[buf]);
  const double *Dinv = d->D[buf] + c->n_free;
  const int nf = int(c->fronts.size());
  // persistent grids: every resident CTA (at most one per task)
  static int per_sm[2] = {0, 0};
  if (!per_sm[0]) {
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm[0], fwd_kernel<TF, TV>, 256, 0);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm[1], bwd_kernel<TF, TV>, 256, 0);
  }
  int sms = 0;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, d->device);
  // while a lagged factorisation is in flight, leave apply_sm_share of the
  // CTA slots to its kernels (tasks are taken from a queue in topological
  // order, so any grid size gives the same result)
  const double keep = d->factor_pending >= 0 ? 1.0 - c->opt.apply_sm_share : 1.0;
  const int64_t slots_f = std::max<int64_t>(1, int64_t(double(int64_t(sms) * std::max(1, per_sm[0])) * keep));
  const int64_t slots_b = std::max<int64_t>(1, int64_t(double(int64_t(sms) * std::max(1, per_sm[1])) * keep));
  const unsigned gf = unsigned(std::max<int64_t>(1, std::min<int64_t>(d->n_apply_fwd, slots_f)));
  const unsigned gb = unsigned(std::max<int64_t>(1, std::min<int64_t>(d->n_apply_bwd, slots_b)));
  {
    // a pending test hold applies to the next application that runs, never
    // to one captured into a graph (the whole-step graph applies it before
    // its launch)
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    cudaStreamIsCapturing(s, &cs);
    if (cs == cudaStreamCaptureStatusNone) launch_pending_hold(d, s);
  }
  d->launches += 2;
  fwd_kernel<TF, TV><<<gf, 256, 0, s>>>(reinterpret_cast<const int4 *>(d->apply_fwd), d->n_apply_fwd, d->fronts, Y,
                                        Dinv, d->perm, d->wsrc_ptr, d->wsrc, r, u, yp, part_f, tick_f, d->df_pend,
                                        d->df_bdone, d->df_ctl, nf, flags, wait_ns_of(c), done);
  bwd_kernel<TF, TV><<<gb, 256, 0, s>>>(reinterpret_cast<const int4 *>(d->apply_bwd), d->n_apply_bwd, d->fronts, Y,
                                        d->perm, d->upd_rows_old, yp, z, part_b, tick_b, d->df_pend, d->df_pend0,
                                        d->df_bdone, d->df_ctl, nf, flags, wait_ns_of(c), done);
}

template <typename TF, typename TV>
static void apply_levels(const fe_ctx *c, const DeviceState *d, int buf, const TV *r, TV *z, cudaStream_t s,
                         const double *done) {
  apply_levels_with<TF, TV>(c, d, buf, r, z, reinterpret_cast<TV *>(d->ubuf), reinterpret_cast<TV *>(d->yperm),
                            reinterpret_cast<TV *>(d->part_f), reinterpret_cast<TV *>(d->part_b), d->tick_f,
                            d->tick_b, d->flags, s, done);
}

// Forward solves of nrhs right-hand sides in one launch, over a subset of
// the fronts (closed under taking parents) outside which every right-hand
// side is zero.  tasks: the subset's forward tasks in topological order, each
// repeated for the right-hand sides k < nrhs with k in the front id's high
// byte; every right-hand side k has its own input r + k n, pivot output
// yp + k n_free, update vectors u + k u_total, partial sums, tickets and
// per-front counters (pend, nf each, set from pend_init: the forward tasks of
// each front's children in the subset), and the launch has its
// own control words, so the context's application state is not touched.  The
// caller clears yp and u once (outside the subset they stay zero) and the
// tickets once (the last CTA of a split block resets its ticket).
void apply_forward_multi_enqueue(const fe_ctx *c, const DeviceState *d, int buf, bool fp32, const void *r, void *yp,
                                 const int32_t *tasks, int64_t ntask, const int *pend_init, int *pend,
                                 int *bdone, int *ctl, void *u, void *part, int *tickets, int nrhs, cudaStream_t s) {
  const int nf = int(c->fronts.size());
  const int64_t total = int64_t(nf) * nrhs;
  multi_reset_kernel<<<unsigned(std::min<int64_t>(1024, (total + 255) / 256)), 256, 0, s>>>(pend_init, pend,
                                                                                           ctl, nf, total);
  int sms = 0;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, d->device);
  const unsigned g = unsigned(std::max<int64_t>(1, std::min<int64_t>(ntask, int64_t(sms) * 4)));
  const int4 *tk = reinterpret_cast<const int4 *>(tasks);
  const double *Dinv = d->D[buf] + c->n_free;
  const RhsStrides rs{c->n, std::max<int64_t>(c->u_total, 1), c->n_free,
                      std::max<int64_t>(c->fwd_slots, 1) * fwd_rows(c->opt), std::max<int64_t>(c->fwd_slots, 1), nf};
  d->launches += 2;
  if (fp32 && c->opt.precond_fp16)
    fwd_kernel<__half, float><<<g, 256, 0, s>>>(tk, ntask, d->fronts, static_cast<const __half *>(d->Yh[buf]), Dinv,
                                                d->perm, d->wsrc_ptr, d->wsrc, static_cast<const float *>(r),
                                                static_cast<float *>(u), static_cast<float *>(yp),
                                                static_cast<float *>(part), tickets, pend, bdone, ctl, nf,
                                                d->flags, wait_ns_of(c), nullptr, rs);
  else if (fp32)
    fwd_kernel<float, float><<<g, 256, 0, s>>>(tk, ntask, d->fronts, static_cast<const float *>(d->Y[buf]), Dinv,
                                               d->perm, d->wsrc_ptr, d->wsrc, static_cast<const float *>(r),
                                               static_cast<float *>(u), static_cast<float *>(yp),
                                               static_cast<float *>(part), tickets, pend, bdone, ctl, nf,
                                               d->flags, wait_ns_of(c), nullptr, rs);
  else
    fwd_kernel<double, double><<<g, 256, 0, s>>>(tk, ntask, d->fronts, static_cast<const double *>(d->Y[buf]), Dinv,
                                                 d->perm, d->wsrc_ptr, d->wsrc, static_cast<const double *>(r),
                                                 static_cast<double *>(u), static_cast<double *>(yp),
                                                 static_cast<double *>(part), tickets, pend, bdone, ctl, nf,
                                                 d->flags, wait_ns_of(c), nullptr, rs);
}

void apply_enqueue(const fe_ctx *c, const DeviceState *d, int buf, bool fp32, const void *r, void *z,
                   cudaStream_t s, const double *done) {
  if (fp32 && c->opt.precond_fp16)
    apply_levels<__half, float>(c, d, buf, reinterpret_cast<const float *>(r), reinterpret_cast<float *>(z), s,
                                done);
  else if (fp32)
    apply_levels<float, float>(c, d, buf, reinterpret_cast<const float *>(r), reinterpret_cast<float *>(z), s, done);
  else
    apply_levels<double, double>(c, d, buf, reinterpret_cast<const double *>(r), reinterpret_cast<double *>(z), s,
                                 done);
}


// ============================================= allocation-free application
// For callers that cannot call cudaMalloc: a real-time loop (an interactive
// simulator's haptic or servo loop, where cudaMalloc's implicit device
// synchronisation and unbounded latency would break the frame budget), or a
// host whose device memory is already fully reserved by another allocator.
// The work vectors of one preconditioner application live in this
// file-scope array instead; the context's factor is only read.
namespace {
constexpr size_t kNoAllocScratchBytes = size_t(64) << 20;  // 64 MiB, held by every GPU that loads the library
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];
std::mutex g_noalloc_mutex;
void *g_noalloc_base[64] = {nullptr};  // device address of the array, per device

size_t round256(size_t b) { return (b + 255) / 256 * 256; }

// Byte offsets of the work vectors inside the array: the same vectors the
// context allocates for fe_apply_preconditioner (the input and output in the
// solve's precision, the update vectors, the permuted pivot vector, the split
// tasks' partial sums and tickets), each 256-byte aligned.
struct NoAllocLayout {
  size_t r, z, u, yp, pf, pb, tk, need;
};
NoAllocLayout noalloc_layout(const fe_ctx *c) {
  const size_t ts = c->opt.precision == FE_MIXED ? sizeof(float) : sizeof(double);
  NoAllocLayout L{};
  size_t o = 0;
  L.r = o; o += round256(size_t(c->n) * ts);
  L.z = o; o += round256(size_t(c->n) * ts);
  L.u = o; o += round256(size_t(std::max<int64_t>(c->u_total, 1)) * ts);
  L.yp = o; o += round256(size_t(std::max<int64_t>(c->n_free, 1)) * ts);
  L.pf = o; o += round256(size_t(std::max<int64_t>(c->fwd_slots, 1)) * size_t(fwd_rows(c->opt)) * ts);
  L.pb = o; o += round256(size_t(std::max<int64_t>(c->bwd_slots, 1)) * kBwdCols * ts);
  L.tk = o; o += round256(size_t(std::max<int64_t>(c->fwd_slots + c->bwd_slots, 1)) * sizeof(int));
  L.need = o;
  return L;
}

}  // namespace

int64_t noalloc_scratch_bytes(const fe_ctx *c) { return c->built ? int64_t(noalloc_layout(c).need) : 0; }
int64_t noalloc_scratch_limit() { return int64_t(kNoAllocScratchBytes); }

}  // namespace fe

extern "C" int fe_apply_preconditioner_noalloc(fe_ctx *c, const double *r, double *z, void *stream) {
  using namespace fe;
  if (!c || !r || !z) return FE_ERR_ARG;
  if (!c->built) return set_error(c, FE_ERR_STATE, "fe_build_pattern has not run");
  // the size check needs only the setup products: no GPU is touched
  const NoAllocLayout L = noalloc_layout(c);
  if (L.need > kNoAllocScratchBytes)
    return set_error(c, FE_ERR_ARG, "this mesh needs " + std::to_string(L.need) +
                                        " bytes of scratch; the allocation-free path holds " +
                                        std::to_string(kNoAllocScratchBytes));
  DeviceState *d = c->dev;
  if (!d || !d->have_factor) return set_error(c, FE_ERR_STATE, "no factor: call fe_factor_now or fe_step first");
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev != d->device || dev < 0 || dev >= 64) {
    cudaGetLastError();
    return set_error(c, FE_ERR_ARG, "the context's device must be current");
  }
  const bool fp32 = c->opt.precision == FE_MIXED;
  void *base = nullptr;
  {
    std::lock_guard<std::mutex> lock(g_noalloc_mutex);
    if (!g_noalloc_base[dev]) {
      cudaError_t e = cudaGetSymbolAddress(&g_noalloc_base[dev], g_noalloc_scratch);
      if (e != cudaSuccess) {
        g_noalloc_base[dev] = nullptr;
        cudaGetLastError();
        return set_error(c, FE_ERR_CUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
      }
    }
    base = g_noalloc_base[dev];
  }
  unsigned char *p = static_cast<unsigned char *>(base);
  void *rT = p + L.r, *zT = p + L.z, *ub = p + L.u, *yp = p + L.yp, *pf = p + L.pf, *pb = p + L.pb;
  int *tf = reinterpret_cast<int *>(p + L.tk);
  int *tb = tf + c->fwd_slots;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  // The application shares the context's per-front counters, task queues and
  // factor buffer with the context's own steps and applications, which run
  // on the context's stream: start after everything queued there (a factor
  // swap included), and make the context's stream (and through it the next
  // refactorisation, which snapshots on that stream) wait for this call.
  cudaError_t e = cudaEventRecord(d->ev_main_tail, d->stream);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(s, d->ev_main_tail, 0);
  // z keeps the last call's values on fixed DOFs unless cleared; the split
  // tasks' tickets start at zero
  if (e == cudaSuccess) e = cudaMemsetAsync(zT, 0, size_t(c->n) * (fp32 ? sizeof(float) : sizeof(double)), s);
  if (e == cudaSuccess) e = cudaMemsetAsync(tf, 0, L.need - L.tk, s);
  if (e != cudaSuccess) return set_error(c, FE_ERR_CUDA, cudaGetErrorString(e));
  // a dependency wait that runs out raises FLAG_APPLY_TIMEOUT in flags[1],
  // which the context's next step reports
  int *flags = d->flags + 1;
  launch_convert(r, false, rT, fp32, c->n, s);
  if (fp32 && c->opt.precond_fp16)
    apply_levels_with<__half, float>(c, d, d->cur, static_cast<const float *>(rT), static_cast<float *>(zT),
                                     static_cast<float *>(ub), static_cast<float *>(yp), static_cast<float *>(pf),
                                     static_cast<float *>(pb), tf, tb, flags, s);
  else if (fp32)
    apply_levels_with<float, float>(c, d, d->cur, static_cast<const float *>(rT), static_cast<float *>(zT),
                                    static_cast<float *>(ub), static_cast<float *>(yp), static_cast<float *>(pf),
                                    static_cast<float *>(pb), tf, tb, flags, s);
  else
    apply_levels_with<double, double>(c, d, d->cur, static_cast<const double *>(rT), static_cast<double *>(zT),
                                      static_cast<double *>(ub), static_cast<double *>(yp),
                                      static_cast<double *>(pf), static_cast<double *>(pb), tf, tb, flags, s);
  launch_convert(zT, fp32, z, false, c->n, s);
  e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaEventRecord(d->ev_noalloc_done, s);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(d->stream, d->ev_noalloc_done, 0);
  if (e != cudaSuccess) return set_error(c, FE_ERR_CUDA, cudaGetErrorString(e));
  return FE_OK;
}
