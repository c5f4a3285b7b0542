// Hyperelastic laws of Section 3.1 on the device, written in terms of the
// displacement gradient H = F - I so that FP32 arithmetic keeps the stress
// accurate relative to its own size (no cancellation of F against I):
//   E = (H + H^T + H^T H)/2, J - 1 = tr H + ((tr H)^2 - tr H^2)/2 + det H,
//   F - F^{-T} = H + F^{-T} H^T, 2F - (2/3) I1 F^{-T} = 4 F^{-T} dev E, ...
// The tangent CC_iJkL = dP_iJ/dF_kL is evaluated one 3x3 block
// C_ik[J][L] = CC_iJkL at a time.
#pragma once

#include "../../include/fe_hotpath.h"
#include "fe_df.cuh"

namespace fe {

template <typename T>
struct M3 {
  T a[3][3];
};

template <typename T>
__device__ __forceinline__ T tr3(const T m[3][3]) { return m[0][0] + m[1][1] + m[2][2]; }

template <typename T>
__device__ __forceinline__ T det3d(const T m[3][3]) {
  return m[0][0] * (m[1][1] * m[2][2] - m[1][2] * m[2][1]) -
         m[0][1] * (m[1][0] * m[2][2] - m[1][2] * m[2][0]) +
         m[0][2] * (m[1][0] * m[2][1] - m[1][1] * m[2][0]);
}

template <typename T>
__device__ __forceinline__ T mlog1p(T x);
template <>
__device__ __forceinline__ double mlog1p<double>(double x) { return log1p(x); }
template <>
__device__ __forceinline__ float mlog1p<float>(float x) { return log1pf(x); }
template <typename T>
__device__ __forceinline__ T mexp(T x);
template <>
__device__ __forceinline__ double mexp<double>(double x) { return exp(x); }
template <>
__device__ __forceinline__ float mexp<float>(float x) { return expf(x); }
// double-float: through FP64 (one transcendental per evaluation, outside the
// laws' matrix arithmetic; the Mooney-Rivlin powers of J avoid it, mr_jpow)
template <>
__device__ __forceinline__ dfloat mlog1p<dfloat>(dfloat x) { return dfloat(log1p(double(x))); }
template <>
__device__ __forceinline__ dfloat mexp<dfloat>(dfloat x) { return dfloat(exp(double(x))); }

// Kinematics common to every law.
template <typename T>
struct Kin {
  T F[3][3], E[3][3], G[3][3];  // F, Green strain, F^{-T}
  T trE, Jm1, J;
  __device__ void init(const T H[3][3]) {
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
      for (int j = 0; j < 3; ++j) {
        T s = H[i][j] + H[j][i];
#pragma unroll
        for (int k = 0; k < 3; ++k) s += H[k][i] * H[k][j];
        E[i][j] = T(0.5) * s;
        F[i][j] = H[i][j] + (i == j ? T(1) : T(0));
      }
    trE = tr3(E);
    T trH = tr3(H);
    T trHH = T(0);
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
      for (int k = 0; k < 3; ++k) trHH += H[i][k] * H[k][i];
    Jm1 = trH + T(0.5) * (trH * trH - trHH) + det3d(H);
    J = T(1) + Jm1;
    // G = F^{-T} = cof(F) / J
    T iJ = T(1) / J;
    G[0][0] = (F[1][1] * F[2][2] - F[1][2] * F[2][1]) * iJ;
    G[0][1] = (F[1][2] * F[2][0] - F[1][0] * F[2][2]) * iJ;
    G[0][2] = (F[1][0] * F[2][1] - F[1][1] * F[2][0]) * iJ;
    G[1][0] = (F[0][2] * F[2][1] - F[0][1] * F[2][2]) * iJ;
    G[1][1] = (F[0][0] * F[2][2] - F[0][2] * F[2][0]) * iJ;
    G[1][2] = (F[0][1] * F[2][0] - F[0][0] * F[2][1]) * iJ;
    G[2][0] = (F[0][1] * F[1][2] - F[0][2] * F[1][1]) * iJ;
    G[2][1] = (F[0][2] * F[1][0] - F[0][0] * F[1][2]) * iJ;
    G[2][2] = (F[0][0] * F[1][1] - F[0][1] * F[1][0]) * iJ;
  }
};

template <int MODEL, typename T>
struct Law;

// St Venant-Kirchhoff: psi = mu tr(E^2) + lambda/2 (tr E)^2, P = F S.
template <typename T>
struct Law<FE_SVK, T> {
  T F[3][3], S[3][3], B[3][3];
  T mu, lam;
  __device__ void init(const Kin<T> &k, const T H[3][3], T p0, T p1, T, T P[3][3]) {
    mu = p0;
    lam = p1;
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
      for (int j = 0; j < 3; ++j) {
        F[i][j] = k.F[i][j];
        S[i][j] = T(2) * mu * k.E[i][j] + (i == j ? lam * k.trE : T(0));
      }
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
      for (int j = 0; j < 3; ++j) {
        T s = T(0), bb = T(0);
#pragma unroll
        for (int l = 0; l < 3; ++l) {
          s += F[i][l] * S[l][j];
          bb += F[i][l] * F[j][l];
        }
        P[i][j] = s;
        B[i][j] = bb;
      }
  }
  __device__ __forceinline__ void block(int i, int k, T C[3][3]) const {
#pragma unroll
    for (int J = 0; J < 3; ++J)
#pragma unroll
      for (int L = 0; L < 3; ++L)
        C[J][L] = (i == k ? S[L][J] : T(0)) + mu * (F[i][L] * F[k][J] + (J == L ? B[i][k] : T(0))) +
                  lam * F[i][J] * F[k][L];
  }
};

// Compressible neo-Hookean: psi = mu/2 (I1 - 3) - mu ln J + lambda/2 (ln J)^2,
// P = mu (F - F^{-T}) + lambda ln J F^{-T}.
template <typename T>
struct Law<FE_NEOHOOKE, T> {
  T G[3][3];
  T mu, lam, c1;
  __device__ void init(const Kin<T> &k, const T H[3][3], T p0, T p1, T, T P[3][3]) {
    mu = p0;
    lam = p1;
    T lnJ = mlog1p(k.Jm1);
    c1 = mu - lam * lnJ;
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
      for (int j = 0; j < 3; ++j) G[i][j] = k.G[i][j];
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
      for (int j = 0; j < 3; ++j) {
        T gh = T(0);  // (F^{-T} H^T)_ij
#pragma unroll
        for (int l = 0; l < 3; ++l) gh += G[i][l] * H[j][l];
        P[i][j] = mu * (H[i][j] + gh) + lam * lnJ * G[i][j];
      }
  }
  __device__ __forceinline__ void block(int i, int k, T C[3][3]) const {
#pragma unroll
    for (int J = 0; J < 3; ++J)
#pragma unroll
      for (int L = 0; L < 3; ++L)
        C[J][L] = (i == k && J == L ? mu : T(0)) + c1 * G[i][L] * G[k][J] + lam * G[i][J] * G[k][L];
  }
};

// J^{-2/3} and J^{-4/3} of the Mooney-Rivlin law: exp(-(2/3) log1p(J - 1))
// (accurate for J near 1); in double-float, J^{-1/3} from the FP32 reciprocal
// cube root refined by one Newton step t <- t + t (1 - J t^3) / 3 with the
// residual in double-float (quadratic convergence: about 1e-7 -> 1e-14),
// no transcendental.
template <typename T>
__device__ __forceinline__ void mr_jpow(const Kin<T> &k, T &j23, T &j43) {
  const T lnJ = mlog1p(k.Jm1);
  j23 = mexp(T(-2.0 / 3.0) * lnJ);
  j43 = mexp(T(-4.0 / 3.0) * lnJ);
}
template <>
__device__ __forceinline__ void mr_jpow<dfloat>(const Kin<dfloat> &k, dfloat &j23, dfloat &j43) {
  const dfloat t0(rcbrtf(k.J.hi), 0.f);
  const dfloat e = dfloat(1) - k.J * (t0 * t0 * t0);
  const dfloat t = t0 + t0 * e * dfloat(1.0 / 3.0);
  j23 = t * t;
  j43 = j23 * j23;
}

// Decoupled Mooney-Rivlin: psi = C10 (J^{-2/3} I1 - 3) + C01 (J^{-4/3} I2 - 3)
// + kappa/2 (J - 1)^2, with I1 = tr C, I2 = ((tr C)^2 - tr C^2)/2.
template <typename T>
struct Law<FE_MOONEY_RIVLIN, T> {
  T F[3][3], G[3][3], R[3][3], Cm[3][3], B[3][3];
  T cdd, gam, cff, cxg, cm;
  __device__ void init(const Kin<T> &k, const T H[3][3], T c10, T c01, T kap, T P[3][3]) {
    T j23, j43;
    mr_jpow(k, j23, j43);
    T a = c10 * j23;
    T b = c01 * j43;
    T J = k.J;
    // stress: P = G (4a devE + b Q) + kappa (J-1) J G,
    // Q = 4 devE + 8 trE devE - 8 dev(E^2)
    T E2[3][3];
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
      for (int j = 0; j < 3; ++j) {
        T s = T(0);
#pragma unroll
        for (int l = 0; l < 3; ++l) s += k.E[i][l] * k.E[l][j];
        E2[i][j] = s;
      }
    T trE2 = tr3(E2);
    T M[3][3];
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
      for (int j = 0; j < 3; ++j) {
        T dE = k.E[i][j] - (i == j ? k.trE / T(3) : T(0));
        T dE2 = E2[i][j] - (i == j ? trE2 / T(3) : T(0));
        M[i][j] = T(4) * a * dE + b * (T(4) * dE + T(8) * k.trE * dE - T(8) * dE2);
      }
    T pj = kap * k.Jm1 * J;
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
      for (int j = 0; j < 3; ++j) {
        T s = T(0);
#pragma unroll
        for (int l = 0; l < 3; ++l) s += k.G[i][l] * M[l][j];
        P[i][j] = s + pj * k.G[i][j];
      }
    // tangent coefficients
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
      for (int j = 0; j < 3; ++j) {
        F[i][j] = k.F[i][j];
        G[i][j] = k.G[i][j];
        Cm[i][j] = T(2) * k.E[i][j] + (i == j ? T(1) : T(0));
      }
    T I1 = tr3(Cm);
    T trC2 = T(0);
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
      for (int j = 0; j < 3; ++j) trC2 += Cm[i][j] * Cm[j][i];
    T I2 = T(0.5) * (I1 * I1 - trC2);
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
      for (int j = 0; j < 3; ++j) {
        T fc = T(0), bb = T(0);
#pragma unroll
        for (int l = 0; l < 3; ++l) {
          fc += F[i][l] * Cm[l][j];
          bb += F[i][l] * F[j][l];
        }
        B[i][j] = bb;
        R[i][j] = T(-4.0 / 3.0) * a * F[i][j] + T(-8.0 / 3.0) * b * (I1 * F[i][j] - fc);
      }
    cdd = T(2) * a + T(2) * b * I1;
    gam = T(4.0 / 9.0) * a * I1 + T(16.0 / 9.0) * b * I2 + kap * (T(2) * J - T(1)) * J;
    cff = T(4) * b;
    cxg = T(2.0 / 3.0) * a * I1 + T(4.0 / 3.0) * b * I2 - kap * (J * J - J);
    cm = T(-2) * b;
  }
  __device__ __forceinline__ void block(int i, int k, T C[3][3]) const {
#pragma unroll
    for (int J = 0; J < 3; ++J)
#pragma unroll
      for (int L = 0; L < 3; ++L)
        C[J][L] = (i == k && J == L ? cdd : T(0)) + R[i][J] * G[k][L] + G[i][J] * R[k][L] +
                  gam * G[i][J] * G[k][L] + cff * F[i][J] * F[k][L] + cxg * G[i][L] * G[k][J] +
                  cm * (F[i][L] * F[k][J] + (i == k ? Cm[L][J] : T(0)) + (J == L ? B[i][k] : T(0)));
  }
};

// Co-rotational linear elasticity (Section 3.1, Eq. "eqmodel": the rest
// stiffness int B^T D B rotated per element).  R is the rotation of the polar
// decomposition F = R S of the element's mean deformation gradient (one F for
// a tet, the volume average over the Gauss points for a hex).  With the
// local strain eps = sym(R^T F) - I and sigma = lambda tr(eps) I + 2 mu eps,
// P = R sigma and CC_iJkL = lambda R_iJ R_kL + mu (d_ik d_JL + R_iL R_kJ),
// i.e. K_e = Rb K0_e Rb^T and f_e = Rb K0_e (Rb^T x_e - X_e).  Without
// cancellation: S - I = Z is the Biot strain of the mean Green strain E
// ((I + Z)^2 = I + 2E, Newton iterations Z <- (I + Z)^{-1} (Z^2/2 + E) from
// Z = E), R = F (I + Z)^{-1}, and at a Gauss point
// eps = Z + sym(R^T (H - Hbar)).
template <typename T>
__device__ __forceinline__ void inv3(const T m[3][3], T r[3][3]) {
  const T c00 = m[1][1] * m[2][2] - m[1][2] * m[2][1], c01 = m[1][2] * m[2][0] - m[1][0] * m[2][2],
          c02 = m[1][0] * m[2][1] - m[1][1] * m[2][0];
  const T id = T(1) / (m[0][0] * c00 + m[0][1] * c01 + m[0][2] * c02);
  r[0][0] = c00 * id;
  r[1][0] = c01 * id;
  r[2][0] = c02 * id;
  r[0][1] = (m[0][2] * m[2][1] - m[0][1] * m[2][2]) * id;
  r[1][1] = (m[0][0] * m[2][2] - m[0][2] * m[2][0]) * id;
  r[2][1] = (m[0][1] * m[2][0] - m[0][0] * m[2][1]) * id;
  r[0][2] = (m[0][1] * m[1][2] - m[0][2] * m[1][1]) * id;
  r[1][2] = (m[0][2] * m[1][0] - m[0][0] * m[1][2]) * id;
  r[2][2] = (m[0][0] * m[1][1] - m[0][1] * m[1][0]) * id;
}

template <typename T>
struct Law<FE_COROTATIONAL, T> {
  T R[3][3], Z[3][3], Hb[3][3];
  T mu, lam;
  // the element's frame from its mean displacement gradient
  __device__ void set_frame(const T H[3][3]) {
    T E[3][3];
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
      for (int j = 0; j < 3; ++j) {
        Hb[i][j] = H[i][j];
        T s = H[i][j] + H[j][i];
#pragma unroll
        for (int k = 0; k < 3; ++k) s += H[k][i] * H[k][j];
        E[i][j] = T(0.5) * s;
        Z[i][j] = E[i][j];
      }
#pragma unroll 1
    for (int it = 0; it < 8; ++it) {
      T A[3][3], Ai[3][3], Bm[3][3];
#pragma unroll
      for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) {
          A[i][j] = Z[i][j] + (i == j ? T(1) : T(0));
          T zz = T(0);
#pragma unroll
          for (int k = 0; k < 3; ++k) zz += Z[i][k] * Z[k][j];
          Bm[i][j] = T(0.5) * zz + E[i][j];
        }
      inv3(A, Ai);
      T N[3][3];
#pragma unroll
      for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) {
          T s = T(0);
#pragma unroll
          for (int k = 0; k < 3; ++k) s += Ai[i][k] * Bm[k][j];
          N[i][j] = s;
        }
#pragma unroll
      for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) Z[i][j] = T(0.5) * (N[i][j] + N[j][i]);
    }
    T A[3][3], Ai[3][3];
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
      for (int j = 0; j < 3; ++j) A[i][j] = Z[i][j] + (i == j ? T(1) : T(0));
    inv3(A, Ai);
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
      for (int j = 0; j < 3; ++j) {
        T s = Ai[i][j];  // (I + H) (I + Z)^{-1}
#pragma unroll
        for (int k = 0; k < 3; ++k) s += H[i][k] * Ai[k][j];
        R[i][j] = s;
      }
  }
  __device__ void init(const Kin<T> &, const T H[3][3], T p0, T p1, T, T P[3][3]) {
    mu = p0;
    lam = p1;
    T D[3][3], ep[3][3];
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
      for (int j = 0; j < 3; ++j) D[i][j] = H[i][j] - Hb[i][j];
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
      for (int j = 0; j < 3; ++j) {
        T a = T(0), b = T(0);  // (R^T D)_ij, (R^T D)_ji
#pragma unroll
        for (int k = 0; k < 3; ++k) {
          a += R[k][i] * D[k][j];
          b += R[k][j] * D[k][i];
        }
        ep[i][j] = Z[i][j] + T(0.5) * (a + b);
      }
    const T tre = tr3(ep);
    T sg[3][3];
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
      for (int j = 0; j < 3; ++j) sg[i][j] = T(2) * mu * ep[i][j] + (i == j ? lam * tre : T(0));
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
      for (int j = 0; j < 3; ++j) {
        T s = T(0);
#pragma unroll
        for (int k = 0; k < 3; ++k) s += R[i][k] * sg[k][j];
        P[i][j] = s;
      }
  }
  __device__ __forceinline__ void block(int i, int k, T C[3][3]) const {
#pragma unroll
    for (int J = 0; J < 3; ++J)
#pragma unroll
      for (int L = 0; L < 3; ++L)
        C[J][L] = lam * R[i][J] * R[k][L] + mu * ((i == k && J == L ? T(1) : T(0)) + R[i][L] * R[k][J]);
  }
};

}  // namespace fe
