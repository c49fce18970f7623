// dvbm_q16.cuh -- the total-energy split (I) on the D2Q16 lattice: lattice,
// moments, equilibria and quasi-equilibria, Grad expansion (double and block
// fixed point).  Shared by the D2Q16 step kernel (dvbm_d2q16.cu) and the
// lattice-templated auxiliary kernels (dvbm_aux.cu).
//
// Same time step as the D2Q25 / split II kernels (Eq. finalDiscretePDE), with
//  * the D2Q16 Gauss--Hermite lattice (App. G, Table "D2Q16"): 1-D nodes
//    +-sqrt(3 -+ sqrt 6) with weights (3 +- sqrt 6)/12;
//  * E = sum g (Eq. eq_quadratur3 (I)), f^eq to third order and g^eq to
//    second order (Sec. II.D.3, App. E), g^eq built from the split-I moments
//    of App. A: M0 = E, M1 = u (E + rho R T), M2 = rho R T uu + (E + rho R T)(uu + R T I);
//  * the split-I quasi-equilibria of Table I: Pr < 1: f* = f^eq,
//    M1(g*) = M1(g) - u.(M2(f) - M2(f^eq)); Pr > 1: M2(f*) = M2(f),
//    M1(g*) = M1(g^eq) + u.(M2(f) - M2(f^eq)); Pr = 1: equilibria.
// Populations: c = 4 p + q for f (0..15), 16 + 4 p + q for g, x-node p and
// y-node q in the order (+a, -a, +b, -b), a = sqrt(3 - sqrt 6), b = sqrt(3 + sqrt 6).
// FP64 storage; advection in block floating point on the integer pipe.
#pragma once
#include "dvbm_device.cuh"

namespace dvbm {
namespace q16 {

constexpr double YA = 0.7419637843027258;   // sqrt(3 - sqrt 6)
constexpr double YB = 2.3344142183389773;   // sqrt(3 + sqrt 6)
constexpr double VA = 0.45412414523193151;  // (3 + sqrt 6)/12
constexpr double VB = 0.045875854768068492; // (3 - sqrt 6)/12
constexpr int NP = 32;

__host__ __device__ constexpr double xi(int k) { return k == 0 ? YA : k == 1 ? -YA : k == 2 ? YB : -YB; }
__host__ __device__ constexpr double w(int k) { return k < 2 ? VA : VB; }
__host__ __device__ constexpr int sgn(int k) { return (k % 2 == 0) ? 1 : -1; }
__host__ __device__ constexpr double khq(int k, int n) { return w(k) * he(n, xi(k)) * inv_fact(n); }

struct Mom { double m00, m10, m01, m20, m11, m02, g00, g10, g01; };
struct Co {
  double f00, f10, f01, f20, f11, f02, f30, f21, f12, f03;
  double g00, g10, g01, g20, g11, g02;  // physical energy units
  double a1;
  bool bad;
};

template <int p>
__device__ __forceinline__ void accumulate(Mom& m, const double (&f)[4], const double (&g)[4]) {
  const double sA = f[0] + f[1], dA = f[0] - f[1], sB = f[2] + f[3], dB = f[2] - f[3];
  const double m0 = sA + sB;
  const double m1 = fma(YA, dA, YB * dB);
  const double m2 = fma(YA * YA, sA, (YB * YB) * sB);
  const double n0 = (g[0] + g[1]) + (g[2] + g[3]);
  const double n1 = fma(YA, g[0] - g[1], YB * (g[2] - g[3]));
  constexpr double x = xi(p);
  m.m00 += m0; m.m01 += m1; m.m02 += m2;
  m.m10 = fma(x, m0, m.m10);
  m.m11 = fma(x, m1, m.m11);
  m.m20 = fma(x * x, m0, m.m20);
  m.g00 += n0; m.g01 += n1;
  m.g10 = fma(x, n0, m.g10);
}

struct Eq3 { double a00, a10, a01, a20, a11, a02, a30, a21, a12, a03; };
struct EqG { double A00, A10, A01, A20, A11, A02; };

__device__ __forceinline__ Eq3 eq_f3(double rho, double ux, double uy, double s) {
  Eq3 e;
  const double rs = rho * s;
  e.a00 = rho; e.a10 = rho * ux; e.a01 = rho * uy;
  e.a20 = fma(e.a10, ux, rs); e.a11 = e.a10 * uy; e.a02 = fma(e.a01, uy, rs);
  e.a30 = fma(e.a20, ux, 2.0 * s * e.a10); e.a03 = fma(e.a02, uy, 2.0 * s * e.a01);
  e.a21 = e.a20 * uy; e.a12 = e.a02 * ux;
  return e;
}

// g^eq coefficients of split I in physical units: E the total energy, pRT = rho R T
__device__ __forceinline__ EqG eq_g1(double E, double pRT, double ux, double uy, double theta) {
  EqG q;
  const double Ep = E + pRT;
  q.A00 = E;
  q.A10 = ux * Ep;
  q.A01 = uy * Ep;
  q.A20 = fma(pRT, ux * ux, Ep * fma(ux, ux, theta)) - E;
  q.A11 = (pRT + Ep) * ux * uy;
  q.A02 = fma(pRT, uy * uy, Ep * fma(uy, uy, theta)) - E;
  return q;
}

template <int PRC>
__device__ __forceinline__ Co coeffs(const Mom& m, const Phys& P) {
  Co C;
  const double rho = m.m00;
  const double irho = 1.0 / rho;
  const double ux = m.m10 * irho, uy = m.m01 * irho;
  const double E = m.g00;
  const double theta = P.gm1 * fma(-0.5, fma(ux, ux, uy * uy), E * P.inv_c2 * irho);
  const double s = theta - 1.0;
  C.bad = !(rho > 0.0) || !(theta > 0.0) || !(fabs(E) < 1e300);
  const double pRT = rho * P.c2 * theta;
  double k1, k2;
  if (PRC <= 0) { k1 = P.dt_mu * pRT; k2 = k1 * P.Pr; }
  else          { k2 = P.dt_mu * pRT; k1 = k2 * P.Pr; }
  const double s1 = k1 - k2;
  C.a1 = 1.0 - k1;
  const Eq3 e = eq_f3(rho, ux, uy, s);
  const EqG q = eq_g1(E, pRT, ux, uy, theta);
  double d20 = 0, d11 = 0, d02 = 0, dg10 = 0, dg01 = 0;
  if (PRC != 0) {
    const double Dxx = (m.m20 - rho) - e.a20, Dxy = m.m11 - e.a11, Dyy = (m.m02 - rho) - e.a02;
    const double ux_ = P.c2 * fma(ux, Dxx, uy * Dxy), uy_ = P.c2 * fma(ux, Dxy, uy * Dyy);  // c^2 (u . Delta)
    if (PRC < 0) {
      dg10 = (m.g10 - ux_) - q.A10;
      dg01 = (m.g01 - uy_) - q.A01;
    } else {
      d20 = Dxx; d11 = Dxy; d02 = Dyy;
      dg10 = ux_; dg01 = uy_;
    }
  }
  C.f00 = k1 * e.a00; C.f10 = k1 * e.a10; C.f01 = k1 * e.a01;
  C.f20 = fma(s1, d20, k1 * e.a20); C.f11 = fma(s1, d11, k1 * e.a11); C.f02 = fma(s1, d02, k1 * e.a02);
  C.f30 = k1 * e.a30; C.f21 = k1 * e.a21; C.f12 = k1 * e.a12; C.f03 = k1 * e.a03;
  C.g00 = k1 * q.A00;
  C.g10 = fma(s1, dg10, k1 * q.A10); C.g01 = fma(s1, dg01, k1 * q.A01);
  C.g20 = k1 * q.A20; C.g11 = k1 * q.A11; C.g02 = k1 * q.A02;
  return C;
}

// equilibrium populations (k1 = 1, no quasi-equilibrium part)
__device__ __forceinline__ Co equilibrium(double rho, double ux, double uy, double theta, const Phys& P) {
  Co C;
  const Eq3 e = eq_f3(rho, ux, uy, theta - 1.0);
  const double pRT = rho * P.c2 * theta;
  const double E = rho * P.c2 * (theta / P.gm1 + 0.5 * fma(ux, ux, uy * uy));
  const EqG q = eq_g1(E, pRT, ux, uy, theta);
  C.f00 = e.a00; C.f10 = e.a10; C.f01 = e.a01; C.f20 = e.a20; C.f11 = e.a11; C.f02 = e.a02;
  C.f30 = e.a30; C.f21 = e.a21; C.f12 = e.a12; C.f03 = e.a03;
  C.g00 = q.A00; C.g10 = q.A10; C.g01 = q.A01; C.g20 = q.A20; C.g11 = q.A11; C.g02 = q.A02;
  C.a1 = 0.0;
  C.bad = false;
  return C;
}

template <int p>
__device__ __forceinline__ void hf(const Co& C, double (&h)[4]) {
  h[0] = fma(khq(p, 3), C.f30, fma(khq(p, 2), C.f20, fma(khq(p, 1), C.f10, khq(p, 0) * C.f00)));
  h[1] = fma(khq(p, 2), C.f21, fma(khq(p, 1), C.f11, khq(p, 0) * C.f01));
  h[2] = fma(khq(p, 1), C.f12, khq(p, 0) * C.f02);
  h[3] = khq(p, 0) * C.f03;
}
template <int p>
__device__ __forceinline__ void hg(const Co& C, double (&h)[4]) {
  h[0] = fma(khq(p, 2), C.g20, fma(khq(p, 1), C.g10, khq(p, 0) * C.g00));
  h[1] = fma(khq(p, 1), C.g11, khq(p, 0) * C.g01);
  h[2] = khq(p, 0) * C.g02;
  h[3] = 0.0;
}
// t_q = W_q sum_b h^b He_b(xi_q)/b!, nodes (+a, -a, +b, -b)
__device__ __forceinline__ void expand(const double (&h)[4], double (&t)[4]) {
  const double EA = fma(khq(0, 2), h[2], khq(0, 0) * h[0]);
  const double OA = fma(khq(0, 3), h[3], khq(0, 1) * h[1]);
  const double EB = fma(khq(2, 2), h[2], khq(2, 0) * h[0]);
  const double OB = fma(khq(2, 3), h[3], khq(2, 1) * h[1]);
  t[0] = EA + OA; t[1] = EA - OA; t[2] = EB + OB; t[3] = EB - OB;
}

__device__ __forceinline__ Mom cell_moments(const double* s, long long PL) {
  Mom m = {};
  double f[4], g[4];
#define Q16_MOM(p)                                                     \
  _Pragma("unroll") for (int q = 0; q < 4; ++q) {                     \
    f[q] = __ldg(s + (4 * p + q) * PL);                                \
    g[q] = __ldg(s + (16 + 4 * p + q) * PL);                           \
  }                                                                    \
  accumulate<p>(m, f, g);
  Q16_MOM(0) Q16_MOM(1) Q16_MOM(2) Q16_MOM(3)
#undef Q16_MOM
  return m;
}

__device__ __forceinline__ void macro(const Mom& m, const Phys& P, double c, double T_ref, double& rho, double& ux,
                                      double& uy, double& T) {
  rho = m.m00;
  const double irho = 1.0 / rho;
  const double a = m.m10 * irho, b = m.m01 * irho;
  const double theta = P.gm1 * fma(-0.5, fma(a, a, b * b), m.g00 * P.inv_c2 * irho);
  ux = a * c;
  uy = b * c;
  T = theta * T_ref;
}

// write the expansion of C (plus optional per-population additions)
__device__ __forceinline__ void write_expansion(double* d, long long PL, const Co& C, const double* addf,
                                                const double* addg) {
#define Q16_EXP(p)                                                     \
  {                                                                    \
    double h[4], t[4], hh[4], tt[4];                                   \
    hf<p>(C, h); expand(h, t); hg<p>(C, hh); expand(hh, tt);           \
    _Pragma("unroll") for (int q = 0; q < 4; ++q) {                    \
      d[(4 * p + q) * PL] = t[q] + (addf ? addf[4 * p + q] : 0.0);     \
      d[(16 + 4 * p + q) * PL] = tt[q] + (addg ? addg[4 * p + q] : 0.0); \
    }                                                                  \
  }
  Q16_EXP(0) Q16_EXP(1) Q16_EXP(2) Q16_EXP(3)
#undef Q16_EXP
}

// ---- fixed-point expansion (as in dvbm_device.cuh for D2Q25) -------------
// node constants khq(k, n) 2^(63 + kdq(k)) (|khq| < 0.46; the +-sqrt(3 + sqrt 6)
// nodes carry the small weight and gain two bits)
__host__ __device__ constexpr int kdq(int k) { return k < 2 ? 0 : 2; }
__host__ __device__ constexpr long long khqfix(int k, int n) {
  return (long long)(khq(k, n) * 9223372036854775808.0 * (double)(1 << kdq(k)));
}
struct CoFix {
  long long f00, f10, f01, f20, f11, f02, f30, f21, f12, f03;
  long long g00, g10, g01, g20, g11, g02;
  int Ef, Eg;  // value = X 2^(E - 1082)
};
__device__ __forceinline__ CoFix to_fix(const Co& C) {
  CoFix X;
  const int Ef = max(max(max(max(bexp(C.f00), bexp(C.f10)), max(bexp(C.f01), bexp(C.f20))),
                         max(max(bexp(C.f11), bexp(C.f02)), max(bexp(C.f30), bexp(C.f21)))),
                     max(bexp(C.f12), bexp(C.f03)));
  const int Eg = max(max(max(bexp(C.g00), bexp(C.g10)), max(bexp(C.g01), bexp(C.g20))),
                     max(bexp(C.g11), bexp(C.g02)));
  X.f00 = to_block_fixed(C.f00, Ef); X.f10 = to_block_fixed(C.f10, Ef); X.f01 = to_block_fixed(C.f01, Ef);
  X.f20 = to_block_fixed(C.f20, Ef); X.f11 = to_block_fixed(C.f11, Ef); X.f02 = to_block_fixed(C.f02, Ef);
  X.f30 = to_block_fixed(C.f30, Ef); X.f21 = to_block_fixed(C.f21, Ef); X.f12 = to_block_fixed(C.f12, Ef);
  X.f03 = to_block_fixed(C.f03, Ef);
  X.g00 = to_block_fixed(C.g00, Eg); X.g10 = to_block_fixed(C.g10, Eg); X.g01 = to_block_fixed(C.g01, Eg);
  X.g20 = to_block_fixed(C.g20, Eg); X.g11 = to_block_fixed(C.g11, Eg); X.g02 = to_block_fixed(C.g02, Eg);
  X.Ef = Ef;
  X.Eg = Eg;
  return X;
}
// t_q = sum_b h^b khq(q, b) with the +-xi symmetry (nodes +a, -a, +b, -b)
__device__ __forceinline__ void expand_fix(const long long (&h)[4], long long (&t)[4]) {
  const long long EA = mhk(h[0], khqfix(0, 0)) + mhk(h[2], khqfix(0, 2));
  const long long OA = mhk(h[1], khqfix(0, 1)) + mhk(h[3], khqfix(0, 3));
  const long long EB = mhk(h[0], khqfix(2, 0)) + mhk(h[2], khqfix(2, 2));
  const long long OB = mhk(h[1], khqfix(2, 1)) + mhk(h[3], khqfix(2, 3));
  t[0] = EA + OA; t[1] = EA - OA; t[2] = EB + OB; t[3] = EB - OB;
}
__device__ __forceinline__ void expand3_fix(const long long (&h)[3], long long (&t)[4]) {
  const long long EA = mhk(h[0], khqfix(0, 0)) + mhk(h[2], khqfix(0, 2));
  const long long OA = mhk(h[1], khqfix(0, 1));
  const long long EB = mhk(h[0], khqfix(2, 0)) + mhk(h[2], khqfix(2, 2));
  const long long OB = mhk(h[1], khqfix(2, 1));
  t[0] = EA + OA; t[1] = EA - OA; t[2] = EB + OB; t[3] = EB - OB;
}

}  // namespace q16

namespace q16 {
// populations of the equilibrium coefficient set C (a1 = 0) by the step
// kernel's fixed-point expansion (FP64-or-better precision): initial conditions
__device__ __forceinline__ void write_equilibrium_fix16(double* d, long long PL, const Co& C) {
  const CoFix X = to_fix(C);
#pragma unroll
  for (int p = 0; p < 4; ++p) {
    const long long k0 = khqfix(p, 0), k1 = khqfix(p, 1), k2 = khqfix(p, 2), k3 = khqfix(p, 3);
    long long h[4], hh[3], xf[4], xg[4];
    h[0] = mhk(X.f00, k0) + mhk(X.f10, k1) + mhk(X.f20, k2) + mhk(X.f30, k3);
    h[1] = mhk(X.f01, k0) + mhk(X.f11, k1) + mhk(X.f21, k2);
    h[2] = mhk(X.f02, k0) + mhk(X.f12, k1);
    h[3] = mhk(X.f03, k0);
    hh[0] = mhk(X.g00, k0) + mhk(X.g10, k1) + mhk(X.g20, k2);
    hh[1] = mhk(X.g01, k0) + mhk(X.g11, k1);
    hh[2] = mhk(X.g02, k0);
    const int sf = renorm_fix(h), sg = renorm_fix(hh);
    expand_fix(h, xf);
    expand3_fix(hh, xg);
    const int dp = kdq(p);
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      d[(4 * p + q) * PL] = X.Ef >= 100 ? ll_to_double_rn(xf[q], X.Ef - 1080 - dp - sf - kdq(q)) : 0.0;
      d[(16 + 4 * p + q) * PL] = X.Eg >= 100 ? ll_to_double_rn(xg[q], X.Eg - 1080 - dp - sg - kdq(q)) : 0.0;
    }
  }
}
}  // namespace q16

}  // namespace dvbm
