// dvbm_device.cuh -- device-side building blocks of the GB300 DVBM step.
//
// Model: double-distribution quasi-equilibrium BGK on the D2Q25 Gauss--Hermite
// lattice, internal non-translational energy split (II).  Everything here is
// written in units of c = sqrt(R T_ref): xi = v / c, theta = T / T_ref,
// Hermite coefficients A_ab = a_{x^a y^b} / c^(a+b), so that the Grad
// expansion (Sec. II.D.2, Eq. Grad_g; App. D) factorises into 1-D
// probabilists' Hermite polynomials:
//     F_pq = W_p W_q sum_{a+b<=N} A_ab He_a(xi_p) He_b(xi_q) / (a! b!).
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace dvbm {

// ---- D2Q25 lattice (App. G): 1-D nodes are the roots of He_5 ---------------
// node k: 0, +sqrt(5 - sqrt 10), -sqrt(5 - sqrt 10), +sqrt(5 + sqrt 10), -sqrt(5 + sqrt 10)
constexpr double XA = 1.3556261799742659;   // sqrt(5 - sqrt(10))
constexpr double XB = 2.8569700138728056;   // sqrt(5 + sqrt(10))
// 1-D Gauss--Hermite weights: 8/15 and (7 +- 2 sqrt 10)/60
constexpr double W0 = 0.53333333333333333;  // 8/15
constexpr double WA = 0.22207592200561264;  // (7 + 2 sqrt(10)) / 60
constexpr double WB = 0.011257411327720689; // (7 - 2 sqrt(10)) / 60

constexpr int Q = 25;
constexpr int NPOP = 50;  // f (0..24) and g (25..49); population c = 5 p + q

__host__ __device__ constexpr double xi_of(int k) {
  return k == 0 ? 0.0 : k == 1 ? XA : k == 2 ? -XA : k == 3 ? XB : -XB;
}
__host__ __device__ constexpr double w_of(int k) {
  return k == 0 ? W0 : (k <= 2 ? WA : WB);
}
__host__ __device__ constexpr int sgn_of(int k) { return k == 0 ? 0 : (k == 1 || k == 3) ? 1 : -1; }
// probabilists' Hermite polynomials He_n(x), n <= 4
__host__ __device__ constexpr double he(int n, double x) {
  return n == 0 ? 1.0 : n == 1 ? x : n == 2 ? x * x - 1.0 : n == 3 ? x * x * x - 3.0 * x
                                                                      : x * x * x * x - 6.0 * x * x + 3.0;
}
__host__ __device__ constexpr double inv_fact(int n) {
  return n == 0 ? 1.0 : n == 1 ? 1.0 : n == 2 ? 0.5 : n == 3 ? 1.0 / 6.0 : 1.0 / 24.0;
}
// W_k He_n(xi_k) / n!
__host__ __device__ constexpr double kh(int k, int n) { return w_of(k) * he(n, xi_of(k)) * inv_fact(n); }

// ---- launch-invariant parameters (passed by value, constant bank) ---------
struct Geom {
  int Nx, Ny;
  int pitch;             // elements per row (ghost columns included)
  int xoff;              // element offset of x = 0 inside a row
  long long plane;       // elements per population plane = (Ny + 4) * pitch
};

struct Phys {
  double c2, inv_c2;     // R T_ref and 1 / (R T_ref)
  double gm1;            // gamma - 1 = R / C_v
  double epsf;           // C_v/R - D/2 = (2 - gamma)/(gamma - 1): eps/(R T) of split II
  double dt, mu, Pr;
  double dt_mu;          // dt / mu
  int prc;               // -1: Pr < 1, 0: Pr == 1, +1: Pr > 1
  double hb;             // beta / 2
  long long hq;          // round(beta/2 * 2^62), integer-pipe limiter (general beta)
  int lp, lq;            // beta = lp / lq exactly (lq <= 64), or lq = 0: use hq
  double kxr[5], kyr[5]; // kxv / (4 lq), kyv / (4 lq): flux factors of the scaled differences
  double kxv[5], kyv[5]; // dt/dx * c * xi_k and dt/dy * c * xi_k
  float kxvf[5], kyvf[5];
  double fref0, gref0;   // FP32DEV reference: f_ref = w rho0, g_ref = w rho0 (C_v - R) T0
  double rho_ref_mom;    // unused padding for alignment
};

__device__ __forceinline__ long long cell_index(const Geom& G, int y, int x) {
  return (long long)(y + 2) * G.pitch + x + G.xoff;
}

// ---- macroscopic state and collision coefficients -------------------------
// Raw dimensionless moments of f (mu_ab = sum_i xi_x^a xi_y^b f_i, a + b <= 3)
// and of g (physical units: G00 = sum g, G10/G01 = sum xi g).
struct Moments {
  double m00, m10, m01, m20, m11, m02, m30, m21, m12, m03;
  double g00, g10, g01;
};

// Combined expansion coefficients of one collision:
//   F_new = a1 F + W W sum C_ab He He/(a! b!) - advection,
// with C = (dt/tau1) A^eq + (dt/tau1 - dt/tau2) (A* - A^eq), which equals
// F - (dt/tau1)(F - F*) - (dt/tau2)(F* - F^eq) by linearity of the expansion.
struct Coeffs {
  double f00, f10, f01, f20, f11, f02, f30, f21, f12, f03, f40, f31, f22, f13, f04;
  double g00, g10, g01, g20, g11, g02;  // physical units of g
  double a1;                            // 1 - dt/tau1
  double k1;                            // dt/tau1
  bool bad;                             // rho <= 0, theta <= 0 or not finite
};

// Equilibrium coefficients of f (App. D theta-form) for rho, u (in units of
// c) and s = theta - 1, via the 1-D Hermite recurrences
//   A_{n+1} = u A_n + n s A_{n-1} along each axis.
struct EqF { double a00, a10, a01, a20, a11, a02, a30, a21, a12, a03, a40, a31, a22, a13, a04; };

__device__ __forceinline__ EqF eq_f(double rho, double ux, double uy, double s) {
  EqF e;
  double rs = rho * s;
  e.a00 = rho;
  e.a10 = rho * ux;
  e.a01 = rho * uy;
  e.a20 = fma(e.a10, ux, rs);
  e.a11 = e.a10 * uy;
  e.a02 = fma(e.a01, uy, rs);
  e.a30 = fma(e.a20, ux, 2.0 * s * e.a10);
  e.a03 = fma(e.a02, uy, 2.0 * s * e.a01);
  e.a21 = e.a20 * uy;
  e.a12 = e.a02 * ux;
  e.a40 = fma(e.a30, ux, 3.0 * s * e.a20);
  e.a04 = fma(e.a03, uy, 3.0 * s * e.a02);
  e.a31 = e.a30 * uy;
  e.a13 = e.a03 * ux;
  e.a22 = e.a20 * fma(uy, uy, s);
  return e;
}

// Collision coefficients from the moments (Sec. II.C relaxation times,
// Table I split-II quasi-equilibria).  PRC selects the Prandtl case at
// compile time: -1 (Pr < 1), 0 (Pr = 1), +1 (Pr > 1).
//   Pr < 1: A*_3 = H_3(f) - S(u, Delta); A*_g1 = sum xi g; else equilibrium.
//   Pr > 1: A*_2 = A^eq_2 + Delta', A*_3 = A^eq_3 + S(u, Delta'),
//           A*_4 = A^eq_4 - [Delta' delta]_cyc; g* = g^eq,
// with Delta = H_2(f) - A^eq_2, Delta' its traceless part and
// S(u, A)_abc = [u_a A_bc]_cyc - tr(A)/(D+2) [u_a d_bc]_cyc, the symmetric
// tensor whose contraction is the heat-flux constraint 2 (A u)_a.
template <int PRC>
__device__ __forceinline__ Coeffs collision_coeffs(const Moments& m, const Phys& P) {
  Coeffs C;
  const double rho = m.m00;
  const double irho = 1.0 / rho;
  const double ux = m.m10 * irho, uy = m.m01 * irho;
  const double Et = fma(0.5, m.m20 + m.m02, m.g00 * P.inv_c2);        // E / c^2
  const double theta = P.gm1 * fma(-0.5, fma(ux, ux, uy * uy), Et * irho);
  const double s = theta - 1.0;
  C.bad = !(rho > 0.0) || !(theta > 0.0) || !(fabs(Et) < 1e300);
  const double p = rho * P.c2 * theta;                                   // rho R T
  double k1, k2;                                                         // dt/tau1, dt/tau2
  if (PRC <= 0) { k1 = P.dt_mu * p; k2 = k1 * P.Pr; }
  else          { k2 = P.dt_mu * p; k1 = k2 * P.Pr; }
  const double s1 = k1 - k2;
  C.a1 = 1.0 - k1;
  C.k1 = k1;
  EqF e = eq_f(rho, ux, uy, s);
  // deviations dA = A* - A^eq (zero where Table I keeps equilibrium moments)
  double d20 = 0, d11 = 0, d02 = 0, d30 = 0, d21 = 0, d12 = 0, d03 = 0;
  double d40 = 0, d31 = 0, d13 = 0, d04 = 0, dg10 = 0, dg01 = 0;
  const double reps = rho * P.epsf * theta;                               // rho eps / c^2
  if (PRC != 0) {
    // Delta = H_2(f) - A^eq_2 with H_20 = mu_20 - rho, H_11 = mu_11, H_02 = mu_02 - rho
    const double Dxx = (m.m20 - rho) - e.a20;
    const double Dxy = m.m11 - e.a11;
    const double Dyy = (m.m02 - rho) - e.a02;
    if (PRC < 0) {
      const double kap = 0.25 * (Dxx + Dyy);                            // tr(Delta)/(D+2)
      const double Px = Dxx - kap, Py = Dyy - kap;
      // H_3(f): mu_30 - 3 mu_10, mu_21 - mu_01, mu_12 - mu_10, mu_03 - 3 mu_01
      d30 = (fma(-3.0, m.m10, m.m30) - e.a30) - 3.0 * ux * Px;
      d21 = ((m.m21 - m.m01) - e.a21) - fma(2.0 * ux, Dxy, uy * Px);
      d12 = ((m.m12 - m.m10) - e.a12) - fma(2.0 * uy, Dxy, ux * Py);
      d03 = (fma(-3.0, m.m01, m.m03) - e.a03) - 3.0 * uy * Py;
      // g*: first moment of g (in units of c^2), minus its equilibrium value
      dg10 = m.g10 * P.inv_c2 - reps * ux;
      dg01 = m.g01 * P.inv_c2 - reps * uy;
    } else {
      const double Tx = 0.5 * (Dxx - Dyy);                              // Delta'_xx = -Delta'_yy
      d20 = Tx; d11 = Dxy; d02 = -Tx;
      d30 = 3.0 * ux * Tx;
      d21 = fma(uy, Tx, 2.0 * ux * Dxy);
      d12 = fma(-ux, Tx, 2.0 * uy * Dxy);
      d03 = -3.0 * uy * Tx;
      d40 = -6.0 * Tx; d31 = -3.0 * Dxy; d13 = -3.0 * Dxy; d04 = 6.0 * Tx;
    }
  }
  C.f00 = k1 * e.a00;
  C.f10 = k1 * e.a10;
  C.f01 = k1 * e.a01;
  C.f20 = fma(s1, d20, k1 * e.a20);
  C.f11 = fma(s1, d11, k1 * e.a11);
  C.f02 = fma(s1, d02, k1 * e.a02);
  C.f30 = fma(s1, d30, k1 * e.a30);
  C.f21 = fma(s1, d21, k1 * e.a21);
  C.f12 = fma(s1, d12, k1 * e.a12);
  C.f03 = fma(s1, d03, k1 * e.a03);
  C.f40 = fma(s1, d40, k1 * e.a40);
  C.f31 = fma(s1, d31, k1 * e.a31);
  C.f22 = k1 * e.a22;
  C.f13 = fma(s1, d13, k1 * e.a13);
  C.f04 = fma(s1, d04, k1 * e.a04);
  // g^eq (split II): A00 = rho eps, A10 = rho eps ux, A20 = rho eps (ux^2 + s) ...
  // (units of c^2; multiplied back by c^2 for physical g)
  const double kg = k1 * P.c2;
  const double sg = s1 * P.c2;
  C.g00 = kg * reps;
  C.g10 = fma(sg, dg10, kg * reps * ux);
  C.g01 = fma(sg, dg01, kg * reps * uy);
  C.g20 = kg * reps * fma(ux, ux, s);
  C.g11 = kg * reps * ux * uy;
  C.g02 = kg * reps * fma(uy, uy, s);
  return C;
}

// Pure equilibrium coefficients (for initial conditions and wall ghosts):
// same layout as Coeffs with C = A^eq, physical g.
__device__ __forceinline__ Coeffs equilibrium_coeffs(double rho, double ux, double uy, double theta,
                                                     const Phys& P) {
  Coeffs C;
  const double s = theta - 1.0;
  EqF e = eq_f(rho, ux, uy, s);
  C.f00 = e.a00; C.f10 = e.a10; C.f01 = e.a01; C.f20 = e.a20; C.f11 = e.a11; C.f02 = e.a02;
  C.f30 = e.a30; C.f21 = e.a21; C.f12 = e.a12; C.f03 = e.a03;
  C.f40 = e.a40; C.f31 = e.a31; C.f22 = e.a22; C.f13 = e.a13; C.f04 = e.a04;
  const double reps = rho * P.epsf * theta * P.c2;
  C.g00 = reps; C.g10 = reps * ux; C.g01 = reps * uy;
  C.g20 = reps * fma(ux, ux, s); C.g11 = reps * ux * uy; C.g02 = reps * fma(uy, uy, s);
  C.a1 = 0.0; C.k1 = 1.0; C.bad = false;
  return C;
}

// Macroscopic values (rho, u in physical units, T) from moments.
__device__ __forceinline__ void macro_from_moments(const Moments& m, const Phys& P, double c, double T_ref,
                                                   double& rho, double& ux, double& uy, double& T) {
  rho = m.m00;
  const double irho = 1.0 / rho;
  const double uxd = m.m10 * irho, uyd = m.m01 * irho;
  const double Et = fma(0.5, m.m20 + m.m02, m.g00 * P.inv_c2);
  const double theta = P.gm1 * fma(-0.5, fma(uxd, uxd, uyd * uyd), Et * irho);
  ux = uxd * c;
  uy = uyd * c;
  T = theta * T_ref;
}

// ---- sum-factorised moment accumulation -----------------------------------
// Accumulate the contribution of the five populations (p, q = 0..4) of one
// x-node p.  f[q] and g[q] are the values (double).
template <int p>
__device__ __forceinline__ void accumulate_moments(Moments& m, const double (&f)[5], const double (&g)[5]) {
  const double sA = f[1] + f[2], dA = f[1] - f[2], sB = f[3] + f[4], dB = f[3] - f[4];
  const double m0 = f[0] + sA + sB;
  const double m1 = fma(XA, dA, XB * dB);
  const double m2 = fma(XA * XA, sA, (XB * XB) * sB);
  const double m3 = fma(XA * XA * XA, dA, (XB * XB * XB) * dB);
  const double n0 = g[0] + (g[1] + g[2]) + (g[3] + g[4]);
  const double n1 = fma(XA, g[1] - g[2], XB * (g[3] - g[4]));
  m.m00 += m0; m.m01 += m1; m.m02 += m2; m.m03 += m3;
  m.g00 += n0; m.g01 += n1;
  if (p != 0) {
    constexpr double x = xi_of(p);
    m.m10 = fma(x, m0, m.m10);
    m.m11 = fma(x, m1, m.m11);
    m.m12 = fma(x, m2, m.m12);
    m.m20 = fma(x * x, m0, m.m20);
    m.m21 = fma(x * x, m1, m.m21);
    m.m30 = fma(x * x * x, m0, m.m30);
    m.g10 = fma(x, n0, m.g10);
  }
}

// ---- sum-factorised Grad expansion ----------------------------------------
// h^b_p = W_p sum_a C_ab He_a(xi_p)/a!  for the f expansion (N = 4).
template <int p>
__device__ __forceinline__ void hf_of(const Coeffs& C, double (&h)[5]) {
  if (p != 0) {
    h[0] = fma(kh(p, 4), C.f40, fma(kh(p, 3), C.f30, fma(kh(p, 2), C.f20, fma(kh(p, 1), C.f10, kh(p, 0) * C.f00))));
    h[1] = fma(kh(p, 3), C.f31, fma(kh(p, 2), C.f21, fma(kh(p, 1), C.f11, kh(p, 0) * C.f01)));
    h[2] = fma(kh(p, 2), C.f22, fma(kh(p, 1), C.f12, kh(p, 0) * C.f02));
    h[3] = fma(kh(p, 1), C.f13, kh(p, 0) * C.f03);
  } else {  // He_1(0) = He_3(0) = 0
    h[0] = fma(kh(p, 4), C.f40, fma(kh(p, 2), C.f20, kh(p, 0) * C.f00));
    h[1] = fma(kh(p, 2), C.f21, kh(p, 0) * C.f01);
    h[2] = fma(kh(p, 2), C.f22, kh(p, 0) * C.f02);
    h[3] = kh(p, 0) * C.f03;
  }
  h[4] = kh(p, 0) * C.f04;
}
template <int p>
__device__ __forceinline__ void hg_of(const Coeffs& C, double (&h)[3]) {
  if (p != 0) {
    h[0] = fma(kh(p, 2), C.g20, fma(kh(p, 1), C.g10, kh(p, 0) * C.g00));
    h[1] = fma(kh(p, 1), C.g11, kh(p, 0) * C.g01);
  } else {
    h[0] = fma(kh(p, 2), C.g20, kh(p, 0) * C.g00);
    h[1] = kh(p, 0) * C.g01;
  }
  h[2] = kh(p, 0) * C.g02;
}
// t_q = W_q sum_b h^b He_b(xi_q)/b! for the five y-nodes, using the +-xi
// symmetry: even part E and odd part O, t(+xi) = E + O, t(-xi) = E - O.
__device__ __forceinline__ void expand_q5(const double (&h)[5], double (&t)[5]) {
  t[0] = fma(kh(0, 4), h[4], fma(kh(0, 2), h[2], kh(0, 0) * h[0]));
  const double EA = fma(kh(1, 4), h[4], fma(kh(1, 2), h[2], kh(1, 0) * h[0]));
  const double OA = fma(kh(1, 3), h[3], kh(1, 1) * h[1]);
  const double EB = fma(kh(3, 4), h[4], fma(kh(3, 2), h[2], kh(3, 0) * h[0]));
  const double OB = fma(kh(3, 3), h[3], kh(3, 1) * h[1]);
  t[1] = EA + OA; t[2] = EA - OA; t[3] = EB + OB; t[4] = EB - OB;
}
__device__ __forceinline__ void expand_q3(const double (&h)[3], double (&t)[5]) {
  t[0] = fma(kh(0, 2), h[2], kh(0, 0) * h[0]);
  const double EA = fma(kh(1, 2), h[2], kh(1, 0) * h[0]);
  const double OA = kh(1, 1) * h[1];
  const double EB = fma(kh(3, 2), h[2], kh(3, 0) * h[0]);
  const double OB = kh(3, 1) * h[1];
  t[1] = EA + OA; t[2] = EA - OA; t[3] = EB + OB; t[4] = EB - OB;
}

// ---- limited slope of the NND reconstruction (Sec. III.A.2) --------------
// sigma(a, b) = (b/2) phi(a/b) = 1/2 minmod3(beta a, (a+b)/2, beta b)
//             = minmod3(hb a, (a+b)/4, hb b),  hb = beta/2,
// (division-free; 0 if a and b differ in sign; b = 0 gives 0).  This float
// form serves the FP32-deviation storage; FP64 storage runs the same limiter
// exactly on integers (below).
__device__ __forceinline__ float limited_slope(float a, float b, float hb) {
  const float x = hb * a, z = hb * b, y = 0.25f * (a + b);
  const float mn = fminf(fminf(fabsf(x), fabsf(y)), fabsf(z));
  return ((__float_as_int(a) ^ __float_as_int(b)) >= 0) ? copysignf(mn, a) : 0.0f;
}

// ---- FP64 advection in block floating point on the integer pipe ----------
// GB300 runs FP64 at 1/64 of the FP32 rate, while integer ops are cheap.  The
// four values of one upwind stencil are brought to their largest exponent E
// as 60-bit integers X = M 2^(e - E + 7) (M the 53-bit significand), so that
// differences, the beta/2 scaling, the minmod selection and the flux
// difference are exact integer arithmetic (truncation only below 2^-60 of the
// largest value); only the result is converted back to double.  The
// conversions are pure bit manipulation.
__device__ __forceinline__ int bexp(double v) { return (__double2hiint(v) >> 20) & 0x7ff; }

// Zero (and subnormal) inputs need no special case: their shift E - e is 63
// whenever E >= 61, which leaves 0; every caller treats E < 64 as "all values
// negligible" and returns 0 before using the result.
__device__ __forceinline__ long long to_block_fixed(double v, int E) {
  const int hi = __double2hiint(v);
  const unsigned lo = (unsigned)__double2loint(v);
  const int e = (hi >> 20) & 0x7ff;
  const unsigned long long m = ((unsigned long long)((unsigned)(hi & 0xfffff) | 0x100000u) << 32) | lo;
  const unsigned long long mag = (m << 7) >> min(E - e, 63);
  return hi < 0 ? -(long long)mag : (long long)mag;
}

// int64 -> double by bit manipulation (the hardware conversion runs at the FP64
// rate on GB300): |F| is normalised with a count of leading zeros, its top 53
// bits become the significand (truncating the rest, < 2^-52 relative), and
// the exponent is that of F times 2^scale.  F = 0 gives 0.
__device__ __forceinline__ double ll_to_double_scaled(long long F, int scale) {
  if (F == 0) return 0.0;
  const unsigned long long mag = F < 0 ? (unsigned long long)(-F) : (unsigned long long)F;
  const int lz = __clzll(mag);
  const unsigned long long norm = mag << lz;           // leading one at bit 63
  const unsigned long long frac = (norm >> 11) & 0x000fffffffffffffull;
  const int ex = 1023 + 63 - lz + scale;
  const unsigned hi = (unsigned)(frac >> 32) | ((unsigned)ex << 20) | (F < 0 ? 0x80000000u : 0u);
  return __hiloint2double((int)hi, (int)(unsigned)frac);
}

// ---- fixed-point Grad expansion (FP64 storage) ----------------------------
// The expansion t = W W sum C He He /(a! b!) is a fixed linear map of the
// collision coefficients.  On GB300 the FP64 pipe (2 ops / clock / SM) is the
// bottleneck of the step, so the expansion runs in block fixed point on the
// integer pipe: the coefficients of one cell share an exponent (f and g
// separately) as 60-bit integers, the node constants kh(k, n) (all |kh| < 0.54)
// are fractions scaled per node to 62-63 bits (kh(k, n) 2^(63 + kd(k)); the
// outer nodes carry the small weight W_B and gain four bits), each product is
// the high word of the 128-bit product, and the h values of each x-node are
// renormalised to 60 bits before the y-expansion.  Truncation stays below
// 2^-56 of the largest term at each stage; the result is rounded to nearest
// when it goes back to double, so the collision target carries no
// systematic bias into the conserved sums.
__host__ __device__ constexpr int kd(int k) { return k == 0 ? 0 : (k <= 2 ? 1 : 4); }
__host__ __device__ constexpr long long khfix(int k, int n) {
  return (long long)(kh(k, n) * 9223372036854775808.0 * (double)(1 << kd(k)));  // exact power-of-two scaling
}

// int64 -> double rounded to nearest (ties away from zero), value F 2^scale
__device__ __forceinline__ double ll_to_double_rn(long long F, int scale) {
  if (F == 0) return 0.0;
  const unsigned long long mag = F < 0 ? (unsigned long long)(-F) : (unsigned long long)F;
  const int lz = __clzll(mag);
  const unsigned long long norm = mag << lz;                     // leading one at bit 63
  const unsigned long long r = (norm >> 11) + ((norm >> 10) & 1ull);  // 53 or 54 bits after rounding
  const int carry = (int)(r >> 53);                               // rounding reached 2^53
  const unsigned long long frac = (r >> carry) & 0x000fffffffffffffull;
  const int ex = 1023 + 63 - lz + scale + carry;
  const unsigned hi = (unsigned)(frac >> 32) | ((unsigned)ex << 20) | (F < 0 ? 0x80000000u : 0u);
  return __hiloint2double((int)hi, (int)(unsigned)frac);
}

struct CoeffsFix {
  long long f00, f10, f01, f20, f11, f02, f30, f21, f12, f03, f40, f31, f22, f13, f04;
  long long g00, g10, g01, g20, g11, g02;
  int Ef, Eg;  // block exponents: value = X 2^(E - 1082)
};

__device__ __forceinline__ CoeffsFix coeffs_to_fix(const Coeffs& C) {
  CoeffsFix X;
  const int Ef = max(max(max(max(bexp(C.f00), bexp(C.f10)), max(bexp(C.f01), bexp(C.f20))),
                         max(max(bexp(C.f11), bexp(C.f02)), max(bexp(C.f30), bexp(C.f21)))),
                     max(max(max(bexp(C.f12), bexp(C.f03)), max(bexp(C.f40), bexp(C.f31))),
                         max(max(bexp(C.f22), bexp(C.f13)), bexp(C.f04))));
  const int Eg = max(max(max(bexp(C.g00), bexp(C.g10)), max(bexp(C.g01), bexp(C.g20))),
                     max(bexp(C.g11), bexp(C.g02)));
  X.f00 = to_block_fixed(C.f00, Ef); X.f10 = to_block_fixed(C.f10, Ef); X.f01 = to_block_fixed(C.f01, Ef);
  X.f20 = to_block_fixed(C.f20, Ef); X.f11 = to_block_fixed(C.f11, Ef); X.f02 = to_block_fixed(C.f02, Ef);
  X.f30 = to_block_fixed(C.f30, Ef); X.f21 = to_block_fixed(C.f21, Ef); X.f12 = to_block_fixed(C.f12, Ef);
  X.f03 = to_block_fixed(C.f03, Ef); X.f40 = to_block_fixed(C.f40, Ef); X.f31 = to_block_fixed(C.f31, Ef);
  X.f22 = to_block_fixed(C.f22, Ef); X.f13 = to_block_fixed(C.f13, Ef); X.f04 = to_block_fixed(C.f04, Ef);
  X.g00 = to_block_fixed(C.g00, Eg); X.g10 = to_block_fixed(C.g10, Eg); X.g01 = to_block_fixed(C.g01, Eg);
  X.g20 = to_block_fixed(C.g20, Eg); X.g11 = to_block_fixed(C.g11, Eg); X.g02 = to_block_fixed(C.g02, Eg);
  X.Ef = Ef;
  X.Eg = Eg;
  return X;
}

__device__ __forceinline__ long long mhk(long long x, long long k) { return __mul64hi(x, k); }

// shift the N values so that the largest magnitude has its top bit at 2^60;
// returns the shift (value of h after the call = h 2^(-sh) of its old scale)
template <int N>
__device__ __forceinline__ int renorm_fix(long long (&h)[N]) {
  unsigned long long m = 0;
#pragma unroll
  for (int i = 0; i < N; ++i) m |= (unsigned long long)(h[i] < 0 ? -h[i] : h[i]);
  const int sh = m == 0ull ? 0 : __clzll((long long)m) - 3;
#pragma unroll
  for (int i = 0; i < N; ++i)
    h[i] = sh >= 0 ? (long long)((unsigned long long)h[i] << sh) : (h[i] >> (-sh));
  return sh;
}

// y-expansion of one x-node in fixed point, with the +-xi symmetry as in
// expand_q5 / expand_q3 (value of t_q = t_q 2^(E - 1080 - kd(p) - sh - kd(q)))
__device__ __forceinline__ void expand_q5_fix(const long long (&h)[5], long long (&t)[5]) {
  t[0] = mhk(h[0], khfix(0, 0)) + mhk(h[2], khfix(0, 2)) + mhk(h[4], khfix(0, 4));
  const long long EA = mhk(h[0], khfix(1, 0)) + mhk(h[2], khfix(1, 2)) + mhk(h[4], khfix(1, 4));
  const long long OA = mhk(h[1], khfix(1, 1)) + mhk(h[3], khfix(1, 3));
  const long long EB = mhk(h[0], khfix(3, 0)) + mhk(h[2], khfix(3, 2)) + mhk(h[4], khfix(3, 4));
  const long long OB = mhk(h[1], khfix(3, 1)) + mhk(h[3], khfix(3, 3));
  t[1] = EA + OA; t[2] = EA - OA; t[3] = EB + OB; t[4] = EB - OB;
}
__device__ __forceinline__ void expand_q3_fix(const long long (&h)[3], long long (&t)[5]) {
  t[0] = mhk(h[0], khfix(0, 0)) + mhk(h[2], khfix(0, 2));
  const long long EA = mhk(h[0], khfix(1, 0)) + mhk(h[2], khfix(1, 2));
  const long long OA = mhk(h[1], khfix(1, 1));
  const long long EB = mhk(h[0], khfix(3, 0)) + mhk(h[2], khfix(3, 2));
  const long long OB = mhk(h[1], khfix(3, 1));
  t[1] = EA + OA; t[2] = EA - OA; t[3] = EB + OB; t[4] = EB - OB;
}

// h^b of x-node p (f: N = 4, g: N = 2) from fixed-point coefficients X, any
// view with X(k) = field k in CoeffsFix order (f00, f10, f01, f20, f11, f02,
// f30, f21, f12, f03, f40, f31, f22, f13, f04, g00, g10, g01, g20, g11, g02);
// k0..k4 = khfix(p, 0..4) (value of h = h 2^(E - 1081 - kd(p)))
template <class V>
__device__ __forceinline__ void hf_fix(const V& X, long long k0, long long k1, long long k2, long long k3,
                                       long long k4, long long (&hf)[5]) {
  hf[0] = mhk(X(0), k0) + mhk(X(1), k1) + mhk(X(3), k2) + mhk(X(6), k3) + mhk(X(10), k4);
  hf[1] = mhk(X(2), k0) + mhk(X(4), k1) + mhk(X(7), k2) + mhk(X(11), k3);
  hf[2] = mhk(X(5), k0) + mhk(X(8), k1) + mhk(X(12), k2);
  hf[3] = mhk(X(9), k0) + mhk(X(13), k1);
  hf[4] = mhk(X(14), k0);
}
template <class V>
__device__ __forceinline__ void hg_fix(const V& X, long long k0, long long k1, long long k2, long long (&hg)[3]) {
  hg[0] = mhk(X(15), k0) + mhk(X(16), k1) + mhk(X(18), k2);
  hg[1] = mhk(X(17), k0) + mhk(X(19), k1);
  hg[2] = mhk(X(20), k0);
}
template <class V>
__device__ __forceinline__ void hfg_fix(const V& X, long long k0, long long k1, long long k2, long long k3,
                                        long long k4, long long (&hf)[5], long long (&hg)[3]) {
  hf_fix(X, k0, k1, k2, k3, k4, hf);
  hg_fix(X, k0, k1, k2, hg);
}

// int64 -> float rounded to nearest (ties away from zero), value F 2^scale;
// results below the normal float range flush to zero
__device__ __forceinline__ float ll_to_float_rn(long long F, int scale) {
  if (F == 0) return 0.0f;
  const unsigned long long mag = F < 0 ? (unsigned long long)(-F) : (unsigned long long)F;
  const int lz = __clzll(mag);
  const unsigned long long norm = mag << lz;                          // leading one at bit 63
  const unsigned r = (unsigned)(norm >> 40) + (unsigned)((norm >> 39) & 1ull);  // 24 or 25 bits
  const int carry = (int)(r >> 24);
  const unsigned frac = (r >> carry) & 0x7fffffu;
  const int ex = 127 + 63 - lz + scale + carry;
  if (ex <= 0) return 0.0f;
  return __uint_as_float((unsigned)min(ex, 255) << 23 | (ex >= 255 ? 0u : frac) | (F < 0 ? 0x80000000u : 0u));
}

// Populations of coefficient set C (a pure equilibrium: a1 = 0, k1 = 1) at one
// padded offset, by the step kernel's fixed-point expansion instead of FP64
// arithmetic: initial conditions (Sec. III.A.3) at FP64-or-better precision.
// FP32-deviation storage: the reference populations w rho0 and w G0 carry
// only a zeroth Hermite coefficient, so they are taken off C first and the
// deviations come straight out of the expansion.
struct RegView {
  const long long* v;
  __device__ __forceinline__ long long operator()(int k) const { return v[k]; }
};
template <class S, int p>
__device__ __forceinline__ void write_node_fix(S* d, long long PL, const RegView& X, int Ef, int Eg) {
  long long hf[5], hg[3], xf[5], xg[5];
  hfg_fix(X, khfix(p, 0), khfix(p, 1), khfix(p, 2), khfix(p, 3), khfix(p, 4), hf, hg);
  const int sf = renorm_fix(hf), sg = renorm_fix(hg);
  expand_q5_fix(hf, xf);
  expand_q3_fix(hg, xg);
  const int scf = Ef - 1080 - sf - kd(p), scg = Eg - 1080 - sg - kd(p);
#pragma unroll
  for (int q = 0; q < 5; ++q) {
    if constexpr (sizeof(S) == 8) {
      d[(5 * p + q) * PL] = Ef >= 100 ? ll_to_double_rn(xf[q], scf - kd(q)) : 0.0;
      d[(25 + 5 * p + q) * PL] = Eg >= 100 ? ll_to_double_rn(xg[q], scg - kd(q)) : 0.0;
    } else {
      d[(5 * p + q) * PL] = Ef >= 100 ? ll_to_float_rn(xf[q], scf - kd(q)) : 0.0f;
      d[(25 + 5 * p + q) * PL] = Eg >= 100 ? ll_to_float_rn(xg[q], scg - kd(q)) : 0.0f;
    }
  }
}
template <class S>
__device__ __forceinline__ void write_equilibrium_fix(S* d, long long PL, Coeffs C, const Phys& P) {
  if constexpr (sizeof(S) == 4) {
    C.f00 -= P.fref0;
    C.g00 -= P.gref0;
  }
  const CoeffsFix F = coeffs_to_fix(C);
  const long long v[21] = {F.f00, F.f10, F.f01, F.f20, F.f11, F.f02, F.f30, F.f21, F.f12, F.f03, F.f40,
                           F.f31, F.f22, F.f13, F.f04, F.g00, F.g10, F.g01, F.g20, F.g11, F.g02};
  const RegView X{v};
  write_node_fix<S, 0>(d, PL, X, F.Ef, F.Eg);
  write_node_fix<S, 1>(d, PL, X, F.Ef, F.Eg);
  write_node_fix<S, 2>(d, PL, X, F.Ef, F.Eg);
  write_node_fix<S, 3>(d, PL, X, F.Ef, F.Eg);
  write_node_fix<S, 4>(d, PL, X, F.Ef, F.Eg);
}

// float -> double by bit manipulation (exact; the hardware conversion runs on
// the FP64 pipe on GB300).  Zero and subnormal floats give a signed zero;
// infinities and NaNs keep their class.
__device__ __forceinline__ double f2d_bits(float v) {
  const unsigned u = __float_as_uint(v);
  const unsigned e = (u >> 23) & 0xffu;
  const unsigned sign = u & 0x80000000u;
  const unsigned m = u & 0x7fffffu;
  unsigned hi = sign | ((e + 896u) << 20) | (m >> 3);
  unsigned lo = m << 29;
  if (e == 0u) { hi = sign; lo = 0u; }
  if (e == 255u) hi = sign | 0x7ff00000u | (m >> 3);
  return __hiloint2double((int)hi, (int)lo);
}

// value of integer F at block exponent E: F 2^(E - 1082)
__device__ __forceinline__ double from_block_fixed(long long F, int E) {
  if (E < 64) return 0.0;
  return ll_to_double_scaled(F, E - 1082);
}

// limited slope on integers: minmod3(hb Da, (Da + Db)/4, hb Db); Hq = hb 2^62
__device__ __forceinline__ long long slope_int(long long Da, long long Db, long long ra, long long rb) {
  const long long y = (Da + Db) >> 2;
  const long long mn = min(min(ra, y), rb), mx = max(max(ra, y), rb);
  const bool same = (Da ^ Db) >= 0;
  return same ? (Da >= 0 ? mn : mx) : 0ll;
}

// F_{j+1/2} - F_{j-1/2} (general beta) from the stencil values a0..a3 (v > 0:
// cells j-2..j+1; v < 0: cells j-1..j+2)
__device__ __forceinline__ double flux_difference_int_v(double a0, double a1, double a2, double a3, long long Hq,
                                                        int sgn) {
  const int E = max(max(bexp(a0), bexp(a1)), max(bexp(a2), bexp(a3)));
  const long long x0 = to_block_fixed(a0, E), x1 = to_block_fixed(a1, E), x2 = to_block_fixed(a2, E),
                  x3 = to_block_fixed(a3, E);
  const long long Da = x1 - x0, Db = x2 - x1, Dc = x3 - x2;
  const long long ra = __mul64hi(Da << 2, Hq), rb = __mul64hi(Db << 2, Hq), rc = __mul64hi(Dc << 2, Hq);
  const long long s_ab = slope_int(Da, Db, ra, rb);  // slope of the cell between a and b faces
  const long long s_bc = slope_int(Db, Dc, rb, rc);
  // v > 0 (cells j-2..j+1): dF = D_j + sigma_j - sigma_{j-1} = Db + s_bc - s_ab
  // v < 0 (cells j-1..j+2): dF = D_{j+1} - sigma_{j+1} + sigma_j = Db - s_bc + s_ab
  const long long F = sgn > 0 ? Db + s_bc - s_ab : Db - s_bc + s_ab;
  return from_block_fixed(F, E);
}


// Rational limiter: with beta = lp/lq the scaled slope 4 lq sigma equals
// minmod3(2 lp Da, lq (Da + Db), 2 lp Db) exactly, so the flux difference
// scaled by 4 lq needs only small-integer multiplies.  Values enter with a
// 52-bit significand (X = value 2^(1074 - E)) to leave headroom for the
// factors (lp <= 128, lq <= 64).
__device__ __forceinline__ long long slope_rat(long long Da, long long Db, long long lp2, long long lq) {
  const long long ra = lp2 * Da, rb = lp2 * Db, y = lq * (Da + Db);
  const long long mn = min(min(ra, y), rb), mx = max(max(ra, y), rb);
  return ((Da ^ Db) >= 0) ? (Da >= 0 ? mn : mx) : 0ll;
}

// 52-bit variant: value = X 2^(E - 1074); the magnitude is truncated (toward
// zero) in one shift of the significand
__device__ __forceinline__ long long to_block_fixed52(double v, int E) {
  const int hi = __double2hiint(v);
  const unsigned lo = (unsigned)__double2loint(v);
  const int e = (hi >> 20) & 0x7ff;
  const unsigned long long m = ((unsigned long long)((unsigned)(hi & 0xfffff) | 0x100000u) << 32) | lo;
  const unsigned long long mag = m >> min(E - e + 1, 63);
  return hi < 0 ? -(long long)mag : (long long)mag;
}

// 4 lq (F_{j+1/2} - F_{j-1/2}) as a double (the caller folds 1/(4 lq)) from
// the stencil values a0..a3 (v > 0: cells j-2..j+1; v < 0: cells j-1..j+2)
__device__ __forceinline__ double flux_difference_rat_v(double a0, double a1, double a2, double a3, int lp, int lq,
                                                        int sgn) {
  const int E = max(max(bexp(a0), bexp(a1)), max(bexp(a2), bexp(a3)));
  const long long x0 = to_block_fixed52(a0, E), x1 = to_block_fixed52(a1, E), x2 = to_block_fixed52(a2, E),
                  x3 = to_block_fixed52(a3, E);
  const long long Da = x1 - x0, Db = x2 - x1, Dc = x3 - x2;
  const long long lp2 = 2 * lp, q4 = 4 * lq;
  const long long s_ab = slope_rat(Da, Db, lp2, lq);
  const long long s_bc = slope_rat(Db, Dc, lp2, lq);
  const long long F = sgn > 0 ? q4 * Db + s_bc - s_ab : q4 * Db - s_bc + s_ab;
  if (E < 64) return 0.0;
  return ll_to_double_scaled(F, E - 1074);  // value = F 2^(E - 1074)
}

// slope_rat together with the minmod branch it took: 0 (a and b differ in
// sign), 1 (2 lp Da), 2 (lq (Da + Db)), 3 (2 lp Db), ties resolved in that
// order.  The value equals slope_rat's.
__device__ __forceinline__ long long slope_rat_code(long long Da, long long Db, long long lp2, long long lq,
                                                    int& code) {
  const long long ra = lp2 * Da, rb = lp2 * Db, y = lq * (Da + Db);
  int br;
  if (Da >= 0) br = (ra <= y && ra <= rb) ? 1 : (y <= rb ? 2 : 3);
  else br = (ra >= y && ra >= rb) ? 1 : (y >= rb ? 2 : 3);
  if ((Da ^ Db) < 0) br = 0;
  code = br;
  return br == 0 ? 0ll : (br == 1 ? ra : (br == 2 ? y : rb));
}

// flux_difference_rat_v that also returns the branch code of the cell's own
// slope sigma_j (first argument its backward, second its forward difference):
// s_bc for v > 0, s_ab for v < 0.  The adjoint reads these codes instead of
// re-deriving them from the state.
__device__ __forceinline__ double flux_difference_rat_code_v(double a0, double a1, double a2, double a3, int lp,
                                                             int lq, int sgn, int& code) {
  const int E = max(max(bexp(a0), bexp(a1)), max(bexp(a2), bexp(a3)));
  const long long x0 = to_block_fixed52(a0, E), x1 = to_block_fixed52(a1, E), x2 = to_block_fixed52(a2, E),
                  x3 = to_block_fixed52(a3, E);
  const long long Da = x1 - x0, Db = x2 - x1, Dc = x3 - x2;
  const long long lp2 = 2 * lp, q4 = 4 * lq;
  int c_ab, c_bc;
  const long long s_ab = slope_rat_code(Da, Db, lp2, lq, c_ab);
  const long long s_bc = slope_rat_code(Db, Dc, lp2, lq, c_bc);
  code = sgn > 0 ? c_bc : c_ab;
  const long long F = sgn > 0 ? q4 * Db + s_bc - s_ab : q4 * Db - s_bc + s_ab;
  if (E < 64) return 0.0;
  return ll_to_double_scaled(F, E - 1074);
}

// Flux difference F_{j+1/2} - F_{j-1/2} of the upwind-limited face values
// along a stride (float, FP32-deviation storage); SGN = sign of the velocity
// component (never 0 here).
//   v > 0: faces f_{j-1} + sigma_{j-1}, f_j + sigma_j
//   v < 0: faces f_j - sigma_j, f_{j+1} - sigma_{j+1}
template <int SGN, class T>
__device__ __forceinline__ T flux_difference(const T* __restrict__ ptr, long long stride, T hb) {
  static_assert(sizeof(T) == 4, "FP64 storage uses the integer flux differences");
  if (SGN > 0) {
    const T fm2 = __ldg(ptr - 2 * stride), fm1 = __ldg(ptr - stride), f0 = __ldg(ptr), fp1 = __ldg(ptr + stride);
    const T Dm = fm1 - fm2, D0 = f0 - fm1, Dp = fp1 - f0;
    return D0 + limited_slope(D0, Dp, hb) - limited_slope(Dm, D0, hb);
  } else {
    const T fm1 = __ldg(ptr - stride), f0 = __ldg(ptr), fp1 = __ldg(ptr + stride), fp2 = __ldg(ptr + 2 * stride);
    const T D0 = f0 - fm1, Dp = fp1 - f0, Dpp = fp2 - fp1;
    return Dp - limited_slope(Dp, Dpp, hb) + limited_slope(D0, Dp, hb);
  }
}

}  // namespace dvbm
