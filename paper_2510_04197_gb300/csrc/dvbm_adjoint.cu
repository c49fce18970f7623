// dvbm_adjoint.cu -- hand-written discrete adjoint of the FP64 time step.
//
// For the map X^{n+1} = Phi(X^n; mu, Pr, gamma) of Eq. finalDiscretePDE (FP64
// storage, periodic domain) the kernels compute lambda^n = (dPhi/dX^n)^T
// lambda^{n+1} and the per-cell contributions to dL/d(mu, Pr, gamma):
//
//  * local (collision) part: with a1 = 1 - dt/tau1 and the combined Grad
//    coefficients C (dvbm_device.cuh), X^{n+1}_k = a1 X_k + W_k sum C H_k - adv_k,
//      lambda^n_i = a1 lambda_i + sum_j mbar_j dm_j/dX_i,
//    where (abar1, Cbar) = (sum_k lambda_k X_k, sum_k lambda_k W_k H_k) are
//    pulled back through the coefficient function by the reverse pass
//    collision_coeffs_rev (the forward statements in reverse order), giving
//    the moment adjoints mbar and the parameter adjoints;
//  * advection part, written as a gather: the flux difference of cell c',
//    F(c') = D_c' + sigma_c' - sigma_{c'-1} (v > 0) or
//    D_{c'+1} - sigma_{c'+1} + sigma_c' (v < 0), with D_k = X_k - X_{k-1} and
//    sigma_k = minmod3(hb D_k, (D_k + D_{k+1})/4, hb D_{k+1}); its adjoint
//    needs X and lambda at c-2 .. c+2 only.  The minmod branch of each slope
//    gives the partial derivatives (hb, 0), (1/4, 1/4), (0, hb) or (0, 0).
//    As in the forward kernel the linear combinations run in block floating
//    point on the integer pipe.
#include <algorithm>

#include "dvbm_device.cuh"
#include "dvbm_cellmom.cuh"
#include "dvbm_internal.h"

namespace dvbm {

// ---------------------------------------------------------------- reverse pass
struct ParamBar { double dt_mu, Pr, gm1, epsf; };

// Reverse of collision_coeffs<PRC> for the outputs C (f, g) and a1.
template <int PRC>
__device__ __forceinline__ double collision_coeffs_rev(const Moments& m, const Phys& P, const Coeffs& Cb,
                                                       double a1b, Moments& mb, ParamBar& pb) {
  // ---- forward recomputation of the intermediates
  const double rho = m.m00;
  const double irho = 1.0 / rho;
  const double ux = m.m10 * irho, uy = m.m01 * irho;
  const double Et = fma(0.5, m.m20 + m.m02, m.g00 * P.inv_c2);
  const double q = fma(ux, ux, uy * uy);
  const double w = fma(-0.5, q, Et * irho);
  const double theta = P.gm1 * w;
  const double s = theta - 1.0;
  const double p = rho * P.c2 * theta;
  double k1, k2;
  if (PRC <= 0) { k1 = P.dt_mu * p; k2 = k1 * P.Pr; }
  else          { k2 = P.dt_mu * p; k1 = k2 * P.Pr; }
  const double s1 = k1 - k2;
  const EqF e = eq_f(rho, ux, uy, s);
  const double reps = rho * P.epsf * theta;
  double Dxx = 0, Dxy = 0, Dyy = 0, kap = 0, Px = 0, Py = 0, Tx = 0;
  double d20 = 0, d11 = 0, d02 = 0, d30 = 0, d21 = 0, d12 = 0, d03 = 0, d40 = 0, d31 = 0, d13 = 0, d04 = 0;
  double dg10 = 0, dg01 = 0;
  if (PRC != 0) {
    Dxx = (m.m20 - rho) - e.a20;
    Dxy = m.m11 - e.a11;
    Dyy = (m.m02 - rho) - e.a02;
    if (PRC < 0) {
      kap = 0.25 * (Dxx + Dyy);
      Px = Dxx - kap; Py = Dyy - kap;
      d30 = (fma(-3.0, m.m10, m.m30) - e.a30) - 3.0 * ux * Px;
      d21 = ((m.m21 - m.m01) - e.a21) - fma(2.0 * ux, Dxy, uy * Px);
      d12 = ((m.m12 - m.m10) - e.a12) - fma(2.0 * uy, Dxy, ux * Py);
      d03 = (fma(-3.0, m.m01, m.m03) - e.a03) - 3.0 * uy * Py;
      dg10 = m.g10 * P.inv_c2 - reps * ux;
      dg01 = m.g01 * P.inv_c2 - reps * uy;
    } else {
      Tx = 0.5 * (Dxx - Dyy);
      d20 = Tx; d11 = Dxy; d02 = -Tx;
      d30 = 3.0 * ux * Tx;
      d21 = fma(uy, Tx, 2.0 * ux * Dxy);
      d12 = fma(-ux, Tx, 2.0 * uy * Dxy);
      d03 = -3.0 * uy * Tx;
      d40 = -6.0 * Tx; d31 = -3.0 * Dxy; d13 = -3.0 * Dxy; d04 = 6.0 * Tx;
    }
  }
  const double kg = k1 * P.c2, sg = s1 * P.c2;
  const double KR = kg * reps;

  // ---- reverse
  double uxb = 0, uyb = 0, sb = 0, rhob = 0, thetab = 0, k1b = 0, k2b = 0, s1b = 0, repsb = 0;
  // g outputs
  double KRb = Cb.g00 + Cb.g10 * ux + Cb.g01 * uy + Cb.g20 * fma(ux, ux, s) + Cb.g11 * ux * uy + Cb.g02 * fma(uy, uy, s);
  double sgb = Cb.g10 * dg10 + Cb.g01 * dg01;
  const double dg10b = Cb.g10 * sg, dg01b = Cb.g01 * sg;
  uxb += KR * (Cb.g10 + 2.0 * ux * Cb.g20 + uy * Cb.g11);
  uyb += KR * (Cb.g01 + 2.0 * uy * Cb.g02 + ux * Cb.g11);
  sb += KR * (Cb.g20 + Cb.g02);
  const double kgb = KRb * reps;
  repsb += KRb * kg;
  k1b += kgb * P.c2;
  s1b += sgb * P.c2;
  // f outputs: C.fab = k1 a_ab + s1 d_ab
  double a00b = Cb.f00 * k1, a10b = Cb.f10 * k1, a01b = Cb.f01 * k1, a20b = Cb.f20 * k1, a11b = Cb.f11 * k1,
         a02b = Cb.f02 * k1, a30b = Cb.f30 * k1, a21b = Cb.f21 * k1, a12b = Cb.f12 * k1, a03b = Cb.f03 * k1,
         a40b = Cb.f40 * k1, a31b = Cb.f31 * k1, a22b = Cb.f22 * k1, a13b = Cb.f13 * k1, a04b = Cb.f04 * k1;
  k1b += Cb.f00 * e.a00 + Cb.f10 * e.a10 + Cb.f01 * e.a01 + Cb.f20 * e.a20 + Cb.f11 * e.a11 + Cb.f02 * e.a02 +
         Cb.f30 * e.a30 + Cb.f21 * e.a21 + Cb.f12 * e.a12 + Cb.f03 * e.a03 + Cb.f40 * e.a40 + Cb.f31 * e.a31 +
         Cb.f22 * e.a22 + Cb.f13 * e.a13 + Cb.f04 * e.a04;
  s1b += Cb.f20 * d20 + Cb.f11 * d11 + Cb.f02 * d02 + Cb.f30 * d30 + Cb.f21 * d21 + Cb.f12 * d12 + Cb.f03 * d03 +
         Cb.f40 * d40 + Cb.f31 * d31 + Cb.f13 * d13 + Cb.f04 * d04;
  const double d20b = Cb.f20 * s1, d11b = Cb.f11 * s1, d02b = Cb.f02 * s1, d30b = Cb.f30 * s1, d21b = Cb.f21 * s1,
               d12b = Cb.f12 * s1, d03b = Cb.f03 * s1, d40b = Cb.f40 * s1, d31b = Cb.f31 * s1, d13b = Cb.f13 * s1,
               d04b = Cb.f04 * s1;
  if (PRC != 0) {
    double Dxxb = 0, Dxyb = 0, Dyyb = 0;
    if (PRC < 0) {
      // dg10 = g10 inv_c2 - reps ux ; dg01 = g01 inv_c2 - reps uy
      mb.g10 += dg10b * P.inv_c2;
      mb.g01 += dg01b * P.inv_c2;
      repsb -= dg10b * ux + dg01b * uy;
      uxb -= dg10b * reps;
      uyb -= dg01b * reps;
      double Pxb = 0, Pyb = 0;
      // d03 = m03 - 3 m01 - a03 - 3 uy Py
      mb.m03 += d03b; mb.m01 -= 3.0 * d03b; a03b -= d03b; uyb -= 3.0 * d03b * Py; Pyb -= 3.0 * d03b * uy;
      // d12 = m12 - m10 - a12 - 2 uy Dxy - ux Py
      mb.m12 += d12b; mb.m10 -= d12b; a12b -= d12b; uyb -= 2.0 * d12b * Dxy; Dxyb -= 2.0 * d12b * uy;
      uxb -= d12b * Py; Pyb -= d12b * ux;
      // d21 = m21 - m01 - a21 - 2 ux Dxy - uy Px
      mb.m21 += d21b; mb.m01 -= d21b; a21b -= d21b; uxb -= 2.0 * d21b * Dxy; Dxyb -= 2.0 * d21b * ux;
      uyb -= d21b * Px; Pxb -= d21b * uy;
      // d30 = m30 - 3 m10 - a30 - 3 ux Px
      mb.m30 += d30b; mb.m10 -= 3.0 * d30b; a30b -= d30b; uxb -= 3.0 * d30b * Px; Pxb -= 3.0 * d30b * ux;
      // Px = Dxx - kap, Py = Dyy - kap, kap = (Dxx + Dyy)/4
      const double kapb = -(Pxb + Pyb);
      Dxxb += Pxb + 0.25 * kapb;
      Dyyb += Pyb + 0.25 * kapb;
    } else {
      const double Txb = d20b - d02b + 3.0 * ux * d30b + uy * d21b - ux * d12b - 3.0 * uy * d03b - 6.0 * d40b + 6.0 * d04b;
      Dxyb += d11b + 2.0 * ux * d21b + 2.0 * uy * d12b - 3.0 * d31b - 3.0 * d13b;
      uxb += 3.0 * Tx * d30b + 2.0 * Dxy * d21b - Tx * d12b;
      uyb += Tx * d21b + 2.0 * Dxy * d12b - 3.0 * Tx * d03b;
      Dxxb += 0.5 * Txb;
      Dyyb -= 0.5 * Txb;
    }
    // Dxx = m20 - rho - a20 ; Dxy = m11 - a11 ; Dyy = m02 - rho - a02
    mb.m20 += Dxxb; rhob -= Dxxb; a20b -= Dxxb;
    mb.m11 += Dxyb; a11b -= Dxyb;
    mb.m02 += Dyyb; rhob -= Dyyb; a02b -= Dyyb;
  }
  // reps = rho epsf theta
  rhob += repsb * P.epsf * theta;
  pb.epsf += repsb * rho * theta;
  thetab += repsb * rho * P.epsf;
  // eq_f reverse (statements in reverse order)
  double rsb = 0;
  a20b += a22b * fma(uy, uy, s); uyb += a22b * e.a20 * 2.0 * uy; sb += a22b * e.a20;
  a03b += a13b * ux; uxb += a13b * e.a03;
  a30b += a31b * uy; uyb += a31b * e.a30;
  a03b += a04b * uy; uyb += a04b * e.a03; sb += 3.0 * a04b * e.a02; a02b += 3.0 * s * a04b;
  a30b += a40b * ux; uxb += a40b * e.a30; sb += 3.0 * a40b * e.a20; a20b += 3.0 * s * a40b;
  a02b += a12b * ux; uxb += a12b * e.a02;
  a20b += a21b * uy; uyb += a21b * e.a20;
  a02b += a03b * uy; uyb += a03b * e.a02; sb += 2.0 * a03b * e.a01; a01b += 2.0 * s * a03b;
  a20b += a30b * ux; uxb += a30b * e.a20; sb += 2.0 * a30b * e.a10; a10b += 2.0 * s * a30b;
  a01b += a02b * uy; uyb += a02b * e.a01; rsb += a02b;
  a10b += a11b * uy; uyb += a11b * e.a10;
  a10b += a20b * ux; uxb += a20b * e.a10; rsb += a20b;
  rhob += a01b * uy; uyb += a01b * rho;
  rhob += a10b * ux; uxb += a10b * rho;
  rhob += a00b;
  rhob += rsb * s; sb += rsb * rho;
  // a1 = 1 - k1 ; s1 = k1 - k2
  k1b += s1b - a1b;
  k2b -= s1b;
  double pbar;
  if (PRC <= 0) {  // k1 = dt_mu p ; k2 = k1 Pr
    k1b += k2b * P.Pr; pb.Pr += k2b * k1;
    pb.dt_mu += k1b * p; pbar = k1b * P.dt_mu;
  } else {         // k2 = dt_mu p ; k1 = k2 Pr
    k2b += k1b * P.Pr; pb.Pr += k1b * k2;
    pb.dt_mu += k2b * p; pbar = k2b * P.dt_mu;
  }
  // p = rho c2 theta
  rhob += pbar * P.c2 * theta;
  thetab += pbar * rho * P.c2;
  // s = theta - 1
  thetab += sb;
  // theta = gm1 w, w = Et irho - q/2
  pb.gm1 += thetab * w;
  const double wb = thetab * P.gm1;
  const double Etb = wb * irho;
  double irhob = wb * Et;
  const double qb = -0.5 * wb;
  uxb += 2.0 * ux * qb;
  uyb += 2.0 * uy * qb;
  mb.m20 += 0.5 * Etb; mb.m02 += 0.5 * Etb; mb.g00 += Etb * P.inv_c2;
  mb.m10 += uxb * irho; irhob += uxb * m.m10;
  mb.m01 += uyb * irho; irhob += uyb * m.m01;
  rhob -= irhob * irho * irho;
  mb.m00 += rhob;
  return 1.0 - k1;  // a1 of the forward step
}

// Reverse of the (rho, T) read-out of the moments (macro_from_moments): given
// dL/drho and dL/dT, accumulate the moment adjoints and dL/d(gamma - 1).
__device__ __forceinline__ void macro_rev(const Moments& m, const Phys& P, double T_ref, double rhob_in, double Tb,
                                          Moments& mb, ParamBar& pb) {
  const double rho = m.m00;
  const double irho = 1.0 / rho;
  const double ux = m.m10 * irho, uy = m.m01 * irho;
  const double Et = fma(0.5, m.m20 + m.m02, m.g00 * P.inv_c2);
  const double w = fma(-0.5, fma(ux, ux, uy * uy), Et * irho);
  const double thetab = Tb * T_ref;
  pb.gm1 += thetab * w;
  const double wb = thetab * P.gm1;
  const double Etb = wb * irho;
  double irhob = wb * Et;
  const double qb = -0.5 * wb;
  const double uxb = 2.0 * ux * qb, uyb = 2.0 * uy * qb;
  mb.m20 += 0.5 * Etb; mb.m02 += 0.5 * Etb; mb.g00 += Etb * P.inv_c2;
  mb.m10 += uxb * irho; irhob += uxb * m.m10;
  mb.m01 += uyb * irho; irhob += uyb * m.m01;
  mb.m00 += rhob_in - irhob * irho * irho;
}

// Reverse of equilibrium_coeffs (initial conditions): from Cbar to the
// adjoints of rho, u (units of c), theta and epsf.
__device__ __forceinline__ void equilibrium_rev(double rho, double ux, double uy, double theta, const Phys& P,
                                                const Coeffs& Cb, double& rhob, double& uxb, double& uyb,
                                                double& thetab, double& epsfb) {
  const double s = theta - 1.0;
  const EqF e = eq_f(rho, ux, uy, s);
  const double reps = rho * P.epsf * theta * P.c2;
  double sb = 0;
  const double repsb = Cb.g00 + Cb.g10 * ux + Cb.g01 * uy + Cb.g20 * fma(ux, ux, s) + Cb.g11 * ux * uy +
                       Cb.g02 * fma(uy, uy, s);
  uxb = reps * (Cb.g10 + 2.0 * ux * Cb.g20 + uy * Cb.g11);
  uyb = reps * (Cb.g01 + 2.0 * uy * Cb.g02 + ux * Cb.g11);
  sb += reps * (Cb.g20 + Cb.g02);
  rhob = repsb * P.epsf * theta * P.c2;
  epsfb = repsb * rho * theta * P.c2;
  thetab = repsb * rho * P.epsf * P.c2;
  double a00b = Cb.f00, a10b = Cb.f10, a01b = Cb.f01, a20b = Cb.f20, a11b = Cb.f11, a02b = Cb.f02, a30b = Cb.f30,
         a21b = Cb.f21, a12b = Cb.f12, a03b = Cb.f03, a40b = Cb.f40, a31b = Cb.f31, a22b = Cb.f22, a13b = Cb.f13,
         a04b = Cb.f04;
  double rsb = 0;
  a20b += a22b * fma(uy, uy, s); uyb += a22b * e.a20 * 2.0 * uy; sb += a22b * e.a20;
  a03b += a13b * ux; uxb += a13b * e.a03;
  a30b += a31b * uy; uyb += a31b * e.a30;
  a03b += a04b * uy; uyb += a04b * e.a03; sb += 3.0 * a04b * e.a02; a02b += 3.0 * s * a04b;
  a30b += a40b * ux; uxb += a40b * e.a30; sb += 3.0 * a40b * e.a20; a20b += 3.0 * s * a40b;
  a02b += a12b * ux; uxb += a12b * e.a02;
  a20b += a21b * uy; uyb += a21b * e.a20;
  a02b += a03b * uy; uyb += a03b * e.a02; sb += 2.0 * a03b * e.a01; a01b += 2.0 * s * a03b;
  a20b += a30b * ux; uxb += a30b * e.a20; sb += 2.0 * a30b * e.a10; a10b += 2.0 * s * a30b;
  a01b += a02b * uy; uyb += a02b * e.a01; rsb += a02b;
  a10b += a11b * uy; uyb += a11b * e.a10;
  a10b += a20b * ux; uxb += a20b * e.a10; rsb += a20b;
  rhob += a01b * uy; uyb += a01b * rho;
  rhob += a10b * ux; uxb += a10b * rho;
  rhob += a00b;
  rhob += rsb * s; sb += rsb * rho;
  thetab += sb;
}

// ------------------------------------------------------- projections / moments
// kh(k, n) 2^63 for every node (no per-node scaling: the projection sums over
// nodes at one scale); |kh| < 0.54
__host__ __device__ constexpr long long c0fix(int k, int n) { return (long long)(kh(k, n) * 9223372036854775808.0); }

// Cbar_ab = sum over the node's populations of lambda W W He_a He_b /(a! b!):
// accumulate the contribution of x-node p (lf, lg: the 5 f and g values).
template <int p>
__device__ __forceinline__ void accumulate_projection(Coeffs& Cb, const double (&lf)[5], const double (&lg)[5]) {
  double hb[5];  // hbar^b_p = sum_q lambda_pq kh(q, b)
  {
    const double sA = lf[1] + lf[2], dA = lf[1] - lf[2], sB = lf[3] + lf[4], dB = lf[3] - lf[4];
    hb[0] = fma(kh(3, 0), sB, fma(kh(1, 0), sA, kh(0, 0) * lf[0]));
    hb[1] = fma(kh(3, 1), dB, kh(1, 1) * dA);
    hb[2] = fma(kh(3, 2), sB, fma(kh(1, 2), sA, kh(0, 2) * lf[0]));
    hb[3] = fma(kh(3, 3), dB, kh(1, 3) * dA);
    hb[4] = fma(kh(3, 4), sB, fma(kh(1, 4), sA, kh(0, 4) * lf[0]));
  }
  Cb.f00 = fma(kh(p, 0), hb[0], Cb.f00);
  Cb.f01 = fma(kh(p, 0), hb[1], Cb.f01);
  Cb.f02 = fma(kh(p, 0), hb[2], Cb.f02);
  Cb.f03 = fma(kh(p, 0), hb[3], Cb.f03);
  Cb.f04 = fma(kh(p, 0), hb[4], Cb.f04);
  Cb.f20 = fma(kh(p, 2), hb[0], Cb.f20);
  Cb.f21 = fma(kh(p, 2), hb[1], Cb.f21);
  Cb.f22 = fma(kh(p, 2), hb[2], Cb.f22);
  Cb.f40 = fma(kh(p, 4), hb[0], Cb.f40);
  if (p != 0) {
    Cb.f10 = fma(kh(p, 1), hb[0], Cb.f10);
    Cb.f11 = fma(kh(p, 1), hb[1], Cb.f11);
    Cb.f12 = fma(kh(p, 1), hb[2], Cb.f12);
    Cb.f13 = fma(kh(p, 1), hb[3], Cb.f13);
    Cb.f30 = fma(kh(p, 3), hb[0], Cb.f30);
    Cb.f31 = fma(kh(p, 3), hb[1], Cb.f31);
  }
  double gb[3];
  {
    const double sA = lg[1] + lg[2], dA = lg[1] - lg[2], sB = lg[3] + lg[4], dB = lg[3] - lg[4];
    gb[0] = fma(kh(3, 0), sB, fma(kh(1, 0), sA, kh(0, 0) * lg[0]));
    gb[1] = fma(kh(3, 1), dB, kh(1, 1) * dA);
    gb[2] = fma(kh(3, 2), sB, fma(kh(1, 2), sA, kh(0, 2) * lg[0]));
  }
  Cb.g00 = fma(kh(p, 0), gb[0], Cb.g00);
  Cb.g01 = fma(kh(p, 0), gb[1], Cb.g01);
  Cb.g02 = fma(kh(p, 0), gb[2], Cb.g02);
  Cb.g20 = fma(kh(p, 2), gb[0], Cb.g20);
  if (p != 0) {
    Cb.g10 = fma(kh(p, 1), gb[0], Cb.g10);
    Cb.g11 = fma(kh(p, 1), gb[1], Cb.g11);
  }
}

// The same projection in block fixed point on the integer pipe (the adjoint
// of the fixed-point expansion of the forward step): lambda of the cell at a
// shared exponent per f / g (60-bit), node constants kh 2^63, products as
// high words; the partial sums of all five x-nodes share one scale, so that
// cbar accumulates across nodes without renormalisation.  Value of cbar_ab:
// cb 2^(E - 1080).  cb: this thread's 21 accumulators in shared memory (f
// fields 0..14 in Coeffs order, g fields 15..20, stride 256).
template <int p>
__device__ __forceinline__ void accumulate_projection_fix(long long* __restrict__ cb, const double (&lf)[5],
                                                          const double (&lg)[5], int Ef, int Eg) {
  long long hb[5];
  {
    const long long l0 = to_block_fixed(lf[0], Ef), l1 = to_block_fixed(lf[1], Ef), l2 = to_block_fixed(lf[2], Ef),
                    l3 = to_block_fixed(lf[3], Ef), l4 = to_block_fixed(lf[4], Ef);
    const long long sA = l1 + l2, dA = l1 - l2, sB = l3 + l4, dB = l3 - l4;
    hb[0] = mhk(l0, c0fix(0, 0)) + mhk(sA, c0fix(1, 0)) + mhk(sB, c0fix(3, 0));
    hb[1] = mhk(dA, c0fix(1, 1)) + mhk(dB, c0fix(3, 1));
    hb[2] = mhk(l0, c0fix(0, 2)) + mhk(sA, c0fix(1, 2)) + mhk(sB, c0fix(3, 2));
    hb[3] = mhk(dA, c0fix(1, 3)) + mhk(dB, c0fix(3, 3));
    hb[4] = mhk(l0, c0fix(0, 4)) + mhk(sA, c0fix(1, 4)) + mhk(sB, c0fix(3, 4));
  }
  // field order f00, f10, f01, f20, f11, f02, f30, f21, f12, f03, f40, f31, f22, f13, f04
  cb[0 * 256] += mhk(hb[0], c0fix(p, 0));
  cb[2 * 256] += mhk(hb[1], c0fix(p, 0));
  cb[5 * 256] += mhk(hb[2], c0fix(p, 0));
  cb[9 * 256] += mhk(hb[3], c0fix(p, 0));
  cb[14 * 256] += mhk(hb[4], c0fix(p, 0));
  cb[3 * 256] += mhk(hb[0], c0fix(p, 2));
  cb[7 * 256] += mhk(hb[1], c0fix(p, 2));
  cb[12 * 256] += mhk(hb[2], c0fix(p, 2));
  cb[10 * 256] += mhk(hb[0], c0fix(p, 4));
  if (p != 0) {
    cb[1 * 256] += mhk(hb[0], c0fix(p, 1));
    cb[4 * 256] += mhk(hb[1], c0fix(p, 1));
    cb[8 * 256] += mhk(hb[2], c0fix(p, 1));
    cb[13 * 256] += mhk(hb[3], c0fix(p, 1));
    cb[6 * 256] += mhk(hb[0], c0fix(p, 3));
    cb[11 * 256] += mhk(hb[1], c0fix(p, 3));
  }
  long long gb[3];
  {
    const long long l0 = to_block_fixed(lg[0], Eg), l1 = to_block_fixed(lg[1], Eg), l2 = to_block_fixed(lg[2], Eg),
                    l3 = to_block_fixed(lg[3], Eg), l4 = to_block_fixed(lg[4], Eg);
    const long long sA = l1 + l2, dA = l1 - l2, sB = l3 + l4, dB = l3 - l4;
    gb[0] = mhk(l0, c0fix(0, 0)) + mhk(sA, c0fix(1, 0)) + mhk(sB, c0fix(3, 0));
    gb[1] = mhk(dA, c0fix(1, 1)) + mhk(dB, c0fix(3, 1));
    gb[2] = mhk(l0, c0fix(0, 2)) + mhk(sA, c0fix(1, 2)) + mhk(sB, c0fix(3, 2));
  }
  // g order g00, g10, g01, g20, g11, g02
  cb[15 * 256] += mhk(gb[0], c0fix(p, 0));
  cb[17 * 256] += mhk(gb[1], c0fix(p, 0));
  cb[20 * 256] += mhk(gb[2], c0fix(p, 0));
  cb[18 * 256] += mhk(gb[0], c0fix(p, 2));
  if (p != 0) {
    cb[16 * 256] += mhk(gb[0], c0fix(p, 1));
    cb[19 * 256] += mhk(gb[1], c0fix(p, 1));
  }
}

// sum_j mbar_j dm_j/dX for the populations (p, q) of one x-node:
// f: sum_{a+b<=3} mbar_ab xi_p^a xi_q^b ; g: gbar00 + gbar10 xi_p + gbar01 xi_q
template <int p>
__device__ __forceinline__ void moment_pullback(const Moments& mb, double (&pf)[5], double (&pg)[5]) {
  constexpr double x = xi_of(p);
  const double b0 = fma(x * x * x, mb.m30, fma(x * x, mb.m20, fma(x, mb.m10, mb.m00)));
  const double b1 = fma(x * x, mb.m21, fma(x, mb.m11, mb.m01));
  const double b2 = fma(x, mb.m12, mb.m02);
  const double b3 = mb.m03;
  const double g0 = fma(x, mb.g10, mb.g00);
#pragma unroll
  for (int q = 0; q < 5; ++q) {
    const double y = xi_of(q);
    pf[q] = fma(y * y * y, b3, fma(y * y, b2, fma(y, b1, b0)));
    pg[q] = fma(y, mb.g01, g0);
  }
}

// ------------------------------------------------------------ advection adjoint
// minmod branch of sigma(Da, Db) with block-fixed integers: 0 zero, 1 hb Da,
// 2 (Da + Db)/4, 3 hb Db.  Ties resolve in the order hb Da, (Da+Db)/4, hb Db.
__device__ __forceinline__ int slope_branch(long long Da, long long Db, long long ra, long long rb) {
  if ((Da ^ Db) < 0) return 0;
  const long long y = (Da + Db) >> 2;
  if (Da >= 0) {
    if (ra <= y && ra <= rb) return 1;
    return y <= rb ? 2 : 3;
  }
  if (ra >= y && ra >= rb) return 1;
  return y >= rb ? 2 : 3;
}
// partial derivatives (first, second argument) times an integer sbar
__device__ __forceinline__ long long slope_d1(int br, long long sbar, long long Hq) {
  return br == 1 ? __mul64hi(sbar << 2, Hq) : (br == 2 ? (sbar >> 2) : 0ll);
}
__device__ __forceinline__ long long slope_d2(int br, long long sbar, long long Hq) {
  return br == 3 ? __mul64hi(sbar << 2, Hq) : (br == 2 ? (sbar >> 2) : 0ll);
}

// lambda values at block exponent with 6 fraction-guard bits less than the
// forward conversion (headroom for the sums below)
__device__ __forceinline__ long long to_block_fixed6(double v, int E) { return to_block_fixed(v, E) >> 1; }

// Adjoint of the flux difference of one population along one axis, gathered
// at cell c: returns sum_{c'} lambda(c') dF(c')/dX(c) (multiply by -k outside).
__device__ __forceinline__ double advection_adjoint(const double* __restrict__ X, const double* __restrict__ L,
                                                    long long stride, long long Hq, int sgn) {
  double xv[5], lv[5];
#pragma unroll
  for (int k = 0; k < 5; ++k) {
    xv[k] = __ldg(X + (k - 2) * stride);
    lv[k] = __ldg(L + (k - 2) * stride);
  }
  const int EX = max(max(max(bexp(xv[0]), bexp(xv[1])), max(bexp(xv[2]), bexp(xv[3]))), bexp(xv[4]));
  long long xi[5];
#pragma unroll
  for (int k = 0; k < 5; ++k) xi[k] = to_block_fixed(xv[k], EX);
  // differences D_{c-1} .. D_{c+2} (index 0..3) and slope branches of
  // sigma_{c-1} (D_{c-1}, D_c), sigma_c (D_c, D_{c+1}), sigma_{c+1} (D_{c+1}, D_{c+2})
  long long D[4], r[4];
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    D[k] = xi[k + 1] - xi[k];
    r[k] = __mul64hi(D[k] << 2, Hq);
  }
  const int bm = slope_branch(D[0], D[1], r[0], r[1]);
  const int b0 = slope_branch(D[1], D[2], r[1], r[2]);
  const int bp = slope_branch(D[2], D[3], r[2], r[3]);
  const int EL = max(max(max(bexp(lv[0]), bexp(lv[1])), max(bexp(lv[2]), bexp(lv[3]))), bexp(lv[4]));
  long long l[5];
#pragma unroll
  for (int k = 0; k < 5; ++k) l[k] = to_block_fixed6(lv[k], EL);
  long long Xb;
  if (sgn > 0) {
    // sbar_k = l_k - l_{k+1}; Dbar_c = l_c + d1(sigma_c) sbar_c + d2(sigma_{c-1}) sbar_{c-1}
    const long long sbm = l[1] - l[2], sb0 = l[2] - l[3], sbp = l[3] - l[4];
    const long long Dc = l[2] + slope_d1(b0, sb0, Hq) + slope_d2(bm, sbm, Hq);
    const long long Dc1 = l[3] + slope_d1(bp, sbp, Hq) + slope_d2(b0, sb0, Hq);
    Xb = Dc - Dc1;
  } else {
    // sbar_k = l_k - l_{k-1}; Dbar_k = l_{k-1} + d1(sigma_k) sbar_k + d2(sigma_{k-1}) sbar_{k-1}
    const long long sbm = l[1] - l[0], sb0 = l[2] - l[1], sbp = l[3] - l[2];
    const long long Dc = l[1] + slope_d1(b0, sb0, Hq) + slope_d2(bm, sbm, Hq);
    const long long Dc1 = l[2] + slope_d1(bp, sbp, Hq) + slope_d2(b0, sb0, Hq);
    Xb = Dc - Dc1;
  }
  // value at exponent EL: Xb 2^(EL - 1081)
  if (EL < 64) return 0.0;
  return ll_to_double_scaled(Xb, EL - 1081);
}

// Rational-beta variant (beta = lp/lq): every partial derivative times 4 lq is
// a small integer (2 lp for beta/2, lq for 1/4), so the adjoint combinations
// are exact integer arithmetic without high multiplies.  Returns 4 lq times
// sum_{c'} lambda(c') dF(c')/dX(c).  lambda enters with a 50-bit significand.
__device__ __forceinline__ int slope_branch_rat(long long Da, long long Db, long long lp2, long long lq) {
  if ((Da ^ Db) < 0) return 0;
  const long long ra = lp2 * Da, rb = lp2 * Db, y = lq * (Da + Db);
  if (Da >= 0) {
    if (ra <= y && ra <= rb) return 1;
    return y <= rb ? 2 : 3;
  }
  if (ra >= y && ra >= rb) return 1;
  return y >= rb ? 2 : 3;
}

// lambda part of the rational-beta advection adjoint, given the minmod branch
// codes bm, b0, bp of the slopes sigma_{c-1}, sigma_c, sigma_{c+1} along the
// stride.  Returns 4 lq sum_{c'} lambda(c') dF(c')/dX(c).
__device__ __forceinline__ double adjoint_combine_rat(const double* __restrict__ L, long long stride, int bm, int b0,
                                                      int bp, int lp, int lq, int sgn) {
  double lv[5];
#pragma unroll
  for (int k = 0; k < 5; ++k) lv[k] = __ldg(L + (k - 2) * stride);
  const long long lp2 = 2 * lp, q = lq, q4 = 4 * lq;
  const int EL = max(max(max(bexp(lv[0]), bexp(lv[1])), max(bexp(lv[2]), bexp(lv[3]))), bexp(lv[4]));
  long long l[5];
#pragma unroll
  for (int k = 0; k < 5; ++k) l[k] = to_block_fixed(lv[k], EL) >> 10;
  auto d1 = [&](int br, long long sb) { return br == 1 ? lp2 * sb : (br == 2 ? q * sb : 0ll); };
  auto d2 = [&](int br, long long sb) { return br == 3 ? lp2 * sb : (br == 2 ? q * sb : 0ll); };
  long long Xb;
  if (sgn > 0) {
    const long long sbm = l[1] - l[2], sb0 = l[2] - l[3], sbp = l[3] - l[4];
    Xb = (q4 * l[2] + d1(b0, sb0) + d2(bm, sbm)) - (q4 * l[3] + d1(bp, sbp) + d2(b0, sb0));
  } else {
    const long long sbm = l[1] - l[0], sb0 = l[2] - l[1], sbp = l[3] - l[2];
    Xb = (q4 * l[1] + d1(b0, sb0) + d2(bm, sbm)) - (q4 * l[2] + d1(bp, sbp) + d2(b0, sb0));
  }
  if (EL < 64) return 0.0;
  return ll_to_double_scaled(Xb, EL - 1072);  // lambda was scaled by 2^(1072 - EL)
}

__device__ __forceinline__ double advection_adjoint_rat(const double* __restrict__ X, const double* __restrict__ L,
                                                        long long stride, int lp, int lq, int sgn) {
  double xv[5];
#pragma unroll
  for (int k = 0; k < 5; ++k) xv[k] = __ldg(X + (k - 2) * stride);
  const int EX = max(max(max(bexp(xv[0]), bexp(xv[1])), max(bexp(xv[2]), bexp(xv[3]))), bexp(xv[4]));
  const long long lp2 = 2 * lp, q = lq;
  long long D[4];
  {
    long long xi[5];
#pragma unroll
    for (int k = 0; k < 5; ++k) xi[k] = to_block_fixed52(xv[k], EX);
#pragma unroll
    for (int k = 0; k < 4; ++k) D[k] = xi[k + 1] - xi[k];
  }
  const int bm = slope_branch_rat(D[0], D[1], lp2, q);
  const int b0 = slope_branch_rat(D[1], D[2], lp2, q);
  const int bp = slope_branch_rat(D[2], D[3], lp2, q);
  return adjoint_combine_rat(L, stride, bm, b0, bp, lp, lq, sgn);
}

// ------------------------------------------------------------------- kernels
// One adjoint step in two launches.
// k_adjoint_local: Lout = a1 Lin + sum_j mbar_j dm_j/dX (collision part) at
// state X; per-block sums of the parameter adjoints (dt_mu, Pr, gm1, epsf)
// into partial[blk*4 + k].
// MOMS: the moments of X come from the recompute step (moms[k][y][x], the
// same sums in the same order) instead of being summed again here.
template <int PRC, bool MOMS>
__global__ void __launch_bounds__(256, 2) k_adjoint_local(const double* __restrict__ X, const double* __restrict__ Lin,
                                                       double* __restrict__ Lout, double* __restrict__ partial,
                                                       const double* __restrict__ moms, Geom G, Phys P) {
  const int x = blockIdx.x * 32 + threadIdx.x;
  const int y = blockIdx.y * 8 + threadIdx.y;
  const bool active = x < G.Nx && y < G.Ny;
  __shared__ long long s_cb[21 * 256];
  const int tid = threadIdx.y * 32 + threadIdx.x;
  ParamBar pb = {0, 0, 0, 0};
  if (active) {
    const long long off = cell_index(G, y, x);
    const double* xs = X + off;
    const double* ls = Lin + off;
    double* lo = Lout + off;
    const long long PL = G.plane;
    Moments m = {};
    Coeffs Cb = {};
    double a1b = 0.0;
    {
      // block exponents of the cell's lambda (f and g) for the fixed-point projection
      int ELf = 0, ELg = 0;
#pragma unroll 5
      for (int c = 0; c < 25; ++c) {
        ELf = max(ELf, bexp(__ldg(ls + c * PL)));
        ELg = max(ELg, bexp(__ldg(ls + (25 + c) * PL)));
      }
      long long* cb = s_cb + tid;
#pragma unroll
      for (int k = 0; k < 21; ++k) cb[k * 256] = 0;
      double f[5], g[5], lf[5], lg[5];
#define DVBM_ADJ_A(p)                                                                  \
      _Pragma("unroll") for (int q = 0; q < 5; ++q) {                                  \
        f[q] = __ldg(xs + (5 * p + q) * PL); g[q] = __ldg(xs + (25 + 5 * p + q) * PL);  \
        lf[q] = __ldg(ls + (5 * p + q) * PL); lg[q] = __ldg(ls + (25 + 5 * p + q) * PL); \
        a1b = fma(lf[q], f[q], fma(lg[q], g[q], a1b));                                \
      }                                                                                \
      if (!MOMS) accumulate_moments<p>(m, f, g);                                       \
      accumulate_projection_fix<p>(cb, lf, lg, ELf, ELg);
      DVBM_ADJ_A(0) DVBM_ADJ_A(1) DVBM_ADJ_A(2) DVBM_ADJ_A(3) DVBM_ADJ_A(4)
#undef DVBM_ADJ_A
      const bool okf = ELf >= 100, okg = ELg >= 100;
      const int sf = ELf - 1080, sg = ELg - 1080;
      auto cv = [](bool ok, long long v, int sc) { return ok ? ll_to_double_rn(v, sc) : 0.0; };
      Cb.f00 = cv(okf, cb[0 * 256], sf); Cb.f10 = cv(okf, cb[1 * 256], sf); Cb.f01 = cv(okf, cb[2 * 256], sf);
      Cb.f20 = cv(okf, cb[3 * 256], sf); Cb.f11 = cv(okf, cb[4 * 256], sf); Cb.f02 = cv(okf, cb[5 * 256], sf);
      Cb.f30 = cv(okf, cb[6 * 256], sf); Cb.f21 = cv(okf, cb[7 * 256], sf); Cb.f12 = cv(okf, cb[8 * 256], sf);
      Cb.f03 = cv(okf, cb[9 * 256], sf); Cb.f40 = cv(okf, cb[10 * 256], sf); Cb.f31 = cv(okf, cb[11 * 256], sf);
      Cb.f22 = cv(okf, cb[12 * 256], sf); Cb.f13 = cv(okf, cb[13 * 256], sf); Cb.f04 = cv(okf, cb[14 * 256], sf);
      Cb.g00 = cv(okg, cb[15 * 256], sg); Cb.g10 = cv(okg, cb[16 * 256], sg); Cb.g01 = cv(okg, cb[17 * 256], sg);
      Cb.g20 = cv(okg, cb[18 * 256], sg); Cb.g11 = cv(okg, cb[19 * 256], sg); Cb.g02 = cv(okg, cb[20 * 256], sg);
    }
    if (MOMS) {
      const long long cp = (long long)G.Nx * G.Ny, ci = (long long)y * G.Nx + x;
      m.m00 = moms[0 * cp + ci]; m.m10 = moms[1 * cp + ci]; m.m01 = moms[2 * cp + ci];
      m.m20 = moms[3 * cp + ci]; m.m11 = moms[4 * cp + ci]; m.m02 = moms[5 * cp + ci];
      m.m30 = moms[6 * cp + ci]; m.m21 = moms[7 * cp + ci]; m.m12 = moms[8 * cp + ci];
      m.m03 = moms[9 * cp + ci]; m.g00 = moms[10 * cp + ci]; m.g10 = moms[11 * cp + ci];
      m.g01 = moms[12 * cp + ci];
    }
    Moments mb = {};
    const double a1 = collision_coeffs_rev<PRC>(m, P, Cb, a1b, mb, pb);
#define DVBM_ADJ_B(p)                                                                       \
    {                                                                                       \
      double pf[5], pg[5];                                                                  \
      moment_pullback<p>(mb, pf, pg);                                                       \
      _Pragma("unroll") for (int q = 0; q < 5; ++q) {                                       \
        lo[(5 * p + q) * PL] = fma(a1, __ldg(ls + (5 * p + q) * PL), pf[q]);                \
        lo[(25 + 5 * p + q) * PL] = fma(a1, __ldg(ls + (25 + 5 * p + q) * PL), pg[q]);      \
      }                                                                                     \
    }
    DVBM_ADJ_B(0) DVBM_ADJ_B(1) DVBM_ADJ_B(2) DVBM_ADJ_B(3) DVBM_ADJ_B(4)
#undef DVBM_ADJ_B
  }
  // block reduction of the parameter adjoints (fixed order)
  __shared__ double sh[4][256];
  const int t = threadIdx.y * 32 + threadIdx.x;
  sh[0][t] = pb.dt_mu; sh[1][t] = pb.Pr; sh[2][t] = pb.gm1; sh[3][t] = pb.epsf;
  __syncthreads();
  for (int w = 128; w > 0; w >>= 1) {
    if (t < w)
#pragma unroll
      for (int k = 0; k < 4; ++k) sh[k][t] += sh[k][t + w];
    __syncthreads();
  }
  if (t == 0) {
    const int b = blockIdx.y * gridDim.x + blockIdx.x;
#pragma unroll
    for (int k = 0; k < 4; ++k) partial[4 * b + k] = sh[k][0];
  }
}

// k_adjoint_adv: Lout += -(dt/dx) v_x sum_c' Lin(c') dF_x(c')/dX(c) - (same in y),
// one thread per (cell, population); blockIdx.z = population.  CODED: the
// minmod branches come from the codes the recomputed forward step recorded
// (periodic neighbours wrap), so X is not read at all.  A band of a
// slab-decomposed grid passes the neighbouring bands' code rows next to its
// edges (glo: the row below y = 0, ghi: the row above y = Ny - 1; [NPOP][Nx]
// each) instead of wrapping in y (BAND).
template <bool RAT, bool CODED, bool BAND = false>
__global__ void __launch_bounds__(256) k_adjoint_adv(const double* __restrict__ X, const double* __restrict__ Lin,
                                                     double* __restrict__ Lout,
                                                     const unsigned char* __restrict__ codes, Geom G, Phys P,
                                                     const unsigned char* __restrict__ glo = nullptr,
                                                     const unsigned char* __restrict__ ghi = nullptr) {
  const int x = blockIdx.x * 32 + threadIdx.x;
  const int y = blockIdx.y * 8 + threadIdx.y;
  const int c = blockIdx.z;
  if (x >= G.Nx || y >= G.Ny) return;
  const int pn = (c % 25) / 5, qn = c % 5;
  const int sx = sgn_of(pn), sy = sgn_of(qn);
  if (sx == 0 && sy == 0) return;
  const long long off = cell_index(G, y, x) + (long long)c * G.plane;
  const double* xc = X + off;
  const double* lc = Lin + off;
  double v = Lout[off];
  if constexpr (CODED) {
    const unsigned char* cp = codes + (long long)c * G.Nx * G.Ny;
    const long long row = (long long)y * G.Nx;
    if (sx != 0) {
      const int xm = x == 0 ? G.Nx - 1 : x - 1, xp = x == G.Nx - 1 ? 0 : x + 1;
      const int bm = __ldg(cp + row + xm) & 3, b0 = __ldg(cp + row + x) & 3, bp = __ldg(cp + row + xp) & 3;
      v = fma(-P.kxr[pn], adjoint_combine_rat(lc, 1, bm, b0, bp, P.lp, P.lq, sx), v);
    }
    if (sy != 0) {
      const int ym = y == 0 ? G.Ny - 1 : y - 1, yp = y == G.Ny - 1 ? 0 : y + 1;
      const unsigned char* pm = (BAND && y == 0 && glo) ? glo + (long long)c * G.Nx + x : cp + (long long)ym * G.Nx + x;
      const unsigned char* pp =
          (BAND && y == G.Ny - 1 && ghi) ? ghi + (long long)c * G.Nx + x : cp + (long long)yp * G.Nx + x;
      const int bm = (__ldg(pm) >> 2) & 3, b0 = (__ldg(cp + row + x) >> 2) & 3, bp = (__ldg(pp) >> 2) & 3;
      v = fma(-P.kyr[qn], adjoint_combine_rat(lc, G.pitch, bm, b0, bp, P.lp, P.lq, sy), v);
    }
  } else if constexpr (RAT) {
    if (sx != 0) v = fma(-P.kxr[pn], advection_adjoint_rat(xc, lc, 1, P.lp, P.lq, sx), v);
    if (sy != 0) v = fma(-P.kyr[qn], advection_adjoint_rat(xc, lc, G.pitch, P.lp, P.lq, sy), v);
  } else {
    if (sx != 0) v = fma(-P.kxv[pn], advection_adjoint(xc, lc, 1, P.hq, sx), v);
    if (sy != 0) v = fma(-P.kyv[qn], advection_adjoint(xc, lc, G.pitch, P.hq, sy), v);
  }
  Lout[off] = v;
}

// lambda^N from dL/drho and dL/dT of the final state; partial: gm1 adjoint
__global__ void __launch_bounds__(256) k_adjoint_final(const double* __restrict__ X, const double* __restrict__ rhob,
                                                       const double* __restrict__ Tb, double* __restrict__ Lout,
                                                       double* __restrict__ partial, Geom G, Phys P, Macro M) {
  const int x = blockIdx.x * 32 + threadIdx.x;
  const int y = blockIdx.y * 8 + threadIdx.y;
  const bool active = x < G.Nx && y < G.Ny;
  ParamBar pb = {0, 0, 0, 0};
  if (active) {
    const long long off = cell_index(G, y, x);
    const long long i = (long long)y * G.Nx + x;
    const Moments m = cell_moments<double>(X + off, G.plane, P);
    Moments mb = {};
    macro_rev(m, P, M.T_ref, rhob ? rhob[i] : 0.0, Tb ? Tb[i] : 0.0, mb, pb);
#define DVBM_FIN(p)                                                          \
    {                                                                        \
      double pf[5], pg[5];                                                   \
      moment_pullback<p>(mb, pf, pg);                                        \
      _Pragma("unroll") for (int q = 0; q < 5; ++q) {                        \
        Lout[off + (5 * p + q) * G.plane] = pf[q];                           \
        Lout[off + (25 + 5 * p + q) * G.plane] = pg[q];                      \
      }                                                                      \
    }
    DVBM_FIN(0) DVBM_FIN(1) DVBM_FIN(2) DVBM_FIN(3) DVBM_FIN(4)
#undef DVBM_FIN
  }
  __shared__ double sh[256];
  const int t = threadIdx.y * 32 + threadIdx.x;
  sh[t] = pb.gm1;
  __syncthreads();
  for (int w = 128; w > 0; w >>= 1) {
    if (t < w) sh[t] += sh[t + w];
    __syncthreads();
  }
  if (t == 0) partial[blockIdx.y * gridDim.x + blockIdx.x] = sh[0];
}

// adjoint of the equilibrium initial condition: per-cell dL/d(rho0, ux0, uy0, T0)
// and per-block epsf adjoints
__global__ void __launch_bounds__(256) k_adjoint_init(const double* __restrict__ L, const double* __restrict__ rho,
                                                      const double* __restrict__ ux, const double* __restrict__ uy,
                                                      const double* __restrict__ T, double* grho, double* gux,
                                                      double* guy, double* gT, double* __restrict__ partial, Geom G,
                                                      Phys P, Macro M) {
  const int x = blockIdx.x * 32 + threadIdx.x;
  const int y = blockIdx.y * 8 + threadIdx.y;
  const bool active = x < G.Nx && y < G.Ny;
  double epsfb = 0.0;
  if (active) {
    const long long off = cell_index(G, y, x);
    const long long i = (long long)y * G.Nx + x;
    Coeffs Cb = {};
    {
      double lf[5], lg[5];
#define DVBM_INI(p)                                                         \
      _Pragma("unroll") for (int q = 0; q < 5; ++q) {                       \
        lf[q] = L[off + (5 * p + q) * G.plane];                             \
        lg[q] = L[off + (25 + 5 * p + q) * G.plane];                        \
      }                                                                     \
      accumulate_projection<p>(Cb, lf, lg);
      DVBM_INI(0) DVBM_INI(1) DVBM_INI(2) DVBM_INI(3) DVBM_INI(4)
#undef DVBM_INI
    }
    double rb, ub, vb, thb;
    equilibrium_rev(rho[i], ux[i] / M.c, uy[i] / M.c, T[i] / M.T_ref, P, Cb, rb, ub, vb, thb, epsfb);
    grho[i] = rb;
    gux[i] = ub / M.c;
    guy[i] = vb / M.c;
    gT[i] = thb / M.T_ref;
  }
  __shared__ double sh[256];
  const int t = threadIdx.y * 32 + threadIdx.x;
  sh[t] = epsfb;
  __syncthreads();
  for (int w = 128; w > 0; w >>= 1) {
    if (t < w) sh[t] += sh[t + w];
    __syncthreads();
  }
  if (t == 0) partial[blockIdx.y * gridDim.x + blockIdx.x] = sh[0];
}

// ------------------------------------------------------------------ wrappers
int adjoint_blocks(const Geom& G) { return ((G.Nx + 31) / 32) * ((G.Ny + 7) / 8); }

// Branch-code rows next to a band's edges: unpack = 0 copies rows y = 0 (to
// lo) and y = Ny - 1 (to hi) of every population's codes, unpack = 1 copies
// lo and hi into the ghost code rows glo, ghi; layouts [NPOP][Nx] bytes; a
// NULL buffer skips its side.
__global__ void k_code_rows(unsigned char* __restrict__ codes, unsigned char* __restrict__ lo,
                            unsigned char* __restrict__ hi, unsigned char* __restrict__ glo,
                            unsigned char* __restrict__ ghi, int unpack, int Nx, int Ny) {
  const long long n = (long long)NPOP * Nx;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const long long c = i / Nx, x = i % Nx;
    if (unpack) {
      if (lo) glo[i] = lo[i];
      if (hi) ghi[i] = hi[i];
    } else {
      if (lo) lo[i] = codes[(c * Ny) * Nx + x];
      if (hi) hi[i] = codes[(c * Ny + Ny - 1) * Nx + x];
    }
  }
}

cudaError_t launch_code_rows(unsigned char* codes, void* lo, void* hi, unsigned char* glo, unsigned char* ghi,
                             int unpack, const Geom& G, cudaStream_t st) {
  const long long n = (long long)NPOP * G.Nx;
  const int blocks = (int)std::min<long long>((n + 255) / 256, 4096);
  k_code_rows<<<blocks, 256, 0, st>>>(codes, (unsigned char*)lo, (unsigned char*)hi, glo, ghi, unpack, G.Nx, G.Ny);
  return cudaGetLastError();
}

cudaError_t launch_adjoint_step(const double* X, const double* Lin, double* Lout, double* partial,
                                const unsigned char* codes, const double* moms, const Geom& G, const Phys& P,
                                cudaStream_t st, const unsigned char* glo, const unsigned char* ghi) {
  dim3 block(32, 8), grid((G.Nx + 31) / 32, (G.Ny + 7) / 8);
  if (moms) {
    if (P.prc < 0) k_adjoint_local<-1, true><<<grid, block, 0, st>>>(X, Lin, Lout, partial, moms, G, P);
    else if (P.prc > 0) k_adjoint_local<1, true><<<grid, block, 0, st>>>(X, Lin, Lout, partial, moms, G, P);
    else k_adjoint_local<0, true><<<grid, block, 0, st>>>(X, Lin, Lout, partial, moms, G, P);
  } else {
    if (P.prc < 0) k_adjoint_local<-1, false><<<grid, block, 0, st>>>(X, Lin, Lout, partial, nullptr, G, P);
    else if (P.prc > 0) k_adjoint_local<1, false><<<grid, block, 0, st>>>(X, Lin, Lout, partial, nullptr, G, P);
    else k_adjoint_local<0, false><<<grid, block, 0, st>>>(X, Lin, Lout, partial, nullptr, G, P);
  }
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  dim3 grid3(grid.x, grid.y, NPOP);
  if (P.lq > 0 && codes && (glo || ghi))
    k_adjoint_adv<true, true, true><<<grid3, block, 0, st>>>(X, Lin, Lout, codes, G, P, glo, ghi);
  else if (P.lq > 0 && codes) k_adjoint_adv<true, true><<<grid3, block, 0, st>>>(X, Lin, Lout, codes, G, P);
  else if (P.lq > 0) k_adjoint_adv<true, false><<<grid3, block, 0, st>>>(X, Lin, Lout, nullptr, G, P);
  else k_adjoint_adv<false, false><<<grid3, block, 0, st>>>(X, Lin, Lout, nullptr, G, P);
  return cudaGetLastError();
}

cudaError_t launch_adjoint_final(const double* X, const double* rhob, const double* Tb, double* Lout, double* partial,
                                 const Geom& G, const Phys& P, const Macro& M, cudaStream_t st) {
  dim3 block(32, 8), grid((G.Nx + 31) / 32, (G.Ny + 7) / 8);
  k_adjoint_final<<<grid, block, 0, st>>>(X, rhob, Tb, Lout, partial, G, P, M);
  return cudaGetLastError();
}

cudaError_t launch_adjoint_init(const double* L, const double* rho, const double* ux, const double* uy,
                                const double* T, double* grho, double* gux, double* guy, double* gT, double* partial,
                                const Geom& G, const Phys& P, const Macro& M, cudaStream_t st) {
  dim3 block(32, 8), grid((G.Nx + 31) / 32, (G.Ny + 7) / 8);
  k_adjoint_init<<<grid, block, 0, st>>>(L, rho, ux, uy, T, grho, gux, guy, gT, partial, G, P, M);
  return cudaGetLastError();
}

}  // namespace dvbm
