// dvbm_d2q16.cu -- the total-energy split (I) on the D2Q16 lattice.
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
#include "dvbm_device.cuh"
#include "dvbm_internal.h"

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

// the node constants as a constant-bank table for the node loop
__constant__ long long c_khqx[4][4] = {
    {q16::khqfix(0, 0), q16::khqfix(0, 1), q16::khqfix(0, 2), q16::khqfix(0, 3)},
    {q16::khqfix(1, 0), q16::khqfix(1, 1), q16::khqfix(1, 2), q16::khqfix(1, 3)},
    {q16::khqfix(2, 0), q16::khqfix(2, 1), q16::khqfix(2, 2), q16::khqfix(2, 3)},
    {q16::khqfix(3, 0), q16::khqfix(3, 1), q16::khqfix(3, 2), q16::khqfix(3, 3)}};

template <int PRC, bool RAT>
__global__ void __launch_bounds__(256) k_step16(const double* __restrict__ src, double* __restrict__ dst, Geom G,
                                                Phys P, unsigned int* __restrict__ flag) {
  using namespace q16;
  const int x = blockIdx.x * 32 + threadIdx.x;
  const int y = blockIdx.y * 8 + threadIdx.y;
  if (x >= G.Nx || y >= G.Ny) return;
  const long long off = cell_index(G, y, x);
  const double* s = src + off;
  double* d = dst + off;
  const long long PL = G.plane, PT = G.pitch;
  const Mom m = cell_moments(s, PL);
  const Co C = coeffs<PRC>(m, P);
  if (C.bad) atomicOr(flag, 1u);
  // fixed-point coefficients in shared memory (field k of thread t at
  // [k * 256 + t]) rather than in 32 registers across the node loop
  __shared__ long long s_fix[16 * 256];
  long long* xs = s_fix + threadIdx.y * 32 + threadIdx.x;
  int Ef, Eg;
  {
    const CoFix Xr = to_fix(C);
    const long long v[16] = {Xr.f00, Xr.f10, Xr.f01, Xr.f20, Xr.f11, Xr.f02, Xr.f30, Xr.f21,
                             Xr.f12, Xr.f03, Xr.g00, Xr.g10, Xr.g01, Xr.g20, Xr.g11, Xr.g02};
#pragma unroll
    for (int k = 0; k < 16; ++k) xs[k * 256] = v[k];
    Ef = Xr.Ef;
    Eg = Xr.Eg;
  }
  // x-nodes p = 0..3 in a run-time loop (one copy of the body: the kernel
  // stays small enough for the instruction cache).
  // The Grad expansion runs in block fixed point on the integer pipe.
#pragma unroll 1
  for (int p = 0; p < 4; ++p) {
    const long long k0 = c_khqx[p][0], k1 = c_khqx[p][1], k2 = c_khqx[p][2], k3 = c_khqx[p][3];
    long long h[4], hh[3], xf[4], xg[4];
    h[0] = mhk(xs[0 * 256], k0) + mhk(xs[1 * 256], k1) + mhk(xs[3 * 256], k2) + mhk(xs[6 * 256], k3);
    h[1] = mhk(xs[2 * 256], k0) + mhk(xs[4 * 256], k1) + mhk(xs[7 * 256], k2);
    h[2] = mhk(xs[5 * 256], k0) + mhk(xs[8 * 256], k1);
    h[3] = mhk(xs[9 * 256], k0);
    hh[0] = mhk(xs[10 * 256], k0) + mhk(xs[11 * 256], k1) + mhk(xs[13 * 256], k2);
    hh[1] = mhk(xs[12 * 256], k0) + mhk(xs[14 * 256], k1);
    hh[2] = mhk(xs[15 * 256], k0);
    const int sf = renorm_fix(h), sg = renorm_fix(hh);
    expand_fix(h, xf);
    expand3_fix(hh, xg);
    const int dp = kdq(p < 2 ? 0 : 2);
    double tf[4], tg[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      // value of t_q = x 2^(E - 1080 - kdq(p) - s - kdq(q))
      tf[q] = Ef >= 100 ? ll_to_double_rn(xf[q], Ef - 1080 - dp - sf - kdq(q)) : 0.0;
      tg[q] = Eg >= 100 ? ll_to_double_rn(xg[q], Eg - 1080 - dp - sg - kdq(q)) : 0.0;
    }
    const int sx = (p & 1) ? -1 : 1;  // nodes +a, -a, +b, -b
    // kx of node p: kxv[1] = -kxv[0] and kxv[3] = -kxv[2] exactly
    const double kb = p < 2 ? (RAT ? P.kxr[0] : P.kxv[0]) : (RAT ? P.kxr[2] : P.kxv[2]);
    const double kx = kb * (double)sx;
    const long long pbase = (long long)(4 * p) * PL;
#pragma unroll 1
    for (int k = 0; k < 2; ++k) {  // f then g: one copy of the body for both
      double tk[4];
#pragma unroll
      for (int q = 0; q < 4; ++q) tk[q] = k == 0 ? tf[q] : tg[q];
#pragma unroll 1
      for (int q = 0; q < 4; ++q) {  // y-nodes rolled too: one copy of the population body
        const long long co = pbase + (long long)(q + 16 * k) * PL;
        const double* pc = s + co;
        double fx, fy;
        if constexpr (RAT) {
          fx = flux_difference_rat(pc, 1, P.lp, P.lq, sx);
          fy = flux_difference_rat(pc, PT, P.lp, P.lq, sgn(q));
        } else {
          fx = flux_difference_int(pc, 1, P.hq, sx);
          fy = flux_difference_int(pc, PT, P.hq, sgn(q));
        }
        double v = fma(C.a1, __ldg(pc), q == 0 ? tk[0] : q == 1 ? tk[1] : q == 2 ? tk[2] : tk[3]);
        v = fma(-kx, fx, v);
        v = fma(RAT ? -P.kyr[q] : -P.kyv[q], fy, v);
        d[co] = v;
      }
    }
  }
}

__global__ void k_init16(double* __restrict__ dst, const double* __restrict__ rho, const double* __restrict__ ux,
                         const double* __restrict__ uy, const double* __restrict__ T, Geom G, Phys P, Macro M) {
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  const int y = blockIdx.y * blockDim.y + threadIdx.y;
  if (x >= G.Nx || y >= G.Ny) return;
  const long long i = (long long)y * G.Nx + x;
  const q16::Co C = q16::equilibrium(rho[i], ux[i] / M.c, uy[i] / M.c, T[i] / M.T_ref, P);
  q16::write_expansion(dst + cell_index(G, y, x), G.plane, C, nullptr, nullptr);
}

__global__ void k_moments16(const double* __restrict__ src, double* rho, double* ux, double* uy, double* T, Geom G,
                            Phys P, Macro M) {
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  const int y = blockIdx.y * blockDim.y + threadIdx.y;
  if (x >= G.Nx || y >= G.Ny) return;
  const q16::Mom m = q16::cell_moments(src + cell_index(G, y, x), G.plane);
  double r, a, b, t;
  q16::macro(m, P, M.c, M.T_ref, r, a, b, t);
  const long long i = (long long)y * G.Nx + x;
  if (rho) rho[i] = r;
  if (ux) ux[i] = a;
  if (uy) uy[i] = b;
  if (T) T[i] = t;
}

__global__ void __launch_bounds__(256) k_totals16(const double* __restrict__ src, double* partial, Geom G, Phys P,
                                                  Macro M) {
  double acc[5] = {0, 0, 0, 0, 0};
  const long long ncell = (long long)G.Nx * G.Ny;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < ncell;
       i += (long long)gridDim.x * blockDim.x) {
    const int y = (int)(i / G.Nx), x = (int)(i % G.Nx);
    const q16::Mom m = q16::cell_moments(src + cell_index(G, y, x), G.plane);
    double r, a, b, t;
    q16::macro(m, P, M.c, M.T_ref, r, a, b, t);
    acc[0] += m.m00;
    acc[1] += m.m10 * M.c;
    acc[2] += m.m01 * M.c;
    acc[3] += m.g00;
    if (!(r > 0.0) || !(t > 0.0) || !(fabs(m.g00) < 1e300)) acc[4] += 1.0;
  }
  __shared__ double sh[5][256];
#pragma unroll
  for (int k = 0; k < 5; ++k) sh[k][threadIdx.x] = acc[k];
  __syncthreads();
  for (int w = 128; w > 0; w >>= 1) {
    if ((int)threadIdx.x < w)
#pragma unroll
      for (int k = 0; k < 5; ++k) sh[k][threadIdx.x] += sh[k][threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0)
    for (int k = 0; k < 5; ++k) partial[blockIdx.x * 6 + k] = sh[k][0];
}

// ghost layers: periodic / zero-gradient copies or the wall closure (Sec. III.E)
// same thread layout as k_ghost: blockIdx.z = population for copied sides,
// the z = 0 slice for wall sides
__global__ void k_ghost16(double* __restrict__ buf, Geom G, Phys P, Macro M, BCDev bc) {
  const int side = blockIdx.y;
  const int kind = bc.kind[side];
  const int pop = blockIdx.z;
  if (kind == 3) return;  // external: the caller supplies these rows (dvbm_halo_unpack)
  if (kind == 2 && pop != 0) return;
  const int len = side < 2 ? G.Ny : G.Nx;
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= 2 * len) return;
  const int k = 1 + t / len;
  const int j = t % len;
  const bool lo = (side % 2) == 0;
  const int n = side < 2 ? G.Nx : G.Ny;
  const int gi = lo ? -k : n - 1 + k;
  int bi;
  if (kind == 0) bi = lo ? n - k : k - 1;
  else if (kind == 1) bi = lo ? 0 : n - 1;
  else bi = lo ? k - 1 : n - k;
  int gx, gy, bx, by;
  if (side < 2) { gx = gi; gy = j; bx = bi; by = j; }
  else          { gx = j; gy = gi; bx = j; by = bi; }
  const long long PL = G.plane;
  double* gptr = buf + cell_index(G, gy, gx);
  const double* bptr = buf + cell_index(G, by, bx);
  if (kind != 2) {
    gptr[pop * PL] = bptr[pop * PL];
    return;
  }
  const q16::Mom m = q16::cell_moments(bptr, PL);
  double rho, ux, uy, T;
  q16::macro(m, P, M.c, M.T_ref, rho, ux, uy, T);
  const q16::Co CB = q16::equilibrium(rho, ux / M.c, uy / M.c, T / M.T_ref, P);
  const q16::Co CG = q16::equilibrium(rho, (2.0 * bc.uw[side][0] - ux) / M.c, (2.0 * bc.uw[side][1] - uy) / M.c,
                                      (2.0 * bc.Tw[side] - T) / M.T_ref, P);
  double neqf[16], neqg[16];
#define Q16_NEQ(p)                                                                     \
  {                                                                                    \
    double h[4], tf[4], hh[4], tg[4];                                                  \
    q16::hf<p>(CB, h); q16::expand(h, tf); q16::hg<p>(CB, hh); q16::expand(hh, tg);    \
    _Pragma("unroll") for (int q = 0; q < 4; ++q) {                                    \
      neqf[4 * p + q] = bptr[(4 * p + q) * PL] - tf[q];                                \
      neqg[4 * p + q] = bptr[(16 + 4 * p + q) * PL] - tg[q];                           \
    }                                                                                  \
  }
  Q16_NEQ(0) Q16_NEQ(1) Q16_NEQ(2) Q16_NEQ(3)
#undef Q16_NEQ
  q16::write_expansion(gptr, PL, CG, neqf, neqg);
}

// ---------------------------------------------------------------- wrappers
cudaError_t launch_step16(const void* src, void* dst, const Geom& G, const Phys& P, unsigned int* flag,
                          cudaStream_t st) {
  dim3 block(32, 8), grid((G.Nx + 31) / 32, (G.Ny + 7) / 8);
  const double* s = (const double*)src;
  double* d = (double*)dst;
  const bool rat = P.lq > 0;
  if (P.prc < 0) {
    if (rat) k_step16<-1, true><<<grid, block, 0, st>>>(s, d, G, P, flag);
    else k_step16<-1, false><<<grid, block, 0, st>>>(s, d, G, P, flag);
  } else if (P.prc > 0) {
    if (rat) k_step16<1, true><<<grid, block, 0, st>>>(s, d, G, P, flag);
    else k_step16<1, false><<<grid, block, 0, st>>>(s, d, G, P, flag);
  } else {
    if (rat) k_step16<0, true><<<grid, block, 0, st>>>(s, d, G, P, flag);
    else k_step16<0, false><<<grid, block, 0, st>>>(s, d, G, P, flag);
  }
  return cudaGetLastError();
}

cudaError_t launch_init16(void* dst, const double* rho, const double* ux, const double* uy, const double* T,
                          const Geom& G, const Phys& P, const Macro& M, cudaStream_t st) {
  dim3 b(32, 4), g((G.Nx + 31) / 32, (G.Ny + 3) / 4);
  k_init16<<<g, b, 0, st>>>((double*)dst, rho, ux, uy, T, G, P, M);
  return cudaGetLastError();
}

cudaError_t launch_moments16(const void* src, double* rho, double* ux, double* uy, double* T, const Geom& G,
                             const Phys& P, const Macro& M, cudaStream_t st) {
  dim3 b(32, 4), g((G.Nx + 31) / 32, (G.Ny + 3) / 4);
  k_moments16<<<g, b, 0, st>>>((const double*)src, rho, ux, uy, T, G, P, M);
  return cudaGetLastError();
}

cudaError_t launch_totals16(const void* src, double* partial, int nblocks, const Geom& G, const Phys& P,
                            const Macro& M, cudaStream_t st) {
  k_totals16<<<nblocks, 256, 0, st>>>((const double*)src, partial, G, P, M);
  return cudaGetLastError();
}

cudaError_t launch_ghost16(void* buf, const Geom& G, const Phys& P, const Macro& M, const BCDev& bc,
                           cudaStream_t st) {
  const int len = G.Nx > G.Ny ? G.Nx : G.Ny;
  dim3 b(128), g((2 * len + 127) / 128, 4, q16::NP);
  k_ghost16<<<g, b, 0, st>>>((double*)buf, G, P, M, bc);
  return cudaGetLastError();
}

}  // namespace dvbm
