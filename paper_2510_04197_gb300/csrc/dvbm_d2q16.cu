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
#include "dvbm_q16.cuh"
#include "dvbm_internal.h"

namespace dvbm {

// the node constants as a constant-bank table for the node loop
__constant__ long long c_khqx[4][4] = {
    {q16::khqfix(0, 0), q16::khqfix(0, 1), q16::khqfix(0, 2), q16::khqfix(0, 3)},
    {q16::khqfix(1, 0), q16::khqfix(1, 1), q16::khqfix(1, 2), q16::khqfix(1, 3)},
    {q16::khqfix(2, 0), q16::khqfix(2, 1), q16::khqfix(2, 2), q16::khqfix(2, 3)},
    {q16::khqfix(3, 0), q16::khqfix(3, 1), q16::khqfix(3, 2), q16::khqfix(3, 3)}};

template <int PRC, bool RAT>
__global__ void __launch_bounds__(256, 4) k_step16(const double* __restrict__ src, double* __restrict__ dst, Geom G,
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
    const int dp = kdq(p < 2 ? 0 : 2);
    const int sx = (p & 1) ? -1 : 1;  // nodes +a, -a, +b, -b
    // kx of node p: kxv[1] = -kxv[0] and kxv[3] = -kxv[2] exactly
    const double kb = p < 2 ? (RAT ? P.kxr[0] : P.kxv[0]) : (RAT ? P.kxr[2] : P.kxv[2]);
    const double kx = kb * (double)sx;
    const long long pbase = (long long)(4 * p) * PL;
#pragma unroll 1
    for (int k = 0; k < 2; ++k) {  // f then g: one copy of the body for both
      // the next population's seven stencil values are loaded one iteration
      // ahead (the rolled loop would leave them exposed)
      double cv = 0, xa = 0, xb = 0, xc = 0, ya = 0, yb = 0, yc = 0;
      auto load_stencil = [&](int qq, double& c0, double& x0, double& x1, double& x3, double& y0, double& y1,
                              double& y3) {
        const double* pq = s + pbase + (long long)(qq + 16 * k) * PL;
        c0 = __ldg(pq);
        const long long ox = sx > 0 ? -2 : -1;
        x0 = __ldg(pq + ox);
        x1 = __ldg(pq + ox + (sx > 0 ? 1 : 2));
        x3 = __ldg(pq + ox + 3);
        const int sq = sgn(qq);
        const long long oy = sq > 0 ? -2 * PT : -PT;
        y0 = __ldg(pq + oy);
        y1 = __ldg(pq + oy + (sq > 0 ? PT : 2 * PT));
        y3 = __ldg(pq + oy + 3 * PT);
      };
      // the first population's stencil is loaded before the collision target
      // below is built, whose integer work then covers the load latency
      load_stencil(0, cv, xa, xb, xc, ya, yb, yc);
      // this half's collision target (f, then g), built at the top of its own
      // pass so that the g targets are not live across the f populations
      double tk[4];
      {
        long long xx[4];
        int sc;
        bool live;
        if (k == 0) {
          long long h[4];
          h[0] = mhk(xs[0 * 256], k0) + mhk(xs[1 * 256], k1) + mhk(xs[3 * 256], k2) + mhk(xs[6 * 256], k3);
          h[1] = mhk(xs[2 * 256], k0) + mhk(xs[4 * 256], k1) + mhk(xs[7 * 256], k2);
          h[2] = mhk(xs[5 * 256], k0) + mhk(xs[8 * 256], k1);
          h[3] = mhk(xs[9 * 256], k0);
          const int sh = renorm_fix(h);
          expand_fix(h, xx);
          sc = Ef - 1080 - dp - sh;
          live = Ef >= 100;
        } else {
          long long h[3];
          h[0] = mhk(xs[10 * 256], k0) + mhk(xs[11 * 256], k1) + mhk(xs[13 * 256], k2);
          h[1] = mhk(xs[12 * 256], k0) + mhk(xs[14 * 256], k1);
          h[2] = mhk(xs[15 * 256], k0);
          const int sh = renorm_fix(h);
          expand3_fix(h, xx);
          sc = Eg - 1080 - dp - sh;
          live = Eg >= 100;
        }
#pragma unroll
        for (int q = 0; q < 4; ++q)  // value of t_q = x 2^(E - 1080 - kdq(p) - s - kdq(q))
          tk[q] = live ? ll_to_double_rn(xx[q], sc - kdq(q)) : 0.0;
      }

#pragma unroll 1
      for (int q = 0; q < 4; ++q) {  // y-nodes rolled too: one copy of the population body
        const long long co = pbase + (long long)(q + 16 * k) * PL;
        const double t = q == 0 ? tk[0] : q == 1 ? tk[1] : q == 2 ? tk[2] : tk[3];
        double nc = 0, nx0 = 0, nx1 = 0, nx3 = 0, ny0 = 0, ny1 = 0, ny3 = 0;
        if (q < 3) load_stencil(q + 1, nc, nx0, nx1, nx3, ny0, ny1, ny3);
        // flux difference of the stencil (a0..a3 = cells j-2..j+1 for v > 0,
        // j-1..j+2 for v < 0): rational or general limiter
        auto fdiff = [&](double a0, double a1, double a2, double a3, int sg) -> double {
          if constexpr (RAT) return flux_difference_rat_v(a0, a1, a2, a3, P.lp, P.lq, sg);
          else return flux_difference_int_v(a0, a1, a2, a3, P.hq, sg);
        };
        const double fx = sx > 0 ? fdiff(xa, xb, cv, xc, 1) : fdiff(xa, cv, xb, xc, -1);
        const double fy = sgn(q) > 0 ? fdiff(ya, yb, cv, yc, 1) : fdiff(ya, cv, yb, yc, -1);
        const double c = cv;
        cv = nc; xa = nx0; xb = nx1; xc = nx3; ya = ny0; yb = ny1; yc = ny3;
        double v = fma(C.a1, c, t);
        v = fma(-kx, fx, v);
        v = fma(RAT ? -P.kyr[q] : -P.kyv[q], fy, v);
        d[co] = v;
      }
    }
  }
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

}  // namespace dvbm
