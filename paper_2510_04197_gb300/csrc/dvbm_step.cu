// dvbm_step.cu -- the fused per-cell time step (Sec. III.A.1, Eq. finalDiscretePDE).
//
// One thread per cell, 32 x 8 cells per CTA.  Phase A reads the cell's 50
// populations and accumulates the sum-factorised moments; the thread then
// forms the combined collision coefficients (dvbm_device.cuh).  Phase B walks
// the populations x-node by x-node: for each it evaluates the collision target
// (sum-factorised Grad expansion, in block fixed point on the integer pipe),
// the upwind-limited flux differences along x and y from the L1-cached
// neighbours, and writes the new value:
//     F_new = (1 - dt/tau1) F + W W sum C He He - (dt/dx) v_x dF_x - (dt/dy) v_y dF_y.
// The storage variant FP32DEV keeps float deviations from a reference state;
// moments, temperature and the collision coefficients stay in double, the
// expansion keeps FP64-or-better precision, the advection runs in float on
// the deviations.
#include "dvbm_device.cuh"
#include "dvbm_internal.h"

namespace dvbm {

template <class S> struct StoreT;
template <> struct StoreT<double> { typedef double adv_t; };
template <> struct StoreT<float> { typedef float adv_t; };

// Load the five populations (p, q = 0..4) of one x-node as doubles (FP32DEV:
// reference added back).
template <class S, int p>
__device__ __forceinline__ void load_node(const S* __restrict__ src, long long plane, const Phys& P,
                                          double (&f)[5], double (&g)[5]) {
#pragma unroll
  for (int q = 0; q < 5; ++q) {
    const int c = 5 * p + q;
    if constexpr (sizeof(S) == 8) {
      f[q] = __ldg(src + c * plane);
      g[q] = __ldg(src + (25 + c) * plane);
    } else {
      f[q] = f2d_bits(__ldg(src + c * plane));
      g[q] = f2d_bits(__ldg(src + (25 + c) * plane));
    }
  }
}

// W_k He_n(xi_k)/n! of the five x-nodes as 63-bit fixed-point fractions
// (khfix), a constant-bank table for the node loop
__constant__ long long c_khx[5][5] = {
    {khfix(0, 0), khfix(0, 1), khfix(0, 2), khfix(0, 3), khfix(0, 4)},
    {khfix(1, 0), khfix(1, 1), khfix(1, 2), khfix(1, 3), khfix(1, 4)},
    {khfix(2, 0), khfix(2, 1), khfix(2, 2), khfix(2, 3), khfix(2, 4)},
    {khfix(3, 0), khfix(3, 1), khfix(3, 2), khfix(3, 3), khfix(3, 4)},
    {khfix(4, 0), khfix(4, 1), khfix(4, 2), khfix(4, 3), khfix(4, 4)}};

// This thread's fixed-point collision coefficients, kept in shared memory
// (field k of thread t at [k * kCta + t]: consecutive threads, consecutive
// words) rather than in 42 registers across the node loop, so that three
// CTAs fit on an SM.  Field order as in CoeffsFix.
constexpr int kFixFields = 21;
constexpr int kTileY = 8;                 // CTA = 32 x kTileY cells
constexpr int kCta = 32 * kTileY;
struct FixView {
  const long long* b;
  __device__ __forceinline__ long long operator()(int k) const { return b[k * kCta]; }
};
__device__ __forceinline__ void fix_to_smem(const CoeffsFix& X, long long* b) {
  const long long v[kFixFields] = {X.f00, X.f10, X.f01, X.f20, X.f11, X.f02, X.f30, X.f21, X.f12, X.f03, X.f40,
                                   X.f31, X.f22, X.f13, X.f04, X.g00, X.g10, X.g01, X.g20, X.g11, X.g02};
#pragma unroll
  for (int k = 0; k < kFixFields; ++k) b[k * kCta] = v[k];
}
// h^b of x-node p from the shared-memory coefficients (value = h 2^(E - 1081 - kd(p)))
__device__ __forceinline__ void hfg_fix_view(const FixView& X, long long k0, long long k1, long long k2, long long k3,
                                             long long k4, long long (&hf)[5], long long (&hg)[3]) {
  hfg_fix(X, k0, k1, k2, k3, k4, hf, hg);
}
__device__ __forceinline__ void hfg_fix_view_centre(const FixView& X, long long (&hf)[5], long long (&hg)[3]) {
  constexpr long long k0 = khfix(0, 0), k2 = khfix(0, 2), k4 = khfix(0, 4);
  hf[0] = mhk(X(0), k0) + mhk(X(3), k2) + mhk(X(10), k4);
  hf[1] = mhk(X(2), k0) + mhk(X(7), k2);
  hf[2] = mhk(X(5), k0) + mhk(X(12), k2);
  hf[3] = mhk(X(9), k0);
  hf[4] = mhk(X(14), k0);
  hg[0] = mhk(X(15), k0) + mhk(X(18), k2);
  hg[1] = mhk(X(17), k0);
  hg[2] = mhk(X(20), k0);
}

// The ten populations (f and g, y-nodes q = 0..4) of x-node p: collision
// target from the sum-factorised expansion, upwind-limited flux differences
// along x (p != 0) and y (q != 0), new value.  CENTER: p = 0 (xi_x = 0, no
// x-flux); otherwise p = 1..4 at run time, so one copy of this body serves
// the four moving x-nodes and the kernel's code stays small enough for the
// instruction cache.
// CODES (FP64, rational limiter only): also store, per population, the
// minmod branch codes of the cell's own x and y slopes as one byte
// (x | y << 2) at cd[pop * cplane]; the adjoint of the step reads them.
// The expansion runs in block fixed point on the integer pipe from X (the
// coefficients C converted once per cell), at FP64-or-better precision, for
// both storage forms.
template <class S, bool RAT, bool CENTER, bool CODES = false>
__device__ __forceinline__ void node_update(int p, const S* __restrict__ s, S* __restrict__ d, long long PL,
                                            long long PT, const Coeffs& C, const FixView& X, int Ef, int Eg,
                                            const Phys& P,
                                            float a1f, unsigned char* __restrict__ cd = nullptr,
                                            long long cplane = 0) {
  typedef typename StoreT<S>::adv_t A;
  // collision target in the storage's arithmetic type (FP32-deviation storage
  // rounds the fixed-point result straight to float).  FP64 storage builds
  // each half's target (f, then g) at the top of its own pass of the f/g loop
  // below, so that the g targets are not live across the f populations (spill
  // 200 -> 16 B per thread, 1007 -> 1086 MLUPS at 4096^2); the arithmetic is
  // the same.  Loading the first population's stencil before this target is
  // built measured 1083.
  constexpr bool SPLIT_T = sizeof(S) == 8;
  const int dp = (CENTER || p == 0) ? 0 : (p <= 2 ? kd(1) : kd(3));
  A tf[5], tg[5];
  if constexpr (!SPLIT_T) {
    long long hf[5], hg[3], xf[5], xg[5];
    if constexpr (CENTER) hfg_fix_view_centre(X, hf, hg);
    else hfg_fix_view(X, c_khx[p][0], c_khx[p][1], c_khx[p][2], c_khx[p][3], c_khx[p][4], hf, hg);  // p = 0 too
    const int sf = renorm_fix(hf), sg = renorm_fix(hg);
    expand_q5_fix(hf, xf);
    expand_q3_fix(hg, xg);
    const int scf = Ef - 1080 - sf - dp, scg = Eg - 1080 - sg - dp;
#pragma unroll
    for (int q = 0; q < 5; ++q) {
      if constexpr (sizeof(S) == 8) {
        tf[q] = Ef >= 100 ? ll_to_double_rn(xf[q], scf - kd(q)) : 0.0;
        tg[q] = Eg >= 100 ? ll_to_double_rn(xg[q], scg - kd(q)) : 0.0;
      } else {
        tf[q] = Ef >= 100 ? ll_to_float_rn(xf[q], scf - kd(q)) : 0.0f;
        tg[q] = Eg >= 100 ? ll_to_float_rn(xg[q], scg - kd(q)) : 0.0f;
      }
    }
  }
  // x-node sign and flux factor (p = 1, 3: +xi; p = 2, 4: -xi); warp-uniform selects
  const int sx = (p & 1) ? 1 : -1;
  const bool xmove = !CENTER && p != 0;  // the centre node has no x-flux
  const int pa = (p + 1) >> 1;  // 1 for p = 1, 2; 2 for p = 3, 4
  double kx = 0.0;
  float kxf = 0.f;
  if constexpr (!CENTER) {
    if constexpr (sizeof(S) == 8) {
      const double k_a = RAT ? P.kxr[1] : P.kxv[1], k_b = RAT ? P.kxr[3] : P.kxv[3];
      kx = (pa == 1 ? k_a : k_b) * (double)sx;  // kxv[2] = -kxv[1], kxv[4] = -kxv[3] exactly
    } else {
      kxf = (pa == 1 ? P.kxvf[1] : P.kxvf[3]) * (float)sx;
    }
  }
  const A hb = (A)P.hb;
  const long long pbase = (long long)(5 * p) * PL;
  // FP64 storage also rolls the y-node loop (one copy of the population body:
  // fewer instruction-cache misses, 964 -> 986 MLUPS at 4096^2, bitwise the same
  // result); FP32-deviation storage keeps it unrolled (1754 vs 1722 MLUPS rolled,
  // 1742 rolled with the stencil loads below, 1734 with the x-neighbours
  // exchanged by warp shuffle instead of loaded)
  constexpr bool ROLLQ = sizeof(S) == 8;
  // The rolled loop would leave each population's stencil loads exposed, so
  // FP64 storage (every limiter form, with or without branch codes) loads the
  // next population's seven stencil values (centre, three along x, three
  // along y) one iteration ahead: 986 -> 1009 MLUPS at 4096^2 for the
  // rational limiter, bitwise the same result.
  constexpr bool PREF = sizeof(S) == 8;
#pragma unroll 1
  for (int k = 0; k < 2; ++k) {  // f then g: one copy of the body for both
    A tk[5];
    if constexpr (SPLIT_T) {
      long long xx[5];
      int sc;
      bool live;
      if (k == 0) {
        long long h[5];
        hf_fix(X, c_khx[p][0], c_khx[p][1], c_khx[p][2], c_khx[p][3], c_khx[p][4], h);
        const int sh = renorm_fix(h);
        expand_q5_fix(h, xx);
        sc = Ef - 1080 - sh - dp;
        live = Ef >= 100;
      } else {
        long long h[3];
        hg_fix(X, c_khx[p][0], c_khx[p][1], c_khx[p][2], h);
        const int sh = renorm_fix(h);
        expand_q3_fix(h, xx);
        sc = Eg - 1080 - sh - dp;
        live = Eg >= 100;
      }
#pragma unroll
      for (int q = 0; q < 5; ++q) tk[q] = live ? (A)ll_to_double_rn(xx[q], sc - kd(q)) : (A)0;
    } else {
#pragma unroll
      for (int q = 0; q < 5; ++q) tk[q] = k == 0 ? tf[q] : tg[q];
    }
    // stencil of population q: centre c, x cells (v > 0: j-2, j-1, j+1; v < 0: j-1, j+1, j+2), y likewise
    double cv = 0, xa = 0, xb = 0, xc = 0, ya = 0, yb = 0, yc = 0;
    auto load_stencil = [&](int qq, double& c0, double& x0, double& x1, double& x3, double& y0, double& y1,
                            double& y3) {
      const double* pq = (const double*)(s + pbase + (long long)(qq + 25 * k) * PL);
      c0 = __ldg(pq);
      if (xmove) {
        const long long o = sx > 0 ? -2 : -1;
        x0 = __ldg(pq + o);
        x1 = __ldg(pq + o + (sx > 0 ? 1 : 2));
        x3 = __ldg(pq + o + 3);
      }
      const int sq = sgn_of(qq);
      if (sq != 0) {
        const long long o = sq > 0 ? -2 * PT : -PT;
        y0 = __ldg(pq + o);
        y1 = __ldg(pq + o + (sq > 0 ? PT : 2 * PT));
        y3 = __ldg(pq + o + 3 * PT);
      }
    };
    if constexpr (PREF) load_stencil(0, cv, xa, xb, xc, ya, yb, yc);
#pragma unroll (ROLLQ ? 1 : 5)
    for (int q = 0; q < 5; ++q) {
      const long long co = pbase + (long long)(q + 25 * k) * PL;
      const A t = ROLLQ ? (q == 0 ? tk[0] : q == 1 ? tk[1] : q == 2 ? tk[2] : q == 3 ? tk[3] : tk[4]) : tk[q];
      if constexpr (PREF) {
        double nc = 0, nx0 = 0, nx1 = 0, nx3 = 0, ny0 = 0, ny1 = 0, ny3 = 0;
        if (q < 4) load_stencil(q + 1, nc, nx0, nx1, nx3, ny0, ny1, ny3);
        // flux difference of the stencil (a0..a3 = cells j-2..j+1 for v > 0,
        // j-1..j+2 for v < 0) in the limiter form of this instantiation
        auto fdiff = [&](double a0, double a1, double a2, double a3, int sg, int& code) -> double {
          if constexpr (CODES) return flux_difference_rat_code_v(a0, a1, a2, a3, P.lp, P.lq, sg, code);
          else if constexpr (RAT) return flux_difference_rat_v(a0, a1, a2, a3, P.lp, P.lq, sg);
          else return flux_difference_int_v(a0, a1, a2, a3, P.hq, sg);
        };
        int cx = 0, cy = 0;
        double v = fma(C.a1, cv, (double)t);
        if (xmove) {
          const double fx2 = sx > 0 ? fdiff(xa, xb, cv, xc, 1, cx) : fdiff(xa, cv, xb, xc, -1, cx);
          v = fma(-kx, fx2, v);
        }
        const int sq = sgn_of(q);
        if (sq != 0) {
          const double fy2 = sq > 0 ? fdiff(ya, yb, cv, yc, 1, cy) : fdiff(ya, cv, yb, yc, -1, cy);
          v = fma(RAT ? -P.kyr[q] : -P.kyv[q], fy2, v);
        }
        if constexpr (CODES) cd[(long long)(5 * p + q + 25 * k) * cplane] = (unsigned char)(cx | (cy << 2));
        d[co] = (S)v;
        cv = nc; xa = nx0; xb = nx1; xc = nx3; ya = ny0; yb = ny1; yc = ny3;
      } else {
        // FP32-deviation storage: float flux differences on the deviations
        const S* pc = s + co;
        A fx = 0, fy = 0;
        if (!CENTER) fx = sx > 0 ? flux_difference<1, S>(pc, 1, (S)hb) : flux_difference<-1, S>(pc, 1, (S)hb);
        if (sgn_of(q) > 0) fy = flux_difference<1, S>(pc, PT, (S)hb);
        if (sgn_of(q) < 0) fy = flux_difference<-1, S>(pc, PT, (S)hb);
        float adv = 0.f;
        if (!CENTER) adv = kxf * (float)fx;
        if (sgn_of(q) != 0) adv = fmaf(P.kyvf[q], (float)fy, adv);
        d[co] = (S)(fmaf(a1f, (float)__ldg(pc), t) - adv);
      }
    }
  }
}

template <class S, int PRC, bool RAT, bool CODES = false>
__global__ void __launch_bounds__(kCta, 1024 / kCta) k_step(const S* __restrict__ src, S* __restrict__ dst, Geom G, Phys P,
                                              unsigned int* __restrict__ flag,
                                              unsigned char* __restrict__ codes = nullptr,
                                              double* __restrict__ moms = nullptr) {
  const int x = blockIdx.x * 32 + threadIdx.x;
  const int y = blockIdx.y * kTileY + threadIdx.y;
  if (x >= G.Nx || y >= G.Ny) return;
  const long long off = cell_index(G, y, x);
  const S* s = src + off;
  S* d = dst + off;
  const long long PL = G.plane;
  const long long PT = G.pitch;

  // ---- phase A: moments -> collision coefficients ----
  Moments m = {};
  {
    double f[5], g[5];
    load_node<S, 0>(s, PL, P, f, g); accumulate_moments<0>(m, f, g);
    load_node<S, 1>(s, PL, P, f, g); accumulate_moments<1>(m, f, g);
    load_node<S, 2>(s, PL, P, f, g); accumulate_moments<2>(m, f, g);
    load_node<S, 3>(s, PL, P, f, g); accumulate_moments<3>(m, f, g);
    load_node<S, 4>(s, PL, P, f, g); accumulate_moments<4>(m, f, g);
  }
  if constexpr (sizeof(S) == 4) {
    // moments of the reference populations w rho0 (f) and w G0 (g):
    // sum w = 1, sum w xi^2 = 1 per axis, odd moments vanish
    m.m00 += P.fref0; m.m20 += P.fref0; m.m02 += P.fref0;
    m.g00 += P.gref0;
  }
  if constexpr (CODES) {
    // the recomputing adjoint also keeps the cell's moments (13 planes of
    // Nx * Ny doubles, Moments field order) for its collision part
    if (moms) {
      const long long cp = (long long)G.Nx * G.Ny, ci = (long long)y * G.Nx + x;
      const double v[13] = {m.m00, m.m10, m.m01, m.m20, m.m11, m.m02, m.m30,
                            m.m21, m.m12, m.m03, m.g00, m.g10, m.g01};
#pragma unroll
      for (int k = 0; k < 13; ++k) moms[k * cp + ci] = v[k];
    }
  }
  Coeffs C = collision_coeffs<PRC>(m, P);
  if (C.bad) atomicOr(flag, 1u);
  if constexpr (sizeof(S) == 4) {
    // the expansion then yields t - (dt/tau1) F_ref directly: the reference
    // populations w rho0 and w G0 have only a zeroth Hermite coefficient
    C.f00 -= C.k1 * P.fref0;
    C.g00 -= C.k1 * P.gref0;
  }
  // FP32DEV: new deviation = a1 * dev + (t - k1 * ref) - advection, with the
  // bracket (equilibrium evaluation minus the relaxed reference) at
  // FP64-or-better precision, rounded to float only in the update
  const float a1f = (float)C.a1;
  __shared__ long long s_fix[kFixFields * kCta];
  const int tid = threadIdx.y * 32 + threadIdx.x;
  int Ef, Eg;
  {
    const CoeffsFix Xr = coeffs_to_fix(C);
    fix_to_smem(Xr, s_fix + tid);
    Ef = Xr.Ef;
    Eg = Xr.Eg;
  }
  const FixView X{s_fix + tid};

  // ---- phase B: populations, x-node by x-node ----
  const long long cplane = (long long)G.Nx * G.Ny;
  unsigned char* cd = CODES ? codes + (long long)y * G.Nx + x : nullptr;
  if constexpr (sizeof(S) == 8) {
    // one loop body for all five x-nodes (the centre node skips its x-flux)
#pragma unroll 1
    for (int p = 0; p < 5; ++p) node_update<S, RAT, false, CODES>(p, s, d, PL, PT, C, X, Ef, Eg, P, a1f, cd, cplane);
  } else {
    node_update<S, RAT, true, CODES>(0, s, d, PL, PT, C, X, Ef, Eg, P, a1f, cd, cplane);
#pragma unroll 1
    for (int p = 1; p < 5; ++p) node_update<S, RAT, false, CODES>(p, s, d, PL, PT, C, X, Ef, Eg, P, a1f, cd, cplane);
  }
}

template <class S>
static cudaError_t launch_step_t(const void* src, void* dst, const Geom& G, const Phys& P, unsigned int* flag,
                                 cudaStream_t st) {
  dim3 block(32, kTileY);
  dim3 grid((G.Nx + 31) / 32, (G.Ny + kTileY - 1) / kTileY);
  const S* s = (const S*)src;
  S* d = (S*)dst;
  // the rational limiter form matters only for FP64 storage
  const bool rat = sizeof(S) == 8 && P.lq > 0;
  if (P.prc < 0) {
    if (rat) k_step<S, -1, true><<<grid, block, 0, st>>>(s, d, G, P, flag);
    else k_step<S, -1, false><<<grid, block, 0, st>>>(s, d, G, P, flag);
  } else if (P.prc > 0) {
    if (rat) k_step<S, 1, true><<<grid, block, 0, st>>>(s, d, G, P, flag);
    else k_step<S, 1, false><<<grid, block, 0, st>>>(s, d, G, P, flag);
  } else {
    if (rat) k_step<S, 0, true><<<grid, block, 0, st>>>(s, d, G, P, flag);
    else k_step<S, 0, false><<<grid, block, 0, st>>>(s, d, G, P, flag);
  }
  return cudaGetLastError();
}

cudaError_t launch_step_codes(const void* src, void* dst, const Geom& G, const Phys& P, unsigned int* flag,
                              unsigned char* codes, double* moms, cudaStream_t st) {
  if (!(P.lq > 0) || !codes) return cudaErrorInvalidValue;
  dim3 block(32, kTileY);
  dim3 grid((G.Nx + 31) / 32, (G.Ny + kTileY - 1) / kTileY);
  const double* s = (const double*)src;
  double* d = (double*)dst;
  if (P.prc < 0) k_step<double, -1, true, true><<<grid, block, 0, st>>>(s, d, G, P, flag, codes, moms);
  else if (P.prc > 0) k_step<double, 1, true, true><<<grid, block, 0, st>>>(s, d, G, P, flag, codes, moms);
  else k_step<double, 0, true, true><<<grid, block, 0, st>>>(s, d, G, P, flag, codes, moms);
  return cudaGetLastError();
}

cudaError_t launch_step(int storage, const void* src, void* dst, const Geom& G, const Phys& P, unsigned int* flag,
                        cudaStream_t st) {
  return storage == 0 ? launch_step_t<double>(src, dst, G, P, flag, st)
                      : launch_step_t<float>(src, dst, G, P, flag, st);
}

}  // namespace dvbm
