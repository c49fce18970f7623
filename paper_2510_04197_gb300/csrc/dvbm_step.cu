// dvbm_step.cu -- the fused per-cell time step (Sec. III.A.1, Eq. finalDiscretePDE).
//
// One thread per cell, 32 x 8 cells per CTA.  Phase A reads the cell's 50
// populations and accumulates the sum-factorised moments; the thread then
// forms the combined collision coefficients (dvbm_device.cuh).  Phase B walks
// the populations x-node by x-node: for each it evaluates the collision target
// (sum-factorised Grad expansion), the upwind-limited flux differences along x
// and y from the L1-cached neighbours, and writes the new value:
//     F_new = (1 - dt/tau1) F + W W sum C He He - (dt/dx) v_x dF_x - (dt/dy) v_y dF_y.
// The storage variant FP32DEV keeps float deviations from a reference state;
// moments, temperature and the equilibrium evaluation stay in double, the
// advection runs in float on the deviations.
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
      f[q] = (double)__ldg(src + c * plane);
      g[q] = (double)__ldg(src + (25 + c) * plane);
    }
  }
}

template <class S, int PRC, bool RAT>
__global__ void __launch_bounds__(256) k_step(const S* __restrict__ src, S* __restrict__ dst, Geom G, Phys P,
                                              unsigned int* __restrict__ flag) {
  const int x = blockIdx.x * 32 + threadIdx.x;
  const int y = blockIdx.y * 8 + threadIdx.y;
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
  Coeffs C = collision_coeffs<PRC>(m, P);
  if (C.bad) atomicOr(flag, 1u);
  if constexpr (sizeof(S) == 4) {
    // the expansion then yields t - (dt/tau1) F_ref directly: the reference
    // populations w rho0 and w G0 have only a zeroth Hermite coefficient
    C.f00 -= C.k1 * P.fref0;
    C.g00 -= C.k1 * P.gref0;
  }

  typedef typename StoreT<S>::adv_t A;
  const A hb = (A)P.hb;
  // FP32DEV: new deviation = a1 * dev + (t - k1 * ref) - advection, with the
  // bracket (equilibrium evaluation minus the relaxed reference) in double
  const float a1f = (float)C.a1;
  constexpr bool rational = RAT;

  // ---- phase B: populations, x-node by x-node ----
#define DVBM_NODE(p)                                                                       \
  {                                                                                         \
    double hf[5], tf[5], hg[3], tg[5];                                                      \
    hf_of<p>(C, hf); expand_q5(hf, tf);                                                     \
    hg_of<p>(C, hg); expand_q3(hg, tg);                                                     \
    _Pragma("unroll") for (int q = 0; q < 5; ++q) {                                         \
      _Pragma("unroll") for (int k = 0; k < 2; ++k) {                                       \
        const int c = 5 * p + q + 25 * k;                                                   \
        const S* pc = s + c * PL;                                                           \
        const double t = k == 0 ? tf[q] : tg[q];                                            \
        A fx = 0, fy = 0;                                                                   \
        if constexpr (sizeof(S) == 8) {                                                     \
          if constexpr (rational) {                                                         \
            if (sgn_of(p) != 0) fx = flux_difference_rat((const double*)pc, 1, P.lp, P.lq, sgn_of(p));   \
            if (sgn_of(q) != 0) fy = flux_difference_rat((const double*)pc, PT, P.lp, P.lq, sgn_of(q));  \
          } else {                                                                          \
            if (sgn_of(p) != 0) fx = flux_difference_int((const double*)pc, 1, P.hq, sgn_of(p)); \
            if (sgn_of(q) != 0) fy = flux_difference_int((const double*)pc, PT, P.hq, sgn_of(q)); \
          }                                                                                 \
        } else {                                                                            \
          if (sgn_of(p) > 0) fx = flux_difference<1, S>(pc, 1, (S)hb);                      \
          if (sgn_of(p) < 0) fx = flux_difference<-1, S>(pc, 1, (S)hb);                     \
          if (sgn_of(q) > 0) fy = flux_difference<1, S>(pc, PT, (S)hb);                     \
          if (sgn_of(q) < 0) fy = flux_difference<-1, S>(pc, PT, (S)hb);                    \
        }                                                                                   \
        if constexpr (sizeof(S) == 8) {                                                     \
          double v = fma(C.a1, (double)__ldg(pc), t);                                       \
          if (sgn_of(p) != 0) v = fma(rational ? -P.kxr[p] : -P.kxv[p], (double)fx, v);    \
          if (sgn_of(q) != 0) v = fma(rational ? -P.kyr[q] : -P.kyv[q], (double)fy, v);    \
          d[c * PL] = (S)v;                                                                 \
        } else {                                                                            \
          const double base = t;                                                            \
          float adv = 0.f;                                                                  \
          if (sgn_of(p) != 0) adv = P.kxvf[p] * (float)fx;                                  \
          if (sgn_of(q) != 0) adv = fmaf(P.kyvf[q], (float)fy, adv);                        \
          d[c * PL] = (S)(fmaf(a1f, (float)__ldg(pc), __double2float_rn(base)) - adv);     \
        }                                                                                   \
      }                                                                                     \
    }                                                                                       \
  }
  DVBM_NODE(0)
  DVBM_NODE(1)
  DVBM_NODE(2)
  DVBM_NODE(3)
  DVBM_NODE(4)
#undef DVBM_NODE
}

template <class S>
static cudaError_t launch_step_t(const void* src, void* dst, const Geom& G, const Phys& P, unsigned int* flag,
                                 cudaStream_t st) {
  dim3 block(32, 8);
  dim3 grid((G.Nx + 31) / 32, (G.Ny + 7) / 8);
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

cudaError_t launch_step(int storage, const void* src, void* dst, const Geom& G, const Phys& P, unsigned int* flag,
                        cudaStream_t st) {
  return storage == 0 ? launch_step_t<double>(src, dst, G, P, flag, st)
                      : launch_step_t<float>(src, dst, G, P, flag, st);
}

}  // namespace dvbm
