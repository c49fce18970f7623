// dvbm_lattice.cuh -- what the auxiliary kernels (initial conditions, ghost
// layers, field and total diagnostics) need from a lattice / energy split, so
// that dvbm_aux.cu writes each of those kernels once for both models:
//   L25: D2Q25, internal non-translational energy split (II), FP64 or
//        FP32-deviation storage;
//   L16: D2Q16, total-energy split (I), FP64 storage.
#pragma once
#include "dvbm_cellmom.cuh"
#include "dvbm_internal.h"
#include "dvbm_q16.cuh"

namespace dvbm {

// macroscopic state of one cell: rho, momentum density jx, jy and total energy
// density E (physical units, per unit volume), velocity u and temperature T
struct CellState {
  double rho, jx, jy, E, ux, uy, T;
};

// write the expansion of coefficient set C (pure equilibrium: a1 = 0, k1 = 1)
// at one padded offset in double arithmetic; addf/addg (nullable) add
// per-population values (the wall closure's non-equilibrium parts)
template <class S>
__device__ __forceinline__ void write_expansion(S* d, long long PL, const Coeffs& C, const Phys& P,
                                                const double* addf, const double* addg) {
#define DVBM_EXP(p)                                                              \
  {                                                                              \
    double hf[5], tf[5], hg[3], tg[5];                                           \
    hf_of<p>(C, hf); expand_q5(hf, tf);                                          \
    hg_of<p>(C, hg); expand_q3(hg, tg);                                          \
    _Pragma("unroll") for (int q = 0; q < 5; ++q) {                              \
      double vf = tf[q], vg = tg[q];                                             \
      if (addf) { vf += addf[5 * p + q]; vg += addg[5 * p + q]; }                \
      if constexpr (sizeof(S) == 8) {                                            \
        d[(5 * p + q) * PL] = vf;                                                \
        d[(25 + 5 * p + q) * PL] = vg;                                           \
      } else {                                                                   \
        const double w = w_of(p) * w_of(q);                                      \
        d[(5 * p + q) * PL] = __double2float_rn(vf - P.fref0 * w);               \
        d[(25 + 5 * p + q) * PL] = __double2float_rn(vg - P.gref0 * w);          \
      }                                                                          \
    }                                                                            \
  }
  DVBM_EXP(0) DVBM_EXP(1) DVBM_EXP(2) DVBM_EXP(3) DVBM_EXP(4)
#undef DVBM_EXP
}

struct L25 {
  static constexpr int NPOP = 50;
  template <class S>
  __device__ static CellState state(const S* p, long long PL, const Phys& P, const Macro& M) {
    const Moments m = cell_moments<S>(p, PL, P);
    CellState c;
    macro_from_moments(m, P, M.c, M.T_ref, c.rho, c.ux, c.uy, c.T);
    c.jx = m.m10 * M.c;
    c.jy = m.m01 * M.c;
    c.E = m.g00 + 0.5 * P.c2 * (m.m20 + m.m02);  // split II: E = sum g + sum v^2/2 f
    return c;
  }
  // equilibrium populations of (rho, u, T) (Sec. III.A.3 initial conditions)
  template <class S>
  __device__ static void write_equilibrium(S* d, long long PL, double rho, double ux, double uy, double T,
                                           const Phys& P, const Macro& M) {
    write_equilibrium_fix<S>(d, PL, equilibrium_coeffs(rho, ux / M.c, uy / M.c, T / M.T_ref, P), P);
  }
  // wall ghost g mirroring interior cell b (Sec. III.E): equilibrium at
  // rho_B, 2 u_W - u_B, 2 T_W - T_B plus the non-equilibrium part of b
  template <class S>
  __device__ static void wall_ghost(S* g, const S* b, long long PL, const Phys& P, const Macro& M, double uwx,
                                    double uwy, double Tw) {
    const Moments m = cell_moments<S>(b, PL, P);
    double rho, ux, uy, T;
    macro_from_moments(m, P, M.c, M.T_ref, rho, ux, uy, T);
    const Coeffs CB = equilibrium_coeffs(rho, ux / M.c, uy / M.c, T / M.T_ref, P);
    const Coeffs CG = equilibrium_coeffs(rho, (2.0 * uwx - ux) / M.c, (2.0 * uwy - uy) / M.c,
                                         (2.0 * Tw - T) / M.T_ref, P);
    double neqf[25], neqg[25];
    {
      double hf[5], tf[5], hg[3], tg[5];
#define DVBM_NEQ(p)                                                                   \
      hf_of<p>(CB, hf); expand_q5(hf, tf); hg_of<p>(CB, hg); expand_q3(hg, tg);       \
      _Pragma("unroll") for (int q = 0; q < 5; ++q) {                                 \
        double w = 0.0;                                                               \
        if constexpr (sizeof(S) == 4) w = w_of(p) * w_of(q);                          \
        neqf[5 * p + q] = ((double)b[(5 * p + q) * PL] + P.fref0 * w) - tf[q];        \
        neqg[5 * p + q] = ((double)b[(25 + 5 * p + q) * PL] + P.gref0 * w) - tg[q];   \
      }
      DVBM_NEQ(0) DVBM_NEQ(1) DVBM_NEQ(2) DVBM_NEQ(3) DVBM_NEQ(4)
#undef DVBM_NEQ
    }
    write_expansion<S>(g, PL, CG, P, neqf, neqg);
  }
};

struct L16 {
  static constexpr int NPOP = 32;
  template <class S>
  __device__ static CellState state(const S* p, long long PL, const Phys& P, const Macro& M) {
    static_assert(sizeof(S) == 8, "the D2Q16 / split I model has FP64 storage only");
    const q16::Mom m = q16::cell_moments(p, PL);
    CellState c;
    q16::macro(m, P, M.c, M.T_ref, c.rho, c.ux, c.uy, c.T);
    c.jx = m.m10 * M.c;
    c.jy = m.m01 * M.c;
    c.E = m.g00;  // split I: E = sum g
    return c;
  }
  template <class S>
  __device__ static void write_equilibrium(S* d, long long PL, double rho, double ux, double uy, double T,
                                           const Phys& P, const Macro& M) {
    q16::write_equilibrium_fix16(d, PL, q16::equilibrium(rho, ux / M.c, uy / M.c, T / M.T_ref, P));
  }
  template <class S>
  __device__ static void wall_ghost(S* g, const S* b, long long PL, const Phys& P, const Macro& M, double uwx,
                                    double uwy, double Tw) {
    const q16::Mom m = q16::cell_moments(b, PL);
    double rho, ux, uy, T;
    q16::macro(m, P, M.c, M.T_ref, rho, ux, uy, T);
    const q16::Co CB = q16::equilibrium(rho, ux / M.c, uy / M.c, T / M.T_ref, P);
    const q16::Co CG = q16::equilibrium(rho, (2.0 * uwx - ux) / M.c, (2.0 * uwy - uy) / M.c,
                                        (2.0 * Tw - T) / M.T_ref, P);
    double neqf[16], neqg[16];
#define Q16_NEQ(p)                                                                     \
    {                                                                                  \
      double h[4], tf[4], hh[4], tg[4];                                                \
      q16::hf<p>(CB, h); q16::expand(h, tf); q16::hg<p>(CB, hh); q16::expand(hh, tg);  \
      _Pragma("unroll") for (int q = 0; q < 4; ++q) {                                  \
        neqf[4 * p + q] = b[(4 * p + q) * PL] - tf[q];                                 \
        neqg[4 * p + q] = b[(16 + 4 * p + q) * PL] - tg[q];                            \
      }                                                                                \
    }
    Q16_NEQ(0) Q16_NEQ(1) Q16_NEQ(2) Q16_NEQ(3)
#undef Q16_NEQ
    q16::write_expansion(g, PL, CG, neqf, neqg);
  }
};

}  // namespace dvbm
