// dvbm_cellmom.cuh -- moments of the 50 populations of one cell (used by the
// auxiliary and adjoint kernels; the step kernel accumulates them inline).
#pragma once
#include "dvbm_device.cuh"

namespace dvbm {

template <class S>
__device__ __forceinline__ double ld_pop(const S* p) {
  return (double)__ldg(p);
}

// moments of the 50 populations at one padded offset
template <class S>
__device__ __forceinline__ Moments cell_moments(const S* s, long long PL, const Phys& P) {
  Moments m = {};
  double f[5], g[5];
#define DVBM_MOM(p)                                                   \
  _Pragma("unroll") for (int q = 0; q < 5; ++q) {                    \
    f[q] = ld_pop(s + (5 * p + q) * PL);                              \
    g[q] = ld_pop(s + (25 + 5 * p + q) * PL);                         \
  }                                                                   \
  accumulate_moments<p>(m, f, g);
  DVBM_MOM(0) DVBM_MOM(1) DVBM_MOM(2) DVBM_MOM(3) DVBM_MOM(4)
#undef DVBM_MOM
  if constexpr (sizeof(S) == 4) {
    m.m00 += P.fref0; m.m20 += P.fref0; m.m02 += P.fref0;
    m.g00 += P.gref0;
  }
  return m;
}

}  // namespace dvbm
