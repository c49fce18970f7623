// dvbm_aux.cu -- initial conditions, ghost layers, diagnostics.
//
//  k_init     equilibrium populations of given (rho, u, T) fields (Sec. III.A.3),
//             by the step kernel's block-fixed-point Grad expansion
//  k_ghost    two ghost layers per non-... side: periodic wrap, zero-gradient copy,
//             or no-slip isothermal wall by ghost node + non-equilibrium
//             extrapolation (Sec. III.E): rho_G = rho_B, u_G = 2 u_W - u_B,
//             T_G = 2 T_W - T_B, F_G = F^eq(G) + (F_B - F^eq(B)); ghost k
//             mirrors interior cell k (k = 1, 2)
//  k_moments  rho, u, T fields
//  k_totals   per-block sums of mass, momentum, total energy (+ bad-cell count)
//  k_speed    per-block maxima of |u| + sqrt(gamma R T) (CFL rule) and of p = rho R T
//             (shortest relaxation time), and a bad-input count
//  k_pack     padded <-> packed [50][Ny][Nx] state copies
#include "dvbm_device.cuh"
#include "dvbm_cellmom.cuh"
#include "dvbm_internal.h"

namespace dvbm {

// write the expansion of coefficient set C (pure equilibrium: a1 = 0, k1 = 1)
// at one padded offset; addf/addg (nullable) add per-population values.
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

template <class S>
__global__ void k_init(S* __restrict__ dst, const double* __restrict__ rho, const double* __restrict__ ux,
                       const double* __restrict__ uy, const double* __restrict__ T, Geom G, Phys P, Macro M) {
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  const int y = blockIdx.y * blockDim.y + threadIdx.y;
  if (x >= G.Nx || y >= G.Ny) return;
  const long long i = (long long)y * G.Nx + x;
  const Coeffs C = equilibrium_coeffs(rho[i], ux[i] / M.c, uy[i] / M.c, T[i] / M.T_ref, P);
  write_equilibrium_fix<S>(dst + cell_index(G, y, x), G.plane, C, P);
}

// one thread per (side, layer k, position along the side, population);
// sides 0..3 = xlo, xhi, ylo, yhi, blockIdx.z = population.  Periodic and
// zero-gradient sides copy one population per thread; a wall side needs all
// populations of its mirror cell and is done by the blockIdx.z = 0 slice.
template <class S>
__global__ void k_ghost(S* __restrict__ buf, Geom G, Phys P, Macro M, BCDev bc) {
  const int side = blockIdx.y;
  const int kind = bc.kind[side];
  const int pop = blockIdx.z;
  if (kind == 3) return;  // external: the caller supplies these rows (dvbm_halo_unpack)
  if (kind == 2 && pop != 0) return;
  const int len = side < 2 ? G.Ny : G.Nx;
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= 2 * len) return;
  const int k = 1 + t / len;        // ghost layer 1 or 2
  const int j = t % len;            // position along the side
  int gx, gy, bx, by;               // ghost cell and source/mirror cell
  const bool lo = (side % 2) == 0;
  const int n = side < 2 ? G.Nx : G.Ny;
  int gi = lo ? -k : n - 1 + k;     // ghost coordinate along the normal
  int bi;
  if (kind == 0) bi = lo ? n - k : k - 1;            // periodic wrap
  else if (kind == 1) bi = lo ? 0 : n - 1;           // zero gradient
  else bi = lo ? k - 1 : n - k;                      // wall: mirror cell
  if (side < 2) { gx = gi; gy = j; bx = bi; by = j; }
  else          { gx = j; gy = gi; bx = j; by = bi; }
  const long long PL = G.plane;
  S* gptr = buf + cell_index(G, gy, gx);
  const S* bptr = buf + cell_index(G, by, bx);
  if (kind != 2) {
    gptr[pop * PL] = bptr[pop * PL];
    return;
  }
  // wall: equilibrium at the ghost state + non-equilibrium part of the mirror cell
  const Moments m = cell_moments<S>(bptr, PL, P);
  double rho, ux, uy, T;
  macro_from_moments(m, P, M.c, M.T_ref, rho, ux, uy, T);
  const Coeffs CB = equilibrium_coeffs(rho, ux / M.c, uy / M.c, T / M.T_ref, P);
  const double uxg = 2.0 * bc.uw[side][0] - ux, uyg = 2.0 * bc.uw[side][1] - uy, Tg = 2.0 * bc.Tw[side] - T;
  const Coeffs CG = equilibrium_coeffs(rho, uxg / M.c, uyg / M.c, Tg / M.T_ref, P);
  double neqf[25], neqg[25];
  {
    double hf[5], tf[5], hg[3], tg[5];
#define DVBM_NEQ(p)                                                                    \
    hf_of<p>(CB, hf); expand_q5(hf, tf); hg_of<p>(CB, hg); expand_q3(hg, tg);          \
    _Pragma("unroll") for (int q = 0; q < 5; ++q) {                                    \
      double w = 0.0;                                                                  \
      if constexpr (sizeof(S) == 4) w = w_of(p) * w_of(q);                             \
      neqf[5 * p + q] = ((double)bptr[(5 * p + q) * PL] + P.fref0 * w) - tf[q];        \
      neqg[5 * p + q] = ((double)bptr[(25 + 5 * p + q) * PL] + P.gref0 * w) - tg[q];   \
    }
    DVBM_NEQ(0) DVBM_NEQ(1) DVBM_NEQ(2) DVBM_NEQ(3) DVBM_NEQ(4)
#undef DVBM_NEQ
  }
  write_expansion<S>(gptr, PL, CG, P, neqf, neqg);
}

template <class S>
__global__ void k_moments(const S* __restrict__ src, double* rho, double* ux, double* uy, double* T, Geom G,
                          Phys P, Macro M) {
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  const int y = blockIdx.y * blockDim.y + threadIdx.y;
  if (x >= G.Nx || y >= G.Ny) return;
  const Moments m = cell_moments<S>(src + cell_index(G, y, x), G.plane, P);
  double r, a, b, t;
  macro_from_moments(m, P, M.c, M.T_ref, r, a, b, t);
  const long long i = (long long)y * G.Nx + x;
  if (rho) rho[i] = r;
  if (ux) ux[i] = a;
  if (uy) uy[i] = b;
  if (T) T[i] = t;
}

// block of 256 threads; grid-stride over cells; fixed-order block reduction
template <class S>
__global__ void __launch_bounds__(256) k_totals(const S* __restrict__ src, double* partial, Geom G, Phys P,
                                                Macro M) {
  double acc[5] = {0, 0, 0, 0, 0};
  const long long ncell = (long long)G.Nx * G.Ny;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < ncell;
       i += (long long)gridDim.x * blockDim.x) {
    const int y = (int)(i / G.Nx), x = (int)(i % G.Nx);
    const Moments m = cell_moments<S>(src + cell_index(G, y, x), G.plane, P);
    const double rho = m.m00;
    const double E = m.g00 + 0.5 * P.c2 * (m.m20 + m.m02);
    double r, a, b, t;
    macro_from_moments(m, P, M.c, M.T_ref, r, a, b, t);
    acc[0] += rho;
    acc[1] += m.m10 * M.c;
    acc[2] += m.m01 * M.c;
    acc[3] += E;
    if (!(r > 0.0) || !(t > 0.0) || !(fabs(E) < 1e300)) acc[4] += 1.0;
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

__global__ void __launch_bounds__(256) k_speed(const double* __restrict__ rho, const double* __restrict__ ux,
                                               const double* __restrict__ uy, const double* __restrict__ T,
                                               long long n, double* partial, Macro M) {
  double mx = 0.0, bad = 0.0, pm = 0.0;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const double r = rho[i], a = ux[i], b = uy[i], t = T[i];
    if (!(r > 0.0) || !(t > 0.0) || !(fabs(a) < 1e300) || !(fabs(b) < 1e300) || !(r < 1e300) || !(t < 1e300)) {
      bad += 1.0;
      continue;
    }
    mx = fmax(mx, sqrt(a * a + b * b) + sqrt(M.gamma * M.R * t));
    pm = fmax(pm, r * M.R * t);
  }
  __shared__ double sm[256], sb[256], sp[256];
  sm[threadIdx.x] = mx;
  sb[threadIdx.x] = bad;
  sp[threadIdx.x] = pm;
  __syncthreads();
  for (int w = 128; w > 0; w >>= 1) {
    if ((int)threadIdx.x < w) {
      sm[threadIdx.x] = fmax(sm[threadIdx.x], sm[threadIdx.x + w]);
      sb[threadIdx.x] += sb[threadIdx.x + w];
      sp[threadIdx.x] = fmax(sp[threadIdx.x], sp[threadIdx.x + w]);
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    partial[3 * blockIdx.x] = sm[0];
    partial[3 * blockIdx.x + 1] = sb[0];
    partial[3 * blockIdx.x + 2] = sp[0];
  }
}

template <class S>
__global__ void k_pack(S* buf, S* packed, int to_packed, Geom G) {
  // one plane per blockIdx.z
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  const int y = blockIdx.y;
  const int c = blockIdx.z;
  if (x >= G.Nx) return;
  const long long pi = ((long long)c * G.Ny + y) * G.Nx + x;
  const long long bi = c * G.plane + cell_index(G, y, x);
  if (to_packed) packed[pi] = buf[bi];
  else buf[bi] = packed[pi];
}

// halo rows of a slab (one thread per element): blockIdx.y = 2 side + row,
// blockIdx.z = population plane
template <class S>
__global__ void k_halo(S* buf, S* lo, S* hi, int unpack, Geom G) {
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  const int side = blockIdx.y >> 1, k = blockIdx.y & 1;
  const int c = blockIdx.z;
  S* ext = side == 0 ? lo : hi;
  if (x >= G.Nx || !ext) return;
  const int yb = unpack ? (side == 0 ? k - 2 : G.Ny + k) : (side == 0 ? k : G.Ny - 2 + k);
  const long long bi = (long long)c * G.plane + cell_index(G, yb, x);
  const long long ei = ((long long)c * 2 + k) * G.Nx + x;
  if (unpack) buf[bi] = ext[ei];
  else ext[ei] = buf[bi];
}

// ---------------------------------------------------------------- wrappers
cudaError_t launch_halo(int elem, void* buf, void* lo, void* hi, int unpack, const Geom& G, int npop,
                        cudaStream_t st) {
  dim3 b(128), g((G.Nx + 127) / 128, 4, npop);
  if (elem == 8) k_halo<double><<<g, b, 0, st>>>((double*)buf, (double*)lo, (double*)hi, unpack, G);
  else k_halo<float><<<g, b, 0, st>>>((float*)buf, (float*)lo, (float*)hi, unpack, G);
  return cudaGetLastError();
}

cudaError_t launch_init(int storage, void* dst, const double* rho, const double* ux, const double* uy,
                        const double* T, const Geom& G, const Phys& P, const Macro& M, cudaStream_t st) {
  dim3 b(32, 4), g((G.Nx + 31) / 32, (G.Ny + 3) / 4);
  if (storage == 0) k_init<double><<<g, b, 0, st>>>((double*)dst, rho, ux, uy, T, G, P, M);
  else k_init<float><<<g, b, 0, st>>>((float*)dst, rho, ux, uy, T, G, P, M);
  return cudaGetLastError();
}

cudaError_t launch_ghost(int storage, void* buf, const Geom& G, const Phys& P, const Macro& M, const BCDev& bc,
                         cudaStream_t st) {
  const int len = G.Nx > G.Ny ? G.Nx : G.Ny;
  dim3 b(128), g((2 * len + 127) / 128, 4, NPOP);
  if (storage == 0) k_ghost<double><<<g, b, 0, st>>>((double*)buf, G, P, M, bc);
  else k_ghost<float><<<g, b, 0, st>>>((float*)buf, G, P, M, bc);
  return cudaGetLastError();
}

cudaError_t launch_moments(int storage, const void* src, double* rho, double* ux, double* uy, double* T,
                           const Geom& G, const Phys& P, const Macro& M, cudaStream_t st) {
  dim3 b(32, 4), g((G.Nx + 31) / 32, (G.Ny + 3) / 4);
  if (storage == 0) k_moments<double><<<g, b, 0, st>>>((const double*)src, rho, ux, uy, T, G, P, M);
  else k_moments<float><<<g, b, 0, st>>>((const float*)src, rho, ux, uy, T, G, P, M);
  return cudaGetLastError();
}

cudaError_t launch_totals(int storage, const void* src, double* partial, int nblocks, const Geom& G, const Phys& P,
                          const Macro& M, cudaStream_t st) {
  if (storage == 0) k_totals<double><<<nblocks, 256, 0, st>>>((const double*)src, partial, G, P, M);
  else k_totals<float><<<nblocks, 256, 0, st>>>((const float*)src, partial, G, P, M);
  return cudaGetLastError();
}

cudaError_t launch_speed(const double* rho, const double* ux, const double* uy, const double* T, long long n,
                         double* partial, int nblocks, const Macro& M, cudaStream_t st) {
  k_speed<<<nblocks, 256, 0, st>>>(rho, ux, uy, T, n, partial, M);
  return cudaGetLastError();
}

cudaError_t launch_pack(int storage, const void* buf, void* packed, int to_packed, const Geom& G, int npop,
                        cudaStream_t st) {
  dim3 b(128), g((G.Nx + 127) / 128, G.Ny, npop);
  if (storage == 0) k_pack<double><<<g, b, 0, st>>>((double*)buf, (double*)packed, to_packed, G);
  else k_pack<float><<<g, b, 0, st>>>((float*)buf, (float*)packed, to_packed, G);
  return cudaGetLastError();
}

}  // namespace dvbm
