// dvbm_aux.cu -- initial conditions, ghost layers, diagnostics.
//
// Each kernel below is written once for both models: templated on the
// lattice traits L25 / L16 of dvbm_lattice.cuh and on the storage type.
//
//  k_init     equilibrium populations of given (rho, u, T) fields (Sec. III.A.3),
//             by the step kernels' block-fixed-point Grad expansion
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
#include "dvbm_lattice.cuh"

namespace dvbm {

template <class L, class S>
__global__ void k_init(S* __restrict__ dst, const double* __restrict__ rho, const double* __restrict__ ux,
                       const double* __restrict__ uy, const double* __restrict__ T, Geom G, Phys P, Macro M) {
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  const int y = blockIdx.y * blockDim.y + threadIdx.y;
  if (x >= G.Nx || y >= G.Ny) return;
  const long long i = (long long)y * G.Nx + x;
  L::template write_equilibrium<S>(dst + cell_index(G, y, x), G.plane, rho[i], ux[i], uy[i], T[i], P, M);
}

// one thread per (side, layer k, position along the side, population);
// sides 0..3 = xlo, xhi, ylo, yhi, blockIdx.z = population.  Periodic and
// zero-gradient sides copy one population per thread; a wall side needs all
// populations of its mirror cell and is done by the blockIdx.z = 0 slice.
template <class L, class S>
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
  L::template wall_ghost<S>(gptr, bptr, PL, P, M, bc.uw[side][0], bc.uw[side][1], bc.Tw[side]);
}

template <class L, class S>
__global__ void k_moments(const S* __restrict__ src, double* rho, double* ux, double* uy, double* T, Geom G,
                          Phys P, Macro M) {
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  const int y = blockIdx.y * blockDim.y + threadIdx.y;
  if (x >= G.Nx || y >= G.Ny) return;
  const CellState c = L::template state<S>(src + cell_index(G, y, x), G.plane, P, M);
  const long long i = (long long)y * G.Nx + x;
  if (rho) rho[i] = c.rho;
  if (ux) ux[i] = c.ux;
  if (uy) uy[i] = c.uy;
  if (T) T[i] = c.T;
}

// block of 256 threads; grid-stride over cells; fixed-order block reduction
template <class L, class S>
__global__ void __launch_bounds__(256) k_totals(const S* __restrict__ src, double* partial, Geom G, Phys P,
                                                Macro M) {
  double acc[5] = {0, 0, 0, 0, 0};
  const long long ncell = (long long)G.Nx * G.Ny;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < ncell;
       i += (long long)gridDim.x * blockDim.x) {
    const int y = (int)(i / G.Nx), x = (int)(i % G.Nx);
    const CellState c = L::template state<S>(src + cell_index(G, y, x), G.plane, P, M);
    acc[0] += c.rho;
    acc[1] += c.jx;
    acc[2] += c.jy;
    acc[3] += c.E;
    if (!(c.rho > 0.0) || !(c.T > 0.0) || !(fabs(c.E) < 1e300)) acc[4] += 1.0;
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

// lattice 0: D2Q25 (storage 0 FP64, 1 FP32-deviation); lattice 1: D2Q16 (FP64)
cudaError_t launch_init(int lattice, int storage, void* dst, const double* rho, const double* ux, const double* uy,
                        const double* T, const Geom& G, const Phys& P, const Macro& M, cudaStream_t st) {
  dim3 b(32, 4), g((G.Nx + 31) / 32, (G.Ny + 3) / 4);
  if (lattice == 1) k_init<L16, double><<<g, b, 0, st>>>((double*)dst, rho, ux, uy, T, G, P, M);
  else if (storage == 0) k_init<L25, double><<<g, b, 0, st>>>((double*)dst, rho, ux, uy, T, G, P, M);
  else k_init<L25, float><<<g, b, 0, st>>>((float*)dst, rho, ux, uy, T, G, P, M);
  return cudaGetLastError();
}

cudaError_t launch_ghost(int lattice, int storage, void* buf, const Geom& G, const Phys& P, const Macro& M,
                         const BCDev& bc, cudaStream_t st) {
  const int len = G.Nx > G.Ny ? G.Nx : G.Ny;
  dim3 b(128), g((2 * len + 127) / 128, 4, lattice == 1 ? L16::NPOP : L25::NPOP);
  if (lattice == 1) k_ghost<L16, double><<<g, b, 0, st>>>((double*)buf, G, P, M, bc);
  else if (storage == 0) k_ghost<L25, double><<<g, b, 0, st>>>((double*)buf, G, P, M, bc);
  else k_ghost<L25, float><<<g, b, 0, st>>>((float*)buf, G, P, M, bc);
  return cudaGetLastError();
}

cudaError_t launch_moments(int lattice, int storage, const void* src, double* rho, double* ux, double* uy, double* T,
                           const Geom& G, const Phys& P, const Macro& M, cudaStream_t st) {
  dim3 b(32, 4), g((G.Nx + 31) / 32, (G.Ny + 3) / 4);
  if (lattice == 1) k_moments<L16, double><<<g, b, 0, st>>>((const double*)src, rho, ux, uy, T, G, P, M);
  else if (storage == 0) k_moments<L25, double><<<g, b, 0, st>>>((const double*)src, rho, ux, uy, T, G, P, M);
  else k_moments<L25, float><<<g, b, 0, st>>>((const float*)src, rho, ux, uy, T, G, P, M);
  return cudaGetLastError();
}

cudaError_t launch_totals(int lattice, int storage, const void* src, double* partial, int nblocks, const Geom& G,
                          const Phys& P, const Macro& M, cudaStream_t st) {
  if (lattice == 1) k_totals<L16, double><<<nblocks, 256, 0, st>>>((const double*)src, partial, G, P, M);
  else if (storage == 0) k_totals<L25, double><<<nblocks, 256, 0, st>>>((const double*)src, partial, G, P, M);
  else k_totals<L25, float><<<nblocks, 256, 0, st>>>((const float*)src, partial, G, P, M);
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
