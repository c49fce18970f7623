// dvbm_internal.h -- launch wrappers shared by the translation units of libdvbm.
#pragma once
#include <cuda_runtime.h>
#include "dvbm_device.cuh"

namespace dvbm {

struct BCDev {
  int kind[4];          // xlo, xhi, ylo, yhi (0 periodic, 1 zero-gradient, 2 wall, 3 external: not filled here)
  double uw[4][2];      // wall velocity
  double Tw[4];         // wall temperature
};

struct Macro {          // constants needed to turn moments into physical fields
  double c, T_ref, R, gamma;
};

cudaError_t launch_step(int storage, const void* src, void* dst, const Geom& G, const Phys& P,
                        unsigned int* flag, cudaStream_t st);
// FP64 step with the rational limiter that also records the minmod branch
// codes of every population's x and y slopes: codes[pop][y][x] = x | y << 2
// moms (nullable): also store the 13 moments of each cell of the input state,
// moms[k][y][x] in Moments field order
cudaError_t launch_step_codes(const void* src, void* dst, const Geom& G, const Phys& P, unsigned int* flag,
                              unsigned char* codes, double* moms, cudaStream_t st);
// auxiliary kernels, written once for both models: lattice 0 = D2Q25 / split II
// (storage 0 FP64, 1 FP32-deviation), lattice 1 = D2Q16 / split I (FP64)
cudaError_t launch_init(int lattice, int storage, void* dst, const double* rho, const double* ux, const double* uy,
                        const double* T, const Geom& G, const Phys& P, const Macro& M, cudaStream_t st);
cudaError_t launch_ghost(int lattice, int storage, void* buf, const Geom& G, const Phys& P, const Macro& M,
                         const BCDev& bc, cudaStream_t st);
cudaError_t launch_moments(int lattice, int storage, const void* src, double* rho, double* ux, double* uy, double* T,
                           const Geom& G, const Phys& P, const Macro& M, cudaStream_t st);
// per-block partial sums: out[blk*6 + {mass, momx, momy, energy, bad, 0}]
cudaError_t launch_totals(int lattice, int storage, const void* src, double* partial, int nblocks, const Geom& G,
                          const Phys& P, const Macro& M, cudaStream_t st);
// per-block maxima of |u| + sqrt(gamma R T) and of p = rho R T, and a bad-input count:
// out[blk*3 + {max speed, bad, max p}]
cudaError_t launch_speed(const double* rho, const double* ux, const double* uy, const double* T, long long n,
                         double* partial, int nblocks, const Macro& M, cudaStream_t st);
// halo rows of a slab: unpack = 0: rows y = 0, 1 -> lo and y = Ny - 2, Ny - 1 -> hi;
// unpack = 1: lo -> ghost rows y = -2, -1 and hi -> y = Ny, Ny + 1; layout [npop][2][Nx]
// of elem-byte elements (8: double, 4: float); a NULL buffer skips its side
cudaError_t launch_halo(int elem, void* buf, void* lo, void* hi, int unpack, const Geom& G, int npop,
                        cudaStream_t st);
cudaError_t launch_pack(int storage, const void* buf, void* packed, int to_packed, const Geom& G, int npop,
                        cudaStream_t st);

// D2Q16, total-energy split (I), FP64 storage
cudaError_t launch_step16(const void* src, void* dst, const Geom& G, const Phys& P, unsigned int* flag,
                          cudaStream_t st);

// adjoint (FP64 storage, periodic)
int adjoint_blocks(const Geom& G);
// codes: the branch codes recorded by launch_step_codes for this step, or
// nullptr (the advection adjoint then derives the branches from X)
// glo, ghi: the neighbouring bands' code rows next to a band's edges ([NPOP][Nx]
// each, coded path only), or nullptr: the codes wrap periodically in y
cudaError_t launch_adjoint_step(const double* X, const double* Lin, double* Lout, double* partial,
                                const unsigned char* codes, const double* moms, const Geom& G, const Phys& P,
                                cudaStream_t st, const unsigned char* glo = nullptr,
                                const unsigned char* ghi = nullptr);
// branch-code rows of a band's edges: unpack = 0: rows y = 0 -> lo, y = Ny - 1 -> hi of
// every population's codes; unpack = 1: lo -> glo, hi -> ghi; [NPOP][Nx] bytes, NULL skips
cudaError_t launch_code_rows(unsigned char* codes, void* lo, void* hi, unsigned char* glo, unsigned char* ghi,
                             int unpack, const Geom& G, cudaStream_t st);
cudaError_t launch_adjoint_final(const double* X, const double* rhob, const double* Tb, double* Lout, double* partial,
                                 const Geom& G, const Phys& P, const Macro& M, cudaStream_t st);
cudaError_t launch_adjoint_init(const double* L, const double* rho, const double* ux, const double* uy,
                                const double* T, double* grho, double* gux, double* guy, double* gT, double* partial,
                                const Geom& G, const Phys& P, const Macro& M, cudaStream_t st);

}  // namespace dvbm
