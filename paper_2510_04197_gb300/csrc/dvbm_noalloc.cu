// dvbm_noalloc.cu -- time-step size from device fields without any allocation.
//
// dvbm_cfl_dt_noalloc() computes the same CFL time step as dvbm_init,
//   dt = cfl * h / max(|u| + sqrt(gamma R T)),
// for callers that cannot allocate device memory: code inside a framework
// that owns a fixed device memory budget (a caching allocator that has
// reserved the device's memory, where a cudaMalloc of our own would fail or
// evict), and latency-critical loops where cudaMalloc / cudaFree would
// synchronise the device.  It creates no context and allocates no device
// memory; the caller passes the four field arrays and receives dt on the
// host.  The call waits for its stream (under a host-side time limit of
// kWaitLimitSeconds, the library's default limit) before it returns.
//
// Its per-block partial maxima live in a file-scope device array of fixed
// size (4096 blocks of 256 threads x 64 cells, 64 KiB), which every GPU that loads the
// library holds until the process exits.  Because every call shares that
// array, calls that overlap on the GPU (different streams or threads) race
// and must be serialised by the caller.  Each call writes every slot it reads
// before reading it, so the contents left by an earlier call never leak into
// a result.  The first call on a device looks up the array's device address
// (cudaGetSymbolAddress) once for that device.
#include <chrono>
#include <cmath>
#include <mutex>
#include <thread>
#include <vector>

#include "../../include/dvbm.h"
#include "dvbm_internal.h"

namespace {

constexpr int kThreads = 256;
constexpr int kCellsPerThread = 64;
constexpr int kMaxBlocks = 4096;
constexpr double kWaitLimitSeconds = 600.0;
constexpr long long kMaxCells = (long long)kMaxBlocks * kThreads * kCellsPerThread;
static_assert(kMaxCells == DVBM_NOALLOC_MAX_CELLS, "scratch size and the published maximum must agree");

// scratch: slot 2b = block b's maximum of |u| + c_s, slot 2b + 1 = its count of invalid cells
static __device__ __align__(256) double g_cfl_scratch[2 * kMaxBlocks];

// device address of g_cfl_scratch per device (set up once per device)
constexpr int kMaxDevices = 64;
double* g_scratch_addr[kMaxDevices] = {nullptr};
std::mutex g_setup_mutex;

__global__ void __launch_bounds__(kThreads) k_speed_static(const double* __restrict__ rho,
                                                          const double* __restrict__ ux,
                                                          const double* __restrict__ uy,
                                                          const double* __restrict__ T, long long n,
                                                          double gamma_R, double* __restrict__ partial) {
  double mx = 0.0, bad = 0.0;
  const long long first = (long long)blockIdx.x * kThreads * kCellsPerThread + threadIdx.x;
  for (int k = 0; k < kCellsPerThread; ++k) {
    const long long i = first + (long long)k * kThreads;
    if (i >= n) break;
    const double r = rho[i], a = ux[i], b = uy[i], t = T[i];
    if (!(r > 0.0) || !(t > 0.0) || !(fabs(a) < 1e300) || !(fabs(b) < 1e300) || !(r < 1e300) || !(t < 1e300)) {
      bad += 1.0;
      continue;
    }
    mx = fmax(mx, sqrt(a * a + b * b) + sqrt(gamma_R * t));
  }
  __shared__ double sm[kThreads], sb[kThreads];
  sm[threadIdx.x] = mx;
  sb[threadIdx.x] = bad;
  __syncthreads();
  for (int w = kThreads / 2; w > 0; w >>= 1) {
    if ((int)threadIdx.x < w) {
      sm[threadIdx.x] = fmax(sm[threadIdx.x], sm[threadIdx.x + w]);
      sb[threadIdx.x] += sb[threadIdx.x + w];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    partial[2 * blockIdx.x] = sm[0];
    partial[2 * blockIdx.x + 1] = sb[0];
  }
}

// Resolve the device address of the scratch array for the current device.
// The array's name is only a host-side stand-in in host code; the kernel
// must be given the address returned by cudaGetSymbolAddress.
cudaError_t scratch_for_current_device(double** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_setup_mutex);
  if (!g_scratch_addr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_cfl_scratch);
    if (e != cudaSuccess) return e;
    g_scratch_addr[dev] = (double*)p;
  }
  *out = g_scratch_addr[dev];
  return cudaSuccess;
}

// Poll the stream until it has run everything queued on it, for at most
// kWaitLimitSeconds: DVBM_OK, DVBM_ETIMEOUT (the work stays queued), or
// DVBM_ECUDA for an error the stream reported.
dvbm_status wait_idle(cudaStream_t st) {
  const auto t0 = std::chrono::steady_clock::now();
  for (int spins = 0;; ++spins) {
    const cudaError_t e = cudaStreamQuery(st);
    if (e == cudaSuccess) return DVBM_OK;
    if (e != cudaErrorNotReady) return DVBM_ECUDA;
    if (std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count() > kWaitLimitSeconds)
      return DVBM_ETIMEOUT;
    if (spins > 64) std::this_thread::sleep_for(std::chrono::microseconds(50));
  }
}

}  // namespace

extern "C" dvbm_status dvbm_cfl_dt_noalloc(const double* rho, const double* ux, const double* uy, const double* T,
                                           long long n, double gamma, double R, double cfl, double h, void* stream,
                                           double* dt_out) {
  if (!rho || !ux || !uy || !T || !dt_out) return DVBM_EINVAL;
  if (n <= 0 || n > kMaxCells) return DVBM_EINVAL;
  if (!(gamma > 1.0) || !(R > 0) || !(cfl > 0) || !(h > 0)) return DVBM_EINVAL;
  double* scratch = nullptr;
  if (scratch_for_current_device(&scratch) != cudaSuccess) return DVBM_ECUDA;
  const int blocks = (int)((n + (long long)kThreads * kCellsPerThread - 1) / ((long long)kThreads * kCellsPerThread));
  cudaStream_t st = (cudaStream_t)stream;
  k_speed_static<<<blocks, kThreads, 0, st>>>(rho, ux, uy, T, n, gamma * R, scratch);
  if (cudaGetLastError() != cudaSuccess) return DVBM_ECUDA;
  // the partial maxima are read only once the stream has run the kernel: wait
  // for it under the time limit (a copy into pageable host memory would block
  // the calling thread for as long as the stream takes)
  if (wait_idle(st) != DVBM_OK) return DVBM_ETIMEOUT;
  std::vector<double> host(2 * (size_t)blocks);  // host memory only
  if (cudaMemcpyAsync(host.data(), scratch, sizeof(double) * 2 * blocks, cudaMemcpyDeviceToHost, st) != cudaSuccess)
    return DVBM_ECUDA;
  const dvbm_status w = wait_idle(st);
  if (w != DVBM_OK) return w;
  double vmax = 0.0, bad = 0.0;
  for (int b = 0; b < blocks; ++b) {
    vmax = std::fmax(vmax, host[2 * b]);
    bad += host[2 * b + 1];
  }
  if (bad > 0 || !(vmax > 0)) return DVBM_EINVAL;
  *dt_out = cfl * h / vmax;
  return DVBM_OK;
}
