// dvbm_api.cu -- the C ABI declared in include/dvbm.h.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <string>
#include <thread>
#include <vector>

#include "../../include/dvbm.h"
#include "dvbm_internal.h"

using namespace dvbm;

struct dvbm_ctx {
  int Nx = 0, Ny = 0, storage = 0;
  int lattice = 0;
  int npop = 50;
  double Pr = 0, gamma = 0, mu = 0;
  dvbm_opts opts{};
  dvbm_bc bcs[4]{};
  cudaStream_t stream = nullptr;
  int device = 0;
  Geom G{};
  Phys P{};
  Macro M{};
  BCDev bc{};
  bool any_ghost_kernel = true;
  size_t elem = 8;
  void* buf[2] = {nullptr, nullptr};
  int cur = 0;
  unsigned int* flag = nullptr;
  double* partial = nullptr;
  int nred = 0;
  double dt = 0.0;
  long long steps = 0;
  bool initialised = false;
  std::string err;
  // adjoint recording: checkpoints of the state every record_every steps
  int record_every = 0;
  bool recorded = false;               // checkpoints cover steps 0 .. steps
  std::vector<void*> ckpt;             // ckpt[j] = state at step j * record_every
  std::vector<void*> pool;             // spare state buffers
  double* init_fields = nullptr;       // rho, ux, uy, T of the recorded dvbm_init
  double* stage = nullptr;             // 4 Nx Ny doubles staging host fields (allocated on first use)
  std::vector<void*> in_flight;        // temporaries of calls that timed out, freed by dvbm_destroy
  size_t state_bytes_dev = 0;
  // slab decomposition along y: sides whose ghost rows come from dvbm_halo_unpack
  bool external[2] = {false, false};  // ylo, yhi
  bool halo_fresh = false;             // the external ghost rows hold the current time level
  double pmax = 0.0;                   // largest pressure of the dvbm_init field (relaxation limit of dt)
  // stepwise backward pass (dvbm_adjoint_begin / _advance / _finish)
  struct AdjRun {
    bool active = false;
    void* lam[2] = {nullptr, nullptr};  // adjoint states; lam[a] is the current one
    int a = 0;
    std::vector<void*> seg;              // the states of the segment being processed
    double* part = nullptr;              // per-block partial sums of the parameter adjoints
    long long slot = 0;                  // next partial-sum slot
    long long j = -1;                    // segment being processed (last first)
    int phase = 0;                       // AdjRestore, AdjRecompute, AdjBackward, AdjDone
    long long t = 0, nrec = 0;           // step within the segment; recompute steps of the segment
    void* halo = nullptr;                // buffer whose ghost rows the neighbours fill next
    int halo_kind = 0;                   // 1: rows of a state buffer (halo); 3: branch-code rows of step code_t
    // coded pass (rational limiter): the recompute records branch codes and
    // moments as in dvbm_adjoint; a band also holds its neighbours' code rows
    unsigned char* codes = nullptr;      // [step][NPOP][Ny][Nx]
    double* moms = nullptr;              // [step][13][Ny][Nx]
    unsigned char* gcodes = nullptr;     // [step][lo, hi][NPOP][Nx]
    long long code_t = 0;                // step whose code rows are exchanged next
  } adj;
};

enum { AdjRestore = 0, AdjRecompute = 1, AdjBackward = 2, AdjDone = 3, AdjCodes = 4 };

static bool has_external(const dvbm_ctx* c) { return c->external[0] || c->external[1]; }

// message of the calling thread's last failed dvbm_create (per thread: creating
// contexts on several threads at once does not race on it)
static thread_local std::string g_create_error;

static dvbm_status fail(dvbm_ctx* c, dvbm_status s, const char* fmt, ...) {
  char msg[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(msg, sizeof msg, fmt, ap);
  va_end(ap);
  if (c) c->err = msg; else g_create_error = msg;
  return s;
}

#define CUDA_TRY(ctx, call)                                                                   \
  do {                                                                                        \
    cudaError_t e_ = (call);                                                                  \
    if (e_ != cudaSuccess)                                                                    \
      return fail(ctx, e_ == cudaErrorMemoryAllocation ? DVBM_ENOMEM : DVBM_ECUDA, "%s: %s", \
                  #call, cudaGetErrorString(e_));                                             \
  } while (0)

extern "C" dvbm_status dvbm_default_opts(dvbm_opts* o) {
  if (!o) return DVBM_EINVAL;
  o->Lx = 1.0;
  o->Ly = 0.0;
  o->R = 1.0;
  o->T_ref = 1.0;
  o->rho0 = 1.0;
  o->T0 = 1.0;
  o->beta = 1.2;
  o->cfl = 0.01;
  o->dt = 0.0;
  o->check_every = 0;
  o->timeout_s = 600.0;
  return DVBM_OK;
}

// 1-D node k of the context's lattice (D2Q25: 0, +-sqrt(5 -+ sqrt 10);
// D2Q16: +-sqrt(3 -+ sqrt 6), in the ABI order)
static double node(const dvbm_ctx* c, int k) {
  if (c->lattice == DVBM_D2Q16_SPLIT_I) {
    const double a = std::sqrt(3.0 - std::sqrt(6.0)), b = std::sqrt(3.0 + std::sqrt(6.0));
    const double v[4] = {a, -a, b, -b};
    return k < 4 ? v[k] : 0.0;
  }
  return xi_of(k);
}

// Limits of the explicit scheme on the fixed time step: the fastest population crosses at most
// one cell per step (the upwind stencil's domain of dependence must contain the characteristic),
// and forward-Euler relaxation takes dt <= the shortest relaxation time, min(tau1, tau2) =
// mu / p * min(1, 1/Pr) at the largest pressure p = rho R T of the initial field.  pmax <= 0: no
// field known (set_state without dvbm_init), the relaxation limit is not checked.
static dvbm_status check_dt(dvbm_ctx* c, double dt, double pmax) {
  double xi = 0.0;
  for (int k = 0; k < 5; ++k) xi = std::fmax(xi, std::fabs(node(c, k)));
  const double courant = dt * c->M.c * xi / std::fmin(c->opts.Lx / c->Nx, c->opts.Ly / c->Ny);
  if (!(courant <= 1.0))
    return fail(c, DVBM_EINVAL, "dt = %g moves the fastest population %.3g cells per step (limit 1)", dt, courant);
  if (pmax > 0) {
    const double tau_min = c->mu / pmax * std::fmin(1.0, 1.0 / c->Pr);
    if (!(dt <= tau_min))
      return fail(c, DVBM_EINVAL, "dt = %g exceeds the shortest relaxation time %g of the initial field", dt, tau_min);
  }
  return DVBM_OK;
}

static void set_step_factors(dvbm_ctx* c) {
  const double dx = c->opts.Lx / c->Nx, dy = c->opts.Ly / c->Ny;
  for (int k = 0; k < 5; ++k) {
    c->P.kxv[k] = c->dt / dx * c->M.c * node(c, k);
    c->P.kyv[k] = c->dt / dy * c->M.c * node(c, k);
    c->P.kxvf[k] = (float)c->P.kxv[k];
    if (c->P.lq > 0) {
      c->P.kxr[k] = c->P.kxv[k] / (4.0 * c->P.lq);
      c->P.kyr[k] = c->P.kyv[k] / (4.0 * c->P.lq);
    }
    c->P.kyvf[k] = (float)c->P.kyv[k];
  }
  c->P.dt = c->dt;
  c->P.dt_mu = c->dt / c->mu;
}

extern "C" dvbm_status dvbm_create(dvbm_ctx** out, int lattice, int Nx, int Ny, double Pr, double gamma,
                                   double mu, const dvbm_bc bcs[4], int storage, const dvbm_opts* opts,
                                   void* stream) {
  if (!out) return fail(nullptr, DVBM_EINVAL, "out is NULL");
  *out = nullptr;
  if (lattice != DVBM_D2Q25_SPLIT_II && lattice != DVBM_D2Q16_SPLIT_I)
    return fail(nullptr, DVBM_EINVAL, "unsupported lattice %d", lattice);
  if (storage != DVBM_FP64 && storage != DVBM_FP32DEV) return fail(nullptr, DVBM_EINVAL, "bad storage %d", storage);
  if (lattice == DVBM_D2Q16_SPLIT_I && storage != DVBM_FP64)
    return fail(nullptr, DVBM_EINVAL, "the D2Q16 / split I lattice is built for FP64 storage");
  if (Nx < 4 || Ny < 4 || Nx > (1 << 20) || Ny > 65535 || (long long)Nx * Ny > (1ll << 31))
    return fail(nullptr, DVBM_EINVAL, "grid %d x %d out of range (4 <= N, Ny <= 65535)", Nx, Ny);
  if (!(Pr > 0) || !std::isfinite(Pr)) return fail(nullptr, DVBM_EINVAL, "Pr must be > 0");
  if (!(gamma > 1.0) || !(gamma <= 2.0)) return fail(nullptr, DVBM_EINVAL, "gamma must be in (1, 2] for split II");
  if (!(mu > 0) || !std::isfinite(mu)) return fail(nullptr, DVBM_EINVAL, "mu must be > 0");
  dvbm_opts o;
  dvbm_default_opts(&o);
  if (opts) o = *opts;
  if (!(o.Lx > 0)) return fail(nullptr, DVBM_EINVAL, "Lx must be > 0");
  if (!(o.Ly > 0)) o.Ly = o.Lx * Ny / Nx;
  if (!(o.R > 0) || !(o.T_ref > 0) || !(o.rho0 > 0) || !(o.T0 > 0))
    return fail(nullptr, DVBM_EINVAL, "R, T_ref, rho0, T0 must be > 0");
  if (!(o.beta >= 1.0 && o.beta <= 2.0)) return fail(nullptr, DVBM_EINVAL, "beta must be in [1, 2]");
  if (!(o.cfl > 0) && !(o.dt > 0)) return fail(nullptr, DVBM_EINVAL, "need cfl > 0 or dt > 0");
  if (!(o.timeout_s > 0)) o.timeout_s = 600.0;
  dvbm_bc b[4];
  for (int s = 0; s < 4; ++s) {
    if (bcs) b[s] = bcs[s];
    else { b[s].kind = DVBM_BC_PERIODIC; b[s].u_wall[0] = b[s].u_wall[1] = 0; b[s].T_wall = 1; }
    if (b[s].kind < 0 || b[s].kind > 3) return fail(nullptr, DVBM_EINVAL, "bad boundary kind on side %d", s);
    if (b[s].kind == DVBM_BC_EXTERNAL && s < 2)
      return fail(nullptr, DVBM_EINVAL, "external halo rows are supported on the y sides only (slabs along y)");
    if (b[s].kind == DVBM_BC_WALL && !(b[s].T_wall > 0)) return fail(nullptr, DVBM_EINVAL, "wall T must be > 0");
  }
  for (int a = 0; a < 2; ++a)
    if ((b[2 * a].kind == DVBM_BC_PERIODIC) != (b[2 * a + 1].kind == DVBM_BC_PERIODIC))
      return fail(nullptr, DVBM_EINVAL, "periodic boundaries must be paired on axis %d", a);

  dvbm_ctx* c = new dvbm_ctx();
  c->Nx = Nx; c->Ny = Ny; c->storage = storage;
  c->lattice = lattice;
  c->npop = lattice == DVBM_D2Q16_SPLIT_I ? 32 : NPOP;
  c->Pr = Pr; c->gamma = gamma; c->mu = mu;
  c->opts = o;
  for (int s = 0; s < 4; ++s) c->bcs[s] = b[s];
  c->external[0] = b[DVBM_YLO].kind == DVBM_BC_EXTERNAL;
  c->external[1] = b[DVBM_YHI].kind == DVBM_BC_EXTERNAL;
  c->stream = (cudaStream_t)stream;
  const cudaError_t ed = cudaGetDevice(&c->device);
  if (ed != cudaSuccess) {
    cudaGetLastError();
    delete c;  // nothing allocated yet
    return fail(nullptr, DVBM_ECUDA, "no usable CUDA device: %s", cudaGetErrorString(ed));
  }
  c->elem = storage == DVBM_FP64 ? 8 : 4;
  const int align = 128 / (int)c->elem;  // elements per 128 B
  c->G.Nx = Nx; c->G.Ny = Ny;
  c->G.xoff = align;
  c->G.pitch = ((Nx + align + 2 + align - 1) / align) * align;
  c->G.plane = (long long)(Ny + 4) * c->G.pitch;
  const double c2 = o.R * o.T_ref;
  c->M.c = std::sqrt(c2); c->M.T_ref = o.T_ref; c->M.R = o.R; c->M.gamma = gamma;
  c->P.c2 = c2; c->P.inv_c2 = 1.0 / c2;
  c->P.gm1 = gamma - 1.0;
  c->P.epsf = 1.0 / (gamma - 1.0) - 1.0;
  c->P.mu = mu; c->P.Pr = Pr;
  c->P.prc = Pr < 1.0 ? -1 : (Pr > 1.0 ? 1 : 0);
  c->P.hb = 0.5 * o.beta;
  c->P.hq = (long long)std::llround(std::ldexp(0.5 * o.beta, 62));
  c->P.lp = 0;
  c->P.lq = 0;
  for (int q = 1; q <= 64; ++q) {  // beta = lp / lq exactly (to double precision)?
    const double pq = o.beta * q;
    if (std::fabs(pq - std::nearbyint(pq)) < 1e-12 * pq) {
      c->P.lp = (int)std::nearbyint(pq);
      c->P.lq = q;
      break;
    }
  }
  c->P.fref0 = o.rho0;
  c->P.gref0 = o.rho0 * (o.R / (gamma - 1.0) - o.R) * o.T0;
  for (int s = 0; s < 4; ++s) {
    c->bc.kind[s] = b[s].kind;
    c->bc.uw[s][0] = b[s].u_wall[0]; c->bc.uw[s][1] = b[s].u_wall[1];
    c->bc.Tw[s] = b[s].T_wall;
  }
  const size_t bytes = (size_t)c->npop * c->G.plane * c->elem;
  c->state_bytes_dev = bytes;
  for (int k = 0; k < 2; ++k) {
    cudaError_t e = cudaMalloc(&c->buf[k], bytes);
    if (e != cudaSuccess) {
      cudaGetLastError();
      dvbm_destroy(c);
      return fail(nullptr, e == cudaErrorMemoryAllocation ? DVBM_ENOMEM : DVBM_ECUDA,
                  "cudaMalloc of %zu bytes failed: %s", bytes, cudaGetErrorString(e));
    }
  }
  int sms = 0;  // reduction grids: four blocks per SM (grid-stride loops, any count is correct)
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, c->device) != cudaSuccess || sms <= 0) {
    cudaGetLastError();
    sms = 152;
  }
  c->nred = 4 * sms;
  if (cudaMalloc(&c->flag, sizeof(unsigned int)) != cudaSuccess ||
      cudaMalloc(&c->partial, sizeof(double) * 6 * c->nred) != cudaSuccess) {
    cudaGetLastError();
    dvbm_destroy(c);
    return fail(nullptr, DVBM_ENOMEM, "cudaMalloc of work buffers failed");
  }
  if (cudaMemsetAsync(c->buf[0], 0, bytes, c->stream) != cudaSuccess ||
      cudaMemsetAsync(c->buf[1], 0, bytes, c->stream) != cudaSuccess ||
      cudaMemsetAsync(c->flag, 0, sizeof(unsigned int), c->stream) != cudaSuccess) {
    cudaGetLastError();
    dvbm_destroy(c);
    return fail(nullptr, DVBM_ECUDA, "buffer initialisation failed");
  }
  // no wait here: the caller's stream may hold earlier work, and every later
  // call of this context is ordered after the memsets on the same stream
  *out = c;
  return DVBM_OK;
}

// stream-ordered wait with a host-side time limit
static dvbm_status wait_stream(dvbm_ctx* c) {
  cudaEvent_t ev;
  CUDA_TRY(c, cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
  cudaError_t e = cudaEventRecord(ev, c->stream);
  if (e != cudaSuccess) { cudaEventDestroy(ev); return fail(c, DVBM_ECUDA, "cudaEventRecord: %s", cudaGetErrorString(e)); }
  const auto t0 = std::chrono::steady_clock::now();
  int spins = 0;
  for (;;) {
    e = cudaEventQuery(ev);
    if (e == cudaSuccess) break;
    if (e != cudaErrorNotReady) { cudaEventDestroy(ev); return fail(c, DVBM_ECUDA, "stream error: %s", cudaGetErrorString(e)); }
    const double el = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    if (el > c->opts.timeout_s) { cudaEventDestroy(ev); return fail(c, DVBM_ETIMEOUT, "stream did not finish within %g s", c->opts.timeout_s); }
    if (++spins > 64) std::this_thread::sleep_for(std::chrono::microseconds(50));
  }
  cudaEventDestroy(ev);
  return DVBM_OK;
}

// Device -> host copy under the time limit. A copy into pageable host memory returns only once
// it has completed, i.e. once the stream has run everything queued before it, so a hung or slow
// stream would block inside the copy, past timeout_s. The queued work is therefore waited for
// first, under the limit; the copy then finds the stream idle.
static dvbm_status drain_then_copy(dvbm_ctx* c, void* dst, const void* src, size_t bytes) {
  dvbm_status s = wait_stream(c);
  if (s != DVBM_OK) return s;
  const cudaError_t e = cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDeviceToHost, c->stream);
  if (e != cudaSuccess) return fail(c, DVBM_ECUDA, "device to host copy: %s", cudaGetErrorString(e));
  return wait_stream(c);
}

// A temporary that queued work may still use after a timeout is not freed here (cudaFree would
// wait for that work, past the limit): dvbm_destroy frees it after synchronising the stream.
static void release_temporary(dvbm_ctx* c, void* p, dvbm_status s) {
  if (s == DVBM_ETIMEOUT) c->in_flight.push_back(p);
  else cudaFree(p);
}

static dvbm_status check_flag(dvbm_ctx* c) {
  unsigned int h = 0;
  dvbm_status s = drain_then_copy(c, &h, c->flag, sizeof h);
  if (s != DVBM_OK) return s;
  if (h) return fail(c, DVBM_EUNSTABLE, "a cell reached rho <= 0, T <= 0 or a non-finite value (after %lld steps)", c->steps);
  return DVBM_OK;
}

static dvbm_status fill_ghosts(dvbm_ctx* c, void* b) {
  CUDA_TRY(c, launch_ghost(c->lattice, c->storage, b, c->G, c->P, c->M, c->bc, c->stream));
  return DVBM_OK;
}

// lattice dispatch of the per-step and diagnostic kernels
static cudaError_t l_step(dvbm_ctx* c, const void* src, void* dst) {
  return c->lattice == DVBM_D2Q16_SPLIT_I ? launch_step16(src, dst, c->G, c->P, c->flag, c->stream)
                                          : launch_step(c->storage, src, dst, c->G, c->P, c->flag, c->stream);
}
static cudaError_t l_init(dvbm_ctx* c, void* dst, const double* const* F) {
  return launch_init(c->lattice, c->storage, dst, F[0], F[1], F[2], F[3], c->G, c->P, c->M, c->stream);
}
static cudaError_t l_moments(dvbm_ctx* c, const void* src, double* r, double* a, double* b, double* t) {
  return launch_moments(c->lattice, c->storage, src, r, a, b, t, c->G, c->P, c->M, c->stream);
}
static cudaError_t l_totals(dvbm_ctx* c, const void* src) {
  return launch_totals(c->lattice, c->storage, src, c->partial, c->nred, c->G, c->P, c->M, c->stream);
}

// device copies of host field arrays (or pass-through for device pointers)
struct DevFields {
  const double* p[4] = {nullptr, nullptr, nullptr, nullptr};
  double* owned = nullptr;
  ~DevFields() { if (owned) cudaFree(owned); }
};

static dvbm_status stage_fields(dvbm_ctx* c, DevFields& F, const double* const in[4], int on_device) {
  const size_t n = (size_t)c->Nx * c->Ny;
  for (int k = 0; k < 4; ++k)
    if (!in[k]) return fail(c, DVBM_EINVAL, "field pointer %d is NULL", k);
  if (on_device) {
    for (int k = 0; k < 4; ++k) F.p[k] = in[k];
    return DVBM_OK;
  }
  // one staging buffer per context, reused (stream-ordered) by every host transfer
  if (!c->stage) CUDA_TRY(c, cudaMalloc(&c->stage, 4 * n * sizeof(double)));
  // a copy from pageable host memory may wait for the stream: drain it first, under the limit
  dvbm_status s = wait_stream(c);
  if (s != DVBM_OK) return s;
  for (int k = 0; k < 4; ++k) {
    CUDA_TRY(c, cudaMemcpyAsync(c->stage + k * n, in[k], n * sizeof(double), cudaMemcpyHostToDevice, c->stream));
    F.p[k] = c->stage + k * n;
  }
  return DVBM_OK;
}

static dvbm_status take_buffer(dvbm_ctx* c, void** out) {
  if (!c->pool.empty()) {
    *out = c->pool.back();
    c->pool.pop_back();
    return DVBM_OK;
  }
  CUDA_TRY(c, cudaMalloc(out, c->state_bytes_dev));
  return DVBM_OK;
}

static void adj_release(dvbm_ctx* c, dvbm_status s);

// also ends a stepwise backward pass: it reads the checkpoints being discarded
static void clear_record(dvbm_ctx* c) {
  if (c->adj.active) adj_release(c, DVBM_OK);
  for (void* p : c->ckpt) c->pool.push_back(p);
  c->ckpt.clear();
  c->recorded = false;
}

static dvbm_status push_checkpoint(dvbm_ctx* c) {
  void* b = nullptr;
  dvbm_status s = take_buffer(c, &b);
  if (s != DVBM_OK) return s;
  CUDA_TRY(c, cudaMemcpyAsync(b, c->buf[c->cur], c->state_bytes_dev, cudaMemcpyDeviceToDevice, c->stream));
  c->ckpt.push_back(b);
  return DVBM_OK;
}

extern "C" dvbm_status dvbm_record(dvbm_ctx* c, int every) {
  if (!c) return DVBM_EINVAL;
  if (every < 0) return fail(c, DVBM_EINVAL, "record interval must be >= 0");
  if (every > 0 && c->storage != DVBM_FP64) return fail(c, DVBM_EINVAL, "the adjoint needs FP64 storage");
  if (every > 0 && c->lattice != DVBM_D2Q25_SPLIT_II)
    return fail(c, DVBM_EINVAL, "the adjoint is built for the D2Q25 / split II model");
  for (int s = 0; s < 4 && every > 0; ++s) {
    // a band of a y-periodic grid has EXTERNAL y sides (the stepwise adjoint)
    const bool band_side = s >= DVBM_YLO && c->bcs[s].kind == DVBM_BC_EXTERNAL;
    if (c->bcs[s].kind != DVBM_BC_PERIODIC && !band_side)
      return fail(c, DVBM_EINVAL, "the adjoint is built for periodic domains");
  }
  clear_record(c);
  c->record_every = every;
  return DVBM_OK;
}

extern "C" dvbm_status dvbm_init(dvbm_ctx* c, const double* rho, const double* ux, const double* uy,
                                 const double* T, int on_device) {
  if (!c) return DVBM_EINVAL;
  CUDA_TRY(c, cudaSetDevice(c->device));
  const double* in[4] = {rho, ux, uy, T};
  DevFields F;
  dvbm_status s = stage_fields(c, F, in, on_device);
  if (s != DVBM_OK) return s;
  const long long n = (long long)c->Nx * c->Ny;
  CUDA_TRY(c, launch_speed(F.p[0], F.p[1], F.p[2], F.p[3], n, c->partial, c->nred, c->M, c->stream));
  std::vector<double> h(3 * c->nred);
  s = drain_then_copy(c, h.data(), c->partial, h.size() * sizeof(double));
  if (s != DVBM_OK) return s;
  double vmax = 0.0, bad = 0.0, pmax = 0.0;
  for (int b = 0; b < c->nred; ++b) {
    vmax = std::fmax(vmax, h[3 * b]);
    bad += h[3 * b + 1];
    pmax = std::fmax(pmax, h[3 * b + 2]);
  }
  if (bad > 0) return fail(c, DVBM_EINVAL, "%.0f cells with rho <= 0, T <= 0 or non-finite values", bad);
  const double dt = c->opts.dt > 0 ? c->opts.dt
                                   : c->opts.cfl * std::fmin(c->opts.Lx / c->Nx, c->opts.Ly / c->Ny) / vmax;
  s = check_dt(c, dt, pmax);  // before any change to the context
  if (s != DVBM_OK) return s;
  c->dt = dt;
  c->pmax = pmax;
  set_step_factors(c);
  c->cur = 0;
  c->halo_fresh = false;
  CUDA_TRY(c, l_init(c, c->buf[0], F.p));
  s = fill_ghosts(c, c->buf[0]);
  if (s != DVBM_OK) return s;
  CUDA_TRY(c, cudaMemsetAsync(c->flag, 0, sizeof(unsigned int), c->stream));
  clear_record(c);
  if (c->record_every > 0) {
    const size_t n = (size_t)c->Nx * c->Ny;
    if (!c->init_fields) CUDA_TRY(c, cudaMalloc(&c->init_fields, 4 * n * sizeof(double)));
    for (int k = 0; k < 4; ++k)
      CUDA_TRY(c, cudaMemcpyAsync(c->init_fields + k * n, F.p[k], n * sizeof(double), cudaMemcpyDeviceToDevice,
                                  c->stream));
    s = push_checkpoint(c);
    if (s != DVBM_OK) return s;
    c->recorded = true;
  }
  s = wait_stream(c);  // the staged host copies are freed on return
  if (s != DVBM_OK) return s;
  c->steps = 0;
  c->initialised = true;
  return DVBM_OK;
}

extern "C" dvbm_status dvbm_step(dvbm_ctx* c, int n) {
  if (!c) return DVBM_EINVAL;
  if (!c->initialised) return fail(c, DVBM_ESTATE, "dvbm_step before dvbm_init / dvbm_set_state");
  if (n < 0) return fail(c, DVBM_EINVAL, "n must be >= 0");
  if (has_external(c) && n > 1)
    return fail(c, DVBM_EINVAL, "a context with external halo rows advances one step per halo exchange (n <= 1)");
  if (has_external(c) && n == 1 && !c->halo_fresh)
    return fail(c, DVBM_ESTATE, "the external halo rows are stale: call dvbm_halo_unpack before each step");
  const int every = c->opts.check_every;
  // new steps change the recorded run a stepwise backward pass is working through
  if (n > 0 && c->adj.active) adj_release(c, DVBM_OK);
  for (int i = 0; i < n; ++i) {
    void* src = c->buf[c->cur];
    void* dst = c->buf[1 - c->cur];
    CUDA_TRY(c, l_step(c, src, dst));
    dvbm_status s = fill_ghosts(c, dst);
    if (s != DVBM_OK) return s;
    c->cur = 1 - c->cur;
    ++c->steps;
    c->halo_fresh = false;
    if (c->recorded && c->steps % c->record_every == 0) {
      s = push_checkpoint(c);
      if (s != DVBM_OK) return s;
    }
    if (every > 0 && (i + 1) % every == 0) {
      s = check_flag(c);
      if (s != DVBM_OK) return s;
    }
  }
  if (every == 0 && n > 0) return check_flag(c);
  return DVBM_OK;
}

extern "C" dvbm_status dvbm_moments(dvbm_ctx* c, double* rho, double* ux, double* uy, double* T, int on_device) {
  if (!c) return DVBM_EINVAL;
  if (!c->initialised) return fail(c, DVBM_ESTATE, "no state yet");
  const size_t n = (size_t)c->Nx * c->Ny;
  double* outs[4] = {rho, ux, uy, T};
  if (on_device) {
    CUDA_TRY(c, l_moments(c, c->buf[c->cur], rho, ux, uy, T));
    return DVBM_OK;
  }
  if (!c->stage) CUDA_TRY(c, cudaMalloc(&c->stage, 4 * n * sizeof(double)));
  double* tmp = c->stage;
  CUDA_TRY(c, l_moments(c, c->buf[c->cur], tmp, tmp + n, tmp + 2 * n, tmp + 3 * n));
  // drained first, under the limit: a copy into pageable memory would otherwise wait unbounded
  dvbm_status s = wait_stream(c);
  if (s != DVBM_OK) return s;
  for (int k = 0; k < 4; ++k)
    if (outs[k]) CUDA_TRY(c, cudaMemcpyAsync(outs[k], tmp + k * n, n * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
  return wait_stream(c);
}

extern "C" dvbm_status dvbm_totals(dvbm_ctx* c, double out[4]) {
  if (!c || !out) return DVBM_EINVAL;
  if (!c->initialised) return fail(c, DVBM_ESTATE, "no state yet");
  CUDA_TRY(c, l_totals(c, c->buf[c->cur]));
  std::vector<double> h(6 * c->nred);
  dvbm_status s = drain_then_copy(c, h.data(), c->partial, h.size() * sizeof(double));
  if (s != DVBM_OK) return s;
  double acc[5] = {0, 0, 0, 0, 0};
  for (int b = 0; b < c->nred; ++b)
    for (int k = 0; k < 5; ++k) acc[k] += h[6 * b + k];
  const double dV = (c->opts.Lx / c->Nx) * (c->opts.Ly / c->Ny);
  for (int k = 0; k < 4; ++k) out[k] = acc[k] * dV;
  if (acc[4] > 0) return fail(c, DVBM_EUNSTABLE, "%.0f cells with rho <= 0, T <= 0 or non-finite values", acc[4]);
  return DVBM_OK;
}

extern "C" size_t dvbm_state_bytes(const dvbm_ctx* c) {
  if (!c) return 0;
  return (size_t)c->npop * c->Nx * c->Ny * c->elem + 8;
}

extern "C" dvbm_status dvbm_get_state(dvbm_ctx* c, void* buf, size_t bytes, int on_device) {
  if (!c || !buf) return DVBM_EINVAL;
  if (!c->initialised) return fail(c, DVBM_ESTATE, "no state yet");
  if (bytes != dvbm_state_bytes(c)) return fail(c, DVBM_EINVAL, "state buffer must be %zu bytes", dvbm_state_bytes(c));
  const size_t pb = bytes - 8;
  void* dev = buf;
  if (!on_device) CUDA_TRY(c, cudaMalloc(&dev, pb));
  cudaError_t e = launch_pack(c->storage, c->buf[c->cur], dev, 1, c->G, c->npop, c->stream);
  dvbm_status s = e == cudaSuccess ? DVBM_OK : fail(c, DVBM_ECUDA, "get_state: %s", cudaGetErrorString(e));
  if (s == DVBM_OK && !on_device) {
    s = drain_then_copy(c, buf, dev, pb);
    if (s == DVBM_OK) std::memcpy((char*)buf + pb, &c->steps, 8);
  } else if (s == DVBM_OK) {
    s = wait_stream(c);
    if (s == DVBM_OK) e = cudaMemcpyAsync((char*)buf + pb, &c->steps, 8, cudaMemcpyHostToDevice, c->stream);
    if (s == DVBM_OK) s = e == cudaSuccess ? wait_stream(c) : fail(c, DVBM_ECUDA, "get_state: %s", cudaGetErrorString(e));
  }
  if (!on_device) release_temporary(c, dev, s);
  return s;
}

extern "C" dvbm_status dvbm_set_state(dvbm_ctx* c, const void* buf, size_t bytes, int on_device) {
  if (!c || !buf) return DVBM_EINVAL;
  if (bytes != dvbm_state_bytes(c)) return fail(c, DVBM_EINVAL, "state buffer must be %zu bytes", dvbm_state_bytes(c));
  if (!(c->dt > 0)) {
    if (!(c->opts.dt > 0)) return fail(c, DVBM_ESTATE, "set_state needs dt: call dvbm_init first or set opts.dt");
    const dvbm_status sd = check_dt(c, c->opts.dt, 0.0);
    if (sd != DVBM_OK) return sd;
    c->dt = c->opts.dt;
    set_step_factors(c);
  }
  const size_t pb = bytes - 8;
  void* dev = (void*)buf;
  if (!on_device) {
    CUDA_TRY(c, cudaMalloc(&dev, pb));
  }
  // a copy from pageable host memory may wait for the stream: drain it first, under the limit
  dvbm_status s = on_device ? DVBM_OK : wait_stream(c);
  cudaError_t e = cudaSuccess;
  if (s == DVBM_OK && !on_device) e = cudaMemcpyAsync(dev, buf, pb, cudaMemcpyHostToDevice, c->stream);
  if (s == DVBM_OK && e == cudaSuccess) e = launch_pack(c->storage, c->buf[c->cur], dev, 0, c->G, c->npop, c->stream);
  // a new state: an instability raised by the replaced one no longer applies
  if (s == DVBM_OK && e == cudaSuccess) e = cudaMemsetAsync(c->flag, 0, sizeof(unsigned int), c->stream);
  if (s == DVBM_OK)
    s = e == cudaSuccess ? fill_ghosts(c, c->buf[c->cur]) : fail(c, DVBM_ECUDA, "set_state: %s", cudaGetErrorString(e));
  long long st = 0;
  if (s == DVBM_OK) {
    if (on_device) s = drain_then_copy(c, &st, (const char*)buf + pb, 8);
    else {
      std::memcpy(&st, (const char*)buf + pb, 8);
      s = wait_stream(c);
    }
  }
  if (!on_device) release_temporary(c, dev, s);
  if (s != DVBM_OK) return s;
  c->steps = st;
  c->initialised = true;
  c->halo_fresh = false;
  clear_record(c);
  return DVBM_OK;
}

extern "C" size_t dvbm_halo_bytes(const dvbm_ctx* c) {
  if (!c) return 0;
  return (size_t)2 * c->Nx * c->npop * c->elem;
}

extern "C" dvbm_status dvbm_halo_pack(dvbm_ctx* c, void* lo, void* hi) {
  if (!c) return DVBM_EINVAL;
  if (!c->initialised) return fail(c, DVBM_ESTATE, "no state yet");
  if (!lo && !hi) return DVBM_OK;
  CUDA_TRY(c, launch_halo(c->storage == DVBM_FP64 ? 8 : 4, c->buf[c->cur], lo, hi, 0, c->G, c->npop, c->stream));
  return DVBM_OK;
}

extern "C" dvbm_status dvbm_halo_unpack(dvbm_ctx* c, const void* lo, const void* hi) {
  if (!c) return DVBM_EINVAL;
  if (!c->initialised) return fail(c, DVBM_ESTATE, "no state yet");
  const void* in[2] = {lo, hi};
  for (int s = 0; s < 2; ++s) {
    if (c->external[s] && !in[s]) return fail(c, DVBM_EINVAL, "side %s is external: its halo buffer is required", s ? "yhi" : "ylo");
    if (!c->external[s] && in[s]) return fail(c, DVBM_EINVAL, "side %s is not external: pass NULL", s ? "yhi" : "ylo");
  }
  if (lo || hi)
    CUDA_TRY(c, launch_halo(c->storage == DVBM_FP64 ? 8 : 4, c->buf[c->cur], (void*)lo, (void*)hi, 1, c->G,
                            c->npop, c->stream));
  c->halo_fresh = true;
  return DVBM_OK;
}

extern "C" dvbm_status dvbm_set_dt(dvbm_ctx* c, double dt) {
  if (!c) return DVBM_EINVAL;
  if (!c->initialised) return fail(c, DVBM_ESTATE, "no state yet");
  if (!(dt > 0) || !std::isfinite(dt)) return fail(c, DVBM_EINVAL, "dt must be > 0 and finite");
  // the adjoint recomputes the recorded run with the context's dt
  if (c->recorded && c->steps > 0 && dt != c->dt)
    return fail(c, DVBM_ESTATE, "the recorded run has taken steps with dt = %g: it cannot change now", c->dt);
  const dvbm_status s = check_dt(c, dt, c->pmax);
  if (s != DVBM_OK) return s;
  c->dt = dt;
  set_step_factors(c);
  return DVBM_OK;
}

// dL/d(mu, Pr, gamma) from the per-block partial sums of a backward pass:
// slot 0: final read-out (gm1 adjoint per block); slots 1 .. slot-2: steps
// (dt_mu, Pr, gm1, epsf); last slot: initial condition (epsf adjoint per block)
static void params_from_partials(const dvbm_ctx* c, const std::vector<double>& h, long long slot, int nblk,
                                 double g_params[3]) {
  double dtmu_b = 0, Pr_b = 0, gm1_b = 0, epsf_b = 0;
  for (int b = 0; b < nblk; ++b) gm1_b += h[b];
  for (long long t = 1; t < slot - 1; ++t)
    for (int b = 0; b < nblk; ++b) {
      const double* q = &h[(t * nblk + b) * 4];
      dtmu_b += q[0]; Pr_b += q[1]; gm1_b += q[2]; epsf_b += q[3];
    }
  for (int b = 0; b < nblk; ++b) epsf_b += h[((slot - 1) * nblk) * 4 + b];
  const double gm1 = c->gamma - 1.0;
  g_params[0] = -dtmu_b * c->dt / (c->mu * c->mu);   // d(dt/mu)/dmu = -dt/mu^2
  g_params[1] = Pr_b;
  g_params[2] = gm1_b - epsf_b / (gm1 * gm1);        // epsf = 1/(gamma-1) - 1
}

// Backward pass over the recorded forward run: lambda^N from dL/d(rho, T) of
// the current state, then segment by segment (last first) a recompute of the
// segment's states from its checkpoint and the adjoint steps through it,
// finally the adjoint of the equilibrium initial condition.
extern "C" dvbm_status dvbm_adjoint(dvbm_ctx* c, const double* dL_drho, const double* dL_dT, double* g_rho0,
                                    double* g_ux0, double* g_uy0, double* g_T0, double g_params[3]) {
  if (!c) return DVBM_EINVAL;
  if (!c->recorded || c->ckpt.empty() || !c->init_fields)
    return fail(c, DVBM_ESTATE, "no recorded forward run: call dvbm_record(ctx, k) before dvbm_init, then dvbm_step");
  if (!g_rho0 || !g_ux0 || !g_uy0 || !g_T0 || !g_params) return fail(c, DVBM_EINVAL, "null gradient pointer");
  if (has_external(c))
    return fail(c, DVBM_EINVAL, "a band of a decomposed grid needs its neighbours at every adjoint step: "
                                "use dvbm_adjoint_begin / _advance / _finish with halo exchanges");
  CUDA_TRY(c, cudaSetDevice(c->device));
  const long long n = c->steps;
  const int k = c->record_every;
  const int nblk = adjoint_blocks(c->G);
  const size_t ncell = (size_t)c->Nx * c->Ny;
  // work buffers: two adjoint states, k segment states (k + 1 when the
  // recompute records minmod branch codes: the segment's last state is stepped
  // too), the codes of k steps (NPOP bytes per cell and step), partial sums
  void* lam[2] = {nullptr, nullptr};
  std::vector<void*> seg;
  double* part = nullptr;
  unsigned char* codes = nullptr;
  double* moms = nullptr;  // the moments of each recomputed state (13 doubles per cell and step)
  const long long nslots = (n + 2) * (long long)nblk * 4;
  const size_t code_step = (size_t)NPOP * ncell;
  bool coded = c->P.lq > 0;
  if (coded && cudaMalloc(&codes, (size_t)k * code_step) != cudaSuccess) {
    cudaGetLastError();  // not enough memory for the codes: derive the branches from the states instead
    codes = nullptr;
    coded = false;
  }
  const size_t mom_step = (size_t)13 * ncell;
  if (coded && cudaMalloc(&moms, (size_t)k * mom_step * sizeof(double)) != cudaSuccess) {
    cudaGetLastError();  // not enough memory: the adjoint sums the moments itself
    moms = nullptr;
  }
  dvbm_status s = DVBM_OK;
  auto cleanup = [&]() {
    for (int i = 0; i < 2; ++i) if (lam[i]) c->pool.push_back(lam[i]);
    for (void* p : seg) c->pool.push_back(p);
    if (part) release_temporary(c, part, s);
    if (codes) release_temporary(c, codes, s);
    if (moms) release_temporary(c, moms, s);
  };
  for (int i = 0; i < 2 && s == DVBM_OK; ++i) s = take_buffer(c, &lam[i]);
  for (int i = 0; i < k + (coded ? 1 : 0) && s == DVBM_OK; ++i) {
    void* b = nullptr;
    s = take_buffer(c, &b);
    if (s == DVBM_OK) seg.push_back(b);
  }
  if (s == DVBM_OK && cudaMalloc(&part, nslots * sizeof(double)) != cudaSuccess) {
    cudaGetLastError();
    s = fail(c, DVBM_ENOMEM, "cudaMalloc of adjoint partial sums failed");
  }
  if (s == DVBM_OK && cudaMemsetAsync(part, 0, nslots * sizeof(double), c->stream) != cudaSuccess)
    s = fail(c, DVBM_ECUDA, "memset failed");
  if (s != DVBM_OK) { cleanup(); return s; }
  // periodic ghost copies for the adjoint buffers
  BCDev per = c->bc;
  for (int i = 0; i < 4; ++i) per.kind[i] = DVBM_BC_PERIODIC;
  cudaError_t e = cudaSuccess;
  int a = 0;
  long long slot = 0;
  e = launch_adjoint_final((const double*)c->buf[c->cur], dL_drho, dL_dT, (double*)lam[a], part + slot * nblk * 4,
                           c->G, c->P, c->M, c->stream);
  ++slot;
  if (e == cudaSuccess) e = launch_ghost(DVBM_D2Q25_SPLIT_II, 0, lam[a], c->G, c->P, c->M, per, c->stream);
  const long long nseg = (n + k - 1) / k;
  for (long long j = nseg - 1; j >= 0 && e == cudaSuccess; --j) {
    const long long S = j * k, E = std::min<long long>((j + 1) * k, n);
    e = cudaMemcpyAsync(seg[0], c->ckpt[j], c->state_bytes_dev, cudaMemcpyDeviceToDevice, c->stream);
    const long long nrec = coded ? E - S : E - S - 1;
    for (long long t = 0; t < nrec && e == cudaSuccess; ++t) {
      if (coded)
        e = launch_step_codes(seg[t], seg[t + 1], c->G, c->P, c->flag, codes + t * code_step,
                              moms ? moms + t * mom_step : nullptr, c->stream);
      else e = launch_step(0, seg[t], seg[t + 1], c->G, c->P, c->flag, c->stream);
      if (e == cudaSuccess && t + 1 < E - S) e = launch_ghost(DVBM_D2Q25_SPLIT_II, 0, seg[t + 1], c->G, c->P, c->M, c->bc, c->stream);
    }
    for (long long t = E - S - 1; t >= 0 && e == cudaSuccess; --t) {
      e = launch_adjoint_step((const double*)seg[t], (const double*)lam[a], (double*)lam[1 - a],
                              part + slot * nblk * 4, coded ? codes + t * code_step : nullptr,
                              moms ? moms + t * mom_step : nullptr, c->G, c->P, c->stream);
      ++slot;
      a = 1 - a;
      if (e == cudaSuccess) e = launch_ghost(DVBM_D2Q25_SPLIT_II, 0, lam[a], c->G, c->P, c->M, per, c->stream);
    }
  }
  const double* F0 = c->init_fields;
  if (e == cudaSuccess)
    e = launch_adjoint_init((const double*)lam[a], F0, F0 + ncell, F0 + 2 * ncell, F0 + 3 * ncell, g_rho0, g_ux0,
                            g_uy0, g_T0, part + slot * nblk * 4, c->G, c->P, c->M, c->stream);
  ++slot;
  if (e != cudaSuccess) { cleanup(); return fail(c, DVBM_ECUDA, "adjoint: %s", cudaGetErrorString(e)); }
  std::vector<double> h(slot * nblk * 4);
  s = drain_then_copy(c, h.data(), part, h.size() * sizeof(double));
  cleanup();
  if (s != DVBM_OK) return s;
  params_from_partials(c, h, slot, nblk, g_params);
  return DVBM_OK;
}

// ---- stepwise backward pass (a band of a slab-decomposed grid) -------------
// The same sequence as dvbm_adjoint with the branch codes derived from the
// states, cut at every point where a buffer's ghost rows must come from the
// neighbouring bands: after lambda^N, after each restored or recomputed
// segment state, after each adjoint step.

// return the pass's buffers to the pool (stream-ordered reuse) and end it
static void adj_release(dvbm_ctx* c, dvbm_status s) {
  auto& A = c->adj;
  for (int i = 0; i < 2; ++i)
    if (A.lam[i]) {
      c->pool.push_back(A.lam[i]);
      A.lam[i] = nullptr;
    }
  for (void* p : A.seg) c->pool.push_back(p);
  A.seg.clear();
  if (A.part) release_temporary(c, A.part, s);
  if (A.codes) release_temporary(c, A.codes, s);
  if (A.moms) release_temporary(c, A.moms, s);
  if (A.gcodes) release_temporary(c, A.gcodes, s);
  A.part = nullptr;
  A.codes = nullptr;
  A.moms = nullptr;
  A.gcodes = nullptr;
  A.active = false;
  A.halo = nullptr;
  A.halo_kind = 0;
}

extern "C" dvbm_status dvbm_adjoint_begin(dvbm_ctx* c, const double* dL_drho, const double* dL_dT) {
  if (!c) return DVBM_EINVAL;
  if (!c->recorded || c->ckpt.empty() || !c->init_fields)
    return fail(c, DVBM_ESTATE, "no recorded forward run: call dvbm_record(ctx, k) before dvbm_init, then dvbm_step");
  CUDA_TRY(c, cudaSetDevice(c->device));
  auto& A = c->adj;
  if (A.active) adj_release(c, DVBM_OK);  // a pass begun earlier is abandoned
  const long long n = c->steps;
  const int k = c->record_every;
  const int nblk = adjoint_blocks(c->G);
  // Rational limiter: the coded pass of dvbm_adjoint (the recompute records
  // branch codes and moments; the segment's last state is stepped too), with
  // the neighbouring bands' code rows exchanged after each recompute step.
  // Otherwise, or without the memory for the codes, the adjoint derives the
  // branches from the states.
  const size_t ncell = (size_t)c->Nx * c->Ny;
  if (c->P.lq > 0) {
    if (cudaMalloc(&A.codes, (size_t)k * NPOP * ncell) != cudaSuccess ||
        cudaMalloc(&A.moms, (size_t)k * 13 * ncell * sizeof(double)) != cudaSuccess ||
        cudaMalloc(&A.gcodes, (size_t)k * 2 * NPOP * c->Nx) != cudaSuccess) {
      cudaGetLastError();
      if (A.codes) cudaFree(A.codes);
      if (A.moms) cudaFree(A.moms);
      A.codes = nullptr;
      A.moms = nullptr;
      A.gcodes = nullptr;
    }
  }
  const bool coded = A.codes != nullptr;
  dvbm_status s = DVBM_OK;
  for (int i = 0; i < 2 && s == DVBM_OK; ++i) s = take_buffer(c, &A.lam[i]);
  for (int i = 0; i < k + (coded ? 1 : 0) && s == DVBM_OK; ++i) {
    void* b = nullptr;
    s = take_buffer(c, &b);
    if (s == DVBM_OK) A.seg.push_back(b);
  }
  const long long nslots = (n + 2) * (long long)nblk * 4;
  if (s == DVBM_OK && cudaMalloc(&A.part, nslots * sizeof(double)) != cudaSuccess) {
    cudaGetLastError();
    A.part = nullptr;
    s = fail(c, DVBM_ENOMEM, "cudaMalloc of adjoint partial sums failed");
  }
  cudaError_t e = cudaSuccess;
  if (s == DVBM_OK) e = cudaMemsetAsync(A.part, 0, nslots * sizeof(double), c->stream);
  if (s == DVBM_OK && e == cudaSuccess)
    e = launch_adjoint_final((const double*)c->buf[c->cur], dL_drho, dL_dT, (double*)A.lam[0], A.part, c->G, c->P,
                             c->M, c->stream);
  // ghost columns (periodic x) now; EXTERNAL ghost rows come from the neighbours
  if (s == DVBM_OK && e == cudaSuccess)
    e = launch_ghost(DVBM_D2Q25_SPLIT_II, 0, A.lam[0], c->G, c->P, c->M, c->bc, c->stream);
  if (s == DVBM_OK && e != cudaSuccess) s = fail(c, DVBM_ECUDA, "adjoint_begin: %s", cudaGetErrorString(e));
  if (s != DVBM_OK) {
    adj_release(c, s);
    return s;
  }
  A.active = true;
  A.a = 0;
  A.slot = 1;
  A.j = (n + k - 1) / k - 1;
  A.phase = A.j >= 0 ? AdjRestore : AdjDone;
  A.halo = A.lam[0];
  A.halo_kind = 1;
  return DVBM_OK;
}

extern "C" dvbm_status dvbm_adjoint_advance(dvbm_ctx* c, int* halo) {
  if (!c || !halo) return DVBM_EINVAL;
  auto& A = c->adj;
  if (!A.active) return fail(c, DVBM_ESTATE, "no backward pass begun: call dvbm_adjoint_begin");
  const long long n = c->steps;
  const int k = c->record_every;
  const int nblk = adjoint_blocks(c->G);
  const size_t ncell = (size_t)c->Nx * c->Ny;
  const size_t code_step = (size_t)NPOP * ncell, mom_step = (size_t)13 * ncell, gcode_step = (size_t)2 * NPOP * c->Nx;
  const bool coded = A.codes != nullptr;
  const long long S = A.j * k, E = std::min<long long>((A.j + 1) * k, n);
  cudaError_t e = cudaSuccess;
  switch (A.phase) {
    case AdjRestore:  // the segment's first state from its checkpoint
      e = cudaMemcpyAsync(A.seg[0], c->ckpt[A.j], c->state_bytes_dev, cudaMemcpyDeviceToDevice, c->stream);
      // the adjoint of step t needs the state at t (states 0 .. E-S-1); the
      // coded pass also steps the last one (its step records its codes)
      A.nrec = coded ? E - S : E - S - 1;
      A.t = A.nrec > 0 ? 0 : E - S - 1;
      A.phase = A.nrec > 0 ? AdjRecompute : AdjBackward;
      A.halo = A.seg[0];
      A.halo_kind = 1;
      *halo = 1;
      break;
    case AdjRecompute:  // one forward step of the segment
      if (coded)
        e = launch_step_codes(A.seg[A.t], A.seg[A.t + 1], c->G, c->P, c->flag, A.codes + A.t * code_step,
                              A.moms + A.t * mom_step, c->stream);
      else
        e = launch_step(0, A.seg[A.t], A.seg[A.t + 1], c->G, c->P, c->flag, c->stream);
      if (e == cudaSuccess)
        e = launch_ghost(DVBM_D2Q25_SPLIT_II, 0, A.seg[A.t + 1], c->G, c->P, c->M, c->bc, c->stream);
      A.code_t = A.t;
      ++A.t;
      A.halo = A.seg[A.t];
      A.halo_kind = 1;
      if (coded) {
        A.phase = AdjCodes;  // next: the code rows of the step just taken
      } else if (A.t == A.nrec) {
        A.phase = AdjBackward;  // the adjoint starts at the segment's last state
        A.t = E - S - 1;
      }
      *halo = 1;
      break;
    case AdjCodes:  // no work: the neighbours' code rows of step code_t are exchanged
      A.halo = nullptr;
      A.halo_kind = 3;
      if (A.t == A.nrec) {
        A.phase = AdjBackward;
        A.t = E - S - 1;
      } else {
        A.phase = AdjRecompute;
      }
      *halo = 3;
      break;
    case AdjBackward: {  // one adjoint step back through the state at step S + t
      const int a = A.a;
      const bool band = has_external(c);
      unsigned char* gl = coded && band ? A.gcodes + A.t * gcode_step : nullptr;
      e = launch_adjoint_step((const double*)A.seg[A.t], (const double*)A.lam[a], (double*)A.lam[1 - a],
                              A.part + A.slot * nblk * 4, coded ? A.codes + A.t * code_step : nullptr,
                              coded ? A.moms + A.t * mom_step : nullptr, c->G, c->P, c->stream,
                              gl && c->external[0] ? gl : nullptr,
                              gl && c->external[1] ? gl + (size_t)NPOP * c->Nx : nullptr);
      ++A.slot;
      A.a = 1 - a;
      if (e == cudaSuccess)
        e = launch_ghost(DVBM_D2Q25_SPLIT_II, 0, A.lam[A.a], c->G, c->P, c->M, c->bc, c->stream);
      A.halo = A.lam[A.a];
      A.halo_kind = 1;
      if (A.t == 0) {
        --A.j;
        A.phase = A.j >= 0 ? AdjRestore : AdjDone;
      } else {
        --A.t;
      }
      *halo = 2;
      break;
    }
    default:
      *halo = 0;
      return DVBM_OK;
  }
  if (e != cudaSuccess) {
    const dvbm_status s = fail(c, DVBM_ECUDA, "adjoint_advance: %s", cudaGetErrorString(e));
    adj_release(c, s);
    return s;
  }
  return DVBM_OK;
}

// halo rows of what the last begin / advance produced: a state buffer's two
// rows per side, or the branch-code row per side of step code_t
static dvbm_status adj_halo(dvbm_ctx* c, const void* lo, const void* hi, int unpack) {
  if (!c) return DVBM_EINVAL;
  auto& A = c->adj;
  if (!A.active || !A.halo_kind) return fail(c, DVBM_ESTATE, "no backward pass begun: call dvbm_adjoint_begin");
  if (unpack) {
    const void* in[2] = {lo, hi};
    for (int s = 0; s < 2; ++s) {
      if (c->external[s] && !in[s]) return fail(c, DVBM_EINVAL, "side %s is external: its halo buffer is required", s ? "yhi" : "ylo");
      if (!c->external[s] && in[s]) return fail(c, DVBM_EINVAL, "side %s is not external: pass NULL", s ? "yhi" : "ylo");
    }
  }
  if (!lo && !hi) return DVBM_OK;
  if (A.halo_kind == 3) {
    const size_t gcode_step = (size_t)2 * NPOP * c->Nx;
    unsigned char* g = A.gcodes + A.code_t * gcode_step;
    CUDA_TRY(c, launch_code_rows(A.codes + A.code_t * (size_t)NPOP * c->Nx * c->Ny, (void*)lo, (void*)hi, g,
                                 g + (size_t)NPOP * c->Nx, unpack, c->G, c->stream));
  } else {
    CUDA_TRY(c, launch_halo(8, A.halo, (void*)lo, (void*)hi, unpack, c->G, c->npop, c->stream));
  }
  return DVBM_OK;
}
extern "C" dvbm_status dvbm_adjoint_halo_pack(dvbm_ctx* c, void* lo, void* hi) { return adj_halo(c, lo, hi, 0); }
extern "C" dvbm_status dvbm_adjoint_halo_unpack(dvbm_ctx* c, const void* lo, const void* hi) {
  return adj_halo(c, lo, hi, 1);
}

extern "C" dvbm_status dvbm_adjoint_finish(dvbm_ctx* c, double* g_rho0, double* g_ux0, double* g_uy0, double* g_T0,
                                           double g_params[3]) {
  if (!c) return DVBM_EINVAL;
  auto& A = c->adj;
  if (!A.active) return fail(c, DVBM_ESTATE, "no backward pass begun: call dvbm_adjoint_begin");
  if (A.phase != AdjDone) return fail(c, DVBM_ESTATE, "the backward pass is not complete: call dvbm_adjoint_advance");
  if (!g_rho0 || !g_ux0 || !g_uy0 || !g_T0 || !g_params) return fail(c, DVBM_EINVAL, "null gradient pointer");
  const int nblk = adjoint_blocks(c->G);
  const size_t ncell = (size_t)c->Nx * c->Ny;
  const double* F0 = c->init_fields;
  cudaError_t e = launch_adjoint_init((const double*)A.lam[A.a], F0, F0 + ncell, F0 + 2 * ncell, F0 + 3 * ncell,
                                      g_rho0, g_ux0, g_uy0, g_T0, A.part + A.slot * nblk * 4, c->G, c->P, c->M,
                                      c->stream);
  ++A.slot;
  if (e != cudaSuccess) {
    const dvbm_status s = fail(c, DVBM_ECUDA, "adjoint_finish: %s", cudaGetErrorString(e));
    adj_release(c, s);
    return s;
  }
  std::vector<double> h(A.slot * nblk * 4);
  dvbm_status s = drain_then_copy(c, h.data(), A.part, h.size() * sizeof(double));
  const long long slot = A.slot;
  adj_release(c, s);
  if (s != DVBM_OK) return s;
  params_from_partials(c, h, slot, nblk, g_params);
  return DVBM_OK;
}

extern "C" double dvbm_dt(const dvbm_ctx* c) { return c ? c->dt : 0.0; }
extern "C" long long dvbm_steps_taken(const dvbm_ctx* c) { return c ? c->steps : 0; }
extern "C" const char* dvbm_last_error(const dvbm_ctx* c) { return c ? c->err.c_str() : g_create_error.c_str(); }

extern "C" void dvbm_destroy(dvbm_ctx* c) {
  if (!c) return;
  if (c->stream || c->buf[0]) cudaStreamSynchronize(c->stream);
  if (c->adj.active) adj_release(c, DVBM_OK);  // an unfinished stepwise adjoint: its buffers go to the pool
  for (int k = 0; k < 2; ++k) if (c->buf[k]) cudaFree(c->buf[k]);
  if (c->flag) cudaFree(c->flag);
  if (c->partial) cudaFree(c->partial);
  for (void* p : c->ckpt) cudaFree(p);
  for (void* p : c->pool) cudaFree(p);
  if (c->init_fields) cudaFree(c->init_fields);
  if (c->stage) cudaFree(c->stage);
  for (void* p : c->in_flight) cudaFree(p);
  delete c;
}
