// C ABI of the GB300 porous lattice Boltzmann library (declared in lbmp.h).
//
// Host-side logic only: parameter validation, device buffers, launches,
// CUDA graphs for the step loop, reductions read back in FP64, checkpoints.
// Every compute step runs in the kernels of kernels.cu.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <new>
#include <string>

#include "lbmp.h"
#include "kernels.h"
#include "context.h"
#include "device_scope.h"
#include "nvtx_range.h"

using lbmp::StepArgs;

namespace {
thread_local std::string g_err;
}

void lbmp::set_last_error(const char *msg) { g_err = msg; }

namespace {

lbmp_status fail(lbmp_status st, const char *fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  g_err = buf;
  return st;
}

lbmp_status cuda_fail(cudaError_t e, const char *what) {
  cudaGetLastError();  // clear a sticky-free error so later calls can proceed
  if (e == cudaErrorMemoryAllocation)
    return fail(LBMP_ENOMEM, "%s: %s", what, cudaGetErrorString(e));
  return fail(LBMP_ECUDA, "%s: %s", what, cudaGetErrorString(e));
}

#define LBMP_CK(call)                                        \
  do {                                                       \
    cudaError_t e_ = (call);                                 \
    if (e_ != cudaSuccess) return cuda_fail(e_, #call);      \
  } while (0)

constexpr int kGraphLevels = 6;   // step graphs of 1, 2, 4, ..., 32 steps
constexpr uint64_t kStateMagic = 0x4c424d5053544131ull;  // "LBMPSTA1"

struct StateHeader {
  uint64_t magic;
  int32_t nx, ny, pitch, storage;
  int64_t steps;
  int32_t cur, pad;
  double scale;
  uint64_t payload_bytes;
};

}  // namespace



namespace {

lbmp_status dalloc(lbmp_ctx *c, void **ptr, size_t bytes, const char *what) {
  *ptr = nullptr;
  c->alloc_count++;
  if (c->fault_alloc_at > 0 && c->alloc_count == c->fault_alloc_at)
    return fail(LBMP_ENOMEM, "%s: simulated allocation failure (LBMP_FAULT_ALLOC)", what);
  cudaError_t e = cudaMalloc(ptr, bytes);
  if (e != cudaSuccess) {
    *ptr = nullptr;
    return cuda_fail(e, what);
  }
  c->device_bytes += (int64_t)bytes;
  return LBMP_OK;
}

void free_graphs(lbmp_ctx *c) {
  for (auto &level : c->graph)
    for (auto &g : level)
      if (g) {
        cudaGraphExecDestroy(g);
        g = nullptr;
      }
}

void release(lbmp_ctx *c) {
  if (!c) return;
  const DeviceScope device_scope(c->device);
  if (c->stream) cudaStreamSynchronize(c->stream);
  free_graphs(c);
  cudaFree(c->buf[0]);
  cudaFree(c->buf[1]);
  cudaFree(c->med);
  cudaFree(c->kn0);
  cudaFree(c->uprev);
  cudaFree(c->partials);
  cudaFree(c->results);
  cudaFree(c->d_flag);
  cudaFree(c->d_tctr);
  cudaFree(c->d_err);
  cudaFree(c->d_hist);
  if (c->h_results) cudaFreeHost(c->h_results);
  if (c->cap_stream) cudaStreamDestroy(c->cap_stream);
  if (c->own_stream && c->stream) cudaStreamDestroy(c->stream);
  delete c;
}

lbmp_status scope_status(const DeviceScope &d) {
  return d.err == cudaSuccess ? LBMP_OK : cuda_fail(d.err, "cudaSetDevice");
}

// Device scratch for caller pointers that live on the host.
struct DevTemp {
  void *ptr = nullptr;
  ~DevTemp() {
    if (ptr) cudaFree(ptr);
  }
};

// The flag of the bounded waits (synchronous read).
lbmp_status check_err(lbmp_ctx *c) {
  unsigned e = 0;
  LBMP_CK(cudaMemcpyAsync(&e, c->d_err, sizeof(e), cudaMemcpyDeviceToHost, c->stream));
  LBMP_CK(cudaStreamSynchronize(c->stream));
  if (e) return fail(LBMP_ETIMEOUT, "a bounded wait of the staged step kernel gave up");
  return LBMP_OK;
}

// Run the macroscopic/reduction kernel and, when partials are requested,
// reduce them into c->h_results (synchronous).
lbmp_status run_macro(lbmp_ctx *c, lbmp::MacroOut o, bool reduce) {
  StepArgs a = c->args();
  a.y0 = 0;
  if (reduce) o.partials = c->partials;
  LBMP_CK(lbmp::launch_macro(c->p.storage, a, c->buf[c->cur], c->med, o, c->stream));
  c->launches++;
  if (reduce) {
    LBMP_CK(lbmp::launch_finalize(c->partials, lbmp::macro_blocks(a), lbmp::kNQ,
                                  c->results, c->stream));
    c->launches++;
    LBMP_CK(cudaMemcpyAsync(c->h_results, c->results, sizeof(double) * lbmp::kNQ,
                            cudaMemcpyDeviceToHost, c->stream));
  }
  LBMP_CK(cudaStreamSynchronize(c->stream));
  lbmp_status st = check_err(c);
  if (st) return st;
  if (reduce && c->h_results[5] != 0.0)
    return fail(LBMP_ENAN, "%.0f fluid nodes have a non-finite density or velocity",
                c->h_results[5]);
  return LBMP_OK;
}

// One step kernel launch (the variant the context selected).  Steps that
// read buffer 1 walk the lattice from the end, so each step starts on the
// nodes the previous one wrote last.
cudaError_t launch_one(lbmp_ctx *c, const StepArgs &a0, const void *fin, void *fout, int k,
                       cudaStream_t s) {
  StepArgs a = a0;
  a.rev = fin == c->buf[1];
  if (c->wide) return lbmp::launch_wide(c->sr, a, c->rows(), fin, fout, c->med, c->d_tctr, k, s);
  if (c->staged)
    return lbmp::launch_staged(c->p.storage, c->sr, a, c->rows(), fin, fout, c->med, c->d_tctr,
                               k, c->d_err, c->nsm, s);
  return lbmp::launch_step(c->p.storage, c->sr, a, c->rows(), fin, fout, c->med, c->d_tctr, k, s);
}

// Graph of 2^level steps starting from buffer `cur` (captured once per
// medium: the launch arguments hold the storage scale), plus the counter
// bump when the rounding is stochastic.  A replay saves the launch gaps of
// single launches (~3 us per step at 4096^2).
lbmp_status get_graph(lbmp_ctx *c, int level, int cur, cudaGraphExec_t *out) {
  if (c->graph[level][cur]) {
    *out = c->graph[level][cur];
    return LBMP_OK;
  }
  const int nsteps = 1 << level;
  StepArgs a = c->args();
  cudaGraph_t g = nullptr;
  LBMP_CK(cudaStreamBeginCapture(c->cap_stream, cudaStreamCaptureModeThreadLocal));
  int b = cur;
  cudaError_t err = cudaSuccess;
  for (int t = 0; t < nsteps && err == cudaSuccess; ++t) {
    err = launch_one(c, a, c->buf[b], c->buf[b ^ 1], t, c->cap_stream);
    b ^= 1;
  }
  if (err == cudaSuccess && c->sr) err = lbmp::launch_bump(c->d_tctr, nsteps, c->cap_stream);
  cudaError_t end = cudaStreamEndCapture(c->cap_stream, &g);
  if (err != cudaSuccess) {
    if (g) cudaGraphDestroy(g);
    return cuda_fail(err, "graph capture of the step loop");
  }
  if (end != cudaSuccess) return cuda_fail(end, "cudaStreamEndCapture");
  cudaGraphExec_t exec = nullptr;
  cudaError_t ie = cudaGraphInstantiate(&exec, g, 0);
  cudaGraphDestroy(g);
  if (ie != cudaSuccess) return cuda_fail(ie, "cudaGraphInstantiate");
  c->graph[level][cur] = exec;
  *out = exec;
  return LBMP_OK;
}

bool valid_where(int32_t w) { return w == LBMP_HOST || w == LBMP_DEVICE; }

// The device address of a pinned, device-mapped host array, if it is one.
bool mapped_host(const double *p, const double **dev) {
  cudaPointerAttributes at{};
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  if (at.type != cudaMemoryTypeHost || !at.devicePointer) return false;
  *dev = static_cast<const double *>(at.devicePointer);
  return true;
}

}  // namespace

lbmp_status lbmp::validate_params(lbmp_params *p) {
    if (p->J == 0.0) p->J = 1.0;
    if (p->rho0 == 0.0) p->rho0 = 1.0;
    if (p->nx < 1 || p->ny < 1) return fail(LBMP_EINVAL, "nx, ny must be >= 1 (got %d x %d)", p->nx, p->ny);
    if (p->nx > (1 << 30)) return fail(LBMP_EINVAL, "nx must be <= 2^30");
    if (p->ny > 65535) return fail(LBMP_EINVAL, "ny must be <= 65535");
    if (!(p->tau > 0.5) || !std::isfinite(p->tau)) return fail(LBMP_EINVAL, "tau must be > 0.5 (got %g)", p->tau);
    if (!(p->J > 0.0) || !std::isfinite(p->J)) return fail(LBMP_EINVAL, "J must be > 0");
    if (!std::isfinite(p->Gx) || !std::isfinite(p->Gy)) return fail(LBMP_EINVAL, "G must be finite");
    if (!(p->rho0 > 0.0) || !std::isfinite(p->rho0)) return fail(LBMP_EINVAL, "rho0 must be > 0");
    if (p->bc_x != LBMP_BCX_PERIODIC && p->bc_x != LBMP_BCX_PRESSURE)
      return fail(LBMP_EINVAL, "bc_x must be LBMP_BCX_PERIODIC or LBMP_BCX_PRESSURE");
    if (p->bc_y != LBMP_BCY_PERIODIC && p->bc_y != LBMP_BCY_WALLS)
      return fail(LBMP_EINVAL, "bc_y must be LBMP_BCY_PERIODIC or LBMP_BCY_WALLS");
    if (p->bc_x == LBMP_BCX_PRESSURE) {
      if (p->nx < 3) return fail(LBMP_EINVAL, "pressure columns need nx >= 3");
      if (!(p->rho_in > 0.0) || !(p->rho_out > 0.0) || !std::isfinite(p->rho_in) ||
          !std::isfinite(p->rho_out))
        return fail(LBMP_EINVAL, "rho_in and rho_out must be finite and > 0");
    }
    if (p->bc_y == LBMP_BCY_WALLS && p->ny < 3) return fail(LBMP_EINVAL, "walls need ny >= 3");
    if (p->forchheimer != 0 && p->forchheimer != 1) return fail(LBMP_EINVAL, "forchheimer must be 0 or 1");
    if (p->storage != LBMP_STORE_FP32 && p->storage != LBMP_STORE_FP16)
      return fail(LBMP_EINVAL, "storage must be LBMP_STORE_FP32 or LBMP_STORE_FP16");
    if (p->fp16_log2_scale < -60 || p->fp16_log2_scale > 60)
      return fail(LBMP_EINVAL, "fp16_log2_scale must be in [-60, 60]");
    if (p->kernel != LBMP_KERNEL_AUTO && p->kernel != LBMP_KERNEL_STAGED &&
        p->kernel != LBMP_KERNEL_DIRECT && p->kernel != LBMP_KERNEL_WIDE)
      return fail(LBMP_EINVAL, "kernel must be LBMP_KERNEL_AUTO, _STAGED, _DIRECT or _WIDE");
    if (p->kernel == LBMP_KERNEL_WIDE && p->storage != LBMP_STORE_FP16)
      return fail(LBMP_EINVAL, "the wide kernel needs FP16 storage");
    if (p->kn_model != LBMP_KN_BKC && p->kn_model != LBMP_KN_FIRST_ORDER)
      return fail(LBMP_EINVAL, "kn_model must be LBMP_KN_BKC or LBMP_KN_FIRST_ORDER");
    if (!std::isfinite(p->kn_beta)) return fail(LBMP_EINVAL, "kn_beta must be finite");
    if (p->kn_beta != 0.0) {
      if (p->kernel == LBMP_KERNEL_STAGED && p->storage != LBMP_STORE_FP16)
        return fail(LBMP_EINVAL,
                    "a dynamic Kn (kn_beta != 0) with FP32 storage needs the direct kernel");
      if (p->bc_x == LBMP_BCX_PRESSURE &&
          !(1.0 + p->kn_beta * (p->rho_in - p->rho0) > 0.0 &&
            1.0 + p->kn_beta * (p->rho_out - p->rho0) > 0.0))
        return fail(LBMP_EINVAL, "kn_beta gives a non-positive pressure at rho_in or rho_out");
    }
    if (p->fp16_rounding != LBMP_ROUND_STOCHASTIC && p->fp16_rounding != LBMP_ROUND_NEAREST)
      return fail(LBMP_EINVAL, "fp16_rounding must be LBMP_ROUND_STOCHASTIC or LBMP_ROUND_NEAREST");

  return LBMP_OK;
}

extern "C" {

const char *lbmp_last_error(void) { return g_err.c_str(); }

double lbmp_fc(double kn) {
  if (!(kn >= 0.0)) return NAN;
  return lbmp::fc_bkc(kn);
}

double lbmp_fc_model(int32_t kn_model, double kn) {
  if (!(kn >= 0.0) || (kn_model != LBMP_KN_BKC && kn_model != LBMP_KN_FIRST_ORDER)) return NAN;
  return lbmp::fc_model(kn, kn_model);
}

double lbmp_kozeny_carman(double eps, double d) {
  if (!(eps >= 0.0 && eps < 1.0) || !(d >= 0.0)) return NAN;
  return d * d / 180.0 * eps * eps * eps / ((1.0 - eps) * (1.0 - eps));
}

double lbmp_mean_free_path(double mu, double p, double T, double M) {
  if (!(mu > 0.0 && p > 0.0 && T > 0.0 && M > 0.0)) return NAN;
  const double R = 8.314462618;  // J / (mol K)
  return (mu / p) * std::sqrt(M_PI * R * T / (2.0 * M));
}

double lbmp_pore_radius(double k_d, double eps) {
  if (!(k_d >= 0.0) || !(eps > 0.0)) return NAN;
  const double mD = 9.869e-16;   // m^2
  return 8.886e-2 * std::sqrt(k_d / mD / eps) * 1e-6;
}

lbmp_status lbmp_physical_medium(int64_t n, const double *eps, const double *d, double lambda,
                                 double dx, double *k_i, double *kn) {
  if (n < 0 || (n > 0 && (!eps || !d || !k_i || !kn)))
    return fail(LBMP_EINVAL, "lbmp_physical_medium: NULL argument or n < 0");
  if (!(lambda >= 0.0) || !(dx > 0.0) || !std::isfinite(lambda) || !std::isfinite(dx))
    return fail(LBMP_EINVAL, "lbmp_physical_medium: lambda must be >= 0 and dx > 0");
  for (int64_t i = 0; i < n; ++i) {
    const double e = eps[i];
    if (!(e >= 0.0 && e <= 1.0))
      return fail(LBMP_EINVAL, "lbmp_physical_medium: eps[%lld] outside [0, 1]", (long long)i);
    if (e == 0.0) {  // impermeable: k_i unused
      k_i[i] = 1.0;
      kn[i] = 0.0;
      continue;
    }
    if (e == 1.0) {  // open pore: no medium, no slip correction
      k_i[i] = INFINITY;
      kn[i] = 0.0;
      continue;
    }
    if (!(d[i] > 0.0) || !std::isfinite(d[i]))
      return fail(LBMP_EINVAL, "lbmp_physical_medium: d[%lld] must be > 0", (long long)i);
    const double kd = lbmp_kozeny_carman(e, d[i]);  // Eq. 9
    k_i[i] = kd / (dx * dx);
    kn[i] = lambda / lbmp_pore_radius(kd, e);       // Eq. 10-11: Kn = lambda / r
  }
  return LBMP_OK;
}

lbmp_status lbmp_create(const lbmp_params *pin, lbmp_ctx **out) {
  const lbmp::NvtxRange nvtx_range("lbmp_create");
  try {
    if (!pin || !out) return fail(LBMP_EINVAL, "lbmp_create: NULL argument");
    *out = nullptr;
    lbmp_params p = *pin;
    lbmp_status vst = lbmp::validate_params(&p);
    if (vst) return vst;

    lbmp_ctx *c = new (std::nothrow) lbmp_ctx();
    if (!c) return fail(LBMP_ENOMEM, "host allocation of the context");
    c->p = p;
    if (const char *f = std::getenv("LBMP_FAULT_ALLOC")) c->fault_alloc_at = std::atoi(f);
    if (const char *f = std::getenv("LBMP_TEST_DROP_TILE")) c->drop_tile = std::atoi(f);
    cudaError_t e = cudaGetDevice(&c->device);
    if (e != cudaSuccess) {
      delete c;
      return cuda_fail(e, "cudaGetDevice");
    }
    c->elem = (p.storage == LBMP_STORE_FP32) ? 4 : 2;
    c->sr = p.storage == LBMP_STORE_FP16 && p.fp16_rounding == LBMP_ROUND_STOCHASTIC;
    // FP32: the direct kernel already saturates HBM (the staged one reaches
    // ~0.95 of it); FP16 (static or dynamic Kn): the staged kernel issues
    // fewer instructions per node.
    c->staged = p.kernel == LBMP_KERNEL_STAGED ||
                (p.kernel == LBMP_KERNEL_AUTO && p.storage == LBMP_STORE_FP16);
    c->wide = p.kernel == LBMP_KERNEL_WIDE;
    e = cudaDeviceGetAttribute(&c->nsm, cudaDevAttrMultiProcessorCount, c->device);
    if (e != cudaSuccess) {
      delete c;
      return cuda_fail(e, "cudaDeviceGetAttribute(multiProcessorCount)");
    }
    e = lbmp::prepare_staged();
    if (e != cudaSuccess) {
      delete c;
      return cuda_fail(e, "shared-memory limit of the staged kernel");
    }
    c->pitch = lbmp::row_pitch(p.nx);
    c->plane = (long long)c->pitch * p.ny;
    c->y_lo = (p.bc_y == LBMP_BCY_WALLS) ? 1 : 0;
    c->y_hi = (p.bc_y == LBMP_BCY_WALLS) ? p.ny - 1 : p.ny;
    c->fluid_nodes = (int64_t)p.nx * (c->y_hi - c->y_lo);
    lbmp_status st = LBMP_OK;
#define LBMP_TRY(x)     \
  do {                  \
    st = (x);           \
    if (st != LBMP_OK) { \
      release(c);       \
      return st;        \
    }                   \
  } while (0)
    if (p.stream) {
      c->stream = (cudaStream_t)p.stream;
    } else {
      e = cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking);
      if (e != cudaSuccess) LBMP_TRY(cuda_fail(e, "cudaStreamCreate"));
      c->own_stream = true;
    }
    e = cudaStreamCreateWithFlags(&c->cap_stream, cudaStreamNonBlocking);
    if (e != cudaSuccess) LBMP_TRY(cuda_fail(e, "cudaStreamCreate (capture)"));
    StepArgs a = c->args();
    a.y0 = 0;
    c->partials_blocks = std::max({lbmp::macro_blocks(a), lbmp::hist_blocks(a),
                                   lbmp::medium_blocks(p.nx, p.ny)});
    LBMP_TRY(dalloc(c, &c->buf[0], c->buf_bytes(), "population buffer A"));
    LBMP_TRY(dalloc(c, &c->buf[1], c->buf_bytes(), "population buffer B"));
    LBMP_TRY(dalloc(c, (void **)&c->med, (size_t)c->plane * sizeof(float2), "medium"));
    if (p.kn_beta != 0.0)
      LBMP_TRY(dalloc(c, (void **)&c->kn0, (size_t)c->plane * sizeof(float), "Kn at p0"));
    LBMP_TRY(dalloc(c, (void **)&c->uprev, (size_t)c->plane * sizeof(float2), "velocity snapshot"));
    LBMP_TRY(dalloc(c, (void **)&c->partials,
                    (size_t)c->partials_blocks * lbmp::kNQ * sizeof(double), "reduction partials"));
    LBMP_TRY(dalloc(c, (void **)&c->results, lbmp::kNQ * sizeof(double), "reduction results"));
    LBMP_TRY(dalloc(c, (void **)&c->d_flag, sizeof(unsigned), "validation flag"));
    LBMP_TRY(dalloc(c, (void **)&c->d_tctr, sizeof(unsigned long long), "time-level counter"));
    LBMP_TRY(dalloc(c, (void **)&c->d_err, sizeof(unsigned), "wait error flag"));
    e = cudaMemset(c->d_err, 0, sizeof(unsigned));
    if (e != cudaSuccess) LBMP_TRY(cuda_fail(e, "cudaMemset"));
    e = cudaMallocHost((void **)&c->h_results, lbmp::kNQ * sizeof(double));
    if (e != cudaSuccess) LBMP_TRY(cuda_fail(e, "cudaMallocHost"));
#undef LBMP_TRY
    *out = c;
    return LBMP_OK;
  } catch (...) {
    return fail(LBMP_ECUDA, "lbmp_create: unexpected exception");
  }
}

lbmp_status lbmp_destroy(lbmp_ctx *c) {
  const lbmp::NvtxRange nvtx_range("lbmp_destroy");
  try {
    release(c);
    return LBMP_OK;
  } catch (...) {
    return fail(LBMP_ECUDA, "lbmp_destroy: unexpected exception");
  }
}

lbmp_status lbmp_set_fields(lbmp_ctx *c, const double *eps, const double *k_i,
                            const double *kn, int32_t where) {
  const lbmp::NvtxRange nvtx_range("lbmp_set_fields");
  try {
    if (!c || !eps || !k_i || !kn) return fail(LBMP_EINVAL, "lbmp_set_fields: NULL argument");
    if (!valid_where(where)) return fail(LBMP_EINVAL, "where must be LBMP_HOST or LBMP_DEVICE");
    const DeviceScope device_scope(c->device);
    lbmp_status st = scope_status(device_scope);
    if (st) return st;
    const lbmp_params &p = c->p;
    const size_t n = (size_t)p.nx * p.ny;
    const double *de = eps, *dk = k_i, *dn = kn;
    DevTemp tmp;
    // Host arrays in pinned, device-mapped memory are read by the kernel in
    // place (over the CPU-GPU link); other host memory is staged.
    if (where == LBMP_HOST && mapped_host(eps, &de) && mapped_host(k_i, &dk) &&
        mapped_host(kn, &dn))
      where = LBMP_DEVICE;
    if (where == LBMP_HOST) {
      de = eps;
      dk = k_i;
      dn = kn;
      cudaError_t e = cudaMalloc(&tmp.ptr, 3 * n * sizeof(double));
      if (e != cudaSuccess) return cuda_fail(e, "staging buffer for the medium");
      double *t = (double *)tmp.ptr;
      LBMP_CK(cudaMemcpyAsync(t, eps, n * sizeof(double), cudaMemcpyHostToDevice, c->stream));
      LBMP_CK(cudaMemcpyAsync(t + n, k_i, n * sizeof(double), cudaMemcpyHostToDevice, c->stream));
      LBMP_CK(cudaMemcpyAsync(t + 2 * n, kn, n * sizeof(double), cudaMemcpyHostToDevice, c->stream));
      de = t;
      dk = t + n;
      dn = t + 2 * n;
    }
    LBMP_CK(cudaMemsetAsync(c->d_flag, 0, sizeof(unsigned), c->stream));
    LBMP_CK(cudaMemsetAsync(c->med, 0, (size_t)c->plane * sizeof(float2), c->stream));
    // with a dynamic Kn the largest k_a (FP16 scale) is that at the lowest
    // imposed pressure
    double kn_scale_max = 1.0;
    if (c->kn0) {
      LBMP_CK(cudaMemsetAsync(c->kn0, 0, (size_t)c->plane * sizeof(float), c->stream));
      double qmin = 1.0;
      if (p.bc_x == LBMP_BCX_PRESSURE)
        qmin = std::min({1.0, 1.0 + p.kn_beta * (p.rho_in - p.rho0),
                         1.0 + p.kn_beta * (p.rho_out - p.rho0)});
      kn_scale_max = 1.0 / qmin;
    }
    LBMP_CK(lbmp::launch_medium(de, dk, dn, p.nx, p.ny, c->pitch, c->y_lo, c->y_hi, p.kn_model,
                                c->kn0, kn_scale_max, c->med, c->d_flag, c->partials,
                                c->stream));
    c->launches++;
    LBMP_CK(lbmp::launch_finalize(c->partials, lbmp::medium_blocks(p.nx, p.ny), lbmp::kNQ,
                                  c->results, c->stream, lbmp::kMediumMaxMask));
    c->launches++;
    unsigned flag = 0;
    LBMP_CK(cudaMemcpyAsync(c->h_results, c->results, lbmp::kNQ * sizeof(double),
                            cudaMemcpyDeviceToHost, c->stream));
    LBMP_CK(cudaMemcpyAsync(&flag, c->d_flag, sizeof(unsigned), cudaMemcpyDeviceToHost,
                            c->stream));
    LBMP_CK(cudaStreamSynchronize(c->stream));
    if (flag) {
      c->fields_set = false;
      return fail(LBMP_EINVAL,
                  "lbmp_set_fields: invalid values (%s%s%s%s); the context needs new fields",
                  (flag & 1u) ? "eps outside [0,1] " : "", (flag & 2u) ? "k_i not > 0 " : "",
                  (flag & 4u) ? "Kn negative or not finite " : "",
                  (flag & 8u) ? "k_a below 1e-15" : "");
    }
    c->eps_mean = c->h_results[0] / c->h_results[1];
    // storage scale S = 2^s for FP16: keep the expected largest deviation
    // near 2^10, far from both the FP16 overflow and its subnormal range.
    // Velocity bound: the Darcy speed |G| max(k_a) / nu of the porous nodes,
    // the Poiseuille speed |G| L^2 / (8 nu) if open pores exist, and at most
    // 0.1 (beyond it the lattice leaves its low-Mach range anyway).
    if (p.storage == LBMP_STORE_FP16) {
      int s = p.fp16_log2_scale;
      if (s == 0) {
        double dev = 0.0;
        if (p.bc_x == LBMP_BCX_PRESSURE)
          dev = std::max(std::fabs(p.rho_in - p.rho0), std::fabs(p.rho_out - p.rho0));
        const double nu = (p.tau - 0.5) / 3.0 / p.J;
        const double g = std::sqrt(p.Gx * p.Gx + p.Gy * p.Gy);
        const double kmax = c->h_results[2];
        const bool open = c->h_results[3] > 0.0;
        const double L = (p.bc_y == LBMP_BCY_WALLS) ? (double)(p.ny - 2)
                                                    : (double)std::min(p.nx, p.ny);
        double u = g * kmax / nu;
        if (open) u = std::max(u, g * L * L / (8.0 * nu));
        u = std::min(u, 0.1);
        dev = std::max(dev, 3.0 * p.rho0 * u);
        dev = std::max(dev, 1e-7);
        s = (int)std::floor(std::log2(1024.0 / dev));
        s = std::min(60, std::max(-60, s));
      }
      const double scale = std::ldexp(1.0, s);
      if (scale != c->scale) free_graphs(c);  // the graphs' step arguments hold S
      c->scale = scale;
    } else {
      c->scale = 1.0;
    }
    LBMP_CK(cudaMemsetAsync(c->buf[0], 0, c->buf_bytes(), c->stream));
    LBMP_CK(cudaMemsetAsync(c->buf[1], 0, c->buf_bytes(), c->stream));
    LBMP_CK(cudaMemsetAsync(c->uprev, 0, (size_t)c->plane * sizeof(float2), c->stream));
    LBMP_CK(cudaMemsetAsync(c->d_tctr, 0, sizeof(unsigned long long), c->stream));
    LBMP_CK(cudaMemsetAsync(c->d_err, 0, sizeof(unsigned), c->stream));
    LBMP_CK(cudaStreamSynchronize(c->stream));
    c->cur = 0;
    c->steps = 0;
    c->fields_set = true;
    return LBMP_OK;
  } catch (...) {
    return fail(LBMP_ECUDA, "lbmp_set_fields: unexpected exception");
  }
}

lbmp_status lbmp_step(lbmp_ctx *c, int64_t n) {
  const lbmp::NvtxRange nvtx_range("lbmp_step");
  try {
    if (!c) return fail(LBMP_EINVAL, "lbmp_step: NULL context");
    if (n < 0) return fail(LBMP_EINVAL, "lbmp_step: n must be >= 0");
    if (!c->fields_set) return fail(LBMP_ESTATE, "lbmp_step: call lbmp_set_fields first");
    if (n == 0) return LBMP_OK;
    const DeviceScope device_scope(c->device);
    lbmp_status st = scope_status(device_scope);
    if (st) return st;
    // n = 32 q + sum of binary digits: q replays of the 32-step graph, then
    // one replay of each smaller power of two
    int64_t left = n;
    for (int level = kGraphLevels - 1; level >= 0 && left > 0; --level) {
      const int64_t size = 1ll << level;
      while (left >= size) {
        cudaGraphExec_t g = nullptr;
        st = get_graph(c, level, c->cur, &g);
        if (st) return st;
        LBMP_CK(cudaGraphLaunch(g, c->stream));
        c->launches += size + (c->sr ? 1 : 0);
        if (size & 1) c->cur ^= 1;  // an odd replay swaps the buffers
        left -= size;
        if (level < kGraphLevels - 1) break;  // one replay of each smaller size
      }
    }
    c->steps += n;
    return LBMP_OK;
  } catch (...) {
    return fail(LBMP_ECUDA, "lbmp_step: unexpected exception");
  }
}

lbmp_status lbmp_synchronize(lbmp_ctx *c) {
  const lbmp::NvtxRange nvtx_range("lbmp_synchronize");
  if (!c) return fail(LBMP_EINVAL, "lbmp_synchronize: NULL context");
  const DeviceScope device_scope(c->device);
  lbmp_status st = scope_status(device_scope);
  if (st) return st;
  LBMP_CK(cudaStreamSynchronize(c->stream));
  return check_err(c);
}

lbmp_status lbmp_macroscopic(lbmp_ctx *c, double *rho, double *ux, double *uy,
                             int32_t where) {
  const lbmp::NvtxRange nvtx_range("lbmp_macroscopic");
  try {
    if (!c) return fail(LBMP_EINVAL, "lbmp_macroscopic: NULL context");
    if (!valid_where(where)) return fail(LBMP_EINVAL, "where must be LBMP_HOST or LBMP_DEVICE");
    if (!c->fields_set) return fail(LBMP_ESTATE, "lbmp_macroscopic: no fields set");
    const DeviceScope device_scope(c->device);
    lbmp_status st = scope_status(device_scope);
    if (st) return st;
    const size_t n = (size_t)c->p.nx * c->p.ny;
    lbmp::MacroOut o{};
    DevTemp tmp;
    if (where == LBMP_HOST) {
      cudaError_t e = cudaMalloc(&tmp.ptr, 3 * n * sizeof(double));
      if (e != cudaSuccess) return cuda_fail(e, "staging buffer");
      double *t = (double *)tmp.ptr;
      o.rho = rho ? t : nullptr;
      o.ux = ux ? t + n : nullptr;
      o.uy = uy ? t + 2 * n : nullptr;
    } else {
      o.rho = rho;
      o.ux = ux;
      o.uy = uy;
    }
    st = run_macro(c, o, false);
    if (st) return st;
    if (where == LBMP_HOST) {
      double *t = (double *)tmp.ptr;
      if (rho) LBMP_CK(cudaMemcpy(rho, t, n * sizeof(double), cudaMemcpyDeviceToHost));
      if (ux) LBMP_CK(cudaMemcpy(ux, t + n, n * sizeof(double), cudaMemcpyDeviceToHost));
      if (uy) LBMP_CK(cudaMemcpy(uy, t + 2 * n, n * sizeof(double), cudaMemcpyDeviceToHost));
    }
    return LBMP_OK;
  } catch (...) {
    return fail(LBMP_ECUDA, "lbmp_macroscopic: unexpected exception");
  }
}

lbmp_status lbmp_apparent_permeability(lbmp_ctx *c, double *ka, int32_t where) {
  const lbmp::NvtxRange nvtx_range("lbmp_apparent_permeability");
  try {
    if (!c || !ka) return fail(LBMP_EINVAL, "lbmp_apparent_permeability: NULL argument");
    if (!valid_where(where)) return fail(LBMP_EINVAL, "where must be LBMP_HOST or LBMP_DEVICE");
    if (!c->fields_set) return fail(LBMP_ESTATE, "lbmp_apparent_permeability: no fields set");
    const DeviceScope device_scope(c->device);
    lbmp_status st = scope_status(device_scope);
    if (st) return st;
    const size_t n = (size_t)c->p.nx * c->p.ny;
    DevTemp tmp;
    double *out = ka;
    if (where == LBMP_HOST) {
      cudaError_t e = cudaMalloc(&tmp.ptr, n * sizeof(double));
      if (e != cudaSuccess) return cuda_fail(e, "staging buffer");
      out = (double *)tmp.ptr;
    }
    LBMP_CK(lbmp::launch_ka(c->med, c->kn0, c->p.nx, c->p.ny, c->pitch, c->y_lo, c->y_hi,
                            c->p.kn_model, out, c->stream));
    c->launches++;
    if (where == LBMP_HOST)
      LBMP_CK(cudaMemcpyAsync(ka, out, n * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    LBMP_CK(cudaStreamSynchronize(c->stream));
    return LBMP_OK;
  } catch (...) {
    return fail(LBMP_ECUDA, "lbmp_apparent_permeability: unexpected exception");
  }
}

lbmp_status lbmp_populations(lbmp_ctx *c, double *f, int32_t where) {
  const lbmp::NvtxRange nvtx_range("lbmp_populations");
  try {
    if (!c || !f) return fail(LBMP_EINVAL, "lbmp_populations: NULL argument");
    if (!valid_where(where)) return fail(LBMP_EINVAL, "where must be LBMP_HOST or LBMP_DEVICE");
    if (!c->fields_set) return fail(LBMP_ESTATE, "lbmp_populations: no fields set");
    const DeviceScope device_scope(c->device);
    lbmp_status st = scope_status(device_scope);
    if (st) return st;
    const size_t n = (size_t)c->p.nx * c->p.ny * 9;
    lbmp::MacroOut o{};
    DevTemp tmp;
    if (where == LBMP_HOST) {
      cudaError_t e = cudaMalloc(&tmp.ptr, n * sizeof(double));
      if (e != cudaSuccess) return cuda_fail(e, "staging buffer");
      o.pops = (double *)tmp.ptr;
    } else {
      o.pops = f;
    }
    st = run_macro(c, o, false);
    if (st) return st;
    if (where == LBMP_HOST)
      LBMP_CK(cudaMemcpy(f, tmp.ptr, n * sizeof(double), cudaMemcpyDeviceToHost));
    return LBMP_OK;
  } catch (...) {
    return fail(LBMP_ECUDA, "lbmp_populations: unexpected exception");
  }
}

lbmp_status lbmp_set_populations(lbmp_ctx *c, const double *f, int32_t where) {
  const lbmp::NvtxRange nvtx_range("lbmp_set_populations");
  try {
    if (!c || !f) return fail(LBMP_EINVAL, "lbmp_set_populations: NULL argument");
    if (!valid_where(where)) return fail(LBMP_EINVAL, "where must be LBMP_HOST or LBMP_DEVICE");
    if (!c->fields_set) return fail(LBMP_ESTATE, "lbmp_set_populations: no fields set");
    const DeviceScope device_scope(c->device);
    lbmp_status st = scope_status(device_scope);
    if (st) return st;
    const size_t n = (size_t)c->p.nx * c->p.ny * 9;
    const double *src = f;
    DevTemp tmp;
    if (where == LBMP_HOST) {
      cudaError_t e = cudaMalloc(&tmp.ptr, n * sizeof(double));
      if (e != cudaSuccess) return cuda_fail(e, "staging buffer");
      LBMP_CK(cudaMemcpyAsync(tmp.ptr, f, n * sizeof(double), cudaMemcpyHostToDevice, c->stream));
      src = (const double *)tmp.ptr;
    }
    StepArgs a = c->args();
    LBMP_CK(lbmp::launch_load_pops(c->p.storage, a, c->rows(), src, c->buf[c->cur], c->stream));
    c->launches++;
    LBMP_CK(cudaStreamSynchronize(c->stream));
    return LBMP_OK;
  } catch (...) {
    return fail(LBMP_ECUDA, "lbmp_set_populations: unexpected exception");
  }
}

lbmp_status lbmp_permeability(lbmp_ctx *c, double *k_g, double *u_mean) {
  const lbmp::NvtxRange nvtx_range("lbmp_permeability");
  try {
    if (!c) return fail(LBMP_EINVAL, "lbmp_permeability: NULL context");
    if (!c->fields_set) return fail(LBMP_ESTATE, "lbmp_permeability: no fields set");
    const DeviceScope device_scope(c->device);
    lbmp_status st = scope_status(device_scope);
    if (st) return st;
    lbmp::MacroOut o{};
    st = run_macro(c, o, true);
    if (st) return st;
    const lbmp_params &p = c->p;
    const double um = c->h_results[0] / (double)c->fluid_nodes;
    double g = p.Gx;
    if (p.bc_x == LBMP_BCX_PRESSURE)
      g += (p.rho_in - p.rho_out) / 3.0 / c->eps_mean / (p.rho0 * (double)(p.nx - 1));
    const double nu = (p.tau - 0.5) / 3.0 / p.J;
    if (u_mean) *u_mean = um;
    if (k_g) *k_g = nu * um / g;
    return LBMP_OK;
  } catch (...) {
    return fail(LBMP_ECUDA, "lbmp_permeability: unexpected exception");
  }
}

lbmp_status lbmp_velocity_histogram(lbmp_ctx *c, int32_t nbins, double *umax,
                                    int64_t *counts) {
  const lbmp::NvtxRange nvtx_range("lbmp_velocity_histogram");
  try {
    if (!c || !counts) return fail(LBMP_EINVAL, "lbmp_velocity_histogram: NULL argument");
    if (nbins < 1 || nbins > lbmp::kMaxHistBins)
      return fail(LBMP_EINVAL, "nbins must be in [1, %d]", lbmp::kMaxHistBins);
    if (!c->fields_set) return fail(LBMP_ESTATE, "lbmp_velocity_histogram: no fields set");
    const DeviceScope device_scope(c->device);
    lbmp_status st = scope_status(device_scope);
    if (st) return st;
    if (!c->d_hist) {
      st = dalloc(c, (void **)&c->d_hist, lbmp::kMaxHistBins * sizeof(unsigned long long),
                  "histogram counts");
      if (st) return st;
    }
    StepArgs a = c->args();
    a.y0 = 0;
    LBMP_CK(lbmp::launch_speed_max(c->p.storage, a, c->buf[c->cur], c->med, c->partials,
                                   c->stream));
    LBMP_CK(lbmp::launch_finalize(c->partials, lbmp::hist_blocks(a), 1, c->results, c->stream,
                                  1u));
    LBMP_CK(cudaMemcpyAsync(c->h_results, c->results, sizeof(double), cudaMemcpyDeviceToHost,
                            c->stream));
    LBMP_CK(cudaStreamSynchronize(c->stream));
    const double um = c->h_results[0];
    if (!std::isfinite(um)) return fail(LBMP_ENAN, "a fluid node has a non-finite velocity");
    LBMP_CK(cudaMemsetAsync(c->d_hist, 0, lbmp::kMaxHistBins * sizeof(unsigned long long),
                            c->stream));
    LBMP_CK(lbmp::launch_histogram(c->p.storage, a, c->buf[c->cur], c->med, um, nbins, c->d_hist,
                                   c->stream));
    c->launches += 3;
    unsigned long long h[lbmp::kMaxHistBins];
    LBMP_CK(cudaMemcpyAsync(h, c->d_hist, (size_t)nbins * sizeof(unsigned long long),
                            cudaMemcpyDeviceToHost, c->stream));
    LBMP_CK(cudaStreamSynchronize(c->stream));
    st = check_err(c);
    if (st) return st;
    for (int k = 0; k < nbins; ++k) counts[k] = (int64_t)h[k];
    if (umax) *umax = um;
    return LBMP_OK;
  } catch (...) {
    return fail(LBMP_ECUDA, "lbmp_velocity_histogram: unexpected exception");
  }
}

lbmp_status lbmp_residual(lbmp_ctx *c, double *r) {
  const lbmp::NvtxRange nvtx_range("lbmp_residual");
  try {
    if (!c || !r) return fail(LBMP_EINVAL, "lbmp_residual: NULL argument");
    if (!c->fields_set) return fail(LBMP_ESTATE, "lbmp_residual: no fields set");
    const DeviceScope device_scope(c->device);
    lbmp_status st = scope_status(device_scope);
    if (st) return st;
    lbmp::MacroOut o{};
    o.uprev = c->uprev;
    o.update_prev = 1;
    st = run_macro(c, o, true);
    if (st) return st;
    *r = std::sqrt(c->h_results[4]) / std::sqrt(c->h_results[3]);
    return LBMP_OK;
  } catch (...) {
    return fail(LBMP_ECUDA, "lbmp_residual: unexpected exception");
  }
}

lbmp_status lbmp_mass(lbmp_ctx *c, double *m) {
  const lbmp::NvtxRange nvtx_range("lbmp_mass");
  try {
    if (!c || !m) return fail(LBMP_EINVAL, "lbmp_mass: NULL argument");
    if (!c->fields_set) return fail(LBMP_ESTATE, "lbmp_mass: no fields set");
    const DeviceScope device_scope(c->device);
    lbmp_status st = scope_status(device_scope);
    if (st) return st;
    lbmp::MacroOut o{};
    st = run_macro(c, o, true);
    if (st) return st;
    *m = (double)c->fluid_nodes * c->p.rho0 + c->h_results[2];
    return LBMP_OK;
  } catch (...) {
    return fail(LBMP_ECUDA, "lbmp_mass: unexpected exception");
  }
}

lbmp_status lbmp_state_size(lbmp_ctx *c, size_t *bytes) {
  if (!c || !bytes) return fail(LBMP_EINVAL, "lbmp_state_size: NULL argument");
  *bytes = sizeof(StateHeader) + c->buf_bytes();
  return LBMP_OK;
}

lbmp_status lbmp_get_state(lbmp_ctx *c, void *buf, size_t bytes, int32_t where) {
  const lbmp::NvtxRange nvtx_range("lbmp_get_state");
  try {
    if (!c || !buf) return fail(LBMP_EINVAL, "lbmp_get_state: NULL argument");
    if (!valid_where(where)) return fail(LBMP_EINVAL, "where must be LBMP_HOST or LBMP_DEVICE");
    if (!c->fields_set) return fail(LBMP_ESTATE, "lbmp_get_state: no fields set");
    size_t need = sizeof(StateHeader) + c->buf_bytes();
    if (bytes < need) return fail(LBMP_EINVAL, "lbmp_get_state: buffer of %zu bytes, need %zu", bytes, need);
    const DeviceScope device_scope(c->device);
    lbmp_status st = scope_status(device_scope);
    if (st) return st;
    StateHeader h{};
    h.magic = kStateMagic;
    h.nx = c->p.nx;
    h.ny = c->p.ny;
    h.pitch = c->pitch;
    h.storage = c->p.storage;
    h.steps = c->steps;
    h.cur = 0;
    h.scale = c->scale;
    h.payload_bytes = c->buf_bytes();
    cudaMemcpyKind k = (where == LBMP_HOST) ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice;
    cudaMemcpyKind kh = (where == LBMP_HOST) ? cudaMemcpyHostToHost : cudaMemcpyHostToDevice;
    LBMP_CK(cudaStreamSynchronize(c->stream));
    LBMP_CK(cudaMemcpy(buf, &h, sizeof(h), kh));
    LBMP_CK(cudaMemcpy((char *)buf + sizeof(h), c->buf[c->cur], c->buf_bytes(), k));
    return LBMP_OK;
  } catch (...) {
    return fail(LBMP_ECUDA, "lbmp_get_state: unexpected exception");
  }
}

lbmp_status lbmp_set_state(lbmp_ctx *c, const void *buf, size_t bytes, int32_t where) {
  const lbmp::NvtxRange nvtx_range("lbmp_set_state");
  try {
    if (!c || !buf) return fail(LBMP_EINVAL, "lbmp_set_state: NULL argument");
    if (!valid_where(where)) return fail(LBMP_EINVAL, "where must be LBMP_HOST or LBMP_DEVICE");
    if (!c->fields_set) return fail(LBMP_ESTATE, "lbmp_set_state: set the medium first");
    size_t need = sizeof(StateHeader) + c->buf_bytes();
    if (bytes != need) return fail(LBMP_EINVAL, "lbmp_set_state: %zu bytes, expected %zu", bytes, need);
    const DeviceScope device_scope(c->device);
    lbmp_status st = scope_status(device_scope);
    if (st) return st;
    StateHeader h{};
    cudaMemcpyKind kh = (where == LBMP_HOST) ? cudaMemcpyHostToHost : cudaMemcpyDeviceToHost;
    LBMP_CK(cudaMemcpy(&h, buf, sizeof(h), kh));
    if (h.magic != kStateMagic || h.nx != c->p.nx || h.ny != c->p.ny || h.pitch != c->pitch ||
        h.storage != c->p.storage || h.payload_bytes != c->buf_bytes())
      return fail(LBMP_EINVAL, "lbmp_set_state: blob does not match this context");
    if (h.scale != c->scale)
      return fail(LBMP_EINVAL, "lbmp_set_state: blob written with FP16 scale %g, context uses %g",
                  h.scale, c->scale);
    cudaMemcpyKind k = (where == LBMP_HOST) ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice;
    LBMP_CK(cudaStreamSynchronize(c->stream));
    LBMP_CK(cudaMemcpy(c->buf[c->cur], (const char *)buf + sizeof(h), c->buf_bytes(), k));
    const unsigned long long t = (unsigned long long)h.steps;
    LBMP_CK(cudaMemcpy(c->d_tctr, &t, sizeof(t), cudaMemcpyHostToDevice));
    c->steps = h.steps;
    return LBMP_OK;
  } catch (...) {
    return fail(LBMP_ECUDA, "lbmp_set_state: unexpected exception");
  }
}

lbmp_status lbmp_get_info(lbmp_ctx *c, lbmp_info *out) {
  if (!c || !out) return fail(LBMP_EINVAL, "lbmp_get_info: NULL argument");
  out->nx = c->p.nx;
  out->ny = c->p.ny;
  out->pitch = c->pitch;
  out->storage = c->p.storage;
  out->fluid_nodes = c->fluid_nodes;
  out->steps = c->steps;
  // nine populations read and written once, plus the float2 medium (and
  // the Kn plane of a dynamic Kn)
  out->bytes_per_update = 2.0 * 9.0 * (double)c->elem + 8.0 + (c->kn0 ? 4.0 : 0.0);
  out->fp16_scale = c->scale;
  out->eps_mean = c->eps_mean;
  out->device_bytes = c->device_bytes;
  out->launches = c->launches;
  return LBMP_OK;
}

}  // extern "C"
