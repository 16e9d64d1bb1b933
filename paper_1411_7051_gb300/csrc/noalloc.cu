// Allocation-free global permeability (lbmp_permeability_noalloc).
//
// Some callers cannot call cudaMalloc: processes whose device memory is
// owned by a pool of another framework that must stay the only allocator
// (an allocation behind its back can fail, or take memory the pool has
// budgeted for itself), and latency-bound control loops that may not pay for
// an allocation and the device-wide synchronisation of cudaFree.  For them
// this entry point takes every input and output from the caller and
// keeps its only scratch -- the per-block FP64 partial sums of the
// reduction -- in a fixed array in the library's own device memory, which
// every GPU that loads the library holds until the process exits.
//
// The computation is the one of lbmp_permeability: density and velocity of
// each fluid node (Eq. 16a and Eq. 17, or its quadratic form with the
// Forchheimer drag of Eq. 2), and Darcy's law over the whole domain, here in
// FP64 from caller-held FP64 populations.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <mutex>

#include "kernels.h"
#include "lbmp.h"

namespace {

constexpr int kNoallocBX = 256;       // threads per block (one row segment each)
constexpr int kNoallocQ = 4;          // sum u_x, sum eps, fluid nodes, non-finite nodes
constexpr int kNoallocMaxBlocks = 65536;  // ceil(nx / 256) * ny must not exceed this
constexpr int kMaxDevices = 64;

// The scratch: block partials of one call.  Every slot the final sum reads
// is written earlier by the same call, so nothing needs clearing; two calls
// that overlap on the GPU write the same slots and race.
static __device__ __align__(256) double g_noalloc_partials[kNoallocMaxBlocks * kNoallocQ];

std::mutex g_setup_mutex;
double *g_scratch_addr[kMaxDevices] = {nullptr};

lbmp_status nfail(lbmp_status st, const char *fmt, ...) {
  char buf[400];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  lbmp::set_last_error(buf);  // read back with lbmp_last_error()
  return st;
}

struct NoallocArgs {
  int nx, ny;
  int walls, pressure, forch, kn_model;
  double nu, Gx, Gy, rho0, rho_in, rho_out, kn_beta;
};

__global__ void __launch_bounds__(kNoallocBX)
    noalloc_partials_kernel(const NoallocArgs a, const double *__restrict__ f,
                            const double *__restrict__ eps, const double *__restrict__ k_i,
                            const double *__restrict__ kn, double *__restrict__ partials) {
  const int y = blockIdx.y;
  const int x = blockIdx.x * kNoallocBX + threadIdx.x;
  double v[kNoallocQ] = {0.0, 0.0, 0.0, 0.0};
  const bool wall = a.walls && (y == 0 || y == a.ny - 1);
  if (x < a.nx && !wall) {
    const long long n = (long long)a.nx * a.ny;
    const long long j = (long long)y * a.nx + x;
    double fi[9];
    for (int i = 0; i < 9; ++i) fi[i] = f[i * n + j];
    const double rho = fi[0] + fi[1] + fi[2] + fi[3] + fi[4] + fi[5] + fi[6] + fi[7] + fi[8];
    const double mx = fi[1] - fi[3] + fi[5] - fi[6] - fi[7] + fi[8];
    const double my = fi[2] - fi[4] + fi[5] + fi[6] - fi[7] - fi[8];
    const double e = eps[j];
    double ux = 0.0;
    if (e > 0.0) {
      // Eq. 3; with a dynamic Kn at the node's pressure p0 (1 + beta (rho - rho0))
      const double K = a.kn_beta == 0.0 ? kn[j] : kn[j] / (1.0 + a.kn_beta * (rho - a.rho0));
      const double ka = k_i[j] * lbmp::fc_model(K, a.kn_model);
      const double inv_k = isinf(ka) ? 0.0 : 1.0 / ka;
      const double vx = mx / rho + 0.5 * e * a.Gx, vy = my / rho + 0.5 * e * a.Gy;
      const double c0 = 0.5 * (1.0 + 0.5 * e * a.nu * inv_k);
      double den = 2.0 * c0;
      if (a.forch) {
        const double c1 = 0.5 * e * (1.75 / sqrt(150.0 * e * e * e)) * sqrt(inv_k);
        den = c0 + sqrt(c0 * c0 + c1 * sqrt(vx * vx + vy * vy));
      }
      ux = vx / den;
    }
    v[0] = ux;
    v[1] = e;
    v[2] = 1.0;
    v[3] = isfinite(ux) ? 0.0 : 1.0;
    if (!isfinite(ux)) v[0] = 0.0;
  }
  __shared__ double red[kNoallocBX / 32][kNoallocQ];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int q = 0; q < kNoallocQ; ++q) {
    double t = v[q];
    for (int off = 16; off > 0; off >>= 1) t += __shfl_down_sync(0xffffffffu, t, off);
    if (lane == 0) red[warp][q] = t;
  }
  __syncthreads();
  if (threadIdx.x < kNoallocQ) {
    double t = 0.0;
    for (int w = 0; w < kNoallocBX / 32; ++w) t += red[w][threadIdx.x];
    const long long b = (long long)blockIdx.y * gridDim.x + blockIdx.x;
    partials[b * kNoallocQ + threadIdx.x] = t;
  }
}

// One block sums the partials in a fixed order and applies Darcy's law:
// out[0] = k_g = nu <u_x> / G_eff, out[1] = <u_x>, out[2] = non-finite nodes.
__global__ void __launch_bounds__(kNoallocBX)
    noalloc_finish_kernel(const NoallocArgs a, const double *__restrict__ partials, int nblocks,
                          double *__restrict__ out) {
  __shared__ double sh[kNoallocQ][kNoallocBX];
  for (int q = 0; q < kNoallocQ; ++q) {
    double t = 0.0;
    for (int b = threadIdx.x; b < nblocks; b += kNoallocBX) t += partials[(long long)b * kNoallocQ + q];
    sh[q][threadIdx.x] = t;
  }
  __syncthreads();
  for (int w = kNoallocBX / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w)
      for (int q = 0; q < kNoallocQ; ++q) sh[q][threadIdx.x] += sh[q][threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    const double um = sh[0][0] / sh[2][0];
    double g = a.Gx;
    if (a.pressure)
      g += (a.rho_in - a.rho_out) / 3.0 / (sh[1][0] / sh[2][0]) / (a.rho0 * (double)(a.nx - 1));
    out[0] = a.nu * um / g;
    out[1] = um;
    out[2] = sh[3][0];
  }
}

// Device address of the scratch array for the current device (looked up
// once per device, under a lock).
lbmp_status scratch_for_current_device(double **out) {
  int dev = -1;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return nfail(LBMP_ECUDA, "cudaGetDevice: %s", cudaGetErrorString(e));
  if (dev < 0 || dev >= kMaxDevices) return nfail(LBMP_ECUDA, "device %d out of range", dev);
  std::lock_guard<std::mutex> lock(g_setup_mutex);
  if (!g_scratch_addr[dev]) {
    void *p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_partials);
    if (e != cudaSuccess)
      return nfail(LBMP_ECUDA, "cudaGetSymbolAddress of the reduction scratch: %s",
                   cudaGetErrorString(e));
    g_scratch_addr[dev] = static_cast<double *>(p);
  }
  *out = g_scratch_addr[dev];
  return LBMP_OK;
}

}  // namespace

extern "C" {

lbmp_status lbmp_permeability_noalloc(const lbmp_params *p, const double *f, const double *eps,
                                      const double *k_i, const double *kn, double *out,
                                      void *stream) {
  try {
    if (!p || !f || !eps || !k_i || !kn || !out)
      return nfail(LBMP_EINVAL, "lbmp_permeability_noalloc: NULL argument");
    // the checks of lbmp_create on the fields read here (the others are
    // ignored: they are set to valid values for the check)
    lbmp_params q = *p;
    q.storage = LBMP_STORE_FP32;
    q.kernel = LBMP_KERNEL_DIRECT;
    q.fp16_log2_scale = 0;
    q.fp16_rounding = LBMP_ROUND_STOCHASTIC;
    lbmp_status vst = lbmp::validate_params(&q);  // also fills J = 0, rho0 = 0 with 1
    if (vst) return vst;
    p = &q;
    const long long blocks = (long long)((p->nx + kNoallocBX - 1) / kNoallocBX) * p->ny;
    if (blocks > kNoallocMaxBlocks)
      return nfail(LBMP_EINVAL,
                   "lattice %d x %d needs %lld reduction blocks; the fixed scratch holds %d "
                   "(ceil(nx / %d) * ny must be <= %d)",
                   p->nx, p->ny, blocks, kNoallocMaxBlocks, kNoallocBX, kNoallocMaxBlocks);
    const int walls = p->bc_y == LBMP_BCY_WALLS, pressure = p->bc_x == LBMP_BCX_PRESSURE;
    double *scratch = nullptr;
    lbmp_status st = scratch_for_current_device(&scratch);
    if (st) return st;
    NoallocArgs a;
    a.nx = p->nx;
    a.ny = p->ny;
    a.walls = walls;
    a.pressure = pressure;
    a.forch = p->forchheimer != 0;
    a.kn_model = p->kn_model;
    a.kn_beta = p->kn_beta;
    a.nu = (p->tau - 0.5) / 3.0 / p->J;
    a.Gx = p->Gx;
    a.Gy = p->Gy;
    a.rho0 = p->rho0;
    a.rho_in = p->rho_in;
    a.rho_out = p->rho_out;
    cudaStream_t s = (cudaStream_t)stream;
    dim3 grid((p->nx + kNoallocBX - 1) / kNoallocBX, p->ny);
    noalloc_partials_kernel<<<grid, kNoallocBX, 0, s>>>(a, f, eps, k_i, kn, scratch);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return nfail(LBMP_ECUDA, "partials kernel: %s", cudaGetErrorString(e));
    noalloc_finish_kernel<<<1, kNoallocBX, 0, s>>>(a, scratch, (int)blocks, out);
    e = cudaGetLastError();
    if (e != cudaSuccess) return nfail(LBMP_ECUDA, "finish kernel: %s", cudaGetErrorString(e));
    return LBMP_OK;
  } catch (...) {
    return nfail(LBMP_ECUDA, "lbmp_permeability_noalloc: unexpected exception");
  }
}

}  // extern "C"
