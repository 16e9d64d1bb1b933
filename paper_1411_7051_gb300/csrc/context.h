// The library context behind the opaque lbmp_ctx handle (internal to the
// library: shared by the C ABI and the adjoint translation units).
#pragma once

#include <cuda_runtime.h>

#include <cmath>
#include <cstddef>
#include <cstdint>

#include "kernels.h"
#include "lbmp.h"

struct lbmp_ctx {
  lbmp_params p{};
  int device = 0;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  cudaStream_t cap_stream = nullptr;
  int pitch = 0;
  long long plane = 0;
  int y_lo = 0, y_hi = 0;   // fluid rows [y_lo, y_hi)
  size_t elem = 4;
  void *buf[2] = {nullptr, nullptr};
  int cur = 0;
  float2 *med = nullptr;
  float *kn0 = nullptr;         // dynamic Kn only: Kn at p0 per node
  float2 *uprev = nullptr;
  double *partials = nullptr;
  int partials_blocks = 0;
  double *results = nullptr;    // device, kNQ doubles
  double *h_results = nullptr;  // pinned host, kNQ doubles
  unsigned long long *d_hist = nullptr;  // velocity histogram counts (allocated on first use)
  unsigned *d_flag = nullptr;
  unsigned long long *d_tctr = nullptr;  // time level for the stochastic rounding
  unsigned *d_err = nullptr;             // raised by a bounded wait that gave up
  int nsm = 1;                           // SMs of the device
  bool staged = true;            // staged kernel (else direct or wide)
  bool wide = false;             // wide FP16 kernel
  bool sr = false;
  bool fields_set = false;
  int64_t steps = 0;
  int64_t launches = 0;
  double scale = 1.0;
  double eps_mean = 1.0;
  int64_t fluid_nodes = 0;
  int64_t device_bytes = 0;
  int alloc_count = 0;
  int fault_alloc_at = 0;       // simulated allocation failure (testing)
  int drop_tile = -1;           // withheld tile of the staged kernel (testing)
  // step graphs: [l][cur] replays 2^l steps starting from buffer cur
  cudaGraphExec_t graph[6][2] = {};

  lbmp::StepArgs args() const {
    lbmp::StepArgs a;
    a.nx = p.nx;
    a.ny = p.ny;
    a.pitch = pitch;
    a.y0 = y_lo;
    a.plane = plane;
    a.rho0 = (float)p.rho0;
    a.drho_in = (float)(p.rho_in - p.rho0);
    a.drho_out = (float)(p.rho_out - p.rho0);
    // omega on the grid of multiples of 2^-24 and 1 - omega formed from it:
    // the two then sum to exactly 1 in FP32, so the collision conserves mass
    // and momentum without a per-step (1 + O(2^-24)) factor that would
    // compound over a run (the grid changes 1/tau by at most 2^-25)
    a.omega = (float)(std::nearbyint(std::ldexp(1.0 / p.tau, 24)) * std::ldexp(1.0, -24));
    a.one_m_omega = 1.0f - a.omega;
    a.cforce = (float)(1.0 - 0.5 / p.tau);
    a.nu = (float)((p.tau - 0.5) / 3.0 / p.J);
    a.Gx = (float)p.Gx;
    a.Gy = (float)p.Gy;
    a.fe_half = (float)(0.5 * 1.75 / std::sqrt(150.0));
    a.scale = (float)scale;
    a.inv_scale = (float)(1.0 / scale);
    a.walls = p.bc_y == LBMP_BCY_WALLS;
    a.pressure = p.bc_x == LBMP_BCX_PRESSURE;
    a.forch = p.forchheimer != 0;
    a.seed_lo = (uint32_t)(p.seed & 0xffffffffu);
    a.seed_hi = (uint32_t)(p.seed >> 32);
    a.test_drop_tile = drop_tile;
    a.kn_model = p.kn_model;
    a.kn_beta = (float)p.kn_beta;
    a.kn0 = kn0;
    return a;
  }
  int rows() const { return y_hi - y_lo; }
  size_t buf_bytes() const { return (size_t)plane * 9 * elem; }
};
