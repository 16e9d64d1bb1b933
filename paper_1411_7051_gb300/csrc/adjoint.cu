// Discrete adjoint of the time loop (Section III, Eq. 12-17) for the global
// permeability k_g = nu <u_x> / G_eff of the final time level: gradients
// with respect to ln k_i and eps of every node.
//
// Forward state: f^{n+1} = Phi(f^n; theta), Phi = stream o collide, plus the
// pressure columns f^{n+1}_b = NEEP(f^{n+1}_neighbour; theta) (non-equilibrium
// extrapolation).  The adjoint Lambda^n = dJ/df^n runs backwards:
//   1. NEEP adjoint: Lambda^{n+1} of a pressure column is pushed into its
//      interior neighbour (and into the eps / 1/k_a gradients);
//   2. reverse streaming: lambda*_i(z) = Lambda^{n+1}_i(z + e_i) (bounce-back
//      at plates, zero for values a pressure column overwrites);
//   3. collision transpose: post_i = (1 - 1/tau) f_i + g_i(rho, m; theta), so
//      Lambda^n_j = (1 - 1/tau) lambda*_j + dG/drho + e_j . dG/dm with
//      G = sum_i lambda*_i g_i; dG/d(rho, m, eps, kappa) come from forward-mode
//      dual numbers evaluated on the same formulas as the forward step.
// States f^n are recomputed segment by segment from checkpoints taken every
// `every` steps (sqrt(N) by default); gradients accumulate in FP64.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <vector>

#include "context.h"
#include "kernels.h"
#include "lattice.cuh"
#include "lbmp.h"

namespace lbmp {

// ------------------------------------------------------------ dual numbers
template <int N>
struct Dual {
  float v;
  float d[N];
};

template <int N>
__device__ __forceinline__ Dual<N> dconst(float x) {
  Dual<N> r;
  r.v = x;
#pragma unroll
  for (int k = 0; k < N; ++k) r.d[k] = 0.0f;
  return r;
}
template <int N>
__device__ __forceinline__ Dual<N> dvar(float x, int k0) {
  Dual<N> r = dconst<N>(x);
  r.d[k0] = 1.0f;
  return r;
}
template <int N>
__device__ __forceinline__ Dual<N> operator+(const Dual<N> &a, const Dual<N> &b) {
  Dual<N> r;
  r.v = a.v + b.v;
#pragma unroll
  for (int k = 0; k < N; ++k) r.d[k] = a.d[k] + b.d[k];
  return r;
}
template <int N>
__device__ __forceinline__ Dual<N> operator-(const Dual<N> &a, const Dual<N> &b) {
  Dual<N> r;
  r.v = a.v - b.v;
#pragma unroll
  for (int k = 0; k < N; ++k) r.d[k] = a.d[k] - b.d[k];
  return r;
}
template <int N>
__device__ __forceinline__ Dual<N> operator-(const Dual<N> &a) {
  Dual<N> r;
  r.v = -a.v;
#pragma unroll
  for (int k = 0; k < N; ++k) r.d[k] = -a.d[k];
  return r;
}
template <int N>
__device__ __forceinline__ Dual<N> operator*(const Dual<N> &a, const Dual<N> &b) {
  Dual<N> r;
  r.v = a.v * b.v;
#pragma unroll
  for (int k = 0; k < N; ++k) r.d[k] = fmaf(a.d[k], b.v, a.v * b.d[k]);
  return r;
}
template <int N>
__device__ __forceinline__ Dual<N> operator*(float s, const Dual<N> &a) {
  Dual<N> r;
  r.v = s * a.v;
#pragma unroll
  for (int k = 0; k < N; ++k) r.d[k] = s * a.d[k];
  return r;
}
template <int N>
__device__ __forceinline__ Dual<N> operator+(float s, const Dual<N> &a) {
  Dual<N> r = a;
  r.v = s + a.v;
  return r;
}
template <int N>
__device__ __forceinline__ Dual<N> operator/(const Dual<N> &a, const Dual<N> &b) {
  Dual<N> r;
  const float ib = 1.0f / b.v;
  r.v = a.v * ib;
#pragma unroll
  for (int k = 0; k < N; ++k) r.d[k] = (a.d[k] - r.v * b.d[k]) * ib;
  return r;
}
// sqrt with the zero subgradient at 0
template <int N>
__device__ __forceinline__ Dual<N> dsqrt(const Dual<N> &a) {
  Dual<N> r;
  r.v = sqrtf(a.v);
  const float g = (r.v > 0.0f) ? 0.5f / r.v : 0.0f;
#pragma unroll
  for (int k = 0; k < N; ++k) r.d[k] = g * a.d[k];
  return r;
}

// Velocity (Eq. 17 or the quadratic form with Eq. 2) and force of a node of
// porosity eps > 0 and kappa = 1/k_a, from rho and the momentum m (sum of
// populations times e_i), all as duals.
template <int N>
struct DVel {
  Dual<N> ux, uy, Fx, Fy;
};
template <int N>
__device__ __forceinline__ DVel<N> dvelocity(const Dual<N> &rho, const Dual<N> &mx,
                                             const Dual<N> &my, const Dual<N> &eps,
                                             const Dual<N> &kap, const StepArgs &a) {
  const Dual<N> eGx = a.Gx * eps, eGy = a.Gy * eps;
  const Dual<N> vx = mx / rho + 0.5f * eGx;
  const Dual<N> vy = my / rho + 0.5f * eGy;
  const Dual<N> darcy = a.nu * (eps * kap);
  const Dual<N> c0 = 0.5f + 0.25f * darcy;
  Dual<N> den, drag;
  if (a.forch) {
    const Dual<N> c1 = a.fe_half * dsqrt(kap / eps);
    const Dual<N> vmag = dsqrt(vx * vx + vy * vy);
    den = c0 + dsqrt(c0 * c0 + c1 * vmag);
    drag = darcy + 2.0f * (c1 * (vmag / den));
  } else {
    den = 2.0f * c0;
    drag = darcy;
  }
  DVel<N> r;
  r.ux = vx / den;
  r.uy = vy / den;
  r.Fx = eGx - drag * r.ux;
  r.Fy = eGy - drag * r.uy;
  return r;
}

// Porous equilibrium (Eq. 14) of direction i, physical units.
template <int N>
__device__ __forceinline__ Dual<N> dfeq(int i, const Dual<N> &rho, const Dual<N> &ux,
                                        const Dual<N> &uy, const Dual<N> &ieps) {
  const int ex[9] = {0, 1, 0, -1, 0, 1, -1, -1, 1};
  const int ey[9] = {0, 0, 1, 0, -1, 1, 1, -1, -1};
  const float w = (i == 0) ? kW0 : (i <= 4 ? kW1 : kW2);
  const Dual<N> eu = (float)ex[i] * ux + (float)ey[i] * uy;
  const Dual<N> uu = ux * ux + uy * uy;
  const Dual<N> br = 1.0f + 3.0f * eu + (4.5f * (eu * eu) - 1.5f * uu) * ieps;
  return w * (rho * br);
}

// G = sum_i lam_i (omega feq_i + F_i) of a node with eps > 0 (Eq. 14, 15).
template <int N>
__device__ __forceinline__ Dual<N> dGamma(const float lam[9], const Dual<N> &rho,
                                          const Dual<N> &mx, const Dual<N> &my,
                                          const Dual<N> &eps, const Dual<N> &kap,
                                          const StepArgs &a) {
  const DVel<N> v = dvelocity(rho, mx, my, eps, kap, a);
  const Dual<N> ieps = dconst<N>(1.0f) / eps;
  const int ex[9] = {0, 1, 0, -1, 0, 1, -1, -1, 1};
  const int ey[9] = {0, 0, 1, 0, -1, 1, 1, -1, -1};
  const Dual<N> uF = v.ux * v.Fx + v.uy * v.Fy;
  Dual<N> G = dconst<N>(0.0f);
#pragma unroll
  for (int i = 0; i < 9; ++i) {
    const float w = (i == 0) ? kW0 : (i <= 4 ? kW1 : kW2);
    const Dual<N> eu = (float)ex[i] * v.ux + (float)ey[i] * v.uy;
    const Dual<N> eF = (float)ex[i] * v.Fx + (float)ey[i] * v.Fy;
    const Dual<N> Fi = (w * a.cforce) * (rho * (3.0f * eF + (9.0f * (eu * eF) - 3.0f * uF) * ieps));
    const Dual<N> gi = a.omega * dfeq(i, rho, v.ux, v.uy, ieps) + Fi;
    G = G + lam[i] * gi;
  }
  return G;
}

struct AdjArgs {
  StepArgs a;            // forward parameters (FP32 storage, scale 1)
  float *lam_in;         // Lambda^{n+1}, [9][ny][pitch]
  float *lam_out;        // Lambda^n
  const float *fin;      // forward buffer whose pull is f^n (or f^{n+1} for NEEP)
  const float2 *med;     // (eps, 1/k_a)
  double *g_eps;         // [ny][pitch] accumulated dJ/deps
  double *g_kap;         // [ny][pitch] accumulated dJ/dkappa
  double coef;           // nu / (G_eff * fluid nodes) for the objective seed
};

__device__ __forceinline__ float lam_at(const AdjArgs &A, int i, int x, int y) {
  return A.lam_in[i * A.a.plane + (long long)y * A.a.pitch + x];
}

// Reverse streaming for node (x, y): the adjoint of its post-collision values.
__device__ __forceinline__ void reverse_pull(const AdjArgs &A, int x, int y, float lp[9]) {
  const StepArgs &a = A.a;
  const int ex[9] = {0, 1, 0, -1, 0, 1, -1, -1, 1};
  const int ey[9] = {0, 0, 1, 0, -1, 1, 1, -1, -1};
  const int opp[9] = {0, 3, 4, 1, 2, 7, 8, 5, 6};
  // the pulls of a pressure column are discarded (replaced by the
  // extrapolation), so whatever streams into one carries no adjoint
  const bool col = a.pressure && (x == 0 || x == a.nx - 1);
#pragma unroll
  for (int i = 0; i < 9; ++i) {
    int xd = x + ex[i], yd = y + ey[i];
    if (a.walls && ey[i] != 0 && (yd == 0 || yd == a.ny - 1)) {
      lp[i] = col ? 0.0f : lam_at(A, opp[i], x, y);  // bounced back into the same node
      continue;
    }
    yd = (yd + a.ny) % a.ny;
    if (a.pressure) {
      if (xd <= 0 || xd >= a.nx - 1) {  // lost at the edge or received by a pressure column
        lp[i] = 0.0f;
        continue;
      }
    } else {
      xd = (xd + a.nx) % a.nx;
    }
    lp[i] = lam_at(A, i, xd, yd);
  }
}

// Forward post-stream state of node (x, y) from buffer fin (pull + pressure
// columns), deviations f_i - w_i rho0.
__device__ __forceinline__ void forward_state(const AdjArgs &A, int x, int y, float d[9]) {
  pull_node<StoreF32>(A.fin, A.a, x, y, d);
  if (A.a.pressure && (x == 0 || x == A.a.nx - 1)) {
    const float2 m = A.med[(long long)y * A.a.pitch + x];
    pressure_node<StoreF32>(A.fin, A.med, A.a, x, y, m.x, d);
  }
}

__device__ __forceinline__ void moments(const float d[9], float rho0, float &rho, float &mx,
                                        float &my) {
  const float drho = ((d[0] + (d[1] + d[3])) + (d[2] + d[4])) + ((d[5] + d[7]) + (d[6] + d[8]));
  rho = rho0 + drho;
  mx = (d[1] - d[3]) + ((d[5] - d[7]) + (d[8] - d[6]));
  my = (d[2] - d[4]) + ((d[5] - d[7]) + (d[6] - d[8]));
}

// One reverse step for every fluid node: Lambda^n from Lambda^{n+1}, f^n.
__global__ void __launch_bounds__(128) adjoint_step_kernel(const AdjArgs A) {
  const StepArgs &a = A.a;
  const int y = a.y0 + blockIdx.y;
  const int x = blockIdx.x * 128 + threadIdx.x;
  if (x >= a.nx) return;
  float lp[9], d[9];
  reverse_pull(A, x, y, lp);
  forward_state(A, x, y, d);
  float rho, mx, my;
  moments(d, a.rho0, rho, mx, my);
  const long long j = (long long)y * a.pitch + x;
  const float2 m = A.med[j];
  const int ex[9] = {0, 1, 0, -1, 0, 1, -1, -1, 1};
  const int ey[9] = {0, 0, 1, 0, -1, 1, 1, -1, -1};
  float ar, amx, amy;
  if (m.x > 0.0f) {
    const Dual<5> G = dGamma<5>(lp, dvar<5>(rho, 0), dvar<5>(mx, 1), dvar<5>(my, 2),
                                dvar<5>(m.x, 3), dvar<5>(m.y, 4), a);
    ar = G.d[0];
    amx = G.d[1];
    amy = G.d[2];
    A.g_eps[j] += (double)G.d[3];
    A.g_kap[j] += (double)G.d[4];
  } else {
    // impermeable node: g_i = omega w_i rho - 6 (1 - 1/2tau) w_i e_i . m
    float sw = 0.0f, swx = 0.0f, swy = 0.0f;
#pragma unroll
    for (int i = 0; i < 9; ++i) {
      const float w = (i == 0) ? kW0 : (i <= 4 ? kW1 : kW2);
      sw += w * lp[i];
      swx += w * lp[i] * ex[i];
      swy += w * lp[i] * ey[i];
    }
    ar = a.omega * sw;
    amx = -6.0f * a.cforce * swx;
    amy = -6.0f * a.cforce * swy;
  }
  const float o1 = a.one_m_omega;
#pragma unroll
  for (int i = 0; i < 9; ++i)
    A.lam_out[i * a.plane + j] = fmaf(o1, lp[i], ar + ex[i] * amx + ey[i] * amy);
}

// Pressure columns: push Lambda of column 0 / nx-1 into columns 1 / nx-2
// (in place in lam_in) and into the parameter gradients.  fin is the buffer
// whose pull gives the post-stream state at the same time level.
__global__ void adjoint_neep_kernel(const AdjArgs A) {
  const StepArgs &a = A.a;
  const int y = a.y0 + blockIdx.x * blockDim.x + threadIdx.x;
  const int y_end = a.walls ? a.ny - 1 : a.ny;
  if (y >= y_end) return;
  const int ex[9] = {0, 1, 0, -1, 0, 1, -1, -1, 1};
  const int ey[9] = {0, 0, 1, 0, -1, 1, 1, -1, -1};
  for (int side = 0; side < 2; ++side) {
    const int xb = side ? a.nx - 1 : 0;
    const int xn = side ? a.nx - 2 : 1;
    const long long jb = (long long)y * a.pitch + xb, jn = (long long)y * a.pitch + xn;
    float lb[9], d[9];
#pragma unroll
    for (int i = 0; i < 9; ++i) lb[i] = A.lam_in[i * a.plane + jb];
    pull_node<StoreF32>(A.fin, a, xn, y, d);
    float rho, mx, my;
    moments(d, a.rho0, rho, mx, my);
    const float2 mn = A.med[jn], mb = A.med[jb];
    const float rho_b = a.rho0 + (side ? a.drho_out : a.drho_in);
    float ar = 0.0f, amx = 0.0f, amy = 0.0f;
    if (mn.x > 0.0f) {
      // Psi = sum_i lb_i (feq_i(rho_b, u_n; eps_b) - feq_i(rho_n, u_n; eps_n))
      const Dual<6> R = dvar<6>(rho, 0), MX = dvar<6>(mx, 1), MY = dvar<6>(my, 2);
      const Dual<6> EN = dvar<6>(mn.x, 3), KN = dvar<6>(mn.y, 4), EB = dvar<6>(mb.x, 5);
      const DVel<6> v = dvelocity(R, MX, MY, EN, KN, a);
      const Dual<6> ien = dconst<6>(1.0f) / EN;
      Dual<6> P = dconst<6>(0.0f);
      if (mb.x > 0.0f) {
        const Dual<6> ieb = dconst<6>(1.0f) / EB;
#pragma unroll
        for (int i = 0; i < 9; ++i)
          P = P + lb[i] * (dfeq(i, dconst<6>(rho_b), v.ux, v.uy, ieb) - dfeq(i, R, v.ux, v.uy, ien));
      } else {
#pragma unroll
        for (int i = 0; i < 9; ++i) {
          const float w = (i == 0) ? kW0 : (i <= 4 ? kW1 : kW2);
          P = P + lb[i] * (dconst<6>(w * rho_b) - dfeq(i, R, v.ux, v.uy, ien));
        }
      }
      ar = P.d[0];
      amx = P.d[1];
      amy = P.d[2];
      A.g_eps[jn] += (double)P.d[3];
      A.g_kap[jn] += (double)P.d[4];
      A.g_eps[jb] += (double)P.d[5];
    } else {
      // impermeable neighbour: u_n = 0, f_b = f_n + w (rho_b - rho_n)
      float sw = 0.0f;
#pragma unroll
      for (int i = 0; i < 9; ++i) sw += ((i == 0) ? kW0 : (i <= 4 ? kW1 : kW2)) * lb[i];
      ar = -sw;
    }
#pragma unroll
    for (int i = 0; i < 9; ++i) A.lam_in[i * a.plane + jn] += lb[i] + ar + ex[i] * amx + ey[i] * amy;
  }
}

// Objective seed at the final level: Lambda^N = coef * du_x/df, gradients
// coef * du_x/d(eps, kappa).
__global__ void __launch_bounds__(128) adjoint_seed_kernel(const AdjArgs A) {
  const StepArgs &a = A.a;
  const int y = a.y0 + blockIdx.y;
  const int x = blockIdx.x * 128 + threadIdx.x;
  if (x >= a.nx) return;
  float d[9];
  forward_state(A, x, y, d);
  float rho, mx, my;
  moments(d, a.rho0, rho, mx, my);
  const long long j = (long long)y * a.pitch + x;
  const float2 m = A.med[j];
  const int ex[9] = {0, 1, 0, -1, 0, 1, -1, -1, 1};
  const int ey[9] = {0, 0, 1, 0, -1, 1, 1, -1, -1};
  float cr = 0.0f, cx = 0.0f, cy = 0.0f;
  if (m.x > 0.0f) {
    const DVel<5> v = dvelocity(dvar<5>(rho, 0), dvar<5>(mx, 1), dvar<5>(my, 2),
                                dvar<5>(m.x, 3), dvar<5>(m.y, 4), a);
    const float c = (float)A.coef;
    cr = c * v.ux.d[0];
    cx = c * v.ux.d[1];
    cy = c * v.ux.d[2];
    A.g_eps[j] += A.coef * (double)v.ux.d[3];
    A.g_kap[j] += A.coef * (double)v.ux.d[4];
  }
#pragma unroll
  for (int i = 0; i < 9; ++i) A.lam_out[i * a.plane + j] = cr + ex[i] * cx + ey[i] * cy;
}

// dJ/dln k_i = -kappa dJ/dkappa, dJ/deps (+ the mean-porosity term of the
// pressure drop), into [ny][nx] float64; plate rows read 0.
__global__ void adjoint_assemble_kernel(const AdjArgs A, double eps_term, double *out_logk,
                                        double *out_eps) {
  const StepArgs &a = A.a;
  const int y = blockIdx.y;
  const int x = blockIdx.x * 128 + threadIdx.x;
  if (x >= a.nx) return;
  const long long o = (long long)y * a.nx + x;
  const bool wall = a.walls && (y == 0 || y == a.ny - 1);
  if (wall) {
    out_logk[o] = 0.0;
    out_eps[o] = 0.0;
    return;
  }
  const long long j = (long long)y * a.pitch + x;
  const float2 m = A.med[j];
  out_logk[o] = -(double)m.y * A.g_kap[j];
  out_eps[o] = A.g_eps[j] + eps_term;
}

}  // namespace lbmp

// ------------------------------------------------------------------ driver
namespace {

lbmp_status afail(lbmp_status st, const char *fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  lbmp::set_last_error(buf);  // read back with lbmp_last_error()
  return st;
}

struct DevBuf {
  void *p = nullptr;
  ~DevBuf() {
    if (p) cudaFree(p);
  }
};

#define ACK(call)                                                                        \
  do {                                                                                   \
    cudaError_t e_ = (call);                                                             \
    if (e_ != cudaSuccess) {                                                             \
      cudaGetLastError();                                                                \
      return afail(e_ == cudaErrorMemoryAllocation ? LBMP_ENOMEM : LBMP_ECUDA, "%s: %s", \
                   #call, cudaGetErrorString(e_));                                       \
    }                                                                                    \
  } while (0)

// One forward step with the kernel the context selected.
cudaError_t forward_step(lbmp_ctx *c, const lbmp::StepArgs &a, const void *fin, void *fout,
                         cudaStream_t s) {
  if (c->staged)
    return lbmp::launch_staged(c->p.storage, false, a, c->rows(), fin, fout, c->med, c->d_tctr,
                               0, c->d_err, c->nsm, s);
  return lbmp::launch_step(c->p.storage, false, a, c->rows(), fin, fout, c->med, c->d_tctr, 0, s);
}

}  // namespace

extern "C" lbmp_status lbmp_permeability_gradient(lbmp_ctx *c, int64_t nsteps, int64_t every,
                                                  double *k_g, double *d_logk, double *d_eps,
                                                  int32_t where) {
  using lbmp::AdjArgs;
  using lbmp::StepArgs;
  try {
    if (!c || !d_logk || !d_eps)
      return afail(LBMP_EINVAL, "lbmp_permeability_gradient: NULL argument");
    if (where != LBMP_HOST && where != LBMP_DEVICE)
      return afail(LBMP_EINVAL, "where must be LBMP_HOST or LBMP_DEVICE");
    if (nsteps < 1) return afail(LBMP_EINVAL, "nsteps must be >= 1 (got %lld)", (long long)nsteps);
    if (every < 0) return afail(LBMP_EINVAL, "every must be >= 0 (0: sqrt(nsteps))");
    if (!c->fields_set) return afail(LBMP_ESTATE, "lbmp_permeability_gradient: no fields set");
    if (c->p.storage != LBMP_STORE_FP32)
      return afail(LBMP_EINVAL, "lbmp_permeability_gradient needs FP32 storage");
    ACK(cudaSetDevice(c->device));
    if (every == 0) every = (int64_t)std::ceil(std::sqrt((double)nsteps));
    every = std::min(every, nsteps);
    const int64_t nseg = (nsteps + every - 1) / every;
    const StepArgs a = c->args();
    const int rows = c->rows();
    const size_t state = c->buf_bytes();
    const size_t field = (size_t)c->plane * sizeof(double);
    cudaStream_t s = c->stream;
    // checkpoints (one per segment), the states of one segment, the two
    // adjoint levels, the FP64 gradient fields
    DevBuf ck, seg, lam, grad, outs;
    ACK(cudaMalloc(&ck.p, state * (size_t)nseg));
    ACK(cudaMalloc(&seg.p, state * (size_t)(every + 1)));
    ACK(cudaMalloc(&lam.p, state * 2));
    ACK(cudaMalloc(&grad.p, field * 2));
    ACK(cudaMemsetAsync(lam.p, 0, state * 2, s));
    ACK(cudaMemsetAsync(grad.p, 0, field * 2, s));
    char *ckp = (char *)ck.p, *segp = (char *)seg.p;
    float *lam0 = (float *)lam.p, *lam1 = (float *)((char *)lam.p + state);
    double *g_eps = (double *)grad.p, *g_kap = (double *)((char *)grad.p + field);

    // forward pass from rest in the context's own buffers, checkpointing
    // the first level of every segment
    ACK(cudaMemsetAsync(c->buf[0], 0, state, s));
    ACK(cudaMemsetAsync(c->buf[1], 0, state, s));
    ACK(cudaMemsetAsync(c->d_err, 0, sizeof(unsigned), s));
    int cur = 0;
    for (int64_t sg = 0; sg < nseg; ++sg) {
      ACK(cudaMemcpyAsync(ckp + state * sg, c->buf[cur], state, cudaMemcpyDeviceToDevice, s));
      const int64_t n = std::min(every, nsteps - sg * every);
      for (int64_t t = 0; t < n; ++t) {
        ACK(forward_step(c, a, c->buf[cur], c->buf[cur ^ 1], s));
        cur ^= 1;
      }
    }
    c->cur = cur;
    c->steps = nsteps;
    c->launches += nsteps;
    // J = k_g of level N, exactly as lbmp_permeability reports it
    double J = 0.0;
    lbmp_status st = lbmp_permeability(c, &J, nullptr);
    if (st) return st;
    const lbmp_params &p = c->p;
    const double nu = (p.tau - 0.5) / 3.0 / p.J;
    double geff = p.Gx, kp = 0.0;
    if (p.bc_x == LBMP_BCX_PRESSURE) {
      kp = (p.rho_in - p.rho_out) / 3.0 / c->eps_mean / (p.rho0 * (double)(p.nx - 1));
      geff += kp;
    }
    const double nf = (double)c->fluid_nodes;
    AdjArgs A;
    A.a = a;
    A.med = c->med;
    A.g_eps = g_eps;
    A.g_kap = g_kap;
    A.coef = nu / (geff * nf);
    // seed: Lambda^N = dJ/df^N
    const dim3 blk(128), grd((a.nx + 127) / 128, rows);
    const int nb = (rows + 127) / 128;
    A.fin = (const float *)c->buf[cur];
    A.lam_in = lam1;
    A.lam_out = lam0;
    lbmp::adjoint_seed_kernel<<<grd, blk, 0, s>>>(A);
    ACK(cudaGetLastError());
    // backward, one segment at a time: recompute its levels from the
    // checkpoint, then run the reverse steps over them
    float *lam_next = lam0, *lam_prev = lam1;  // Lambda^{t+1}, Lambda^t
    for (int64_t sg = nseg - 1; sg >= 0; --sg) {
      const int64_t t0 = sg * every, n = std::min(every, nsteps - t0);
      ACK(cudaMemcpyAsync(segp, ckp + state * sg, state, cudaMemcpyDeviceToDevice, s));
      for (int64_t t = 0; t < n; ++t)
        ACK(forward_step(c, a, segp + state * t, segp + state * (t + 1), s));
      for (int64_t t = n - 1; t >= 0; --t) {
        A.lam_in = lam_next;
        A.lam_out = lam_prev;
        if (a.pressure) {  // the pressure columns of level t0 + t + 1
          A.fin = (const float *)(segp + state * (t + 1));
          lbmp::adjoint_neep_kernel<<<nb, 128, 0, s>>>(A);
          ACK(cudaGetLastError());
        }
        A.fin = (const float *)(segp + state * t);
        lbmp::adjoint_step_kernel<<<grd, blk, 0, s>>>(A);
        ACK(cudaGetLastError());
        std::swap(lam_next, lam_prev);
      }
      c->launches += 2 * n + (a.pressure ? n : 0);
    }
    if (a.pressure) {  // the pressure columns of level 0 (the rest state)
      A.lam_in = lam_next;
      A.fin = (const float *)segp;
      lbmp::adjoint_neep_kernel<<<nb, 128, 0, s>>>(A);
      ACK(cudaGetLastError());
    }
    // d/d eps_z of G_eff through the mean porosity (pressure drive only)
    const double eps_term = (kp != 0.0) ? J * kp / (geff * c->eps_mean * nf) : 0.0;
    const size_t nn = (size_t)a.nx * a.ny;
    double *ol = d_logk, *oe = d_eps;
    if (where == LBMP_HOST) {
      ACK(cudaMalloc(&outs.p, 2 * nn * sizeof(double)));
      ol = (double *)outs.p;
      oe = ol + nn;
    }
    const dim3 g2((a.nx + 127) / 128, a.ny);
    lbmp::adjoint_assemble_kernel<<<g2, blk, 0, s>>>(A, eps_term, ol, oe);
    ACK(cudaGetLastError());
    c->launches += 3;
    if (where == LBMP_HOST) {
      ACK(cudaMemcpyAsync(d_logk, ol, nn * sizeof(double), cudaMemcpyDeviceToHost, s));
      ACK(cudaMemcpyAsync(d_eps, oe, nn * sizeof(double), cudaMemcpyDeviceToHost, s));
    }
    ACK(cudaStreamSynchronize(s));
    unsigned err = 0;
    ACK(cudaMemcpy(&err, c->d_err, sizeof(err), cudaMemcpyDeviceToHost));
    if (err) return afail(LBMP_ETIMEOUT, "a bounded wait of the staged step kernel gave up");
    if (k_g) *k_g = J;
    return LBMP_OK;
  } catch (...) {
    return afail(LBMP_ECUDA, "lbmp_permeability_gradient: unexpected exception");
  }
}
