// Device building blocks of the porous lattice Boltzmann step
// (Chen et al., arXiv:1411.7051, Section III, Eq. 12-17 and Eq. 2).
//
// State representation.  After t time steps, population buffer B holds the
// post-collision values f*_i(x, t-1) of every fluid node, stored as the
// shifted deviation d_i = f_i - w_i rho0 (FP32, or FP16 scaled by S = 2^s).
// Pulling B (f_i(x) <- f*_i(x - e_i), Eq. 12's streaming) gives the
// post-stream populations f_i(x, t), from which density and velocity
// (Eq. 16-17) are defined.  The initial buffer is all zeros (f = w_i rho0).
//
// Layout in HBM: 9 planes [9][ny][pitch] (plane = pitch * ny elements,
// pitch a multiple of 64 elements), medium as float2 (eps, 1/k_a) per node
// on the same [ny][pitch] grid.
#pragma once

#include <cuda_fp16.h>
#include <stdint.h>

namespace lbmp {

// D2Q9 weights (the values printed under Eq. 14).
constexpr float kW0 = 4.0f / 9.0f;
constexpr float kW1 = 1.0f / 9.0f;
constexpr float kW2 = 1.0f / 36.0f;

struct StepArgs {
  int nx, ny, pitch;
  int y0;              // first row covered by the launch
  long long plane;     // elements per population plane
  float rho0;          // storage shift and initial density
  float drho_in;       // rho_in - rho0
  float drho_out;      // rho_out - rho0
  float omega;         // 1 / tau
  float cforce;        // 1 - 1 / (2 tau)  (Eq. 15 prefactor)
  float nu;            // nu_e / J
  float Gx, Gy;        // body force of Eq. 2
  float fe_half;       // (1/2) * 1.75 / sqrt(150): eps F_eps / 2 = fe_half / sqrt(eps)
  float scale;         // storage scale S (1 for FP32)
  float inv_scale;     // 1 / S
  int walls;           // rows 0 and ny-1 are plates (halfway bounce-back)
  int pressure;        // columns 0 and nx-1 carry imposed densities
  int forch;           // keep the Forchheimer drag of Eq. 2
};

// ----------------------------------------------------------------- storage
struct StoreF32 {
  using T = float;
  static __device__ __forceinline__ float ld(const float *p, float) { return *p; }
  static __device__ __forceinline__ void st(float *p, float v, float) { *p = v; }
};

struct StoreF16 {
  using T = __half;
  static __device__ __forceinline__ float ld(const __half *p, float inv_s) {
    return __half2float(*p) * inv_s;
  }
  static __device__ __forceinline__ void st(__half *p, float v, float s) {
    *p = __float2half_rn(v * s);
  }
};

// ------------------------------------------------------------------- pull
// Post-stream deviations d[0..8] of node (x, y) from the post-collision
// buffer: f_i(x) = f*_i(x - e_i); a source in a wall row returns the node's
// own population of the opposite direction (halfway bounce-back); periodic
// edges wrap.  Sources outside [0, nx) only occur for the pressure columns,
// whose populations are replaced by the extrapolation afterwards.
template <class S>
__device__ __forceinline__ void pull_node(const typename S::T *__restrict__ fin,
                                          const StepArgs &a, int x, int y,
                                          float d[9]) {
  const int xm = (x == 0) ? a.nx - 1 : x - 1;       // source for e_x = +1
  const int xp = (x == a.nx - 1) ? 0 : x + 1;       // source for e_x = -1
  const int ym = (y == 0) ? a.ny - 1 : y - 1;       // source for e_y = +1
  const int yp = (y == a.ny - 1) ? 0 : y + 1;       // source for e_y = -1
  const bool wm = a.walls && (y - 1 == 0);          // e_y = +1 source is a plate
  const bool wp = a.walls && (y + 1 == a.ny - 1);   // e_y = -1 source is a plate
  const long long P = a.plane;
  const long long r = (long long)y * a.pitch;
  const long long rm = (long long)ym * a.pitch;
  const long long rp = (long long)yp * a.pitch;
  const float is = a.inv_scale;
  d[0] = S::ld(fin + r + x, is);
  d[1] = S::ld(fin + 1 * P + r + xm, is);
  d[3] = S::ld(fin + 3 * P + r + xp, is);
  d[2] = wm ? S::ld(fin + 4 * P + r + x, is) : S::ld(fin + 2 * P + rm + x, is);
  d[5] = wm ? S::ld(fin + 7 * P + r + x, is) : S::ld(fin + 5 * P + rm + xm, is);
  d[6] = wm ? S::ld(fin + 8 * P + r + x, is) : S::ld(fin + 6 * P + rm + xp, is);
  d[4] = wp ? S::ld(fin + 2 * P + r + x, is) : S::ld(fin + 4 * P + rp + x, is);
  d[7] = wp ? S::ld(fin + 5 * P + r + x, is) : S::ld(fin + 7 * P + rp + xp, is);
  d[8] = wp ? S::ld(fin + 6 * P + r + x, is) : S::ld(fin + 8 * P + rp + xm, is);
}

// ---------------------------------------------------- macroscopic state
struct NodeState {
  float drho;   // rho - rho0
  float rho;
  float ux, uy; // physical velocity (Eq. 17 / quadratic form)
  float Fx, Fy; // total force (Eq. 2 / Eq. 8)
};

// Eq. 16a, Eq. 16b solved for u (Eq. 17, or u = v / (c0 + sqrt(c0^2 +
// c1|v|)) with the Forchheimer term), and F of Eq. 2.  eps = 0 is an
// impermeable node: u = 0 and F = -2 m / rho (Eq. 16b with u = 0).
__device__ __forceinline__ NodeState node_state(const float d[9], float eps,
                                                float inv_k, const StepArgs &a) {
  NodeState s;
  s.drho = ((d[0] + (d[1] + d[3])) + (d[2] + d[4])) + ((d[5] + d[7]) + (d[6] + d[8]));
  s.rho = a.rho0 + s.drho;
  // sum_i w_i e_i = 0, so the momentum of the deviations is the momentum.
  const float mx = (d[1] - d[3]) + ((d[5] - d[7]) + (d[8] - d[6]));
  const float my = (d[2] - d[4]) + ((d[5] - d[7]) + (d[6] - d[8]));
  const float inv_rho = 1.0f / s.rho;
  if (eps > 0.0f) {
    const float vx = fmaf(0.5f * eps, a.Gx, mx * inv_rho);
    const float vy = fmaf(0.5f * eps, a.Gy, my * inv_rho);
    const float darcy = eps * a.nu * inv_k;       // eps nu / k_a
    const float c0 = fmaf(0.25f, darcy, 0.5f);    // (1 + eps nu / (2 k_a)) / 2
    float den, forch = 0.0f;
    if (a.forch) {
      // c1 = eps F_eps / (2 sqrt(k_a)), F_eps = 1.75 / sqrt(150 eps^3)
      const float c1 = a.fe_half * sqrtf(inv_k) * rsqrtf(eps);
      const float vmag = sqrtf(fmaf(vx, vx, vy * vy));
      den = c0 + sqrtf(fmaf(c0, c0, c1 * vmag));
      forch = 2.0f * c1;                          // eps F_eps / sqrt(k_a)
    } else {
      den = 2.0f * c0;
    }
    const float inv_den = 1.0f / den;
    s.ux = vx * inv_den;
    s.uy = vy * inv_den;
    const float drag = (a.forch) ? fmaf(forch, sqrtf(fmaf(s.ux, s.ux, s.uy * s.uy)), darcy)
                                 : darcy;
    s.Fx = fmaf(-drag, s.ux, eps * a.Gx);
    s.Fy = fmaf(-drag, s.uy, eps * a.Gy);
  } else {
    s.ux = 0.0f;
    s.uy = 0.0f;
    s.Fx = -2.0f * mx * inv_rho;
    s.Fy = -2.0f * my * inv_rho;
  }
  return s;
}

// Deviation of the porous equilibrium (Eq. 14) from w_i rho0, all nine
// directions: deq_i = w_i (rho - rho0) + w_i rho (3 e.u + (9/2 (e.u)^2 -
// 3/2 u^2) / eps); eps = 0 keeps only w_i (rho - rho0).
__device__ __forceinline__ void equilibrium_dev(float drho, float rho, float ux,
                                                float uy, float eps, float deq[9]) {
  const float inv_eps = (eps > 0.0f) ? 1.0f / eps : 0.0f;
  const float vx = (eps > 0.0f) ? ux : 0.0f;
  const float vy = (eps > 0.0f) ? uy : 0.0f;
  const float usq = 1.5f * inv_eps * fmaf(vx, vx, vy * vy);
  const float q = 4.5f * inv_eps;
  const float r1 = kW1 * rho, r2 = kW2 * rho;
  const float dr1 = kW1 * drho, dr2 = kW2 * drho;
  deq[0] = fmaf(kW0 * rho, -usq, kW0 * drho);
  float eu;
  eu = vx;        deq[1] = fmaf(r1, 3.0f * eu + fmaf(q * eu, eu, -usq), dr1);
  eu = vy;        deq[2] = fmaf(r1, 3.0f * eu + fmaf(q * eu, eu, -usq), dr1);
  eu = -vx;       deq[3] = fmaf(r1, 3.0f * eu + fmaf(q * eu, eu, -usq), dr1);
  eu = -vy;       deq[4] = fmaf(r1, 3.0f * eu + fmaf(q * eu, eu, -usq), dr1);
  eu = vx + vy;   deq[5] = fmaf(r2, 3.0f * eu + fmaf(q * eu, eu, -usq), dr2);
  eu = vy - vx;   deq[6] = fmaf(r2, 3.0f * eu + fmaf(q * eu, eu, -usq), dr2);
  eu = -vx - vy;  deq[7] = fmaf(r2, 3.0f * eu + fmaf(q * eu, eu, -usq), dr2);
  eu = vx - vy;   deq[8] = fmaf(r2, 3.0f * eu + fmaf(q * eu, eu, -usq), dr2);
}

// Eq. 12 with Eq. 14 and Eq. 15 (last term over eps), in place on the
// deviations: d_i <- d_i - (d_i - deq_i) / tau + F_i.
__device__ __forceinline__ void collide(float d[9], const NodeState &s, float eps,
                                        const StepArgs &a) {
  float deq[9];
  equilibrium_dev(s.drho, s.rho, s.ux, s.uy, eps, deq);
  const float inv_eps = (eps > 0.0f) ? 1.0f / eps : 0.0f;
  const float ux = s.ux, uy = s.uy, Fx = s.Fx, Fy = s.Fy;
  const float uF3 = 3.0f * inv_eps * fmaf(ux, Fx, uy * Fy);
  const float g9 = 9.0f * inv_eps;
  const float c = s.rho * a.cforce;
  const float c0 = kW0 * c, c1 = kW1 * c, c2 = kW2 * c;
  const float om = a.omega;
  float eu, eF, Fi;
  Fi = -c0 * uF3;
  d[0] = fmaf(-om, d[0] - deq[0], d[0]) + Fi;
#define LBMP_DIR(I, EU, EF, CW)                                   \
  eu = (EU);                                                      \
  eF = (EF);                                                      \
  Fi = (CW) * (fmaf(g9 * eu, eF, 3.0f * eF) - uF3);               \
  d[I] = fmaf(-om, d[I] - deq[I], d[I]) + Fi;
  LBMP_DIR(1, ux, Fx, c1)
  LBMP_DIR(2, uy, Fy, c1)
  LBMP_DIR(3, -ux, -Fx, c1)
  LBMP_DIR(4, -uy, -Fy, c1)
  LBMP_DIR(5, ux + uy, Fx + Fy, c2)
  LBMP_DIR(6, uy - ux, Fy - Fx, c2)
  LBMP_DIR(7, -ux - uy, -Fx - Fy, c2)
  LBMP_DIR(8, ux - uy, Fx - Fy, c2)
#undef LBMP_DIR
}

// Pressure column (non-equilibrium extrapolation, Guo, Zheng & Shi 2002):
// d_b = d_n + deq(rho_b, u_n; eps_b) - deq(rho_n, u_n; eps_n), where n is the
// adjacent interior node and rho_b the imposed density.
template <class S>
__device__ __forceinline__ void pressure_node(const typename S::T *__restrict__ fin,
                                              const float2 *__restrict__ med,
                                              const StepArgs &a, int xb, int y,
                                              float eps_b, float d[9]) {
  const int xn = (xb == 0) ? 1 : a.nx - 2;
  const float2 mn = med[(long long)y * a.pitch + xn];
  float dn[9];
  pull_node<S>(fin, a, xn, y, dn);
  const NodeState sn = node_state(dn, mn.x, mn.y, a);
  const float drho_b = (xb == 0) ? a.drho_in : a.drho_out;
  float eq_b[9], eq_n[9];
  equilibrium_dev(drho_b, a.rho0 + drho_b, sn.ux, sn.uy, eps_b, eq_b);
  equilibrium_dev(sn.drho, sn.rho, sn.ux, sn.uy, mn.x, eq_n);
#pragma unroll
  for (int i = 0; i < 9; ++i) d[i] = dn[i] + (eq_b[i] - eq_n[i]);
}

}  // namespace lbmp
