// Discrete adjoint of the time loop (Section III, Eq. 12-17) for the global
// permeability k_g = nu <u_x> / G_eff of the final time level (Darcy's law
// over the domain, Section IV.A): gradients with respect to ln k_a and eps
// of every node.
//
// Forward: B_{t+1} = C(E(P(B_t))), B the post-collision buffer (B_0 = rest),
// P the pull (streaming with plates and periodic edges), E the pressure
// column extrapolation (non-equilibrium, from the adjacent interior node),
// C the collision of every fluid node; J depends on f^N = E(P(B_N)).
// Reverse: mu^N = dJ/df^N, then for t = N-1 .. 0
//   lambda*(z) = mu^{t+1}(z + e_i) for each direction (P transposed: a
//                plate returns it to the opposite direction of the same
//                node, a pressure column or the outside returns nothing),
//   mu^t       = C_t^T lambda* at the state f^t, with E^T folded in: a
//                column's adjoint is pushed into its interior neighbour by
//                the thread of that neighbour, which also forms it.
// C_t^T: post_i = (1 - 1/tau) f_i + g_i(rho, m; eps, k_a) with g_i = f_eq_i /
// tau + F_i (Eq. 14, 15), so mu_j = (1 - 1/tau) lambda*_j + dG/drho +
// e_j . dG/dm, G = sum_i lambda*_i g_i.  G is written through the weighted
// moments L0 = sum w lambda, L1 = sum w lambda e, L2 = sum w lambda e e of
// lambda* and differentiated by hand, back through the velocity solve of
// Eq. 16b-17 (with the Forchheimer drag of Eq. 2, the quadratic form).
// States f^t are recomputed segment by segment from checkpoints taken every
// `every` steps (sqrt(N) by default).  Each reverse step adds its parameter
// derivatives to FP32 accumulators, folded into the FP64 gradients every
// kFold steps (a schedule independent of `every`).
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <map>
#include <tuple>

#include "context.h"
#include "device_scope.h"
#include "kernels.h"
#include "lattice.cuh"
#include "lbmp.h"

namespace lbmp {

struct AdjArgs {
  StepArgs a;            // forward parameters (FP32 storage, scale 1)
  const float *lam_in;   // mu^{t+1}, [9][ny][pitch] (pressure columns unused)
  float *lam_out;        // mu^t
  const float *fin;      // forward buffer whose pull gives f^t (seed step)
  const float *mom;      // moments of f^t (rho - rho0, m_x, m_y planes; reverse steps)
  const float2 *med;     // (eps, 1/k_a)
  float2 *acc;           // [ny][pitch] (dJ/d eps, dJ/d ln k_a) of the last few steps, FP32
  double *g_eps;         // [ny][pitch] dJ/d eps, FP64 (acc folded in every kFold steps)
  double *g_lk;          // [ny][pitch] dJ/d ln k_a, FP64
  float coef;            // dJ/du_x of one node: nu / (G_eff * fluid nodes)
};

constexpr int kAdjBX = 128;
constexpr int kFold = 32;  // reverse steps summed in FP32 before the FP64 fold

// Weighted moments of an adjoint population vector.
struct LamMom {
  float L0, Lx, Ly, Lxx, Lxy, Lyy;
};
__device__ __forceinline__ LamMom lam_moments(const float l[9]) {
  const float s1 = l[1] + l[3], s2 = l[2] + l[4];
  const float a57 = l[5] + l[7], a68 = l[6] + l[8];
  const float d57 = l[5] - l[7], d86 = l[8] - l[6];
  LamMom M;
  M.L0 = kW0 * l[0] + kW1 * (s1 + s2) + kW2 * (a57 + a68);
  M.Lx = kW1 * (l[1] - l[3]) + kW2 * (d57 + d86);
  M.Ly = kW1 * (l[2] - l[4]) + kW2 * (d57 - d86);
  M.Lxx = kW1 * s1 + kW2 * (a57 + a68);
  M.Lyy = kW1 * s2 + kW2 * (a57 + a68);
  M.Lxy = kW2 * (a57 - a68);
  return M;
}

// Velocity solve of a node with eps > 0, kept for its adjoint:
// v = m / rho + eps G / 2, u = v / den, F = eps G - drag u, with
// den = c0 + s, s = sqrt(c0^2 + c1 |v|), drag = eps nu / k_a + 2 c1 |v| / den
// (Forchheimer), or den = 2 c0, drag = eps nu / k_a (Darcy only);
// c0 = 1/2 + eps nu / (4 k_a), c1 = (eps F_eps / 2) / sqrt(k_a).
struct Vel {
  float vx, vy, vmag, c0, c1, s, den, id, drag, ux, uy, Fx, Fy;  // id = 1 / den
};
__device__ __forceinline__ Vel vel_forward(float rho, float mx, float my, float eps, float kap,
                                           const StepArgs &a) {
  Vel V;
  const float ir = rcp_approx(rho);
  V.vx = fmaf(mx, ir, 0.5f * eps * a.Gx);
  V.vy = fmaf(my, ir, 0.5f * eps * a.Gy);
  const float darcy = a.nu * eps * kap;
  V.c0 = fmaf(0.25f, darcy, 0.5f);
  if (a.forch) {
    V.c1 = a.fe_half * sqrt_approx(kap * rcp_approx(eps));
    V.vmag = sqrt_approx(fmaf(V.vx, V.vx, V.vy * V.vy));
    V.s = sqrt_approx(fmaf(V.c0, V.c0, V.c1 * V.vmag));
    V.den = V.c0 + V.s;
    V.id = rcp_approx(V.den);
    V.drag = fmaf(2.0f * V.c1, V.vmag * V.id, darcy);
  } else {
    V.c1 = 0.0f;
    V.vmag = 0.0f;
    V.s = 0.0f;
    V.den = 2.0f * V.c0;
    V.id = rcp_approx(V.den);
    V.drag = darcy;
  }
  V.ux = V.vx * V.id;
  V.uy = V.vy * V.id;
  V.Fx = eps * a.Gx - V.drag * V.ux;
  V.Fy = eps * a.Gy - V.drag * V.uy;
  return V;
}

// Sensitivities of a node: d/drho and d/dm of its post-stream moments, and
// the parameter derivatives d/d eps and d/d ln k_a.
struct Bar {
  float rho, mx, my, eps, lk;
};

// Reverse of vel_forward: adds to b the derivatives of ub . u + Fb . F.
__device__ __forceinline__ void vel_adjoint(const Vel &V, float rho, float mx, float my,
                                            float eps, float kap, float ubx, float uby, float Fbx,
                                            float Fby, const StepArgs &a, Bar &b) {
  // F = eps G - drag u
  ubx -= V.drag * Fbx;
  uby -= V.drag * Fby;
  const float dragb = -(Fbx * V.ux + Fby * V.uy);
  b.eps += Fbx * a.Gx + Fby * a.Gy;
  // u = v / den
  const float id = V.id;
  float vbx = ubx * id, vby = uby * id;
  float denb = -(ubx * V.ux + uby * V.uy) * id;
  const float darcy = a.nu * eps * kap;
  float darcyb = dragb, c0b;
  if (a.forch) {
    // drag = darcy + 2 c1 |v| / den
    float c1b = 2.0f * dragb * V.vmag * id;
    float vmagb = 2.0f * dragb * V.c1 * id;
    denb -= 2.0f * dragb * V.c1 * V.vmag * id * id;
    // den = c0 + s, s = sqrt(c0^2 + c1 |v|) >= c0 >= 1/2
    const float is = rcp_approx(V.s);
    c0b = denb * (1.0f + V.c0 * is);
    c1b += 0.5f * denb * V.vmag * is;
    vmagb += 0.5f * denb * V.c1 * is;
    // |v|: at v = 0 the terms it enters vanish with u, so its derivative is
    // not needed there
    if (V.vmag > 0.0f) {
      const float iv = rcp_approx(V.vmag);
      vbx += vmagb * V.vx * iv;
      vby += vmagb * V.vy * iv;
    }
    // c1 = fe_half sqrt(kap / eps): dc1/d ln k_a = -c1 / 2, dc1/d eps = -c1 / (2 eps)
    b.lk -= 0.5f * V.c1 * c1b;
    b.eps -= 0.5f * V.c1 * c1b * rcp_approx(eps);
  } else {
    c0b = 2.0f * denb;
  }
  darcyb += 0.25f * c0b;
  // darcy = nu eps kap: d/d ln k_a = -darcy, d/d eps = nu kap
  b.lk -= darcy * darcyb;
  b.eps += a.nu * kap * darcyb;
  // v = m / rho + eps G / 2
  const float ir = rcp_approx(rho);
  b.mx += vbx * ir;
  b.my += vby * ir;
  b.rho -= (vbx * mx + vby * my) * ir * ir;
  b.eps += 0.5f * (vbx * a.Gx + vby * a.Gy);
}

// Adds to b the derivatives of G = sum_i lam_i g_i(rho, m; eps, k_a) of one
// node.  sum_i lam_i f_eq_i = rho [L0 + 3 u.L1 + (9/2 u.L2.u - 3/2 u^2 L0) /
// eps] (Eq. 14) and sum_i lam_i F_i = (1 - 1/2tau) rho [3 F.L1 + (9 u.L2.F -
// 3 (u.F) L0) / eps] (Eq. 15); eps = 0 keeps f_eq = w rho, u = 0 and
// F = -2 m / rho.
__device__ __forceinline__ void collide_adjoint(const float lam[9], float rho, float mx, float my,
                                                float eps, float kap, const StepArgs &a, Bar &b) {
  const LamMom M = lam_moments(lam);
  const float om = a.omega, cf = a.cforce;
  if (!(eps > 0.0f)) {
    b.rho += om * M.L0;
    b.mx -= 6.0f * cf * M.Lx;
    b.my -= 6.0f * cf * M.Ly;
    return;
  }
  const Vel V = vel_forward(rho, mx, my, eps, kap, a);
  const float ie = rcp_approx(eps);
  const float ux = V.ux, uy = V.uy, Fx = V.Fx, Fy = V.Fy;
  const float L2ux = M.Lxx * ux + M.Lxy * uy, L2uy = M.Lxy * ux + M.Lyy * uy;
  const float L2Fx = M.Lxx * Fx + M.Lxy * Fy, L2Fy = M.Lxy * Fx + M.Lyy * Fy;
  const float qe = 4.5f * (ux * L2ux + uy * L2uy) - 1.5f * (ux * ux + uy * uy) * M.L0;
  const float qf = 9.0f * (ux * L2Fx + uy * L2Fy) - 3.0f * (ux * Fx + uy * Fy) * M.L0;
  const float Seq = M.L0 + 3.0f * (ux * M.Lx + uy * M.Ly) + qe * ie;
  const float SF = 3.0f * (Fx * M.Lx + Fy * M.Ly) + qf * ie;
  b.rho += om * Seq + cf * SF;
  // dSeq/du = dSF/dF
  const float ax = 3.0f * M.Lx + (9.0f * L2ux - 3.0f * ux * M.L0) * ie;
  const float ay = 3.0f * M.Ly + (9.0f * L2uy - 3.0f * uy * M.L0) * ie;
  const float ubx = rho * (om * ax + cf * (9.0f * L2Fx - 3.0f * Fx * M.L0) * ie);
  const float uby = rho * (om * ay + cf * (9.0f * L2Fy - 3.0f * Fy * M.L0) * ie);
  b.eps -= rho * (om * qe + cf * qf) * ie * ie;
  vel_adjoint(V, rho, mx, my, eps, kap, ubx, uby, rho * cf * ax, rho * cf * ay, a, b);
}

// Pressure column b next to interior node n: f_b = f_n + f_eq(rho_b, u_n;
// eps_b) - f_eq(rho_n, u_n; eps_n).  Adds to bn the derivatives of
// sum_i lb_i f_b,i with respect to n's moments and parameters (the identity
// part, lb itself, is added by the caller) and to eb the one of eps_b.
__device__ __forceinline__ void neep_adjoint(const float lb[9], float rho_n, float mx, float my,
                                             float eps_n, float kap_n, float eps_b, float rho_b,
                                             const StepArgs &a, Bar &bn, float &eb) {
  const LamMom M = lam_moments(lb);
  if (!(eps_n > 0.0f)) {  // u_n = 0: f_b = f_n + w (rho_b - rho_n)
    bn.rho -= M.L0;
    return;
  }
  const Vel V = vel_forward(rho_n, mx, my, eps_n, kap_n, a);
  const float ux = V.ux, uy = V.uy;
  const float L2ux = M.Lxx * ux + M.Lxy * uy, L2uy = M.Lxy * ux + M.Lyy * uy;
  const float q = 4.5f * (ux * L2ux + uy * L2uy) - 1.5f * (ux * ux + uy * uy) * M.L0;
  const float cx = 3.0f * M.Lx, cy = 3.0f * M.Ly;
  const float qx = 9.0f * L2ux - 3.0f * ux * M.L0, qy = 9.0f * L2uy - 3.0f * uy * M.L0;
  const float ien = rcp_approx(eps_n);
  bn.rho -= M.L0 + (ux * cx + uy * cy) + q * ien;
  float ubx = -rho_n * (cx + qx * ien), uby = -rho_n * (cy + qy * ien);
  bn.eps += rho_n * q * ien * ien;
  if (eps_b > 0.0f) {
    const float ieb = rcp_approx(eps_b);
    ubx += rho_b * (cx + qx * ieb);
    uby += rho_b * (cy + qy * ieb);
    eb -= rho_b * q * ieb * ieb;
  }
  vel_adjoint(V, rho_n, mx, my, eps_n, kap_n, ubx, uby, 0.0f, 0.0f, a, bn);
}

__device__ __forceinline__ float lam_at(const AdjArgs &A, int i, int x, int y) {
  return A.lam_in[i * A.a.plane + (long long)y * A.a.pitch + x];
}

// Reverse streaming for node (x, y): the adjoint of its post-collision
// values, read where each of them streams to.
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
    yd = (yd < 0) ? yd + a.ny : (yd >= a.ny ? yd - a.ny : yd);
    if (a.pressure) {
      if (xd <= 0 || xd >= a.nx - 1) {  // lost at the edge or received by a pressure column
        lp[i] = 0.0f;
        continue;
      }
    } else {
      xd = (xd < 0) ? xd + a.nx : (xd >= a.nx ? xd - a.nx : xd);
    }
    lp[i] = lam_at(A, i, xd, yd);
  }
}

__device__ __forceinline__ void moments(const float d[9], float rho0, float &rho, float &mx,
                                        float &my) {
  const float drho = ((d[0] + (d[1] + d[3])) + (d[2] + d[4])) + ((d[5] + d[7]) + (d[6] + d[8]));
  rho = rho0 + drho;
  mx = (d[1] - d[3]) + ((d[5] - d[7]) + (d[8] - d[6]));
  my = (d[2] - d[4]) + ((d[5] - d[7]) + (d[6] - d[8]));
}

// Adjoint of the pressure column beside interior node (x, y), formed and
// pushed into the node by the node's own thread: the column's adjoint lb =
// (1 - 1/tau) lambda*_b + its collision adjoint (SEED: the objective's
// dJ/df_b instead), then E^T.  Adds lb to mu and the node's moment and
// parameter sensitivities to bn; writes the column's parameter gradients.
template <bool SEED>
__device__ __forceinline__ void column_adjoint(const AdjArgs &A, int x, int y, float rho,
                                               float mx, float my, float2 mn, float mu[9],
                                               Bar &bn) {
  const StepArgs &a = A.a;
  const int ex[9] = {0, 1, 0, -1, 0, 1, -1, -1, 1};
  const int ey[9] = {0, 0, 1, 0, -1, 1, 1, -1, -1};
#pragma unroll 1
  for (int side = 0; side < 2; ++side) {
    const int xn = side ? a.nx - 2 : 1;
    if (x != xn) continue;
    const int xb = side ? a.nx - 1 : 0;
    const long long jb = (long long)y * a.pitch + xb;
    const float2 mb = A.med[jb];
    float rb, mbx, mby;
    if (SEED) {
      float fb[9];
      pressure_node<StoreF32>(A.fin, A.med, a, xb, y, mb.x, fb);
      moments(fb, a.rho0, rb, mbx, mby);
    } else {  // the column's moments as its forward step stored them
      rb = a.rho0 + A.mom[jb];
      mbx = A.mom[a.plane + jb];
      mby = A.mom[2 * a.plane + jb];
    }
    Bar bb = {0.0f, 0.0f, 0.0f, 0.0f, 0.0f};
    float lb[9];
    if (SEED) {
      if (mb.x > 0.0f) {
        const Vel V = vel_forward(rb, mbx, mby, mb.x, mb.y, a);
        vel_adjoint(V, rb, mbx, mby, mb.x, mb.y, A.coef, 0.0f, 0.0f, 0.0f, a, bb);
      }
#pragma unroll
      for (int i = 0; i < 9; ++i) lb[i] = bb.rho + ex[i] * bb.mx + ey[i] * bb.my;
    } else {
      float lpb[9];
      reverse_pull(A, xb, y, lpb);
      collide_adjoint(lpb, rb, mbx, mby, mb.x, mb.y, a, bb);
#pragma unroll
      for (int i = 0; i < 9; ++i)
        lb[i] = fmaf(a.one_m_omega, lpb[i], bb.rho + ex[i] * bb.mx + ey[i] * bb.my);
    }
    float eb = 0.0f;
    const float rho_b = a.rho0 + (side ? a.drho_out : a.drho_in);
    neep_adjoint(lb, rho, mx, my, mn.x, mn.y, mb.x, rho_b, a, bn, eb);
#pragma unroll
    for (int i = 0; i < 9; ++i) mu[i] += lb[i];
    const float2 g = A.acc[jb];  // only this thread touches the column node
    A.acc[jb] = make_float2(g.x + (bb.eps + eb), g.y + bb.lk);
  }
}

// One reverse step over the fluid rows: mu^t from mu^{t+1} and f^t.
// SEED: the objective instead, mu^N = dJ/df^N.  Pressure-column threads
// return at once (their neighbours handle them).
template <bool SEED>
__global__ void __launch_bounds__(kAdjBX, 8) adjoint_step_kernel(const AdjArgs A) {
  const StepArgs &a = A.a;
  const int y = a.y0 + blockIdx.y;
  const int x = blockIdx.x * kAdjBX + threadIdx.x;
  if (x >= a.nx) return;
  if (a.pressure && (x == 0 || x == a.nx - 1)) return;
  const int ex[9] = {0, 1, 0, -1, 0, 1, -1, -1, 1};
  const int ey[9] = {0, 0, 1, 0, -1, 1, 1, -1, -1};
  const long long j = (long long)y * a.pitch + x;
  // the accumulators are read up front so that their latency overlaps the
  // population loads
  const float2 g0 = A.acc[j];
  const float2 m = __ldg(A.med + j);
  float mu[9];
  float rho, mx, my;
  if (SEED) {
    float d[9];
    pull_node<StoreF32>(A.fin, a, x, y, d);
    moments(d, a.rho0, rho, mx, my);
  } else {  // the moments of f^t, stored by the recompute step (bit for bit
            // the sums above)
    rho = a.rho0 + A.mom[j];
    mx = A.mom[a.plane + j];
    my = A.mom[2 * a.plane + j];
  }
  Bar b = {0.0f, 0.0f, 0.0f, 0.0f, 0.0f};
  if (SEED) {
    if (m.x > 0.0f) {
      const Vel V = vel_forward(rho, mx, my, m.x, m.y, a);
      vel_adjoint(V, rho, mx, my, m.x, m.y, A.coef, 0.0f, 0.0f, 0.0f, a, b);
    }
#pragma unroll
    for (int i = 0; i < 9; ++i) mu[i] = 0.0f;
  } else {
    float lp[9];
    // Away from the lattice edges every destination z + e_i is a plain fluid
    // node at a fixed offset; the edge rules of reverse_pull apply to the rest.
    const bool inner = x >= 2 && x <= a.nx - 3 && y >= 2 && y <= a.ny - 3;
    if (inner) {
      const float *l = A.lam_in + j;
      const long long P = a.plane, R = a.pitch;
      lp[0] = l[0];
      lp[1] = l[P + 1];
      lp[2] = l[2 * P + R];
      lp[3] = l[3 * P - 1];
      lp[4] = l[4 * P - R];
      lp[5] = l[5 * P + R + 1];
      lp[6] = l[6 * P + R - 1];
      lp[7] = l[7 * P - R - 1];
      lp[8] = l[8 * P - R + 1];
    } else {
      reverse_pull(A, x, y, lp);
    }
    collide_adjoint(lp, rho, mx, my, m.x, m.y, a, b);
#pragma unroll
    for (int i = 0; i < 9; ++i) mu[i] = a.one_m_omega * lp[i];
  }
  if (a.pressure && (x == 1 || x == a.nx - 2)) column_adjoint<SEED>(A, x, y, rho, mx, my, m, mu, b);
#pragma unroll
  for (int i = 0; i < 9; ++i)
    A.lam_out[i * a.plane + j] = mu[i] + b.rho + ex[i] * b.mx + ey[i] * b.my;
  A.acc[j] = make_float2(g0.x + b.eps, g0.y + b.lk);
}

// Folds the FP32 accumulators of the fluid rows into the FP64 gradients
// and clears them.
__global__ void __launch_bounds__(kAdjBX) adjoint_fold_kernel(const AdjArgs A) {
  const StepArgs &a = A.a;
  const int y = a.y0 + blockIdx.y;
  const int x = blockIdx.x * kAdjBX + threadIdx.x;
  if (x >= a.nx) return;
  const long long j = (long long)y * a.pitch + x;
  const float2 g = A.acc[j];
  A.g_eps[j] += (double)g.x;
  A.g_lk[j] += (double)g.y;
  A.acc[j] = make_float2(0.0f, 0.0f);
}

// dJ/d ln k_a and dJ/d eps (+ the mean-porosity term of the pressure drop)
// into [ny][nx] float64; plate rows read 0.
__global__ void adjoint_assemble_kernel(const AdjArgs A, double eps_term, double *out_logk,
                                        double *out_eps) {
  const StepArgs &a = A.a;
  const int y = blockIdx.y;
  const int x = blockIdx.x * kAdjBX + threadIdx.x;
  if (x >= a.nx) return;
  const long long o = (long long)y * a.nx + x;
  if (a.walls && (y == 0 || y == a.ny - 1)) {
    out_logk[o] = 0.0;
    out_eps[o] = 0.0;
    return;
  }
  const long long j = (long long)y * a.pitch + x;
  out_logk[o] = A.g_lk[j];
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

// The launches of one backward segment: n recompute steps from the
// checkpoint copy in seg[0] (the two state buffers alternate; level t's
// moments go to mom + t * mom_level), then the n reverse steps from the
// last level down, with an FP64 fold after every kFold-th reverse step of
// the whole sweep (`reversed` of them done before this segment).  lam[0]
// holds Lambda^{t+1} of the segment's last level on entry.
cudaError_t enqueue_segment(const lbmp::AdjArgs &A0, int rows, const float2 *med, char *segp,
                            size_t state, char *momp, size_t mom_level, int64_t n,
                            float *const lam[2], int64_t reversed, cudaStream_t s) {
  lbmp::AdjArgs A = A0;
  const lbmp::StepArgs &a = A.a;
  cudaError_t e = cudaSuccess;
  for (int64_t t = 0; t < n && e == cudaSuccess; ++t)
    e = lbmp::launch_step_moments(a, rows, (const float *)(segp + state * (t & 1)),
                                  (float *)(segp + state * ((t + 1) & 1)), med,
                                  (float *)(momp + mom_level * t), s);
  const dim3 blk(lbmp::kAdjBX), grd((a.nx + lbmp::kAdjBX - 1) / lbmp::kAdjBX, rows);
  int next = 0;
  for (int64_t t = n - 1; t >= 0 && e == cudaSuccess; --t) {
    A.lam_in = lam[next];
    A.lam_out = lam[next ^ 1];
    A.fin = nullptr;
    A.mom = (const float *)(momp + mom_level * t);
    lbmp::adjoint_step_kernel<false><<<grd, blk, 0, s>>>(A);
    e = cudaGetLastError();
    next ^= 1;
    if (e == cudaSuccess && ++reversed % lbmp::kFold == 0) {
      lbmp::adjoint_fold_kernel<<<grd, blk, 0, s>>>(A);
      e = cudaGetLastError();
    }
  }
  return e;
}

// Instantiated backward-segment graphs of one gradient call, keyed by the
// segment length, which adjoint buffer holds Lambda^{t+1} on entry, and
// the fold phase (reversed steps mod kFold): full segments share one graph
// per phase, so a call captures at most kFold + 1 of them.
struct SegmentGraphs {
  std::map<std::tuple<int64_t, int, int>, cudaGraphExec_t> g;
  ~SegmentGraphs() {
    for (auto &kv : g) cudaGraphExecDestroy(kv.second);
  }
};

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
    if (c->p.kn_beta != 0.0)
      return afail(LBMP_EINVAL, "lbmp_permeability_gradient: a dynamic Kn is not available");
    const DeviceScope device_scope(c->device);
    ACK(device_scope.err);
    if (every == 0) every = (int64_t)std::ceil(std::sqrt((double)nsteps));
    every = std::min(every, nsteps);
    const int64_t nseg = (nsteps + every - 1) / every;
    const StepArgs a = c->args();
    const int rows = c->rows();
    const size_t state = c->buf_bytes();
    const size_t field = (size_t)c->plane * sizeof(double);
    cudaStream_t s = c->stream;
    // checkpoints (one per segment), two states for the recompute, the
    // moments of the levels of one segment, the two adjoint levels, the FP64
    // gradient fields
    const size_t mom_level = (size_t)c->plane * 3 * sizeof(float);
    DevBuf ck, seg, mom, lam, grad, outs;
    ACK(cudaMalloc(&ck.p, state * (size_t)nseg));
    ACK(cudaMalloc(&seg.p, state * 2));
    ACK(cudaMalloc(&mom.p, mom_level * (size_t)every));
    ACK(cudaMalloc(&lam.p, state * 2));
    const size_t accb = (size_t)c->plane * sizeof(float2);
    ACK(cudaMalloc(&grad.p, field * 2 + accb));
    ACK(cudaMemsetAsync(lam.p, 0, state * 2, s));
    ACK(cudaMemsetAsync(grad.p, 0, field * 2 + accb, s));
    char *ckp = (char *)ck.p, *segp = (char *)seg.p, *momp = (char *)mom.p;
    float *lam0 = (float *)lam.p, *lam1 = (float *)((char *)lam.p + state);
    double *g_eps = (double *)grad.p, *g_lk = (double *)((char *)grad.p + field);
    float2 *acc = (float2 *)((char *)grad.p + 2 * field);

    // forward pass from rest in the context's own buffers (the step graphs
    // of lbmp_step), checkpointing the first level of every segment
    ACK(cudaMemsetAsync(c->buf[0], 0, state, s));
    ACK(cudaMemsetAsync(c->buf[1], 0, state, s));
    ACK(cudaMemsetAsync(c->d_err, 0, sizeof(unsigned), s));
    c->cur = 0;
    c->steps = 0;
    for (int64_t sg = 0; sg < nseg; ++sg) {
      ACK(cudaMemcpyAsync(ckp + state * sg, c->buf[c->cur], state, cudaMemcpyDeviceToDevice, s));
      lbmp_status fst = lbmp_step(c, std::min(every, nsteps - sg * every));
      if (fst) return fst;
    }
    const int cur = c->cur;
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
    A.g_lk = g_lk;
    A.acc = acc;
    A.coef = (float)(nu / (geff * nf));
    // seed: Lambda^N = dJ/df^N
    const dim3 blk(lbmp::kAdjBX), grd((a.nx + lbmp::kAdjBX - 1) / lbmp::kAdjBX, rows);
    A.fin = (const float *)c->buf[cur];
    A.mom = nullptr;
    A.lam_in = lam1;
    A.lam_out = lam0;
    lbmp::adjoint_step_kernel<true><<<grd, blk, 0, s>>>(A);
    ACK(cudaGetLastError());
    // backward, one segment at a time: recompute its levels from the
    // checkpoint (keeping only their moments), then run the reverse steps
    // over them; each segment replays a captured graph
    float *lams[2] = {lam0, lam1};  // lams[0]: Lambda^{t+1} of the next reverse step
    int64_t reversed = 0;          // the FP32 accumulators fold every kFold reverse steps
    SegmentGraphs graphs;
    for (int64_t sg = nseg - 1; sg >= 0; --sg) {
      const int64_t t0 = sg * every, n = std::min(every, nsteps - t0);
      ACK(cudaMemcpyAsync(segp, ckp + state * sg, state, cudaMemcpyDeviceToDevice, s));
      const auto key = std::make_tuple(n, lams[0] == lam0 ? 0 : 1, (int)(reversed % lbmp::kFold));
      auto it = graphs.g.find(key);
      if (it == graphs.g.end()) {
        cudaGraph_t g = nullptr;
        ACK(cudaStreamBeginCapture(c->cap_stream, cudaStreamCaptureModeThreadLocal));
        cudaError_t ce = enqueue_segment(A, rows, c->med, segp, state, momp, mom_level, n, lams,
                                         reversed, c->cap_stream);
        cudaError_t ee = cudaStreamEndCapture(c->cap_stream, &g);
        if (ce != cudaSuccess || ee != cudaSuccess) {
          if (g) cudaGraphDestroy(g);
          ACK(ce != cudaSuccess ? ce : ee);
        }
        cudaGraphExec_t exec = nullptr;
        cudaError_t ie = cudaGraphInstantiate(&exec, g, 0);
        cudaGraphDestroy(g);
        ACK(ie);
        it = graphs.g.emplace(key, exec).first;
      }
      ACK(cudaGraphLaunch(it->second, s));
      const int64_t folds = (reversed + n) / lbmp::kFold - reversed / lbmp::kFold;
      c->launches += 2 * n + folds;
      reversed += n;
      if (n & 1) std::swap(lams[0], lams[1]);
    }
    lbmp::adjoint_fold_kernel<<<grd, blk, 0, s>>>(A);
    ACK(cudaGetLastError());
    // d/d eps_z of G_eff through the mean porosity (pressure drive only)
    const double eps_term = (kp != 0.0) ? J * kp / (geff * c->eps_mean * nf) : 0.0;
    const size_t nn = (size_t)a.nx * a.ny;
    double *ol = d_logk, *oe = d_eps;
    if (where == LBMP_HOST) {
      ACK(cudaMalloc(&outs.p, 2 * nn * sizeof(double)));
      ol = (double *)outs.p;
      oe = ol + nn;
    }
    const dim3 g2((a.nx + lbmp::kAdjBX - 1) / lbmp::kAdjBX, a.ny);
    lbmp::adjoint_assemble_kernel<<<g2, blk, 0, s>>>(A, eps_term, ol, oe);
    ACK(cudaGetLastError());
    c->launches += 4;
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
