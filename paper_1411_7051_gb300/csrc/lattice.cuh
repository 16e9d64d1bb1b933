// Device building blocks of the porous lattice Boltzmann step
// (Chen et al., arXiv:1411.7051, Section III, Eq. 12-17 and Eq. 2).
//
// State representation.  After t time steps, population buffer B holds the
// post-collision values f*_i(x, t-1) of every fluid node, stored as the
// shifted deviation d_i = f_i - w_i rho0, scaled by S (S = 1 for FP32,
// S = 2^s for FP16).  Pulling B (f_i(x) <- f*_i(x - e_i), the streaming of
// Eq. 12) gives the post-stream populations f_i(x, t), from which density
// and velocity (Eq. 16-17) are defined.  The initial buffer is all zeros.
// Device code works on these "stored units" directly; S enters only through
// a few per-node scalars.
//
// Layout in HBM: 9 planes [9][ny][pitch] (plane = pitch * ny elements,
// pitch a multiple of 64 elements), medium as float2 (eps, 1/k_a) per node
// on the same [ny][pitch] grid (read as float4 for a node pair).
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
  float one_m_omega;   // 1 - 1 / tau
  float cforce;        // 1 - 1 / (2 tau)  (Eq. 15 prefactor)
  float nu;            // nu_e / J
  float Gx, Gy;        // body force of Eq. 2
  float fe_half;       // (1/2) 1.75 / sqrt(150): eps F_eps / 2 = fe_half / sqrt(eps)
  float scale;         // storage scale S (1 for FP32)
  float inv_scale;     // 1 / S
  int walls;           // rows 0 and ny-1 are plates (halfway bounce-back)
  int pressure;        // columns 0 and nx-1 carry imposed densities
  int forch;           // keep the Forchheimer drag of Eq. 2
  uint32_t seed_lo, seed_hi;  // stochastic rounding stream
  int test_drop_tile;   // staged kernel: tile whose copies are withheld (-1: none);
                        // exercises the bounded waits in tests
  int kn_model;         // f_c: 0 Eq. 6-7 (second order), 1 Eq. 4-5 (first order)
  float kn_beta;        // dynamic Kn: p / p0 = 1 + kn_beta (rho - rho0)
  const float *kn0;     // dynamic Kn: [ny][pitch] Kn at p0 (medium then holds 1/k_i);
                        // NULL for a static Kn (medium holds 1/k_a)
  int rev = 0;          // walk the launch's rows (direct) or tiles (staged) from the end:
                        // alternate steps then start where the previous one finished,
                        // on lines it left in L2.  The order of the nodes' updates
                        // changes nothing in their results.
};

// ------------------------------------------------ hardware approximations
// PTX approximate reciprocal and square root (relative error ~2^-23); the
// step needs ~1e-7, and IEEE-exact division would double the instruction
// count of the kernel.
__device__ __forceinline__ float rcp_approx(float x) {
  float r;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}
__device__ __forceinline__ float sqrt_approx(float x) {
  float r;
  asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}

// 32-bit avalanche mix (the finalizer of MurmurHash3), for the counter-based
// stochastic-rounding bits.
__device__ __forceinline__ uint32_t mix32(uint32_t h) {
  h ^= h >> 16;
  h *= 0x85ebca6bu;
  h ^= h >> 13;
  h *= 0xc2b2ae35u;
  h ^= h >> 16;
  return h;
}

// f_c of Eq. 6-7 (b = -1; model 0) or of Eq. 4-5 (model 1) in FP32, any
// Kn >= 0.  At Kn = 0 the power Kn^-0.4348 is +inf, alpha 0 and f_c exactly
// 1; at huge Kn, Kn / (1 + Kn) is taken as 1 (no inf / inf).
__device__ __forceinline__ float fc_f32(float kn, int model) {
  if (model == 1) return fmaf(4.0f, kn, 1.0f);
  const float t = exp2f(-0.4348f * log2f(kn));
  const float alpha = 1.358f / fmaf(0.170f, t, 1.0f);
  const float r = kn < 1e30f ? kn / (1.0f + kn) : 1.0f;
  return fmaf(alpha, kn, 1.0f) * fmaf(4.0f, r, 1.0f);
}

// Kn^-0.4348 for a normal FP32 Kn from the hardware base-2 logarithm and
// power (lg2.approx: absolute error ~2^-22.6, the exponent part exact;
// ex2.approx: relative ~2^-22.5).  The exponent y = -0.4348 log2 Kn is
// carried as y_hi + y_lo (exact product, the constant as hi + lo) and
// 2^y = 2^y_hi (1 + ln2 y_lo): ~3e-7 relative in all, where rounding y to
// one FP32 would alone cost up to 7e-7 at |y| ~ 17.  t enters f_c with a
// sensitivity below 0.08.
__device__ __forceinline__ float kn_power(float K) {
  constexpr float c_hi = -0.4348f;
  constexpr float c_lo = (float)(-0.4348 - (double)c_hi);
  float lg, t;
  asm("lg2.approx.ftz.f32 %0, %1;" : "=f"(lg) : "f"(K));
  const float y_hi = __fmul_rn(lg, c_hi);
  const float y_lo = __fmaf_rn(lg, c_lo, __fmaf_rn(lg, c_hi, -y_hi));
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(t) : "f"(y_hi));
  return __fmaf_rn(__fmul_rn(t, 0.69314718f), y_lo, t);
}

// n / d (d normal, positive) from the approximate reciprocal and one Newton
// correction of the quotient: q0 = n r, q0 + r (n - d q0) with the residual
// exact by fma; within ~1 ulp, where the IEEE division takes a longer
// sequence.
__device__ __forceinline__ float div_newton(float n, float d) {
  float r;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(d));
  const float q = __fmul_rn(n, r);
  return __fmaf_rn(r, __fmaf_rn(-d, q, n), q);
}

// (1/k_i) / f_c(Kn) (Eq. 3) for a node's current Kn, as one fraction:
// f_c = ((a + 1.358 Kn) / a) ((1 + 5 Kn) / (1 + Kn)) with a = 1 + 0.17
// Kn^-0.4348 (Eq. 6-7, b = -1), so one division where the factor form
// takes three; Eq. 4-5: (1/k_i) / (1 + 4 Kn).  Kn = 0 (and subnormal Kn)
// gives f_c = 1; Kn above 1e12 takes fc_f32 (the fraction would overflow).
__device__ __forceinline__ float inv_ka_dynamic(float inv_k, float kn, int model) {
  if (model == 1) return div_newton(inv_k, __fmaf_rn(4.0f, kn, 1.0f));
  if (!(kn >= 1.17549435e-38f)) return inv_k;
  if (kn > 1e12f) return inv_k / fc_f32(kn, 0);
  const float a = __fmaf_rn(0.17f, kn_power(kn), 1.0f);
  const float num = __fmul_rn(__fmul_rn(inv_k, a), __fadd_rn(1.0f, kn));
  const float den = __fmul_rn(__fmaf_rn(1.358f, kn, a), __fmaf_rn(5.0f, kn, 1.0f));
  return div_newton(num, den);
}

// ----------------------------------------------------------------- storage
struct StoreF32 {
  using T = float;
  static __device__ __forceinline__ float ld1(const float *p) { return *p; }
  static __device__ __forceinline__ void ld2(const float *p, float &a, float &b) {
    const float2 v = *reinterpret_cast<const float2 *>(p);
    a = v.x;
    b = v.y;
  }
  static __device__ __forceinline__ void st1(float *p, float v) { *p = v; }
  template <bool SR>
  static __device__ __forceinline__ void st1r(float *p, float v, uint32_t, int) { *p = v; }
  static constexpr bool kHiLo = true;
  template <bool SR>
  static __device__ __forceinline__ void st2(float *p, float a, float b, uint32_t, uint32_t) {
    *reinterpret_cast<float2 *>(p) = make_float2(a, b);
  }
};

struct StoreF16 {
  using T = __half;
  static __device__ __forceinline__ float ld1(const __half *p) { return __half2float(*p); }
  static __device__ __forceinline__ void ld2(const __half *p, float &a, float &b) {
    const float2 v = __half22float2(*reinterpret_cast<const __half2 *>(p));
    a = v.x;
    b = v.y;
  }
  static __device__ __forceinline__ void st1(__half *p, float v) { *p = __float2half_rn(v); }
  static constexpr bool kHiLo = false;
  // Scalar store; with SR the 8 random bits of direction i come from the
  // node hash h times an odd constant of that direction.
  template <bool SR>
  static __device__ __forceinline__ void st1r(__half *p, float v, uint32_t h, int i) {
    if (SR) {
      constexpr uint32_t kC[9] = {0x9e3779b1u, 0x85ebca77u, 0xc2b2ae3du, 0x27d4eb2fu,
                                  0x165667b1u, 0xd3a2646du, 0xfd7046c5u, 0xb55a4f09u,
                                  0x7feb352du};
      const uint32_t r = ((h * kC[i]) >> 24) << 5;  // 8 bits just below the FP16 LSB
      const float sv = __uint_as_float(__float_as_uint(v) + r);
      unsigned short b;
      asm("cvt.rz.f16.f32 %0, %1;" : "=h"(b) : "f"(sv));
      *reinterpret_cast<unsigned short *>(p) = b;
    } else {
      *p = __float2half_rn(v);
    }
  }
  // Node pair -> one 32-bit word.  SR: the hardware stochastic rounding
  // cvt.rs, whose random operand supplies bits 31..16 to the upper half
  // (node b) and bits 15..0 to the lower half (node a); a value between two
  // FP16 neighbours rounds up with probability equal to its distance from
  // the lower one.  Otherwise round to nearest even.
  template <bool SR>
  static __device__ __forceinline__ void st2(__half *p, float a, float b, uint32_t rbits,
                                             uint32_t) {
    uint32_t packed;
    if (SR) {
      asm("cvt.rs.f16x2.f32 %0, %1, %2, %3;" : "=r"(packed) : "f"(b), "f"(a), "r"(rbits));
    } else {
      const __half2 h = __floats2half2_rn(a, b);
      packed = *reinterpret_cast<const uint32_t *>(&h);
    }
    *reinterpret_cast<uint32_t *>(p) = packed;
  }
};

// ------------------------------------------------------------------- pull
// Post-stream values d[0..8] (stored units) of node (x, y): f_i(x) =
// f*_i(x - e_i); a source in a plate row returns the node's own population
// of the opposite direction (halfway bounce-back); periodic edges wrap.
template <class S>
__device__ __forceinline__ void pull_node(const typename S::T *__restrict__ fin,
                                          const StepArgs &a, int x, int y, float d[9]) {
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
  d[0] = S::ld1(fin + r + x);
  d[1] = S::ld1(fin + 1 * P + r + xm);
  d[3] = S::ld1(fin + 3 * P + r + xp);
  d[2] = wm ? S::ld1(fin + 4 * P + r + x) : S::ld1(fin + 2 * P + rm + x);
  d[5] = wm ? S::ld1(fin + 7 * P + r + x) : S::ld1(fin + 5 * P + rm + xm);
  d[6] = wm ? S::ld1(fin + 8 * P + r + x) : S::ld1(fin + 6 * P + rm + xp);
  d[4] = wp ? S::ld1(fin + 2 * P + r + x) : S::ld1(fin + 4 * P + rp + x);
  d[7] = wp ? S::ld1(fin + 5 * P + r + x) : S::ld1(fin + 7 * P + rp + xp);
  d[8] = wp ? S::ld1(fin + 6 * P + r + x) : S::ld1(fin + 8 * P + rp + xm);
}

// ------------------------------------------------- explicit FP32 arithmetic
// The node update is written once over a lane type V: float for one node,
// float2 for a node pair held in the two lanes and computed with the packed
// FP32 instructions of sm_100 and later (add / mul / fma .f32x2), whose
// lanes round exactly as the scalar operations do.  Every operation is
// spelled out (no multiply-add contraction left to the compiler), so a node
// gives the same bits on either path, and the pair path issues about half
// the arithmetic instructions.
__device__ __forceinline__ float vadd(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ float vsub(float a, float b) { return __fsub_rn(a, b); }
__device__ __forceinline__ float vmul(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ float vfma(float a, float b, float c) { return __fmaf_rn(a, b, c); }
__device__ __forceinline__ float vneg(float a) { return -a; }
__device__ __forceinline__ float vrcp(float a) { return rcp_approx(a); }
__device__ __forceinline__ float vsqrt(float a) { return sqrt_approx(a); }

// The packed forms are inline PTX with an explicit .rn.  The code generator
// may still fuse a packed multiply into a packed add that consumes it
// (observed: ~10% of the updates then differ in the last bit from the
// one-node path, and the difference moves with the surrounding code), so
// the update below never adds or subtracts the result of a multiply: each
// such pair is written as one fma on both paths.
#define LBMP_F32X2_2(op)                                                      \
  float2 r;                                                                   \
  asm("{\n\t.reg .b64 p, q, t;\n\t"                                       \
      "mov.b64 p, {%2, %3};\n\tmov.b64 q, {%4, %5};\n\t" op               \
      " t, p, q;\n\tmov.b64 {%0, %1}, t;\n\t}"                            \
      : "=f"(r.x), "=f"(r.y)                                                  \
      : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y));                              \
  return r
__device__ __forceinline__ float2 vadd(float2 a, float2 b) { LBMP_F32X2_2("add.rn.f32x2"); }
__device__ __forceinline__ float2 vsub(float2 a, float2 b) { LBMP_F32X2_2("sub.rn.f32x2"); }
__device__ __forceinline__ float2 vmul(float2 a, float2 b) { LBMP_F32X2_2("mul.rn.f32x2"); }
#undef LBMP_F32X2_2
__device__ __forceinline__ float2 vfma(float2 a, float2 b, float2 c) {
  float2 r;
  asm("{\n\t.reg .b64 p, q, s, t;\n\t"
      "mov.b64 p, {%2, %3};\n\tmov.b64 q, {%4, %5};\n\tmov.b64 s, {%6, %7};\n\t"
      "fma.rn.f32x2 t, p, q, s;\n\tmov.b64 {%0, %1}, t;\n\t}"
      : "=f"(r.x), "=f"(r.y)
      : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y), "f"(c.x), "f"(c.y));
  return r;
}
__device__ __forceinline__ float2 vneg(float2 a) { return make_float2(-a.x, -a.y); }
__device__ __forceinline__ float2 vrcp(float2 a) {
  return make_float2(rcp_approx(a.x), rcp_approx(a.y));
}
__device__ __forceinline__ float2 vsqrt(float2 a) {
  return make_float2(sqrt_approx(a.x), sqrt_approx(a.y));
}

template <class V>
__device__ __forceinline__ V vsplat(float s);
template <>
__device__ __forceinline__ float vsplat<float>(float s) { return s; }
template <>
__device__ __forceinline__ float2 vsplat<float2>(float s) { return make_float2(s, s); }

// ---------------------------------------------------- macroscopic state
template <class V>
struct NodeStateT {
  V drho_s;  // (rho - rho0) * S
  V mx, my;  // momentum sum_i f_i e_i, stored units
  V rho;     // physical density
  V ux, uy;  // physical velocity (Eq. 17 / quadratic form)
  V Fx, Fy;  // total force (Eq. 2 / Eq. 8)
  V rFx, rFy;  // rho S F (stored units): the momentum the force adds
  V ieps;    // 1 / eps (0 for an impermeable node)
};
using NodeState = NodeStateT<float>;

// Velocity and force of a permeable node (eps > 0): v = m / rho + eps G / 2,
// u = v / (c0 + sqrt(c0^2 + c1 |v|)) (Eq. 17 when c1 = 0, i.e. without the
// Forchheimer term), F = eps G - (eps nu / k_a + eps F_eps |u| / sqrt(k_a)) u
// (Eq. 2).  c = 1 / (S rho).
template <class V>
__device__ __forceinline__ void porous_state(NodeStateT<V> &s, V eps, V inv_k, V c,
                                             const StepArgs &a) {
  s.ieps = vrcp(eps);
  const V eGx = vmul(eps, vsplat<V>(a.Gx)), eGy = vmul(eps, vsplat<V>(a.Gy));
  const V vx = vfma(vsplat<V>(0.5f), eGx, vmul(s.mx, c));
  const V vy = vfma(vsplat<V>(0.5f), eGy, vmul(s.my, c));
  const V darcy = vmul(vmul(eps, vsplat<V>(a.nu)), inv_k);  // eps nu / k_a
  const V c0 = vfma(vsplat<V>(0.25f), darcy, vsplat<V>(0.5f));  // (1 + eps nu / (2 k_a)) / 2
  V idn, drag;
  if (a.forch) {
    // c1 = eps F_eps / (2 sqrt(k_a)) with F_eps = 1.75 / sqrt(150 eps^3)
    const V c1 = vmul(vsplat<V>(a.fe_half), vsqrt(vmul(inv_k, s.ieps)));
    const V vmag = vsqrt(vfma(vx, vx, vmul(vy, vy)));
    idn = vrcp(vadd(c0, vsqrt(vfma(c0, c0, vmul(c1, vmag)))));
    // eps nu / k_a + eps F_eps |u| / sqrt(k_a)
    drag = vfma(vmul(vsplat<V>(2.0f), c1), vmul(vmag, idn), darcy);
  } else {
    idn = vrcp(vmul(vsplat<V>(2.0f), c0));
    drag = darcy;
  }
  s.ux = vmul(vx, idn);
  s.uy = vmul(vy, idn);
  s.Fx = vfma(vneg(drag), s.ux, eGx);
  s.Fy = vfma(vneg(drag), s.uy, eGy);
  const V rs = vmul(s.rho, vsplat<V>(a.scale));
  s.rFx = vmul(rs, s.Fx);
  s.rFy = vmul(rs, s.Fy);
}

// An impermeable node (eps = 0): u = 0, F = -2 m / rho (Eq. 16b with u = 0).
// rho F = -2 m exactly: the collision then reverses the momentum of the node
// exactly (a rounded rho * (1 / rho) would make it grow or decay by ~1e-7
// per step, compounding over the run).
template <class V>
__device__ __forceinline__ void solid_state(NodeStateT<V> &s, V c) {
  s.ieps = vsplat<V>(0.0f);
  s.ux = vsplat<V>(0.0f);
  s.uy = vsplat<V>(0.0f);
  s.rFx = vmul(vsplat<V>(-2.0f), s.mx);
  s.rFy = vmul(vsplat<V>(-2.0f), s.my);
  s.Fx = vmul(s.rFx, c);
  s.Fy = vmul(s.rFy, c);
}

// 1/k_a of a node with a dynamic Kn: inv_k is 1/k_i, kn0 the node's Kn at
// p0, drho_s its (rho - rho0) S; p / p0 = 1 + kn_beta (rho - rho0) and
// k_a = k_i f_c(kn0 p0 / p) (Eq. 3).  One node; the pair path applies it
// lane by lane, so both give the same bits.
__device__ __forceinline__ float dynamic_inv_k(float inv_k, float drho_s, float kn0,
                                               const StepArgs &a) {
  const float q = fmaf(a.kn_beta, __fmul_rn(drho_s, a.inv_scale), 1.0f);
  return inv_ka_dynamic(inv_k, div_newton(kn0, q), a.kn_model);
}

// The pair forms: the same operations in the two lanes of the packed
// instructions (which round as the scalar ones; the negations as exact
// products by -1), so each lane gives dynamic_inv_k's bits.
__device__ __forceinline__ float2 rcp2(float2 d) {
  float2 r;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r.x) : "f"(d.x));
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r.y) : "f"(d.y));
  return r;
}
__device__ __forceinline__ float2 div_newton(float2 n, float2 d) {
  const float2 r = rcp2(d);
  const float2 q = vmul(n, r);
  return vfma(r, vfma(vmul(vsplat<float2>(-1.0f), d), q, n), q);
}
__device__ __forceinline__ float2 kn_power(float2 K) {
  constexpr float c_hi = -0.4348f;
  constexpr float c_lo = (float)(-0.4348 - (double)c_hi);
  float2 lg, t;
  asm("lg2.approx.ftz.f32 %0, %1;" : "=f"(lg.x) : "f"(K.x));
  asm("lg2.approx.ftz.f32 %0, %1;" : "=f"(lg.y) : "f"(K.y));
  const float2 y_hi = vmul(lg, vsplat<float2>(c_hi));
  const float2 y_lo = vfma(lg, vsplat<float2>(c_lo),
                           vfma(lg, vsplat<float2>(c_hi), vmul(vsplat<float2>(-1.0f), y_hi)));
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(t.x) : "f"(y_hi.x));
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(t.y) : "f"(y_hi.y));
  return vfma(vmul(t, vsplat<float2>(0.69314718f)), y_lo, t);
}
__device__ __forceinline__ float2 dynamic_inv_k(float2 inv_k, float2 drho_s, float2 kn0,
                                                const StepArgs &a) {
  const float2 q = vfma(vsplat<float2>(a.kn_beta), vmul(drho_s, vsplat<float2>(a.inv_scale)),
                        vsplat<float2>(1.0f));
  const float2 kn = div_newton(kn0, q);
  const bool common = a.kn_model == 0 && kn.x >= 1.17549435e-38f && kn.x <= 1e12f &&
                      kn.y >= 1.17549435e-38f && kn.y <= 1e12f;
  if (!common)  // the one-node form, lane by lane
    return make_float2(inv_ka_dynamic(inv_k.x, kn.x, a.kn_model),
                       inv_ka_dynamic(inv_k.y, kn.y, a.kn_model));
  const float2 one = vsplat<float2>(1.0f);
  const float2 ca = vfma(vsplat<float2>(0.17f), kn_power(kn), one);
  const float2 num = vmul(vmul(inv_k, ca), vadd(one, kn));
  const float2 den = vmul(vfma(vsplat<float2>(1.358f), kn, ca), vfma(vsplat<float2>(5.0f), kn, one));
  return div_newton(num, den);
}

// Moments of Eq. 16a and the state of a node (one node, or a pair of nodes
// in the lanes of V).  DYN: inv_k is 1/k_i and kn0 the node's Kn at p0; its
// apparent permeability k_a = k_i f_c(kn0 p0 / p) (Eq. 3) follows the
// pressure p / p0 = 1 + kn_beta (rho - rho0).
template <class V, bool DYN = false>
__device__ __forceinline__ NodeStateT<V> node_state_t(const V d[9], V eps, V inv_k,
                                                      const StepArgs &a,
                                                      V kn0 = vsplat<V>(0.0f)) {
  NodeStateT<V> s;
  s.drho_s = vadd(vadd(vadd(d[0], vadd(d[1], d[3])), vadd(d[2], d[4])),
                  vadd(vadd(d[5], d[7]), vadd(d[6], d[8])));
  // sum_i w_i e_i = 0, so the momentum of the deviations is the momentum.
  const V d57 = vsub(d[5], d[7]);
  s.mx = vadd(vsub(d[1], d[3]), vadd(d57, vsub(d[8], d[6])));
  s.my = vadd(vsub(d[2], d[4]), vadd(d57, vsub(d[6], d[8])));
  s.rho = vfma(s.drho_s, vsplat<V>(a.inv_scale), vsplat<V>(a.rho0));
  const V c = vmul(vsplat<V>(a.inv_scale), vrcp(s.rho));  // 1 / (S rho)
  if constexpr (sizeof(V) == sizeof(float)) {
    if (eps > 0.0f) {
      if (DYN) inv_k = dynamic_inv_k(inv_k, s.drho_s, kn0, a);
      porous_state(s, eps, inv_k, c, a);
    } else {
      solid_state(s, c);
    }
  } else {
    if (DYN) inv_k = dynamic_inv_k(inv_k, s.drho_s, kn0, a);  // a solid lane's value is unused
    const bool px = eps.x > 0.0f, py = eps.y > 0.0f;
    if (px && py) {  // the common case: two permeable nodes
      porous_state(s, eps, inv_k, c, a);
      return s;
    }
    // otherwise both forms, then each lane keeps its own
    NodeStateT<V> q = s;
    porous_state(s, eps, inv_k, c, a);
    solid_state(q, c);
#define LBMP_PICK(f) s.f = make_float2(px ? s.f.x : q.f.x, py ? s.f.y : q.f.y)
    LBMP_PICK(ieps);
    LBMP_PICK(ux);
    LBMP_PICK(uy);
    LBMP_PICK(Fx);
    LBMP_PICK(Fy);
    LBMP_PICK(rFx);
    LBMP_PICK(rFy);
#undef LBMP_PICK
  }
  return s;
}

// One node (the form every kernel but the staged pair path uses).
template <bool DYN = false>
__device__ __forceinline__ NodeState node_state(const float d[9], float eps, float inv_k,
                                                const StepArgs &a, float kn0 = 0.0f) {
  return node_state_t<float, DYN>(d, eps, inv_k, a, kn0);
}

// Eq. 12 with the equilibrium of Eq. 14 and the forcing of Eq. 15 (last term
// over eps), in stored units, written through moments:
//   d*_i = (1 - 1/tau) d_i + w_i S [A + e_i.P + e_i^T M e_i],
//   A = drho/tau - rho (3 u^2 / (2 eps tau) + (1 - 1/2tau) 3 u.F / eps),
//   P = 3 rho (u / tau + (1 - 1/2tau) F) = 3 (m / tau + rho F),
//   M = rho (9 u u / (2 eps tau) + (1 - 1/2tau) 9 (u F + F u) / (2 eps)),
// which is f_eq / tau + F_i expanded direction by direction.  P uses the
// identity rho u = m + rho F / 2 (Eq. 16b): the momentum the collision hands
// on is then m + rho F exactly, whatever the rounding of u.  The weights are
// applied as hi + lo pairs so that their FP32 representation error does not
// bias the momentum at every node in the same direction.
constexpr float kW0h = 4.0f / 9.0f;
constexpr float kW1h = 1.0f / 9.0f;
constexpr float kW2h = 1.0f / 36.0f;
constexpr float kW0l = (float)(4.0 / 9.0 - (double)kW0h);
constexpr float kW1l = (float)(1.0 / 9.0 - (double)kW1h);
constexpr float kW2l = (float)(1.0 / 36.0 - (double)kW2h);

template <bool HILO, class V>
__device__ __forceinline__ V wmul(float wh, float wl, V t) {
  if (HILO) return vfma(vsplat<V>(wh), t, vmul(vsplat<V>(wl), t));
  return vmul(vsplat<V>(wh), t);
}

// HILO = false drops the lo parts of the weights: for FP16 storage the FP16
// rounding (zero-mean with stochastic rounding) dominates their effect.
template <bool HILO, class V>
__device__ __forceinline__ void collide_t(V d[9], const NodeStateT<V> &s, const StepArgs &a) {
  const V rs = vmul(s.rho, vsplat<V>(a.scale));
  const V ux = s.ux, uy = s.uy, Fx = s.Fx, Fy = s.Fy, ie = s.ieps;
  const V om = vsplat<V>(a.omega), cf = vsplat<V>(a.cforce);
  const V usq = vmul(vmul(vsplat<V>(1.5f), ie), vfma(ux, ux, vmul(uy, uy)));
  const V uF3 = vmul(vmul(vsplat<V>(3.0f), ie), vfma(ux, Fx, vmul(uy, Fy)));
  const V A = vfma(om, s.drho_s, vneg(vmul(rs, vfma(om, usq, vmul(cf, uF3)))));
  // P = 3 (X, Y); every sum with a product below is one fma
  const V X = vfma(om, s.mx, s.rFx), Y = vfma(om, s.my, s.rFy);
  const V three = vsplat<V>(3.0f), mthree = vsplat<V>(-3.0f);
  const V qq = vmul(vmul(vsplat<V>(a.omega * 4.5f), ie), rs);
  const V gg = vmul(vmul(vsplat<V>(a.cforce * 9.0f), ie), rs);
  const V tx = vfma(qq, ux, vmul(gg, Fx)), ty = vfma(qq, uy, vmul(gg, Fy));  // M_xx / u_x, M_yy / u_y
  const V Mxy2 = vfma(vmul(vmul(vsplat<V>(2.0f), qq), ux), uy,
                      vmul(gg, vfma(ux, Fy, vmul(uy, Fx))));  // 2 M_xy
  const V sx = vfma(ux, tx, A), sy = vfma(uy, ty, A), sd = vfma(uy, ty, sx);
  const V s5 = vadd(sd, Mxy2), s6 = vsub(sd, Mxy2);
  const V Py = vmul(three, Y);
  const V pp = vfma(three, X, Py), pm = vfma(three, X, vneg(Py));
  const V o1 = vsplat<V>(a.one_m_omega);
  d[0] = vfma(o1, d[0], wmul<HILO>(kW0h, kW0l, A));
  d[1] = vfma(o1, d[1], wmul<HILO>(kW1h, kW1l, vfma(three, X, sx)));
  d[3] = vfma(o1, d[3], wmul<HILO>(kW1h, kW1l, vfma(mthree, X, sx)));
  d[2] = vfma(o1, d[2], wmul<HILO>(kW1h, kW1l, vfma(three, Y, sy)));
  d[4] = vfma(o1, d[4], wmul<HILO>(kW1h, kW1l, vfma(mthree, Y, sy)));
  d[5] = vfma(o1, d[5], wmul<HILO>(kW2h, kW2l, vadd(s5, pp)));
  d[7] = vfma(o1, d[7], wmul<HILO>(kW2h, kW2l, vsub(s5, pp)));
  d[6] = vfma(o1, d[6], wmul<HILO>(kW2h, kW2l, vsub(s6, pm)));
  d[8] = vfma(o1, d[8], wmul<HILO>(kW2h, kW2l, vadd(s6, pm)));
}

template <bool HILO = true>
__device__ __forceinline__ void collide(float d[9], const NodeState &s, const StepArgs &a) {
  collide_t<HILO, float>(d, s, a);
}

// Deviation of the porous equilibrium (Eq. 14) from w_i rho0, physical
// units: deq_i = w_i (rho - rho0) + w_i rho (3 e.u + (9/2 (e.u)^2 - 3/2 u^2)
// / eps); eps = 0 keeps only w_i (rho - rho0).  Every multiply-add is an
// explicit fmaf, so the pressure columns of every kernel round alike.
__device__ __forceinline__ void equilibrium_dev(float drho, float rho, float ux, float uy,
                                                float eps, float deq[9]) {
  const float inv_eps = (eps > 0.0f) ? 1.0f / eps : 0.0f;
  const float vx = (eps > 0.0f) ? ux : 0.0f;
  const float vy = (eps > 0.0f) ? uy : 0.0f;
  const float usq = 1.5f * inv_eps * fmaf(vx, vx, vy * vy);
  const float q = 4.5f * inv_eps;
  const float r1 = kW1 * rho, r2 = kW2 * rho;
  const float dr1 = kW1 * drho, dr2 = kW2 * drho;
  deq[0] = fmaf(kW0 * rho, -usq, kW0 * drho);
  float eu;
  eu = vx;        deq[1] = fmaf(r1, fmaf(3.0f, eu, fmaf(q * eu, eu, -usq)), dr1);
  eu = vy;        deq[2] = fmaf(r1, fmaf(3.0f, eu, fmaf(q * eu, eu, -usq)), dr1);
  eu = -vx;       deq[3] = fmaf(r1, fmaf(3.0f, eu, fmaf(q * eu, eu, -usq)), dr1);
  eu = -vy;       deq[4] = fmaf(r1, fmaf(3.0f, eu, fmaf(q * eu, eu, -usq)), dr1);
  eu = vx + vy;   deq[5] = fmaf(r2, fmaf(3.0f, eu, fmaf(q * eu, eu, -usq)), dr2);
  eu = vy - vx;   deq[6] = fmaf(r2, fmaf(3.0f, eu, fmaf(q * eu, eu, -usq)), dr2);
  eu = -vx - vy;  deq[7] = fmaf(r2, fmaf(3.0f, eu, fmaf(q * eu, eu, -usq)), dr2);
  eu = vx - vy;   deq[8] = fmaf(r2, fmaf(3.0f, eu, fmaf(q * eu, eu, -usq)), dr2);
}

// Pressure column (non-equilibrium extrapolation, Guo, Zheng & Shi 2002),
// stored units: d_b = d_n + S (deq(rho_b, u_n; eps_b) - deq(rho_n, u_n;
// eps_n)), n the adjacent interior node and rho_b the imposed density.
template <class S, bool DYN = false>
__device__ __forceinline__ void pressure_node(const typename S::T *__restrict__ fin,
                                           const float2 *__restrict__ med, const StepArgs &a,
                                           int xb, int y, float eps_b, float d[9]) {
  const int xn = (xb == 0) ? 1 : a.nx - 2;
  const long long jn = (long long)y * a.pitch + xn;
  const float2 mn = med[jn];
  float dn[9];
  pull_node<S>(fin, a, xn, y, dn);
  const NodeState sn = node_state<DYN>(dn, mn.x, mn.y, a, DYN ? a.kn0[jn] : 0.0f);
  const float drho_b = (xb == 0) ? a.drho_in : a.drho_out;
  float eq_b[9], eq_n[9];
  equilibrium_dev(drho_b, a.rho0 + drho_b, sn.ux, sn.uy, eps_b, eq_b);
  equilibrium_dev(sn.drho_s * a.inv_scale, sn.rho, sn.ux, sn.uy, mn.x, eq_n);
#pragma unroll
  for (int i = 0; i < 9; ++i) d[i] = fmaf(a.scale, eq_b[i] - eq_n[i], dn[i]);
}

}  // namespace lbmp
