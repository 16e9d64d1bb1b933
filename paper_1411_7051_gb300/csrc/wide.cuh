// Vectorised FP16 step: four consecutive nodes of a row per thread (Section
// III, Eq. 12-17; the arithmetic of lattice.cuh).
//
// FP16 storage halves the bytes of a step, so the instruction stream per
// byte doubles; this kernel keeps it short.  Each plane is read with one
// 8-byte load per thread (the four nodes' populations), the e_x = +-1
// directions take the one value they need from the neighbouring thread's
// span through one aligned 4-byte halo load and a byte permutation, and the
// nine results go out as one 8-byte store per plane.  No shared memory, no
// barriers: the bytes in flight come from the many independent 8-byte loads
// of each thread.
//
// Boundaries: the halo of x = 0 and the source of x = nx - 1 wrap across
// the row (periodic edges); rows next to a plate read the opposite
// direction of their own node (halfway bounce-back), a warp-uniform branch;
// pressure columns are extrapolated from their neighbour (pressure_node).
// Nodes x >= nx of the last thread of a row are computed from the row
// padding and written back there; nothing reads the padding as a node.
#pragma once

#include <cuda_fp16.h>
#include <stdint.h>

#include "lattice.cuh"

namespace lbmp {

constexpr int kWideBX = 128;  // threads per block
constexpr int kWideV = 4;     // nodes per thread

__device__ __forceinline__ uint2 ldg_u2(const __half *p) {
  return __ldg(reinterpret_cast<const uint2 *>(p));
}
__device__ __forceinline__ uint32_t ldg_u1(const __half *p) {
  return __ldg(reinterpret_cast<const unsigned int *>(p));
}
__device__ __forceinline__ uint32_t ldg_h(const __half *p) {
  return (uint32_t)__ldg(reinterpret_cast<const unsigned short *>(p));
}

// The four values of direction i for nodes x0 .. x0+3 of row y, as two
// half2 words (nodes x0, x0+1 | x0+2, x0+3).
//   ex  = the direction's e_x; bounce: the source is a plate row, so the
//   values are those of the opposite direction `opp` at the node itself.
// rs is the row of the source (y - e_y, wrapped).
template <int EX>
__device__ __forceinline__ uint2 load_dir(const __half *__restrict__ fin, const StepArgs &a,
                                          int i, int opp, bool bounce, int rs, int y, int x0) {
  if (bounce) return ldg_u2(fin + (long long)opp * a.plane + (long long)y * a.pitch + x0);
  const __half *row = fin + (long long)i * a.plane + (long long)rs * a.pitch;
  const uint2 w = ldg_u2(row + x0);
  if (EX == 0) return w;
  if (EX == 1) {
    // node x takes x - 1: halo word (x0-2, x0-1); at x0 = 0 the source of
    // node 0 is x = nx - 1 (periodic), unused beside a pressure column
    uint32_t h;
    if (x0 > 0) h = ldg_u1(row + x0 - 2);
    else h = a.pressure ? 0u : (ldg_h(row + a.nx - 1) << 16);
    return make_uint2(__byte_perm(h, w.x, 0x5432), __byte_perm(w.x, w.y, 0x5432));
  }
  // EX == -1: node x takes x + 1: halo word (x0+4, x0+5)
  uint32_t h = 0u;
  if (x0 + 4 < a.nx) h = ldg_u1(row + x0 + 4);
  else if (x0 + 3 == a.nx - 1 && !a.pressure) h = ldg_h(row);  // node nx-1 wraps to 0
  uint2 o = make_uint2(__byte_perm(w.x, w.y, 0x5432), __byte_perm(w.y, h, 0x5432));
  if (x0 + 3 > a.nx - 1 && !a.pressure) {
    // node nx - 1 sits inside the span: its source x = nx wraps to 0
    const uint32_t z = ldg_h(row);
    const int k = a.nx - 1 - x0;  // 0, 1 or 2
    if (k == 0) o.x = (o.x & 0xffff0000u) | z;
    else if (k == 1) o.x = (o.x & 0x0000ffffu) | (z << 16);
    else o.y = (o.y & 0xffff0000u) | z;
  }
  return o;
}

__device__ __forceinline__ void unpack(uint32_t w, float &lo, float &hi) {
  const float2 f = __half22float2(*reinterpret_cast<const __half2 *>(&w));
  lo = f.x;
  hi = f.y;
}

template <bool SR>
__device__ __forceinline__ uint32_t pack(float lo, float hi, uint32_t rbits) {
  uint32_t out;
  if (SR) {
    asm("cvt.rs.f16x2.f32 %0, %1, %2, %3;" : "=r"(out) : "f"(hi), "f"(lo), "r"(rbits));
  } else {
    const __half2 h = __floats2half2_rn(lo, hi);
    out = *reinterpret_cast<const uint32_t *>(&h);
  }
  return out;
}

template <bool SR, bool DYN>
__global__ void __launch_bounds__(kWideBX)
    wide_step_kernel(const StepArgs a, const __half *__restrict__ fin, __half *__restrict__ fout,
                     const float2 *__restrict__ med, const unsigned long long *__restrict__ tctr,
                     int k) {
  const int y = a.y0 + blockIdx.y;
  const int x0 = (blockIdx.x * kWideBX + threadIdx.x) * kWideV;
  if (x0 >= a.nx) return;
  const int ym = (y == 0) ? a.ny - 1 : y - 1;    // source row of e_y = +1
  const int yp = (y == a.ny - 1) ? 0 : y + 1;    // source row of e_y = -1
  const bool bm = a.walls && (y - 1 == 0);       // e_y = +1 sources are a plate
  const bool bp = a.walls && (y + 1 == a.ny - 1);
  // direction i: e (0,0) (1,0) (0,1) (-1,0) (0,-1) (1,1) (-1,1) (-1,-1) (1,-1)
  uint2 v[9];
  v[0] = load_dir<0>(fin, a, 0, 0, false, y, y, x0);
  v[1] = load_dir<1>(fin, a, 1, 3, false, y, y, x0);
  v[3] = load_dir<-1>(fin, a, 3, 1, false, y, y, x0);
  v[2] = load_dir<0>(fin, a, 2, 4, bm, ym, y, x0);
  v[5] = load_dir<1>(fin, a, 5, 7, bm, ym, y, x0);
  v[6] = load_dir<-1>(fin, a, 6, 8, bm, ym, y, x0);
  v[4] = load_dir<0>(fin, a, 4, 2, bp, yp, y, x0);
  v[7] = load_dir<-1>(fin, a, 7, 5, bp, yp, y, x0);
  v[8] = load_dir<1>(fin, a, 8, 6, bp, yp, y, x0);
  const long long row = (long long)y * a.pitch;
  const float4 m01 = __ldg(reinterpret_cast<const float4 *>(med + row + x0));
  const float4 m23 = __ldg(reinterpret_cast<const float4 *>(med + row + x0 + 2));
  float4 kn = make_float4(0.f, 0.f, 0.f, 0.f);
  if (DYN) kn = __ldg(reinterpret_cast<const float4 *>(a.kn0 + row + x0));
  uint32_t ts = 0;
  if (SR) {
    const unsigned long long t = *tctr + (unsigned long long)k;
    ts = mix32((uint32_t)t * 0x9e3779b9u ^ a.seed_lo ^ mix32((uint32_t)(t >> 32) ^ a.seed_hi));
  }
  constexpr uint32_t kC[9] = {0x9e3779b1u, 0x85ebca77u, 0xc2b2ae3du, 0x27d4eb2fu, 0x165667b1u,
                              0xd3a2646du, 0xfd7046c5u, 0xb55a4f09u, 0x7feb352du};
  uint2 out[9];
#pragma unroll
  for (int p = 0; p < 2; ++p) {
    float dA[9], dB[9];
#pragma unroll
    for (int i = 0; i < 9; ++i) unpack(p ? v[i].y : v[i].x, dA[i], dB[i]);
    const int xA = x0 + 2 * p;
    const float2 mA = p ? make_float2(m23.x, m23.y) : make_float2(m01.x, m01.y);
    const float2 mB = p ? make_float2(m23.z, m23.w) : make_float2(m01.z, m01.w);
    if (a.pressure) {
      if (xA == 0 || xA == a.nx - 1) pressure_node<StoreF16, DYN>(fin, med, a, xA, y, mA.x, dA);
      if (xA + 1 == a.nx - 1) pressure_node<StoreF16, DYN>(fin, med, a, xA + 1, y, mB.x, dB);
    }
    const NodeState sA = node_state<DYN>(dA, mA.x, mA.y, a, p ? kn.z : kn.x);
    collide<false>(dA, sA, a);
    const NodeState sB = node_state<DYN>(dB, mB.x, mB.y, a, p ? kn.w : kn.y);
    collide<false>(dB, sB, a);
    // the random word of a pair: the hash of the staged kernel's pair index
    const uint32_t h = SR ? mix32((uint32_t)((row + xA) >> 1) ^ ts) : 0u;
#pragma unroll
    for (int i = 0; i < 9; ++i) {
      const uint32_t w = pack<SR>(dA[i], dB[i], SR ? h * kC[i] : 0u);
      if (p) out[i].y = w;
      else out[i].x = w;
    }
  }
  __half *o = fout + row + x0;
#pragma unroll
  for (int i = 0; i < 9; ++i) *reinterpret_cast<uint2 *>(o + (long long)i * a.plane) = out[i];
}

}  // namespace lbmp
