// Staged (asynchronous bulk-copy) variant of the porous lattice Boltzmann
// step (Chen et al., arXiv:1411.7051, Section III, Eq. 12-17).
//
// The fused step moves every population once per time step, so it is
// bound by HBM bandwidth, and bandwidth needs many bytes in flight.  Here
// the bytes in flight do not depend on registers: a persistent CTA per SM
// runs one producer warp that copies tile spans of the nine population
// planes and of the medium into a ring of shared-memory stages with
// cp.async.bulk (completion counted on an mbarrier), while 16 consumer
// warps pull, collide and store from the stage that has landed.
//
// Tile: W consecutive nodes of the padded lattice taken row after row (flat
// index y * pitch + x), so a tile may continue on the next row and no tile
// is left partly empty at a row end.  A stage holds, for each plane i, the
// sources of the tile's nodes, flat [T - e_iy pitch - A, T - e_iy pitch + W
// + A) (A = 16 bytes of halo on each side, so every copy starts and ends on
// a 16-byte boundary): one contiguous span, split where it wraps around the
// plane (the periodic edge in y).  Interior nodes never read across a row
// end.  Sources that the stage cannot hold -- the periodic wrap of column
// 0 / nx-1 and the bounce-back of the rows next to a plate -- are read from
// global memory by the few threads that need them.
//
// Every wait is bounded (kWaitNs of %globaltimer); a wait that gives up
// raises *err and the CTA returns (the host reports LBMP_ETIMEOUT).
#pragma once

#include <cuda_fp16.h>
#include <stdint.h>

#include <type_traits>

#include "lattice.cuh"

namespace lbmp {

constexpr int kConsumerWarps = 16;
constexpr int kStagedThreads = (kConsumerWarps + 1) * 32;
constexpr unsigned long long kWaitNs = 2000000000ull;  // 2 s

template <class S>
struct StageCfg;
template <>
struct StageCfg<StoreF32> {
  static constexpr int W = 1024, H = 1, A = 4, STAGES = 4;
  static constexpr int WARPS = kConsumerWarps;
  static constexpr bool KN0 = false;
};
template <>
struct StageCfg<StoreF16> {
  static constexpr int W = 2048, H = 1, A = 8, STAGES = 4;
  static constexpr int WARPS = kConsumerWarps;
  static constexpr bool KN0 = false;
};
// FP16 with a dynamic Kn: each stage also holds the tile's Kn at p0 (a
// float per node), so the ring is one stage shorter.
struct StageCfgDyn16 {
  static constexpr int W = 2048, H = 1, A = 8, STAGES = 3;
  static constexpr int WARPS = kConsumerWarps;
  static constexpr bool KN0 = true;
};
template <class S, bool DYN>
using StageCfgFor = typename std::conditional<DYN, StageCfgDyn16, StageCfg<S>>::type;

// Shared-memory layout of a stage configuration Cfg (tile width W, halo A,
// STAGES, WARPS consumer warps).
template <class S, class Cfg = StageCfg<S>>
struct StageLayout {
  using C = Cfg;
  using T = typename S::T;
  static constexpr int RW = C::W + 2 * C::A;  // stage row length (elements)
  static constexpr int kPopBytes = 9 * C::H * RW * (int)sizeof(T);
  static constexpr int kMedBytes = C::H * C::W * 8;
  static constexpr int kKnBytes = C::KN0 ? C::H * C::W * 4 : 0;  // Kn at p0 (dynamic Kn)
  static constexpr int kStageBytes = kPopBytes + kMedBytes + kKnBytes;
  static constexpr int kBarBytes = 128;  // full[STAGES], empty[STAGES]
  static constexpr int kSmemBytes = kBarBytes + C::STAGES * kStageBytes;
  static_assert(kPopBytes % 16 == 0 && kMedBytes % 16 == 0 && kKnBytes % 16 == 0,
                "16-byte stage alignment");
  static_assert(RW * (int)sizeof(T) % 16 == 0, "16-byte row alignment");
  static_assert(C::A * (int)sizeof(T) == 16, "halo of 16 bytes");
  static_assert(2 * C::STAGES * 8 <= kBarBytes, "barrier area");
  static_assert((C::H * C::W / 2) % (C::WARPS * 32) == 0, "node pairs per consumer thread");
  static_assert(C::H == 1, "tiles are spans of the flattened lattice");
  static_assert(C::W % 64 == 0, "tile starts stay 16-byte aligned");
  static_assert(C::W % 2 == 0 && C::A % 2 == 0, "pairs stay aligned");
};

// ------------------------------------------------------------- PTX helpers
__device__ __forceinline__ uint32_t smem_u32(const void *p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_arrive_expect_tx(uint32_t bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes)
               : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint32_t bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(bar), "r"(parity)
      : "memory");
  return ok != 0;
}
__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
// Bounded wait for the phase of parity `parity` to complete.
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity, unsigned *err) {
  if (mbar_try_wait(bar, parity)) return true;
  const unsigned long long t0 = global_ns();
  for (uint32_t it = 0; it < (1u << 30); ++it) {
    if (mbar_try_wait(bar, parity)) return true;
    if (global_ns() - t0 > kWaitNs) break;
  }
  atomicOr(err, 1u);
  return false;
}
// Global -> shared bulk copy; completion is counted on mbarrier `bar`.
__device__ __forceinline__ void bulk_g2s(uint32_t dst, const void *src, uint32_t bytes,
                                         uint32_t bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::
          "r"(dst),
      "l"(src), "r"(bytes), "r"(bar)
      : "memory");
}

// --------------------------------------------------------------- helpers
// Post-stream values of node (x, y) at tile position (r, c), stored units.
template <class S, class Cfg = StageCfg<S>>
__device__ __forceinline__ void pull_staged(const typename S::T *__restrict__ sp,
                                            const typename S::T *__restrict__ fin,
                                            const StepArgs &a, int r, int c, int x, int y,
                                            float d[9]) {
  using L = StageLayout<S, Cfg>;
  using C = Cfg;
  constexpr int RW = L::RW, A = C::A, H = C::H;
  const typename S::T *row[9];
#pragma unroll
  for (int i = 0; i < 9; ++i) row[i] = sp + (i * H + r) * RW + A + c;
  // columns with e_x = 0 and the shifted ones
  d[0] = S::ld1(row[0]);
  d[2] = S::ld1(row[2]);
  d[4] = S::ld1(row[4]);
  d[1] = S::ld1(row[1] - 1);
  d[5] = S::ld1(row[5] - 1);
  d[8] = S::ld1(row[8] - 1);
  d[3] = S::ld1(row[3] + 1);
  d[6] = S::ld1(row[6] + 1);
  d[7] = S::ld1(row[7] + 1);
  const bool xlo = !a.pressure && x == 0;           // e_x = +1 sources wrap to nx-1
  const bool xhi = !a.pressure && x == a.nx - 1;    // e_x = -1 sources wrap to 0
  const bool wm = a.walls && y == 1;                // e_y = +1 sources are a plate
  const bool wp = a.walls && y == a.ny - 2;         // e_y = -1 sources are a plate
  if (xlo || xhi || wm || wp) {
    const long long P = a.plane;
    const int ym = (y == 0) ? a.ny - 1 : y - 1;
    const int yp = (y == a.ny - 1) ? 0 : y + 1;
    const long long rr = (long long)y * a.pitch, rm = (long long)ym * a.pitch,
                    rp = (long long)yp * a.pitch;
    if (xlo) {
      const int xs = a.nx - 1;
      d[1] = S::ld1(fin + 1 * P + rr + xs);
      d[5] = S::ld1(fin + 5 * P + rm + xs);
      d[8] = S::ld1(fin + 8 * P + rp + xs);
    }
    if (xhi) {
      d[3] = S::ld1(fin + 3 * P + rr);
      d[6] = S::ld1(fin + 6 * P + rm);
      d[7] = S::ld1(fin + 7 * P + rp);
    }
    if (wm) {
      d[2] = S::ld1(fin + 4 * P + rr + x);
      d[5] = S::ld1(fin + 7 * P + rr + x);
      d[6] = S::ld1(fin + 8 * P + rr + x);
    }
    if (wp) {
      d[4] = S::ld1(fin + 2 * P + rr + x);
      d[7] = S::ld1(fin + 5 * P + rr + x);
      d[8] = S::ld1(fin + 6 * P + rr + x);
    }
  }
}

// The 32 random bits of direction i of a node pair (stochastic rounding).
__device__ __forceinline__ uint32_t pair_bits(uint32_t h, int i) {
  constexpr uint32_t kC[9] = {0x9e3779b1u, 0x85ebca77u, 0xc2b2ae3du, 0x27d4eb2fu, 0x165667b1u,
                              0xd3a2646du, 0xfd7046c5u, 0xb55a4f09u, 0x7feb352du};
  return h * kC[i];
}

// Pressure column xb (0 or nx - 1) at tile position c: non-equilibrium
// extrapolation from the neighbouring interior node (stage position cn).
template <class S, class Cfg = StageCfg<S>, bool DYN = false>
__device__ __forceinline__ void staged_pressure(const typename S::T *__restrict__ sp,
                                                const typename S::T *__restrict__ fin,
                                                const float2 *__restrict__ med, const StepArgs &a,
                                                int cn, int xb, int y, float eps_b, float d[9]) {
  const int xn = (xb == 0) ? 1 : a.nx - 2;
  const long long jn = (long long)y * a.pitch + xn;
  const float2 mn = med[jn];
  float dn[9];
  pull_staged<S, Cfg>(sp, fin, a, 0, cn, xn, y, dn);
  const NodeState sn = node_state<DYN>(dn, mn.x, mn.y, a, DYN ? a.kn0[jn] : 0.0f);
  const float drho_b = (xb == 0) ? a.drho_in : a.drho_out;
  float eq_b[9], eq_n[9];
  equilibrium_dev(drho_b, a.rho0 + drho_b, sn.ux, sn.uy, eps_b, eq_b);
  equilibrium_dev(sn.drho_s * a.inv_scale, sn.rho, sn.ux, sn.uy, mn.x, eq_n);
#pragma unroll
  for (int i = 0; i < 9; ++i) d[i] = fmaf(a.scale, eq_b[i] - eq_n[i], dn[i]);
}

// Update of a node pair that needs more than the stage holds: the periodic
// wrap at x = 0 and nx - 1, the bounce-back next to a plate, the pressure
// columns, the lone last node of an odd row.  These are a few pairs per
// row; keeping them out of line keeps the interior path's registers and
// code lean.  The step arguments come by value: taking the address of the
// kernel parameter would move every read of it to local memory.
template <class S, bool SR, class Cfg = StageCfg<S>, bool DYN = false>
__device__ __noinline__ void staged_edge_pair(const typename S::T *__restrict__ sp,
                                              const typename S::T *__restrict__ fin,
                                              typename S::T *__restrict__ fout,
                                              const float2 *__restrict__ med, const StepArgs a,
                                              int c, int x, int y, float4 m, float2 k0,
                                              uint32_t ts) {
  const bool two = x + 1 < a.nx;
  float dA[9], dB[9];
  pull_staged<S, Cfg>(sp, fin, a, 0, c, x, y, dA);
  if (two) pull_staged<S, Cfg>(sp, fin, a, 0, c + 1, x + 1, y, dB);
  if (a.pressure) {
    if (x == 0 || x == a.nx - 1)
      staged_pressure<S, Cfg, DYN>(sp, fin, med, a, x == 0 ? c + 1 : c - 1, x, y, m.x, dA);
    if (two && x + 1 == a.nx - 1)
      staged_pressure<S, Cfg, DYN>(sp, fin, med, a, c, x + 1, y, m.z, dB);
  }
  const NodeState nA = node_state<DYN>(dA, m.x, m.y, a, k0.x);
  collide<S::kHiLo>(dA, nA, a);
  if (two) {
    const NodeState nB = node_state<DYN>(dB, m.z, m.w, a, k0.y);
    collide<S::kHiLo>(dB, nB, a);
  } else {
    // a last node of an odd row is stored as a pair with a zero in the row
    // padding (x = nx < pitch), drawing its rounding bits as a pair
#pragma unroll
    for (int i = 0; i < 9; ++i) dB[i] = 0.0f;
  }
  const long long o = (long long)y * a.pitch + x;
  const uint32_t h = SR ? mix32((uint32_t)(o >> 1) ^ ts) : 0u;
#pragma unroll
  for (int i = 0; i < 9; ++i)
    S::template st2<SR>(fout + i * a.plane + o, dA[i], dB[i], SR ? pair_bits(h, i) : 0u, 0u);
}

// The populations of pressure column xb from its interior neighbour's pulled
// values dn and state sn (non-equilibrium extrapolation, as staged_pressure).
__device__ __forceinline__ void column_from_neighbour(const StepArgs &a, const float dn[9],
                                                      const NodeState &sn, float eps_n, int xb,
                                                      float eps_b, float d[9]) {
  const float drho_b = (xb == 0) ? a.drho_in : a.drho_out;
  float eq_b[9], eq_n[9];
  equilibrium_dev(drho_b, a.rho0 + drho_b, sn.ux, sn.uy, eps_b, eq_b);
  equilibrium_dev(sn.drho_s * a.inv_scale, sn.rho, sn.ux, sn.uy, eps_n, eq_n);
#pragma unroll
  for (int i = 0; i < 9; ++i) d[i] = fmaf(a.scale, eq_b[i] - eq_n[i], dn[i]);
}

// The same update with both nodes in the lanes of the packed arithmetic,
// and a pressure column taking its neighbour's pull and state from the pair
// (the batched kernel, whose short rows make edge pairs frequent: 125 -> 132
// GLUPS on 256 instances; in the single-lattice kernel, where they are a
// few per row, the scalar form above was the faster one).
template <class S, bool SR, class Cfg = StageCfg<S>>
__device__ __noinline__ void staged_edge_pair_packed(const typename S::T *__restrict__ sp,
                                                     const typename S::T *__restrict__ fin,
                                                     typename S::T *__restrict__ fout,
                                                     const float2 *__restrict__ med,
                                                     const StepArgs a, int c, int x, int y,
                                                     float4 m, uint32_t ts) {
  const bool two = x + 1 < a.nx;
  float dA[9], dB[9];
  pull_staged<S, Cfg>(sp, fin, a, 0, c, x, y, dA);
  if (two) {
    pull_staged<S, Cfg>(sp, fin, a, 0, c + 1, x + 1, y, dB);
  } else {
#pragma unroll
    for (int i = 0; i < 9; ++i) dB[i] = 0.0f;
  }
  if (a.pressure) {
    // a column next to its neighbour in the same pair takes the neighbour's
    // pull and state from here; a lone last node of an odd row pulls its
    // neighbour from the stage
    if (x == 0)
      column_from_neighbour(a, dB, node_state(dB, m.z, m.w, a), m.z, 0, m.x, dA);
    else if (x == a.nx - 1)
      staged_pressure<S, Cfg>(sp, fin, med, a, c - 1, x, y, m.x, dA);
    if (two && x + 1 == a.nx - 1)
      column_from_neighbour(a, dA, node_state(dA, m.x, m.y, a), m.x, a.nx - 1, m.z, dB);
  }
  // both nodes in the two lanes of the packed arithmetic (each lane gives the
  // one-node bits); a lone last node of an odd row is stored as a pair with
  // a zero in the row padding (x = nx < pitch, medium zero there), drawing
  // its rounding bits as a pair
  float2 d[9];
#pragma unroll
  for (int i = 0; i < 9; ++i) d[i] = make_float2(dA[i], dB[i]);
  const NodeStateT<float2> n = node_state_t<float2>(d, make_float2(m.x, m.z),
                                                    make_float2(m.y, m.w), a);
  collide_t<S::kHiLo>(d, n, a);
  const long long o = (long long)y * a.pitch + x;
  const uint32_t h = SR ? mix32((uint32_t)(o >> 1) ^ ts) : 0u;
#pragma unroll
  for (int i = 0; i < 9; ++i)
    S::template st2<SR>(fout + i * a.plane + o, d[i].x, two ? d[i].y : 0.0f,
                        SR ? pair_bits(h, i) : 0u, 0u);
}

// Update of an interior node pair (2 <= x, x + 2 < nx, no plate
// neighbour) at tile position c: every source is in the stage.  The pair is
// computed in the two lanes of float2 values (packed FP32 arithmetic); each
// lane gives the bits of the one-node update.
template <class S, bool SR, class Cfg = StageCfg<S>, bool DYN = false>
__device__ __forceinline__ void staged_interior_pair(const typename S::T *__restrict__ sp,
                                                     typename S::T *__restrict__ fout,
                                                     const StepArgs &a, int c, int x, int y,
                                                     float4 m, uint32_t ts,
                                                     float2 k0 = make_float2(0.0f, 0.0f)) {
  using L = StageLayout<S, Cfg>;
  constexpr int PL = L::RW;  // elements between planes in a stage
  float2 d[9];               // lane x: node x, lane y: node x + 1
  const typename S::T *row = sp + Cfg::A + c;
  // e_x = 0 directions as one vector read per plane
  S::ld2(row, d[0].x, d[0].y);
  S::ld2(row + 2 * PL, d[2].x, d[2].y);
  S::ld2(row + 4 * PL, d[4].x, d[4].y);
  d[1] = make_float2(S::ld1(row + 1 * PL - 1), S::ld1(row + 1 * PL));
  d[5] = make_float2(S::ld1(row + 5 * PL - 1), S::ld1(row + 5 * PL));
  d[8] = make_float2(S::ld1(row + 8 * PL - 1), S::ld1(row + 8 * PL));
  d[3] = make_float2(S::ld1(row + 3 * PL + 1), S::ld1(row + 3 * PL + 2));
  d[6] = make_float2(S::ld1(row + 6 * PL + 1), S::ld1(row + 6 * PL + 2));
  d[7] = make_float2(S::ld1(row + 7 * PL + 1), S::ld1(row + 7 * PL + 2));
  const NodeStateT<float2> n = node_state_t<float2, DYN>(d, make_float2(m.x, m.z),
                                                         make_float2(m.y, m.w), a, k0);
  collide_t<S::kHiLo>(d, n, a);
  const long long o = (long long)y * a.pitch + x;
  const uint32_t h = SR ? mix32((uint32_t)(o >> 1) ^ ts) : 0u;
#pragma unroll
  for (int i = 0; i < 9; ++i)  // 32 random bits per direction and pair
    S::template st2<SR>(fout + i * a.plane + o, d[i].x, d[i].y, SR ? pair_bits(h, i) : 0u, 0u);
}

// The column-edge pairs of a tile: x = 0 and the last pair start
// (nx - 1) & ~1 of every row the tile touches (tile start (xT, yT), rows
// below y_end), for a consumer loop that skips them.  The pass hands them
// out one per thread, so that the long edge path runs in one or two warps
// per tile instead of diverging inside most of the interior warps when rows
// are short (the batched kernel: rows of 256 - 1024 nodes; with rows longer
// than a tile the single-lattice kernel keeps its edges in the loop, where
// they cost no registers).  Item k (row yT + k / 2, column end k % 2) goes
// to consumer thread (k + 32 rot) mod (consumer threads): rot turns with
// the tile, so that no warp is the slow one of every stage.
template <class S, bool SR, class Cfg = StageCfg<S>>
__device__ __forceinline__ void staged_column_edges(const typename S::T *__restrict__ sp,
                                                    const typename S::T *__restrict__ fin,
                                                    typename S::T *__restrict__ fout,
                                                    const float2 *__restrict__ med,
                                                    const StepArgs &a, const float2 *sm, int xT,
                                                    int yT, int y_end, uint32_t ts, int rot) {
  constexpr int kThreads = Cfg::WARPS * 32;
  const int k = (threadIdx.x + kThreads - 32 * rot) % kThreads;
  const int r = k >> 1;
  const int xl = (a.nx - 1) & ~1;
  const int x = (k & 1) ? xl : 0;
  if ((k & 1) && xl == 0) return;  // a row of one pair has one edge pair
  const int y = yT + r;
  if (y >= y_end) return;
  const long long c = (long long)r * a.pitch + x - xT;  // position in the tile
  if (c < 0 || c >= Cfg::W) return;
  const float4 m = *reinterpret_cast<const float4 *>(sm + c);
  staged_edge_pair_packed<S, SR, Cfg>(sp, fin, fout, med, a, (int)c, x, y, m, ts);
}

// ------------------------------------------------------------------ kernel
template <class S, bool SR, bool DYN = false>
__global__ void __launch_bounds__(kStagedThreads, 1)
    staged_step_kernel(const StepArgs a, const typename S::T *__restrict__ fin,
                       typename S::T *__restrict__ fout, const float2 *__restrict__ med,
                       const unsigned long long *__restrict__ tctr, int k, int rows,
                       unsigned *err) {
  using C = StageCfgFor<S, DYN>;
  using L = StageLayout<S, C>;
  static_assert(C::KN0 == DYN, "a dynamic Kn stages the Kn plane");
  using T = typename S::T;
  constexpr int W = C::W, H = C::H, A = C::A, NS = C::STAGES, RW = L::RW;
  extern __shared__ __align__(128) unsigned char smem[];
  const uint32_t sbase = smem_u32(smem);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  auto full = [&](int s) { return sbase + 8u * (uint32_t)s; };
  auto empty = [&](int s) { return sbase + 8u * (uint32_t)(NS + s); };
  if (threadIdx.x == 0) {
    for (int s = 0; s < NS; ++s) {
      mbar_init(full(s), 1);
      mbar_init(empty(s), kConsumerWarps);
    }
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  // Tiles are W consecutive nodes of the padded lattice read row after row
  // (flat index y * pitch + x over the launch rows), so no tile is partly
  // empty at a row end.  The source of plane i for flat index p is
  // p - e_iy * pitch (mod ny * pitch, the periodic wrap in y): the sources of
  // a tile are one contiguous span per plane, split only where it wraps.
  const long long F0 = (long long)a.y0 * a.pitch;
  const long long Fend = (long long)(a.y0 + rows) * a.pitch;
  const long long NP = (long long)a.ny * a.pitch;
  const int ntiles = (int)((Fend - F0 + W - 1) / W);
  const int y_end = a.y0 + rows;

  if (warp == kConsumerWarps) {
    // ------------------------------------------------------- producer
    // Lane i < 9 copies plane i (one or a few segments), lane 9 the medium,
    // lane 10 (dynamic Kn) the Kn at p0, after lane 0 has posted the
    // expected byte count.
    constexpr uint32_t kPlaneBytes = (uint32_t)(RW * sizeof(T));
    int it = 0;
    bool ok = true;
    for (int t = blockIdx.x; t < ntiles; t += gridDim.x, ++it) {
      const int tt = a.rev ? ntiles - 1 - t : t;  // the tile copied
      const int s = it % NS;
      const uint32_t use = (uint32_t)(it / NS);
      if (use > 0) {
        if (lane == 0) ok = mbar_wait(empty(s), (use - 1) & 1u, err);
        ok = __shfl_sync(0xffffffffu, ok ? 1 : 0, 0) != 0;
      }
      if (!ok) {
        // consumers are gone: let the copies already issued land, then leave
        if (lane == 0)
          for (int j = 1; j < NS && j <= it; ++j)
            mbar_wait(full((it - j) % NS), (uint32_t)((it - j) / NS) & 1u, err);
        return;
      }
      const long long T0 = F0 + (long long)tt * W;
      const uint32_t med_bytes = (uint32_t)(min((long long)W, Fend - T0) * 8);
      const uint32_t kn_bytes = DYN ? med_bytes / 2 : 0u;
      if (lane == 0) mbar_arrive_expect_tx(full(s), 9u * kPlaneBytes + med_bytes + kn_bytes);
      __syncwarp();
      if (tt == a.test_drop_tile) continue;  // the consumers' wait must run out
      const uint32_t st = sbase + (uint32_t)L::kBarBytes + (uint32_t)s * (uint32_t)L::kStageBytes;
      if (lane < 9) {
        const int ey = (lane == 2 || lane == 5 || lane == 6) ? 1
                       : ((lane == 4 || lane == 7 || lane == 8) ? -1 : 0);
        long long v = T0 - (long long)ey * a.pitch - A;
        while (v < 0) v += NP;
        while (v >= NP) v -= NP;
        const T *plane = fin + (long long)lane * a.plane;
        uint32_t dst = st + (uint32_t)lane * kPlaneBytes;
        long long left = RW;
        while (left > 0) {
          const long long seg = min(left, NP - v);
          bulk_g2s(dst, plane + v, (uint32_t)(seg * (long long)sizeof(T)), full(s));
          dst += (uint32_t)(seg * (long long)sizeof(T));
          left -= seg;
          v = 0;
        }
      } else if (lane == 9) {
        bulk_g2s(st + (uint32_t)L::kPopBytes, med + T0, med_bytes, full(s));
      } else if (DYN && lane == 10) {
        bulk_g2s(st + (uint32_t)(L::kPopBytes + L::kMedBytes), a.kn0 + T0, kn_bytes, full(s));
      }
    }
    return;
  }

  // --------------------------------------------------------- consumers
  uint32_t ts = 0;
  if (SR) {
    const unsigned long long tl = *tctr + (unsigned long long)k;
    ts = mix32((uint32_t)tl * 0x9e3779b9u ^ a.seed_lo ^ mix32((uint32_t)(tl >> 32) ^ a.seed_hi));
  }
  // Each consumer thread owns node pairs (x0, x0 + 1), x0 even, of the tile.
  constexpr int kPairs = (H * W / 2) / (kConsumerWarps * 32);
  // first node of this block's first tile, and the step between its tiles
  // (backwards when the launch walks the tiles from the end)
  const int t0 = a.rev ? ntiles - 1 - (int)blockIdx.x : (int)blockIdx.x;
  const long long Tb = F0 + (long long)t0 * W;
  int yT = (int)(Tb / a.pitch), xT = (int)(Tb - (long long)yT * a.pitch);
  const long long D = (long long)gridDim.x * W;
  const int dy = (int)(D / a.pitch), dx = (int)(D - (long long)dy * a.pitch);
  int it = 0;
  for (int t = blockIdx.x; t < ntiles; t += gridDim.x, ++it) {
    const int s = it % NS;
    if (!mbar_wait(full(s), (uint32_t)(it / NS) & 1u, err)) return;
    const unsigned char *sb = smem + L::kBarBytes + s * L::kStageBytes;
    const T *sp = reinterpret_cast<const T *>(sb);
    const float2 *sm = reinterpret_cast<const float2 *>(sb + L::kPopBytes);
    const float *sk = reinterpret_cast<const float *>(sb + L::kPopBytes + L::kMedBytes);
#pragma unroll 1
    for (int j = 0; j < kPairs; ++j) {
      const int q = threadIdx.x + j * kConsumerWarps * 32;  // pair index in the tile
      const int c = 2 * q;
      int x = xT + c, y = yT;
      while (x >= a.pitch) {  // at most W / pitch + 1 rows per tile
        x -= a.pitch;
        ++y;
      }
      if (y >= y_end || x >= a.nx) continue;
      const float4 m = *reinterpret_cast<const float4 *>(sm + c);
      const float2 k0 = DYN ? *reinterpret_cast<const float2 *>(sk + c) : make_float2(0.0f, 0.0f);
      if (x == 0 || x + 2 >= a.nx || (a.walls && (y == 1 || y == a.ny - 2))) {
        staged_edge_pair<S, SR, C, DYN>(sp, fin, fout, med, a, c, x, y, m, k0, ts);
        continue;
      }
      staged_interior_pair<S, SR, C, DYN>(sp, fout, a, c, x, y, m, ts, k0);
    }
    __syncwarp();
    if (lane == 0) mbar_arrive(empty(s));
    if (a.rev) {
      xT -= dx;
      yT -= dy;
      if (xT < 0) {
        xT += a.pitch;
        --yT;
      }
    } else {
      xT += dx;
      yT += dy;
      if (xT >= a.pitch) {
        xT -= a.pitch;
        ++yT;
      }
    }
  }
}

}  // namespace lbmp
