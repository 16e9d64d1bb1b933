// Batched sweeps: many lattices (media realizations, Knudsen numbers, sizes)
// advanced together by one persistent launch per time step.
//
// Every instance has its own population buffers, medium and FP16 scale; the
// physics parameters (tau, J, G, boundary kinds, densities, Forchheimer) are
// shared.  The step kernel is the fused pull-collide-store of Eq. 12-17
// (Section III) over a flat work list: work item w is a row segment of
// BX * NPT nodes of instance item_inst[w].  Either one block per item, or a
// persistent grid (SMs x resident blocks) walking contiguous item ranges.
// The launch shape (BX, NPT, grid mode, or the staged bulk-copy kernel over
// a tile list) is picked by lbmp_batch_tune, which times every candidate on
// the batch itself and restores the populations.
// Per-instance global permeabilities are FP64 segmented reductions.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <new>
#include <string>
#include <vector>

#include "kernels.h"
#include "device_scope.h"
#include "nvtx_range.h"
#include "lattice.cuh"
#include "lbmp.h"
#include "staged.cuh"

namespace lbmp {

struct BatchInst {
  StepArgs a;            // geometry (y0 = first fluid row), physics, FP16 scale
  void *buf[2];          // population buffers
  const float2 *med;     // (eps, 1/k_a)
  int rows;              // fluid rows
  int index;             // instance number (mixes the stochastic-rounding stream)
};

__device__ __forceinline__ int find_instance(const long long *__restrict__ cum, int count,
                                             long long w) {
  int lo = 0, hi = count;  // cum[0] = 0, cum[count] = items; largest lo with cum[lo] <= w
  while (hi - lo > 1) {
    const int mid = (lo + hi) >> 1;
    if (cum[mid] <= w) lo = mid; else hi = mid;
  }
  return lo;
}

// One work item: a row segment of BX * NPT nodes of instance ii.
template <class S, bool SR, int BX, int NPT>
__device__ __forceinline__ void batch_item(const BatchInst &I, long long local, int parity,
                                           uint32_t ts) {
  const StepArgs &a = I.a;
  constexpr int chunk = BX * NPT;
  const int xblocks = (a.nx + chunk - 1) / chunk;
  const int y = a.y0 + (int)(local / xblocks);
  const int xb = (int)(local % xblocks) * chunk + threadIdx.x;
  const typename S::T *fin = (const typename S::T *)I.buf[parity];
  typename S::T *fout = (typename S::T *)I.buf[parity ^ 1];
  const long long row = (long long)y * a.pitch;
  float d[NPT][9];
  float2 m[NPT];
#pragma unroll
  for (int j = 0; j < NPT; ++j) {
    const int x = xb + j * BX;
    if (x < a.nx) {
      pull_node<S>(fin, a, x, y, d[j]);
      m[j] = I.med[row + x];
    }
  }
  const uint32_t tsi = SR ? ts ^ mix32((uint32_t)I.index * 0x85ebca77u + 1u) : 0u;
#pragma unroll
  for (int j = 0; j < NPT; ++j) {
    const int x = xb + j * BX;
    if (x >= a.nx) continue;
    if (a.pressure && (x == 0 || x == a.nx - 1))
      pressure_node<S>(fin, I.med, a, x, y, m[j].x, d[j]);
    const NodeState s = node_state(d[j], m[j].x, m[j].y, a);
    collide<S::kHiLo>(d[j], s, a);
    typename S::T *o = fout + row + x;
    const uint32_t h = SR ? mix32((uint32_t)(row + x) ^ tsi) : 0u;
#pragma unroll
    for (int i = 0; i < 9; ++i) S::template st1r<SR>(o + i * a.plane, d[j][i], h, i);
  }
}

// persistent = 0: block b updates work item b (one launch over every item).  persistent = 1: gridDim.x
// resident blocks each walk a contiguous range of items.  item_inst[w] is
// the instance of item w, cum[i] its first item.
template <class S, bool SR, int BX, int NPT>
__global__ void __launch_bounds__(BX)
    batch_step_kernel(const BatchInst *__restrict__ inst, const long long *__restrict__ cum,
                      const int *__restrict__ item_inst, long long items, int persistent,
                      int parity, const unsigned long long *__restrict__ tctr, int k) {
  uint32_t ts = 0;
  if (SR) {
    const StepArgs &a0 = inst[0].a;
    const unsigned long long t = *tctr + (unsigned long long)k;
    ts = mix32((uint32_t)t * 0x9e3779b9u ^ a0.seed_lo ^ mix32((uint32_t)(t >> 32) ^ a0.seed_hi));
  }
  if (!persistent) {
    const long long w = blockIdx.x;
    if (w >= items) return;
    const int ii = item_inst[w];
    batch_item<S, SR, BX, NPT>(inst[ii], w - cum[ii], parity, ts);
    return;
  }
  const long long per = (items + gridDim.x - 1) / gridDim.x;
  const long long w0 = (long long)blockIdx.x * per;
  const long long w1 = w0 + per < items ? w0 + per : items;
  for (long long w = w0; w < w1; ++w) {
    const int ii = item_inst[w];
    batch_item<S, SR, BX, NPT>(inst[ii], w - cum[ii], parity, ts);
  }
}

// --------------------------------------------------- staged batched kernel
// The staged step (staged.cuh) over the tiles of every instance: tile t is
// W consecutive nodes of one instance's padded lattice, tiles[t] = (instance,
// x and y of its first node, end of the instance's fluid rows).  The physics
// shared by all instances comes in `base`; per tile the consumers override
// the instance's geometry and FP16 scale, which then live in registers.
// The producer, which runs stages ahead, looks the tile and its instance up
// and leaves them in a per-stage header next to the copies (published by the
// same mbarrier phase), so the consumers never wait on a global load at a
// tile start.
struct TileHead {
  const void *fin;      // population buffer read this step
  void *fout;           // population buffer written this step
  const float2 *med;    // medium of the instance
  long long plane;      // elements per plane
  int nx, ny, pitch;    // geometry of the instance
  int x, y, y_end;      // first node of the tile, end of the fluid rows
  float scale, inv_scale;  // FP16 scale of the instance
  uint32_t mix;         // stochastic-rounding stream of the instance
  int pad[3];
};
constexpr int kHeadBytes = 128;
static_assert(sizeof(TileHead) <= kHeadBytes && sizeof(TileHead) % 16 == 0, "tile header");

// Row pitch of an instance: nx rounded up to kBatchPitchAlign, without the
// skew a single lattice's pitch gets at multiples of 512.  That skew keeps
// the tile copies of 4096-wide rows from aliasing in the DRAM channels; the
// instances here are at most ~1000 wide and many run at once, and the skew
// only added row padding to the 512- and 1024-wide ones (12.5% and 6% of
// their reads): FP16 on 256 instances 142.5 -> 146.1 GLUPS without it.
// A multiple of 64 elements keeps every bulk copy 16-byte aligned.
constexpr int kBatchPitchAlign = 64;
inline int batch_pitch(int nx) {
  return ((nx + kBatchPitchAlign - 1) / kBatchPitchAlign) * kBatchPitchAlign;
}
// Stage configuration of the batched kernel.  Its consumers hold more per
// tile (the instance's buffers, geometry and scale) than the single-lattice
// ones: ~108 registers a thread.  Registers are split between the SM's four
// schedulers (16 K each) and a block's warps spread over them, so a block of
// 17 warps (16 consumers and the producer) leaves 96 registers a thread and
// spills, while 16 warps leave 128.  FP16: 15 consumer warps, tiles of 2880
// nodes (three pairs a thread), 3 stages (256 instances: 131.7 -> 142.9
// GLUPS against 12 warps x 2304 x 3; the larger tiles also spread the
// per-tile header and column-edge work over more nodes).  FP32: 12 consumer
// warps, 1536-node tiles, two pairs a thread (at the copy roofline).
template <class S>
struct BatchCfg;
template <>
struct BatchCfg<StoreF32> {
  static constexpr int W = 1536, H = 1, A = 4, STAGES = 3;
  static constexpr int WARPS = 12;
  static constexpr bool KN0 = false;  // batches have a static Kn
};
template <>
struct BatchCfg<StoreF16> {
  static constexpr int W = 2880, H = 1, A = 8, STAGES = 3;
  static constexpr int WARPS = 15;
  static constexpr bool KN0 = false;
};
template <class S>
constexpr int batch_threads() {
  return (BatchCfg<S>::WARPS + 1) * 32;
}
template <class S>
constexpr int batch_smem_bytes() {
  return StageLayout<S, BatchCfg<S>>::kSmemBytes + BatchCfg<S>::STAGES * kHeadBytes;
}
static_assert(batch_smem_bytes<StoreF16>() <= 227 * 1024 &&
                  batch_smem_bytes<StoreF32>() <= 227 * 1024,
              "stages and tile headers fit the 227 KB of shared memory of a CTA");

template <class S, bool SR>
__global__ void __launch_bounds__(batch_threads<S>(), 1)
    batch_staged_kernel(const StepArgs base, const BatchInst *__restrict__ inst,
                        const int4 *__restrict__ tiles, int ntiles, int parity,
                        const unsigned long long *__restrict__ tctr, int k, unsigned *err) {
  using C = BatchCfg<S>;
  using L = StageLayout<S, C>;
  using T = typename S::T;
  constexpr int W = C::W, A = C::A, NS = C::STAGES, RW = L::RW;
  constexpr uint32_t kPlaneBytes = (uint32_t)(RW * sizeof(T));
  extern __shared__ __align__(128) unsigned char smem[];
  const uint32_t sbase = smem_u32(smem);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  auto full = [&](int s) { return sbase + 8u * (uint32_t)s; };
  auto empty = [&](int s) { return sbase + 8u * (uint32_t)(NS + s); };
  if (threadIdx.x == 0) {
    for (int s = 0; s < NS; ++s) {
      mbar_init(full(s), 1);
      mbar_init(empty(s), C::WARPS);
    }
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  if (warp == C::WARPS) {
    // ------------------------------------------------------- producer
    int it = 0;
    bool ok = true;
    for (int t = blockIdx.x; t < ntiles; t += gridDim.x, ++it) {
      const int s = it % NS;
      const uint32_t use = (uint32_t)(it / NS);
      if (use > 0) {
        if (lane == 0) ok = mbar_wait(empty(s), (use - 1) & 1u, err);
        ok = __shfl_sync(0xffffffffu, ok ? 1 : 0, 0) != 0;
      }
      if (!ok) {
        if (lane == 0)
          for (int j = 1; j < NS && j <= it; ++j)
            mbar_wait(full((it - j) % NS), (uint32_t)((it - j) / NS) & 1u, err);
        return;
      }
      const int4 tr = tiles[t];
      const BatchInst &I = inst[tr.x];
      const int pitch = I.a.pitch;
      const long long NP = (long long)I.a.ny * pitch;
      const long long T0 = (long long)tr.z * pitch + tr.y;
      const long long Fend = (long long)tr.w * pitch;
      const uint32_t med_bytes = (uint32_t)(min((long long)W, Fend - T0) * 8);
      if (lane == 0) {
        // the header is a plain store ordered before the arrival (release);
        // the consumers' wait on the phase acquires it
        TileHead *h = reinterpret_cast<TileHead *>(smem + L::kSmemBytes + s * kHeadBytes);
        h->fin = I.buf[parity];
        h->fout = I.buf[parity ^ 1];
        h->med = I.med;
        h->plane = I.a.plane;
        h->nx = I.a.nx;
        h->ny = I.a.ny;
        h->pitch = pitch;
        h->x = tr.y;
        h->y = tr.z;
        h->y_end = tr.w;
        h->scale = I.a.scale;
        h->inv_scale = I.a.inv_scale;
        h->mix = mix32((uint32_t)I.index * 0x85ebca77u + 1u);
        mbar_arrive_expect_tx(full(s), 9u * kPlaneBytes + med_bytes);
      }
      __syncwarp();
      if (t == base.test_drop_tile) continue;  // the consumers' wait must run out
      const uint32_t st = sbase + (uint32_t)L::kBarBytes + (uint32_t)s * (uint32_t)L::kStageBytes;
      if (lane < 9) {
        const int ey = (lane == 2 || lane == 5 || lane == 6) ? 1
                       : ((lane == 4 || lane == 7 || lane == 8) ? -1 : 0);
        long long v = T0 - (long long)ey * pitch - A;
        while (v < 0) v += NP;
        while (v >= NP) v -= NP;
        const T *plane = (const T *)I.buf[parity] + (long long)lane * I.a.plane;
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
        bulk_g2s(st + (uint32_t)L::kPopBytes, I.med + T0, med_bytes, full(s));
      }
    }
    return;
  }
  // --------------------------------------------------------- consumers
  uint32_t ts = 0;
  if (SR) {
    const unsigned long long tl = *tctr + (unsigned long long)k;
    ts = mix32((uint32_t)tl * 0x9e3779b9u ^ base.seed_lo ^ mix32((uint32_t)(tl >> 32) ^ base.seed_hi));
  }
  constexpr int kPairs = (W / 2) / (C::WARPS * 32);
  int it = 0;
  for (int t = blockIdx.x; t < ntiles; t += gridDim.x, ++it) {
    const int s = it % NS;
    if (!mbar_wait(full(s), (uint32_t)(it / NS) & 1u, err)) return;
    const TileHead h = *reinterpret_cast<const TileHead *>(smem + L::kSmemBytes + s * kHeadBytes);
    const T *fin = (const T *)h.fin;
    T *fout = (T *)h.fout;
    const float2 *med = h.med;
    const unsigned char *sb = smem + L::kBarBytes + s * L::kStageBytes;
    const T *sp = reinterpret_cast<const T *>(sb);
    const float2 *sm = reinterpret_cast<const float2 *>(sb + L::kPopBytes);
    StepArgs a = base;
    a.nx = h.nx;
    a.ny = h.ny;
    a.pitch = h.pitch;
    a.plane = h.plane;
    a.scale = h.scale;
    a.inv_scale = h.inv_scale;
    const uint32_t tsi = SR ? ts ^ h.mix : 0u;
#pragma unroll 1
    for (int j = 0; j < kPairs; ++j) {
      const int c = 2 * (threadIdx.x + j * C::WARPS * 32);
      int x = h.x + c, y = h.y;
      while (x >= a.pitch) {
        x -= a.pitch;
        ++y;
      }
      if (y >= h.y_end || x >= a.nx) continue;
      if (x == 0 || x + 2 >= a.nx) continue;  // column edges: the pass below
      const float4 m = *reinterpret_cast<const float4 *>(sm + c);
      if (a.walls && (y == 1 || y == a.ny - 2)) {
        staged_edge_pair_packed<S, SR, C>(sp, fin, fout, med, a, c, x, y, m, tsi);
        continue;
      }
      staged_interior_pair<S, SR, C>(sp, fout, a, c, x, y, m, tsi);
    }
    staged_column_edges<S, SR, C>(sp, fin, fout, med, a, sm, h.x, h.y, h.y_end, tsi,
                                  it % C::WARPS);
    __syncwarp();
    if (lane == 0) mbar_arrive(empty(s));
  }
}

template <class S, bool SR>
static cudaError_t launch_batch_staged_t(const StepArgs &base, const BatchInst *inst,
                                         const int4 *tiles, int ntiles, int parity,
                                         const unsigned long long *tctr, int k, unsigned *err,
                                         int nsm, cudaStream_t s) {
  static const cudaError_t attr = cudaFuncSetAttribute(
      batch_staged_kernel<S, SR>, cudaFuncAttributeMaxDynamicSharedMemorySize,
      batch_smem_bytes<S>());
  if (attr != cudaSuccess) return attr;
  if (ntiles <= 0) return cudaSuccess;
  const int grid = ntiles < nsm ? ntiles : nsm;
  batch_staged_kernel<S, SR><<<grid, batch_threads<S>(), batch_smem_bytes<S>(), s>>>(
      base, inst, tiles, ntiles, parity, tctr, k, err);
  return cudaGetLastError();
}

// Tile width of the staged kernel for a storage kind.
inline int staged_tile_width(int storage) {
  return storage == LBMP_STORE_FP32 ? BatchCfg<StoreF32>::W : BatchCfg<StoreF16>::W;
}
// Consumer warps of the staged kernel for a storage kind.
inline int staged_warps(int storage) {
  return storage == LBMP_STORE_FP32 ? BatchCfg<StoreF32>::WARPS : BatchCfg<StoreF16>::WARPS;
}

// Per-instance reductions: block partials over the work list (one 256-node
// segment per item), then one block per instance sums its items in order.
constexpr int kBatchMacroBX = 256;

template <class S>
__global__ void __launch_bounds__(kBatchMacroBX)
    batch_macro_kernel(const BatchInst *__restrict__ inst, const long long *__restrict__ cum,
                       int count, int parity, double *__restrict__ partials) {
  const long long items = cum[count];
  for (long long w = blockIdx.x; w < items; w += gridDim.x) {
    const int ii = find_instance(cum, count, w);
    const BatchInst &I = inst[ii];
    const StepArgs &a = I.a;
    const long long local = w - cum[ii];
    const int xblocks = (a.nx + kBatchMacroBX - 1) / kBatchMacroBX;
    const int y = a.y0 + (int)(local / xblocks);
    const int x = (int)(local % xblocks) * kBatchMacroBX + threadIdx.x;
    const typename S::T *fin = (const typename S::T *)I.buf[parity];
    double v[kNQ] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
    if (x < a.nx) {
      float d[9];
      const float2 m = I.med[(long long)y * a.pitch + x];
      pull_node<S>(fin, a, x, y, d);
      if (a.pressure && (x == 0 || x == a.nx - 1)) pressure_node<S>(fin, I.med, a, x, y, m.x, d);
      const NodeState s = node_state(d, m.x, m.y, a);
      const bool finite = isfinite(s.ux) && isfinite(s.uy) && isfinite(s.rho);
      v[0] = finite ? (double)s.ux : 0.0;
      v[1] = finite ? (double)s.uy : 0.0;
      v[2] = finite ? (double)(s.drho_s * a.inv_scale) : 0.0;
      v[3] = finite ? (double)s.ux * s.ux + (double)s.uy * s.uy : 0.0;
      v[5] = finite ? 0.0 : 1.0;
    }
    __shared__ double red[kBatchMacroBX / 32][kNQ];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int q = 0; q < kNQ; ++q) {
      double t = v[q];
#pragma unroll
      for (int off = 16; off > 0; off >>= 1) t += __shfl_down_sync(0xffffffffu, t, off);
      if (lane == 0) red[warp][q] = t;
    }
    __syncthreads();
    if (threadIdx.x < kNQ) {
      double t = 0.0;
      for (int ww = 0; ww < kBatchMacroBX / 32; ++ww) t += red[ww][threadIdx.x];
      partials[w * kNQ + threadIdx.x] = t;
    }
    __syncthreads();
  }
}

__global__ void __launch_bounds__(256)
    batch_finalize_kernel(const long long *__restrict__ cum, const double *__restrict__ partials,
                          double *__restrict__ out) {
  __shared__ double sh[256];
  const int ii = blockIdx.x;
  const long long b0 = cum[ii], b1 = cum[ii + 1];
  for (int q = 0; q < kNQ; ++q) {
    double t = 0.0;
    for (long long b = b0 + threadIdx.x; b < b1; b += 256) t += partials[b * kNQ + q];
    sh[threadIdx.x] = t;
    __syncthreads();
    for (int s = 128; s > 0; s >>= 1) {
      if (threadIdx.x < s) sh[threadIdx.x] += sh[threadIdx.x + s];
      __syncthreads();
    }
    if (threadIdx.x == 0) out[(long long)ii * kNQ + q] = sh[0];
    __syncthreads();
  }
}

// ------------------------------------------------------------ launch shapes
struct Shape {
  int bx, npt, persistent;
};
// persistent = 2: the staged batched kernel (bx, npt unused)
constexpr Shape kShapes[] = {{128, 1, 0}, {128, 2, 0}, {256, 1, 0}, {256, 2, 0}, {64, 4, 0},
                             {128, 4, 0}, {128, 2, 1}, {256, 2, 1}, {64, 4, 1}, {0, 0, 2}};
constexpr int kNumShapes = (int)(sizeof(kShapes) / sizeof(kShapes[0]));

template <class S, bool SR, int BX, int NPT>
static cudaError_t launch_shape_t(const BatchInst *inst, const long long *cum, const int *item_inst,
                                  int persistent, int parity, const unsigned long long *tctr, int k,
                                  int nsm, long long items, cudaStream_t s) {
  // resident blocks per SM of this instantiation (queried once per process)
  static const int per_sm = [] {
    int v = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&v, batch_step_kernel<S, SR, BX, NPT>, BX,
                                                      0) != cudaSuccess)
      v = 1;
    return std::max(v, 1);
  }();
  long long grid = persistent ? std::min((long long)per_sm * nsm, items) : items;
  if (grid < 1) return cudaSuccess;
  if (grid > 0x7fffffffLL) return cudaErrorInvalidConfiguration;
  batch_step_kernel<S, SR, BX, NPT><<<(unsigned)grid, BX, 0, s>>>(inst, cum, item_inst, items,
                                                                   persistent, parity, tctr, k);
  return cudaGetLastError();
}

template <class S, bool SR>
static cudaError_t launch_shape_s(int shape, const BatchInst *inst, const long long *cum,
                                  const int *item_inst, int parity,
                                  const unsigned long long *tctr, int k, int nsm, long long items,
                                  cudaStream_t s) {
  const int ps = kShapes[shape].persistent;
  switch (kShapes[shape].bx * 16 + kShapes[shape].npt) {
    case 128 * 16 + 1: return launch_shape_t<S, SR, 128, 1>(inst, cum, item_inst, ps, parity, tctr, k, nsm, items, s);
    case 128 * 16 + 2: return launch_shape_t<S, SR, 128, 2>(inst, cum, item_inst, ps, parity, tctr, k, nsm, items, s);
    case 256 * 16 + 1: return launch_shape_t<S, SR, 256, 1>(inst, cum, item_inst, ps, parity, tctr, k, nsm, items, s);
    case 256 * 16 + 2: return launch_shape_t<S, SR, 256, 2>(inst, cum, item_inst, ps, parity, tctr, k, nsm, items, s);
    case 64 * 16 + 4: return launch_shape_t<S, SR, 64, 4>(inst, cum, item_inst, ps, parity, tctr, k, nsm, items, s);
    default: return launch_shape_t<S, SR, 128, 4>(inst, cum, item_inst, ps, parity, tctr, k, nsm, items, s);
  }
}

static cudaError_t launch_batch_step(int storage, bool sr, int shape, const BatchInst *inst,
                                     const long long *cum, const int *item_inst, int parity,
                                     const unsigned long long *tctr, int k, int nsm,
                                     long long items, const StepArgs &base, const int4 *tiles,
                                     int ntiles, unsigned *err, cudaStream_t s) {
  if (kShapes[shape].persistent == 2) {
    if (storage == LBMP_STORE_FP32)
      return launch_batch_staged_t<StoreF32, false>(base, inst, tiles, ntiles, parity, tctr, k, err, nsm, s);
    if (sr) return launch_batch_staged_t<StoreF16, true>(base, inst, tiles, ntiles, parity, tctr, k, err, nsm, s);
    return launch_batch_staged_t<StoreF16, false>(base, inst, tiles, ntiles, parity, tctr, k, err, nsm, s);
  }
  if (storage == LBMP_STORE_FP32)
    return launch_shape_s<StoreF32, false>(shape, inst, cum, item_inst, parity, tctr, k, nsm, items, s);
  if (sr)
    return launch_shape_s<StoreF16, true>(shape, inst, cum, item_inst, parity, tctr, k, nsm, items, s);
  return launch_shape_s<StoreF16, false>(shape, inst, cum, item_inst, parity, tctr, k, nsm, items, s);
}

}  // namespace lbmp

using lbmp::BatchInst;

namespace {

lbmp_status bfail(lbmp_status st, const char *fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  lbmp::set_last_error(buf);
  return st;
}

lbmp_status bcuda(cudaError_t e, const char *what) {
  cudaGetLastError();
  return bfail(e == cudaErrorMemoryAllocation ? LBMP_ENOMEM : LBMP_ECUDA, "%s: %s", what,
               cudaGetErrorString(e));
}

#define BCK(call)                                        \
  do {                                                   \
    cudaError_t e_ = (call);                             \
    if (e_ != cudaSuccess) return bcuda(e_, #call);      \
  } while (0)

constexpr int kBatchGraphSteps = 32;

}  // namespace

struct lbmp_batch {
  lbmp_params p{};
  int device = 0, nsm = 1;
  cudaStream_t stream = nullptr, cap_stream = nullptr;
  bool own_stream = false;
  int count = 0;
  bool sr = false;
  std::vector<BatchInst> h_inst;
  std::vector<int> fields_set;
  std::vector<double> eps_mean;
  std::vector<long long> fluid_nodes;
  BatchInst *d_inst = nullptr;
  long long *d_cum_step = nullptr;   // work list of the chosen shape
  int *d_item_inst = nullptr;        // instance of every work item (chosen shape)
  long long items_cap = 0;           // capacity of d_item_inst
  long long *d_cum_macro = nullptr;  // work list of the reductions
  long long items_step = 0, items_macro = 0;
  double *d_partials = nullptr;      // [items_macro][kNQ]
  double *d_results = nullptr;       // [count][kNQ]
  double *d_med_partials = nullptr;  // set_fields scratch
  double *d_med_results = nullptr;
  unsigned *d_flag = nullptr;
  unsigned *d_err = nullptr;         // raised by a bounded wait of the staged kernel
  int4 *d_tiles = nullptr;           // tile list of the staged kernel
  int ntiles = 0;
  unsigned long long *d_tctr = nullptr;
  int shape = 1;                     // index into kShapes (default 128 x 2)
  int parity = 0;
  int64_t steps = 0, launches = 0, total_nodes = 0, device_bytes = 0;
  cudaGraphExec_t graph[2] = {nullptr, nullptr};
  std::vector<void *> allocs;
};

namespace {

lbmp_status balloc(lbmp_batch *b, void **p, size_t bytes, const char *what) {
  cudaError_t e = cudaMalloc(p, bytes);
  if (e != cudaSuccess) {
    *p = nullptr;
    return bcuda(e, what);
  }
  b->allocs.push_back(*p);
  b->device_bytes += (int64_t)bytes;
  return LBMP_OK;
}

void bfree_graphs(lbmp_batch *b) {
  for (auto &g : b->graph)
    if (g) {
      cudaGraphExecDestroy(g);
      g = nullptr;
    }
}

void brelease(lbmp_batch *b) {
  if (!b) return;
  const DeviceScope device_scope(b->device);
  if (b->stream) cudaStreamSynchronize(b->stream);
  bfree_graphs(b);
  for (void *p : b->allocs) cudaFree(p);
  if (b->cap_stream) cudaStreamDestroy(b->cap_stream);
  if (b->own_stream && b->stream) cudaStreamDestroy(b->stream);
  delete b;
}

// cumulative work items for a chunk of `chunk` nodes per item
std::vector<long long> work_list(const lbmp_batch *b, int chunk) {
  std::vector<long long> cum(b->count + 1, 0);
  for (int i = 0; i < b->count; ++i) {
    const lbmp::StepArgs &a = b->h_inst[i].a;
    const long long xblocks = (a.nx + chunk - 1) / chunk;
    cum[i + 1] = cum[i] + xblocks * (long long)b->h_inst[i].rows;
  }
  return cum;
}

lbmp_status upload_cum(lbmp_batch *b, long long *d_cum, const std::vector<long long> &cum) {
  BCK(cudaMemcpyAsync(d_cum, cum.data(), cum.size() * sizeof(long long),
                      cudaMemcpyHostToDevice, b->stream));
  BCK(cudaStreamSynchronize(b->stream));
  return LBMP_OK;
}

lbmp_status set_shape(lbmp_batch *b, int shape) {
  const lbmp::Shape sh = lbmp::kShapes[shape];
  if (sh.persistent == 2) {  // staged: the tile list is built at creation
    b->shape = shape;
    bfree_graphs(b);
    return LBMP_OK;
  }
  std::vector<long long> cum = work_list(b, sh.bx * sh.npt);
  if (cum.back() > b->items_cap) return bfail(LBMP_ECUDA, "work-item table too small");
  std::vector<int> item_inst((size_t)cum.back());
  for (int i = 0; i < b->count; ++i)
    std::fill(item_inst.begin() + cum[i], item_inst.begin() + cum[i + 1], i);
  BCK(cudaMemcpyAsync(b->d_item_inst, item_inst.data(), item_inst.size() * sizeof(int),
                      cudaMemcpyHostToDevice, b->stream));
  lbmp_status st = upload_cum(b, b->d_cum_step, cum);
  if (st) return st;
  b->items_step = cum.back();
  b->shape = shape;
  bfree_graphs(b);
  return LBMP_OK;
}

lbmp_status launch_steps(lbmp_batch *b, int64_t n, cudaStream_t s, bool count_launches) {
  for (int64_t t = 0; t < n; ++t) {
    BCK(lbmp::launch_batch_step(b->p.storage, b->sr, b->shape, b->d_inst, b->d_cum_step,
                                b->d_item_inst, b->parity, b->d_tctr, (int)t, b->nsm,
                                b->items_step, b->h_inst[0].a, b->d_tiles, b->ntiles, b->d_err, s));
    b->parity ^= 1;
    if (count_launches) b->launches++;
  }
  if (n > 0 && b->sr) {
    BCK(lbmp::launch_bump(b->d_tctr, (int)n, s));
    if (count_launches) b->launches++;
  }
  return LBMP_OK;
}

lbmp_status get_graph(lbmp_batch *b, cudaGraphExec_t *out) {
  const int par = b->parity;
  if (b->graph[par]) {
    *out = b->graph[par];
    return LBMP_OK;
  }
  cudaGraph_t g = nullptr;
  BCK(cudaStreamBeginCapture(b->cap_stream, cudaStreamCaptureModeThreadLocal));
  lbmp_status st = launch_steps(b, kBatchGraphSteps, b->cap_stream, false);
  cudaError_t end = cudaStreamEndCapture(b->cap_stream, &g);
  b->parity = par;  // the capture did not run anything
  if (st) {
    if (g) cudaGraphDestroy(g);
    return st;
  }
  if (end != cudaSuccess) return bcuda(end, "cudaStreamEndCapture");
  cudaGraphExec_t exec = nullptr;
  cudaError_t ie = cudaGraphInstantiate(&exec, g, 0);
  cudaGraphDestroy(g);
  if (ie != cudaSuccess) return bcuda(ie, "cudaGraphInstantiate");
  b->graph[par] = exec;
  *out = exec;
  return LBMP_OK;
}

lbmp_status do_step(lbmp_batch *b, int64_t n) {
  int64_t left = n;
  while (left >= kBatchGraphSteps) {
    cudaGraphExec_t g = nullptr;
    lbmp_status st = get_graph(b, &g);
    if (st) return st;
    BCK(cudaGraphLaunch(g, b->stream));
    b->launches += kBatchGraphSteps + (b->sr ? 1 : 0);
    left -= kBatchGraphSteps;
    // an even number of steps keeps the parity
  }
  lbmp_status st = launch_steps(b, left, b->stream, true);
  if (st) return st;
  b->steps += n;
  return LBMP_OK;
}

bool all_fields(const lbmp_batch *b) {
  for (int f : b->fields_set)
    if (!f) return false;
  return true;
}

// ------------------------------------------------------ tuned-shape cache
// The launch shape tuned for one batch serves every later batch of the same
// class: storage and rounding, boundary kinds, Forchheimer, the node-weighted
// median of ceil(log2 nx) over the instances, floor(log2 of all nodes), and
// the SM count of the device.  Kept per process, and in the file named by
// LBMP_TUNE_CACHE when that is set (one "key shape ms_per_step" line per
// tuning; the last line of a key wins).  File errors are ignored: the cache
// only saves tuning time.
std::string class_key(const lbmp_params &p, int count, const int32_t *nx, const int32_t *ny,
                      int nsm) {
  std::vector<std::pair<int, long long>> cls;  // (ceil(log2 nx), nodes)
  long long total = 0;
  for (int i = 0; i < count; ++i) {
    int c = 0;
    while ((1LL << c) < (long long)nx[i]) ++c;
    const long long n = (long long)nx[i] * ny[i];
    cls.push_back({c, n});
    total += n;
  }
  std::sort(cls.begin(), cls.end());
  int med = cls.back().first;
  long long acc = 0;
  for (const auto &q : cls) {
    acc += q.second;
    if (2 * acc >= total) {
      med = q.first;
      break;
    }
  }
  int tcls = 0;  // floor(log2 total)
  while ((2LL << tcls) <= total) ++tcls;
  const int sr = p.storage == LBMP_STORE_FP16 && p.fp16_rounding == LBMP_ROUND_STOCHASTIC;
  char buf[128];
  snprintf(buf, sizeof(buf), "s%d-r%d-x%d-y%d-f%d-n%d-t%d-m%d", (int)p.storage, sr, (int)p.bc_x,
           (int)p.bc_y, p.forchheimer ? 1 : 0, med, tcls, nsm);
  return buf;
}

struct TuneEntry {
  int shape;
  double ms;
};
std::mutex g_tune_mu;
std::map<std::string, TuneEntry> g_tune_cache;

bool tune_file_lookup(const std::string &key, TuneEntry *out) {
  const char *path = getenv("LBMP_TUNE_CACHE");
  if (!path || !*path) return false;
  FILE *f = fopen(path, "r");
  if (!f) return false;
  char k[128];
  int shape;
  double ms;
  bool found = false;
  while (fscanf(f, "%127s %d %lf", k, &shape, &ms) == 3)
    if (key == k && shape >= 0 && shape < lbmp::kNumShapes) {
      *out = {shape, ms};
      found = true;
    }
  fclose(f);
  return found;
}

void tune_file_append(const std::string &key, const TuneEntry &e) {
  const char *path = getenv("LBMP_TUNE_CACHE");
  if (!path || !*path) return;
  FILE *f = fopen(path, "a");
  if (!f) return;
  fprintf(f, "%s %d %.9g\n", key.c_str(), e.shape, e.ms);
  fclose(f);
}

}  // namespace

extern "C" {

lbmp_status lbmp_batch_class(const lbmp_params *p, int32_t count, const int32_t *nx,
                             const int32_t *ny, int32_t nsm, char *key, int32_t cap) {
  try {
    if (!p || !nx || !ny || !key) return bfail(LBMP_EINVAL, "lbmp_batch_class: NULL argument");
    if (count < 1) return bfail(LBMP_EINVAL, "count must be >= 1");
    if (nsm < 1) return bfail(LBMP_EINVAL, "nsm must be >= 1");
    for (int i = 0; i < count; ++i)
      if (nx[i] < 1 || ny[i] < 1) return bfail(LBMP_EINVAL, "instance %d: nx, ny must be >= 1", i);
    const std::string k = class_key(*p, count, nx, ny, nsm);
    if (cap < (int32_t)k.size() + 1) return bfail(LBMP_EINVAL, "key buffer needs %d bytes", (int)k.size() + 1);
    memcpy(key, k.c_str(), k.size() + 1);
    return LBMP_OK;
  } catch (...) {
    return bfail(LBMP_EINVAL, "lbmp_batch_class: unexpected exception");
  }
}

lbmp_status lbmp_batch_create(const lbmp_params *pin, int32_t count, const int32_t *nx,
                              const int32_t *ny, lbmp_batch **out) {
  const lbmp::NvtxRange nvtx_range("lbmp_batch_create");
  try {
    if (!pin || !nx || !ny || !out) return bfail(LBMP_EINVAL, "lbmp_batch_create: NULL argument");
    *out = nullptr;
    if (count < 1) return bfail(LBMP_EINVAL, "count must be >= 1");
    lbmp_params p = *pin;
    if (p.kn_beta != 0.0)
      return bfail(LBMP_EINVAL, "lbmp_batch_*: a dynamic Kn (kn_beta != 0) is not available");
    if (p.J == 0.0) p.J = 1.0;
    if (p.rho0 == 0.0) p.rho0 = 1.0;
    // validate the shared parameters through the single-lattice rules
    for (int i = 0; i < count; ++i) {
      lbmp_params q = p;
      q.nx = nx[i];
      q.ny = ny[i];
      q.stream = nullptr;
      q.kernel = LBMP_KERNEL_DIRECT;
      lbmp_status st = lbmp::validate_params(&q);
      if (st) return st;
    }
    lbmp_batch *b = new (std::nothrow) lbmp_batch();
    if (!b) return bfail(LBMP_ENOMEM, "host allocation of the batch");
    b->p = p;
    b->count = count;
    b->sr = p.storage == LBMP_STORE_FP16 && p.fp16_rounding == LBMP_ROUND_STOCHASTIC;
    cudaError_t e = cudaGetDevice(&b->device);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&b->nsm, cudaDevAttrMultiProcessorCount, b->device);
    if (e != cudaSuccess) {
      delete b;
      return bcuda(e, "device query");
    }
    lbmp_status st = LBMP_OK;
#define BTRY(x)           \
  do {                    \
    st = (x);             \
    if (st != LBMP_OK) {  \
      brelease(b);        \
      return st;          \
    }                     \
  } while (0)
    if (p.stream) {
      b->stream = (cudaStream_t)p.stream;
    } else {
      e = cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking);
      if (e != cudaSuccess) BTRY(bcuda(e, "cudaStreamCreate"));
      b->own_stream = true;
    }
    e = cudaStreamCreateWithFlags(&b->cap_stream, cudaStreamNonBlocking);
    if (e != cudaSuccess) BTRY(bcuda(e, "cudaStreamCreate (capture)"));
    const size_t elem = p.storage == LBMP_STORE_FP32 ? 4 : 2;
    int drop_tile = -1;
    if (const char *f = std::getenv("LBMP_TEST_DROP_TILE")) drop_tile = std::atoi(f);
    b->h_inst.resize(count);
    b->fields_set.assign(count, 0);
    b->eps_mean.assign(count, 1.0);
    b->fluid_nodes.assign(count, 0);
    for (int i = 0; i < count; ++i) {
      BatchInst &I = b->h_inst[i];
      std::memset(&I, 0, sizeof(I));
      lbmp::StepArgs &a = I.a;
      const int walls = p.bc_y == LBMP_BCY_WALLS;
      a.nx = nx[i];
      a.ny = ny[i];
      a.pitch = lbmp::batch_pitch(nx[i]);
      a.y0 = walls ? 1 : 0;
      a.plane = (long long)a.pitch * ny[i];
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
      a.scale = 1.0f;
      a.inv_scale = 1.0f;
      a.walls = walls;
      a.pressure = p.bc_x == LBMP_BCX_PRESSURE;
      a.forch = p.forchheimer != 0;
      a.seed_lo = (uint32_t)(p.seed & 0xffffffffu);
      a.seed_hi = (uint32_t)(p.seed >> 32);
      // instance 0's arguments are the kernel's shared ones: the staged
      // kernel withholds the copies of that tile (tests of its bounded waits)
      a.test_drop_tile = i == 0 ? drop_tile : -1;
      a.kn_model = p.kn_model;
      a.kn_beta = 0.0f;
      a.kn0 = nullptr;
      I.rows = walls ? ny[i] - 2 : ny[i];
      I.index = i;
      b->fluid_nodes[i] = (long long)nx[i] * I.rows;
      b->total_nodes += b->fluid_nodes[i];
      const size_t pop_bytes = (size_t)a.plane * 9 * elem;
      BTRY(balloc(b, &I.buf[0], pop_bytes, "batch populations A"));
      BTRY(balloc(b, &I.buf[1], pop_bytes, "batch populations B"));
      void *m = nullptr;
      BTRY(balloc(b, &m, (size_t)a.plane * sizeof(float2), "batch medium"));
      I.med = (const float2 *)m;
    }
    const std::vector<long long> cum_macro = work_list(b, lbmp::kBatchMacroBX);
    b->items_macro = cum_macro.back();
    BTRY(balloc(b, (void **)&b->d_inst, sizeof(BatchInst) * count, "batch descriptors"));
    BTRY(balloc(b, (void **)&b->d_cum_step, sizeof(long long) * (count + 1), "work list"));
    BTRY(balloc(b, (void **)&b->d_cum_macro, sizeof(long long) * (count + 1), "work list"));
    {
      int min_chunk = 1 << 30;
      for (const auto &sh : lbmp::kShapes)
        if (sh.persistent != 2) min_chunk = std::min(min_chunk, sh.bx * sh.npt);
      b->items_cap = work_list(b, min_chunk).back();
      BTRY(balloc(b, (void **)&b->d_item_inst, sizeof(int) * (size_t)b->items_cap, "work-item table"));
    }
    BTRY(balloc(b, (void **)&b->d_partials, sizeof(double) * lbmp::kNQ * (size_t)b->items_macro,
                "batch partials"));
    BTRY(balloc(b, (void **)&b->d_results, sizeof(double) * lbmp::kNQ * count, "batch results"));
    int max_mb = 0;
    for (int i = 0; i < count; ++i) max_mb = std::max(max_mb, lbmp::medium_blocks(nx[i], ny[i]));
    BTRY(balloc(b, (void **)&b->d_med_partials, sizeof(double) * lbmp::kNQ * max_mb, "medium partials"));
    BTRY(balloc(b, (void **)&b->d_med_results, sizeof(double) * lbmp::kNQ, "medium results"));
    BTRY(balloc(b, (void **)&b->d_flag, sizeof(unsigned), "validation flag"));
    BTRY(balloc(b, (void **)&b->d_err, sizeof(unsigned), "wait error flag"));
    e = cudaMemset(b->d_err, 0, sizeof(unsigned));
    if (e != cudaSuccess) BTRY(bcuda(e, "cudaMemset"));
    {
      // tile list of the staged kernel: W consecutive nodes of each
      // instance's padded lattice over its fluid rows
      const int W = lbmp::staged_tile_width(p.storage);
      std::vector<int4> tiles;
      for (int i = 0; i < count; ++i) {
        const lbmp::StepArgs &a = b->h_inst[i].a;
        const long long F0 = (long long)a.y0 * a.pitch;
        const long long Fend = (long long)(a.y0 + b->h_inst[i].rows) * a.pitch;
        for (long long T0 = F0; T0 < Fend; T0 += W)
          tiles.push_back(make_int4(i, (int)(T0 % a.pitch), (int)(T0 / a.pitch),
                                    a.y0 + b->h_inst[i].rows));
      }
      if (tiles.size() > 0x7fffffffu) BTRY(bfail(LBMP_EINVAL, "batch too large for the tile list"));
      b->ntiles = (int)tiles.size();
      BTRY(balloc(b, (void **)&b->d_tiles, tiles.size() * sizeof(int4), "tile list"));
      e = cudaMemcpy(b->d_tiles, tiles.data(), tiles.size() * sizeof(int4), cudaMemcpyHostToDevice);
      if (e != cudaSuccess) BTRY(bcuda(e, "tile list upload"));
    }
    BTRY(balloc(b, (void **)&b->d_tctr, sizeof(unsigned long long), "time-level counter"));
    e = cudaMemset(b->d_tctr, 0, sizeof(unsigned long long));
    if (e != cudaSuccess) BTRY(bcuda(e, "cudaMemset"));
    BTRY(upload_cum(b, b->d_cum_macro, cum_macro));
    BTRY(set_shape(b, b->shape));
#undef BTRY
    *out = b;
    return LBMP_OK;
  } catch (...) {
    return bfail(LBMP_ECUDA, "lbmp_batch_create: unexpected exception");
  }
}

lbmp_status lbmp_batch_destroy(lbmp_batch *b) {
  brelease(b);
  return LBMP_OK;
}

lbmp_status lbmp_batch_set_fields(lbmp_batch *b, int32_t i, const double *eps, const double *k_i,
                                  const double *kn, int32_t where) {
  const lbmp::NvtxRange nvtx_range("lbmp_batch_set_fields");
  try {
    if (!b || !eps || !k_i || !kn) return bfail(LBMP_EINVAL, "lbmp_batch_set_fields: NULL argument");
    if (i < 0 || i >= b->count) return bfail(LBMP_EINVAL, "instance %d out of range", i);
    if (where != LBMP_HOST && where != LBMP_DEVICE) return bfail(LBMP_EINVAL, "bad where");
    const DeviceScope device_scope(b->device);
    BCK(device_scope.err);
    BatchInst &I = b->h_inst[i];
    lbmp::StepArgs &a = I.a;
    const size_t n = (size_t)a.nx * a.ny;
    const double *de = eps, *dk = k_i, *dn = kn;
    void *tmp = nullptr;
    if (where == LBMP_HOST) {
      BCK(cudaMalloc(&tmp, 3 * n * sizeof(double)));
      double *t = (double *)tmp;
      cudaMemcpyAsync(t, eps, n * sizeof(double), cudaMemcpyHostToDevice, b->stream);
      cudaMemcpyAsync(t + n, k_i, n * sizeof(double), cudaMemcpyHostToDevice, b->stream);
      cudaMemcpyAsync(t + 2 * n, kn, n * sizeof(double), cudaMemcpyHostToDevice, b->stream);
      de = t;
      dk = t + n;
      dn = t + 2 * n;
    }
    const int y_hi = a.walls ? a.ny - 1 : a.ny;
    unsigned flag = 0;
    double res[lbmp::kNQ];
    cudaError_t e = cudaMemsetAsync(b->d_flag, 0, sizeof(unsigned), b->stream);
    if (e == cudaSuccess)
      e = cudaMemsetAsync((void *)I.med, 0, (size_t)a.plane * sizeof(float2), b->stream);
    if (e == cudaSuccess)
      e = lbmp::launch_medium(de, dk, dn, a.nx, a.ny, a.pitch, a.y0, y_hi, b->p.kn_model,
                              nullptr, 1.0, (float2 *)I.med, b->d_flag, b->d_med_partials,
                              b->stream);
    if (e == cudaSuccess)
      e = lbmp::launch_finalize(b->d_med_partials, lbmp::medium_blocks(a.nx, a.ny), lbmp::kNQ,
                                b->d_med_results, b->stream, lbmp::kMediumMaxMask);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(res, b->d_med_results, sizeof(res), cudaMemcpyDeviceToHost, b->stream);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(&flag, b->d_flag, sizeof(flag), cudaMemcpyDeviceToHost, b->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
    if (tmp) cudaFree(tmp);
    if (e != cudaSuccess) return bcuda(e, "batch medium precompute");
    if (flag) {
      b->fields_set[i] = 0;
      return bfail(LBMP_EINVAL, "lbmp_batch_set_fields: invalid values in instance %d (flags %u)", i, flag);
    }
    b->eps_mean[i] = res[0] / res[1];
    double scale = 1.0;
    const lbmp_params &p = b->p;
    if (p.storage == LBMP_STORE_FP16) {
      int s = p.fp16_log2_scale;
      if (s == 0) {  // the rule of lbmp_set_fields
        double dev = 0.0;
        if (p.bc_x == LBMP_BCX_PRESSURE)
          dev = std::max(std::fabs(p.rho_in - p.rho0), std::fabs(p.rho_out - p.rho0));
        const double nu = (p.tau - 0.5) / 3.0 / p.J;
        const double g = std::sqrt(p.Gx * p.Gx + p.Gy * p.Gy);
        const double L = a.walls ? (double)(a.ny - 2) : (double)std::min(a.nx, a.ny);
        double u = g * res[2] / nu;
        if (res[3] > 0.0) u = std::max(u, g * L * L / (8.0 * nu));
        u = std::min(u, 0.1);
        dev = std::max(std::max(dev, 3.0 * p.rho0 * u), 1e-7);
        s = std::min(60, std::max(-60, (int)std::floor(std::log2(1024.0 / dev))));
      }
      scale = std::ldexp(1.0, s);
    }
    a.scale = (float)scale;
    a.inv_scale = (float)(1.0 / scale);
    const size_t elem = p.storage == LBMP_STORE_FP32 ? 4 : 2;
    BCK(cudaMemsetAsync(I.buf[0], 0, (size_t)a.plane * 9 * elem, b->stream));
    BCK(cudaMemsetAsync(I.buf[1], 0, (size_t)a.plane * 9 * elem, b->stream));
    BCK(cudaMemcpyAsync(b->d_inst + i, &I, sizeof(BatchInst), cudaMemcpyHostToDevice, b->stream));
    BCK(cudaStreamSynchronize(b->stream));
    b->fields_set[i] = 1;
    bfree_graphs(b);
    return LBMP_OK;
  } catch (...) {
    return bfail(LBMP_ECUDA, "lbmp_batch_set_fields: unexpected exception");
  }
}

lbmp_status lbmp_batch_step(lbmp_batch *b, int64_t n) {
  const lbmp::NvtxRange nvtx_range("lbmp_batch_step");
  try {
    if (!b) return bfail(LBMP_EINVAL, "lbmp_batch_step: NULL batch");
    if (n < 0) return bfail(LBMP_EINVAL, "n must be >= 0");
    if (!all_fields(b)) return bfail(LBMP_ESTATE, "lbmp_batch_step: every instance needs its fields");
    if (n == 0) return LBMP_OK;
    const DeviceScope device_scope(b->device);
    BCK(device_scope.err);
    return do_step(b, n);
  } catch (...) {
    return bfail(LBMP_ECUDA, "lbmp_batch_step: unexpected exception");
  }
}

lbmp_status lbmp_batch_synchronize(lbmp_batch *b) {
  const lbmp::NvtxRange nvtx_range("lbmp_batch_synchronize");
  if (!b) return bfail(LBMP_EINVAL, "NULL batch");
  const DeviceScope device_scope(b->device);
  BCK(device_scope.err);
  BCK(cudaStreamSynchronize(b->stream));
  unsigned err = 0;
  BCK(cudaMemcpy(&err, b->d_err, sizeof(err), cudaMemcpyDeviceToHost));
  if (err) return bfail(LBMP_ETIMEOUT, "a bounded wait of the staged batched kernel gave up");
  return LBMP_OK;
}

lbmp_status lbmp_batch_tune_cached(lbmp_batch *b, int32_t steps, int32_t *chosen,
                                   double *ms_per_step, int32_t *from_cache) {
  const lbmp::NvtxRange nvtx_range("lbmp_batch_tune_cached");
  try {
    if (!b) return bfail(LBMP_EINVAL, "NULL batch");
    if (steps < 1) return bfail(LBMP_EINVAL, "steps must be >= 1");
    std::vector<int32_t> nx(b->count), ny(b->count);
    for (int i = 0; i < b->count; ++i) {
      nx[i] = b->h_inst[i].a.nx;
      ny[i] = b->h_inst[i].a.ny;
    }
    const std::string key = class_key(b->p, b->count, nx.data(), ny.data(), b->nsm);
    TuneEntry e{};
    bool hit;
    {
      std::lock_guard<std::mutex> lk(g_tune_mu);
      auto it = g_tune_cache.find(key);
      hit = it != g_tune_cache.end();
      if (hit) e = it->second;
      if (!hit && tune_file_lookup(key, &e)) {
        g_tune_cache[key] = e;
        hit = true;
      }
    }
    if (hit) {
      const lbmp_status st = set_shape(b, e.shape);
      if (st) return st;
    } else {
      int32_t c = 0;
      double ms = 0.0;
      const lbmp_status st = lbmp_batch_tune(b, steps, &c, &ms);
      if (st) return st;
      e = {c, ms};
      std::lock_guard<std::mutex> lk(g_tune_mu);
      g_tune_cache[key] = e;
      tune_file_append(key, e);
    }
    if (chosen) *chosen = e.shape;
    if (ms_per_step) *ms_per_step = e.ms;
    if (from_cache) *from_cache = hit ? 1 : 0;
    return LBMP_OK;
  } catch (...) {
    return bfail(LBMP_ECUDA, "lbmp_batch_tune_cached: unexpected exception");
  }
}

lbmp_status lbmp_batch_tune_cache_clear(void) {
  std::lock_guard<std::mutex> lk(g_tune_mu);
  g_tune_cache.clear();
  return LBMP_OK;
}

lbmp_status lbmp_batch_set_shape(lbmp_batch *b, int32_t shape) {
  try {
    if (!b) return bfail(LBMP_EINVAL, "NULL batch");
    if (shape < 0 || shape >= lbmp::kNumShapes)
      return bfail(LBMP_EINVAL, "shape must be in [0, %d)", lbmp::kNumShapes);
    const DeviceScope device_scope(b->device);
    BCK(device_scope.err);
    return set_shape(b, shape);
  } catch (...) {
    return bfail(LBMP_ECUDA, "lbmp_batch_set_shape: unexpected exception");
  }
}

lbmp_status lbmp_batch_permeability(lbmp_batch *b, double *k_g, double *u_mean) {
  const lbmp::NvtxRange nvtx_range("lbmp_batch_permeability");
  try {
    if (!b) return bfail(LBMP_EINVAL, "NULL batch");
    if (!all_fields(b)) return bfail(LBMP_ESTATE, "every instance needs its fields");
    const DeviceScope device_scope(b->device);
    BCK(device_scope.err);
    cudaError_t e;
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(
        &per_sm, lbmp::batch_macro_kernel<lbmp::StoreF32>, lbmp::kBatchMacroBX, 0);
    if (e != cudaSuccess) return bcuda(e, "occupancy");
    const long long grid = std::min<long long>((long long)std::max(per_sm, 1) * b->nsm, b->items_macro);
    if (b->p.storage == LBMP_STORE_FP32)
      lbmp::batch_macro_kernel<lbmp::StoreF32><<<(unsigned)grid, lbmp::kBatchMacroBX, 0, b->stream>>>(
          b->d_inst, b->d_cum_macro, b->count, b->parity, b->d_partials);
    else
      lbmp::batch_macro_kernel<lbmp::StoreF16><<<(unsigned)grid, lbmp::kBatchMacroBX, 0, b->stream>>>(
          b->d_inst, b->d_cum_macro, b->count, b->parity, b->d_partials);
    BCK(cudaGetLastError());
    lbmp::batch_finalize_kernel<<<b->count, 256, 0, b->stream>>>(b->d_cum_macro, b->d_partials,
                                                                  b->d_results);
    BCK(cudaGetLastError());
    b->launches += 2;
    std::vector<double> res((size_t)b->count * lbmp::kNQ);
    BCK(cudaMemcpyAsync(res.data(), b->d_results, res.size() * sizeof(double),
                        cudaMemcpyDeviceToHost, b->stream));
    BCK(cudaStreamSynchronize(b->stream));
    const lbmp_params &p = b->p;
    const double nu = (p.tau - 0.5) / 3.0 / p.J;
    lbmp_status st = LBMP_OK;
    for (int i = 0; i < b->count; ++i) {
      const double *r = res.data() + (size_t)i * lbmp::kNQ;
      if (r[5] != 0.0) st = bfail(LBMP_ENAN, "instance %d has non-finite velocities", i);
      const double um = r[0] / (double)b->fluid_nodes[i];
      double g = p.Gx;
      if (p.bc_x == LBMP_BCX_PRESSURE)
        g += (p.rho_in - p.rho_out) / 3.0 / b->eps_mean[i] /
             (p.rho0 * (double)(b->h_inst[i].a.nx - 1));
      if (u_mean) u_mean[i] = um;
      if (k_g) k_g[i] = nu * um / g;
    }
    return st;
  } catch (...) {
    return bfail(LBMP_ECUDA, "lbmp_batch_permeability: unexpected exception");
  }
}

lbmp_status lbmp_batch_populations(lbmp_batch *b, int32_t i, double *f, int32_t where) {
  const lbmp::NvtxRange nvtx_range("lbmp_batch_populations");
  try {
    if (!b || !f) return bfail(LBMP_EINVAL, "NULL argument");
    if (i < 0 || i >= b->count) return bfail(LBMP_EINVAL, "instance %d out of range", i);
    if (!b->fields_set[i]) return bfail(LBMP_ESTATE, "instance %d has no fields", i);
    const DeviceScope device_scope(b->device);
    BCK(device_scope.err);
    const BatchInst &I = b->h_inst[i];
    lbmp::StepArgs a = I.a;
    a.y0 = 0;
    const size_t n = (size_t)a.nx * a.ny * 9;
    double *dst = f;
    void *tmp = nullptr;
    if (where == LBMP_HOST) {
      BCK(cudaMalloc(&tmp, n * sizeof(double)));
      dst = (double *)tmp;
    }
    lbmp::MacroOut o{};
    o.pops = dst;
    cudaError_t e = lbmp::launch_macro(b->p.storage, a, I.buf[b->parity], I.med, o, b->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
    if (e == cudaSuccess && tmp) e = cudaMemcpy(f, tmp, n * sizeof(double), cudaMemcpyDeviceToHost);
    if (tmp) cudaFree(tmp);
    if (e != cudaSuccess) return bcuda(e, "batch populations");
    return LBMP_OK;
  } catch (...) {
    return bfail(LBMP_ECUDA, "lbmp_batch_populations: unexpected exception");
  }
}

lbmp_status lbmp_batch_tune(lbmp_batch *b, int32_t steps, int32_t *chosen, double *ms_per_step) {
  const lbmp::NvtxRange nvtx_range("lbmp_batch_tune");
  try {
    if (!b) return bfail(LBMP_EINVAL, "NULL batch");
    if (steps < 1) return bfail(LBMP_EINVAL, "steps must be >= 1");
    if (!all_fields(b)) return bfail(LBMP_ESTATE, "every instance needs its fields");
    const DeviceScope device_scope(b->device);
    BCK(device_scope.err);
    const size_t elem = b->p.storage == LBMP_STORE_FP32 ? 4 : 2;
    // save the current populations and the counter of every instance
    std::vector<void *> saved(b->count, nullptr);
    size_t total = 0;
    for (int i = 0; i < b->count; ++i) total += (size_t)b->h_inst[i].a.plane * 9 * elem;
    void *store = nullptr;
    BCK(cudaMalloc(&store, total));
    size_t off = 0;
    for (int i = 0; i < b->count; ++i) {
      const size_t bytes = (size_t)b->h_inst[i].a.plane * 9 * elem;
      saved[i] = (char *)store + off;
      cudaMemcpyAsync(saved[i], b->h_inst[i].buf[b->parity], bytes, cudaMemcpyDeviceToDevice, b->stream);
      off += bytes;
    }
    unsigned long long tctr0 = 0;
    cudaMemcpyAsync(&tctr0, b->d_tctr, sizeof(tctr0), cudaMemcpyDeviceToHost, b->stream);
    const int parity0 = b->parity;
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    int best = b->shape;
    float best_ms = 1e30f;
    lbmp_status st = LBMP_OK;
    for (int sidx = 0; sidx < lbmp::kNumShapes && st == LBMP_OK; ++sidx) {
      st = set_shape(b, sidx);
      if (st) break;
      st = launch_steps(b, 2, b->stream, false);  // warm-up
      if (st) break;
      cudaEventRecord(e0, b->stream);
      st = launch_steps(b, steps, b->stream, false);
      cudaEventRecord(e1, b->stream);
      if (cudaEventSynchronize(e1) != cudaSuccess) {
        st = bcuda(cudaGetLastError(), "tuning run");
        break;
      }
      float ms = 0.0f;
      cudaEventElapsedTime(&ms, e0, e1);
      if (ms < best_ms) {
        best_ms = ms;
        best = sidx;
      }
    }
    // restore the state
    b->parity = parity0;
    off = 0;
    for (int i = 0; i < b->count; ++i) {
      const size_t bytes = (size_t)b->h_inst[i].a.plane * 9 * elem;
      cudaMemcpyAsync(b->h_inst[i].buf[b->parity], saved[i], bytes, cudaMemcpyDeviceToDevice, b->stream);
      off += bytes;
    }
    cudaMemcpyAsync(b->d_tctr, &tctr0, sizeof(tctr0), cudaMemcpyHostToDevice, b->stream);
    cudaStreamSynchronize(b->stream);
    cudaFree(store);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (st) return st;
    st = set_shape(b, best);
    if (st) return st;
    if (chosen) *chosen = best;
    if (ms_per_step) *ms_per_step = best_ms / steps;
    return LBMP_OK;
  } catch (...) {
    return bfail(LBMP_ECUDA, "lbmp_batch_tune: unexpected exception");
  }
}

lbmp_status lbmp_batch_get_info(lbmp_batch *b, lbmp_batch_info *out) {
  if (!b || !out) return bfail(LBMP_EINVAL, "NULL argument");
  out->count = b->count;
  const lbmp::Shape sh = lbmp::kShapes[b->shape];
  if (sh.persistent == 2) {  // staged: consumer threads and nodes per thread per tile
    const int W = lbmp::staged_tile_width(b->p.storage);
    const int warps = lbmp::staged_warps(b->p.storage);
    out->shape_threads = warps * 32;
    out->shape_nodes_per_thread = W / (warps * 32);
  } else {
    out->shape_threads = sh.bx;
    out->shape_nodes_per_thread = sh.npt;
  }
  out->persistent = sh.persistent;
  out->total_nodes = b->total_nodes;
  out->steps = b->steps;
  out->launches = b->launches;
  out->device_bytes = b->device_bytes;
  out->bytes_per_update = 2.0 * 9.0 * (b->p.storage == LBMP_STORE_FP32 ? 4.0 : 2.0) + 8.0;
  return LBMP_OK;
}

}  // extern "C"
