// CUDA kernels of the porous lattice Boltzmann step for sm_103a
// (Chen et al., arXiv:1411.7051, Section III).
//
// The step is a stencil stream: every population is read once and written
// once per time step, so the roofline is HBM bandwidth (no dense
// contraction, no tensor cores).  One fused kernel pulls the nine
// populations of a node (periodic wrap, halfway bounce-back at plates,
// pressure-column extrapolation), solves Eq. 16-17 for the velocity, forms
// Eq. 2, Eq. 14 and Eq. 15 and writes the nine post-collision values.
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>

#include "kernels.h"
#include "lattice.cuh"
#include "staged.cuh"
#include "wide.cuh"

namespace lbmp {

constexpr int kStepBX = 128;   // threads per block along x
constexpr int kStepNPT = 2;    // nodes per thread, strided by kStepBX
constexpr int kMacroBX = 256;
constexpr int kMediumBX = 256;

// ------------------------------------------------------------- step kernel
// Each thread updates kStepNPT nodes of one row, kStepBX apart, so every
// load and store instruction of a warp touches 32 consecutive elements.
// All loads of a thread are issued before its first collision.  Plate rows
// are block-uniform branches inside pull_node.  The stochastic-rounding
// bits of time level t come from *tctr + k (the counter is advanced by
// bump_kernel after a group of launches).
// DYN: Knudsen number per node and step from the local pressure (the
// medium holds 1/k_i, a.kn0 the Kn at p0).
// MOM: also store each node's post-stream moments (rho - rho0, m_x, m_y;
// three [ny][pitch] planes at mom, a.plane apart) -- all that the reverse
// step of the adjoint needs of the forward state.
template <class S, bool SR, bool DYN, bool MOM = false>
__global__ void __launch_bounds__(kStepBX)
    step_kernel(const StepArgs a, const typename S::T *__restrict__ fin,
                typename S::T *__restrict__ fout, const float2 *__restrict__ med,
                const unsigned long long *__restrict__ tctr, int k,
                float *__restrict__ mom) {
  const int y = a.y0 + (a.rev ? (int)gridDim.y - 1 - (int)blockIdx.y : (int)blockIdx.y);
  const int xb = blockIdx.x * (kStepBX * kStepNPT) + threadIdx.x;
  const long long row = (long long)y * a.pitch;
  float d[kStepNPT][9];
  float2 m[kStepNPT];
  float k0[kStepNPT];
#pragma unroll
  for (int j = 0; j < kStepNPT; ++j) {
    const int x = xb + j * kStepBX;
    k0[j] = 0.0f;
    if (x < a.nx) {
      pull_node<S>(fin, a, x, y, d[j]);
      m[j] = med[row + x];
      if (DYN) k0[j] = a.kn0[row + x];
    }
  }
  uint32_t ts = 0;
  if (SR) {
    const unsigned long long t = *tctr + (unsigned long long)k;
    ts = mix32((uint32_t)t * 0x9e3779b9u ^ a.seed_lo ^ mix32((uint32_t)(t >> 32) ^ a.seed_hi));
  }
#pragma unroll
  for (int j = 0; j < kStepNPT; ++j) {
    const int x = xb + j * kStepBX;
    if (x >= a.nx) continue;
    if (a.pressure && (x == 0 || x == a.nx - 1))
      pressure_node<S, DYN>(fin, med, a, x, y, m[j].x, d[j]);
    const NodeState s = node_state<DYN>(d[j], m[j].x, m[j].y, a, k0[j]);
    if (MOM) {
      float *mo = mom + row + x;
      mo[0] = s.drho_s;
      mo[a.plane] = s.mx;
      mo[2 * a.plane] = s.my;
    }
    collide<S::kHiLo>(d[j], s, a);
    typename S::T *o = fout + row + x;
    const uint32_t h = SR ? mix32((uint32_t)(row + x) ^ ts) : 0u;
#pragma unroll
    for (int i = 0; i < 9; ++i) S::template st1r<SR>(o + i * a.plane, d[j][i], h, i);
  }
}

// Advance the time-level counter of the stochastic rounding by n.
__global__ void bump_kernel(unsigned long long *tctr, int n) { *tctr += (unsigned long long)n; }

cudaError_t launch_step(int storage, bool sr, const StepArgs &a, int rows, const void *fin,
                        void *fout, const float2 *med, const unsigned long long *tctr, int k,
                        cudaStream_t s) {
  if (rows <= 0 || a.nx <= 0) return cudaSuccess;
  dim3 block(kStepBX);
  dim3 grid((a.nx + kStepBX * kStepNPT - 1) / (kStepBX * kStepNPT), rows);
  const bool dyn = a.kn0 != nullptr;
  const float *f32i = (const float *)fin;
  float *f32o = (float *)fout;
  const __half *f16i = (const __half *)fin;
  __half *f16o = (__half *)fout;
  if (storage == 0) {
    if (dyn)
      step_kernel<StoreF32, false, true><<<grid, block, 0, s>>>(a, f32i, f32o, med, tctr, k, nullptr);
    else
      step_kernel<StoreF32, false, false><<<grid, block, 0, s>>>(a, f32i, f32o, med, tctr, k, nullptr);
  } else if (sr) {
    if (dyn)
      step_kernel<StoreF16, true, true><<<grid, block, 0, s>>>(a, f16i, f16o, med, tctr, k, nullptr);
    else
      step_kernel<StoreF16, true, false><<<grid, block, 0, s>>>(a, f16i, f16o, med, tctr, k, nullptr);
  } else {
    if (dyn)
      step_kernel<StoreF16, false, true><<<grid, block, 0, s>>>(a, f16i, f16o, med, tctr, k, nullptr);
    else
      step_kernel<StoreF16, false, false><<<grid, block, 0, s>>>(a, f16i, f16o, med, tctr, k, nullptr);
  }
  return cudaGetLastError();
}

cudaError_t launch_step_moments(const StepArgs &a, int rows, const float *fin, float *fout,
                                const float2 *med, float *mom, cudaStream_t s) {
  if (rows <= 0 || a.nx <= 0) return cudaSuccess;
  dim3 block(kStepBX);
  dim3 grid((a.nx + kStepBX * kStepNPT - 1) / (kStepBX * kStepNPT), rows);
  step_kernel<StoreF32, false, false, true><<<grid, block, 0, s>>>(a, fin, fout, med, nullptr, 0,
                                                                   mom);
  return cudaGetLastError();
}

// -------------------------------------------------------- wide variant
cudaError_t launch_wide(bool sr, const StepArgs &a, int rows, const void *fin, void *fout,
                        const float2 *med, const unsigned long long *tctr, int k,
                        cudaStream_t s) {
  if (rows <= 0 || a.nx <= 0) return cudaSuccess;
  dim3 block(kWideBX);
  dim3 grid((a.nx + kWideBX * kWideV - 1) / (kWideBX * kWideV), rows);
  const __half *i = (const __half *)fin;
  __half *o = (__half *)fout;
  const bool dyn = a.kn0 != nullptr;
  if (sr) {
    if (dyn) wide_step_kernel<true, true><<<grid, block, 0, s>>>(a, i, o, med, tctr, k);
    else wide_step_kernel<true, false><<<grid, block, 0, s>>>(a, i, o, med, tctr, k);
  } else {
    if (dyn) wide_step_kernel<false, true><<<grid, block, 0, s>>>(a, i, o, med, tctr, k);
    else wide_step_kernel<false, false><<<grid, block, 0, s>>>(a, i, o, med, tctr, k);
  }
  return cudaGetLastError();
}

// ------------------------------------------------------ staged variant
template <class S, bool SR, bool DYN>
static cudaError_t launch_staged_t(const StepArgs &a, int rows, const void *fin, void *fout,
                                   const float2 *med, const unsigned long long *tctr, int k,
                                   unsigned *err, int nsm, cudaStream_t s) {
  using C = StageCfgFor<S, DYN>;
  using L = StageLayout<S, C>;
  const long long span = (long long)rows * a.pitch;  // flat nodes of the launch rows
  const int ntiles = (int)((span + C::W - 1) / C::W);
  const int grid = ntiles < nsm ? ntiles : nsm;
  staged_step_kernel<S, SR, DYN><<<grid, kStagedThreads, L::kSmemBytes, s>>>(
      a, (const typename S::T *)fin, (typename S::T *)fout, med, tctr, k, rows, err);
  return cudaGetLastError();
}

template <class S, bool SR, bool DYN>
static cudaError_t staged_smem_attr() {
  return cudaFuncSetAttribute(staged_step_kernel<S, SR, DYN>,
                              cudaFuncAttributeMaxDynamicSharedMemorySize,
                              StageLayout<S, StageCfgFor<S, DYN>>::kSmemBytes);
}

cudaError_t prepare_staged() {
  cudaError_t e;
  if ((e = staged_smem_attr<StoreF32, false, false>()) != cudaSuccess) return e;
  if ((e = staged_smem_attr<StoreF16, false, false>()) != cudaSuccess) return e;
  if ((e = staged_smem_attr<StoreF16, true, false>()) != cudaSuccess) return e;
  if ((e = staged_smem_attr<StoreF16, false, true>()) != cudaSuccess) return e;
  return staged_smem_attr<StoreF16, true, true>();
}

// A dynamic Kn (a.kn0 set) takes the FP16 kernel that also stages the Kn
// plane; with FP32 storage the direct kernel serves it (the context never
// selects the staged one).
cudaError_t launch_staged(int storage, bool sr, const StepArgs &a, int rows, const void *fin,
                          void *fout, const float2 *med, const unsigned long long *tctr, int k,
                          unsigned *err, int nsm, cudaStream_t s) {
  if (rows <= 0 || a.nx <= 0) return cudaSuccess;
  const bool dyn = a.kn0 != nullptr;
  if (storage == 0) {
    if (dyn) return cudaErrorInvalidValue;
    return launch_staged_t<StoreF32, false, false>(a, rows, fin, fout, med, tctr, k, err, nsm, s);
  }
  if (dyn) {
    if (sr) return launch_staged_t<StoreF16, true, true>(a, rows, fin, fout, med, tctr, k, err, nsm, s);
    return launch_staged_t<StoreF16, false, true>(a, rows, fin, fout, med, tctr, k, err, nsm, s);
  }
  if (sr) return launch_staged_t<StoreF16, true, false>(a, rows, fin, fout, med, tctr, k, err, nsm, s);
  return launch_staged_t<StoreF16, false, false>(a, rows, fin, fout, med, tctr, k, err, nsm, s);
}

cudaError_t launch_bump(unsigned long long *tctr, int n, cudaStream_t s) {
  bump_kernel<<<1, 1, 0, s>>>(tctr, n);
  return cudaGetLastError();
}

// ------------------------------------------------- block reduction helper
// Sums kNQ doubles over the block in a fixed order and writes them to
// partials[blockLinear * kNQ + q] (deterministic for a fixed launch shape).
// Quantities whose bit is set in max_mask are reduced by max (values >= 0).
template <int BX>
__device__ __forceinline__ void block_reduce_store(double v[kNQ], double *partials,
                                                   unsigned max_mask = 0u) {
  __shared__ double red[BX / 32][kNQ];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int q = 0; q < kNQ; ++q) {
    const bool mx = (max_mask >> q) & 1u;
    double t = v[q];
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
      const double o = __shfl_down_sync(0xffffffffu, t, off);
      t = mx ? fmax(t, o) : t + o;
    }
    if (lane == 0) red[warp][q] = t;
  }
  __syncthreads();
  if (threadIdx.x < kNQ) {
    const bool mx = (max_mask >> threadIdx.x) & 1u;
    double t = 0.0;
    for (int w = 0; w < BX / 32; ++w) t = mx ? fmax(t, red[w][threadIdx.x]) : t + red[w][threadIdx.x];
    const long long b = (long long)blockIdx.y * gridDim.x + blockIdx.x;
    partials[b * kNQ + threadIdx.x] = t;
  }
}

// ------------------------------------------------ FP32-pair arithmetic
// Pairs of FP32 numbers (value = hi + lo) carrying ~44 significant bits:
// exact sums (Knuth's two-sum) and exact products (fma of the product and
// its negation), the standard error-free transformations.  FP64 arithmetic
// runs at ~1/64 of the FP32 rate on this GPU; the precompute and the
// per-thread parts of the reductions use these pairs instead.
struct F2 {
  float hi, lo;
};
__device__ __forceinline__ F2 two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  const float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
  return {s, e};
}
__device__ __forceinline__ F2 fast_two_sum(float a, float b) {  // |a| >= |b|
  const float s = __fadd_rn(a, b);
  return {s, __fsub_rn(b, __fsub_rn(s, a))};
}
__device__ __forceinline__ F2 two_prod(float a, float b) {
  const float p = __fmul_rn(a, b);
  return {p, __fmaf_rn(a, b, -p)};
}
__device__ __forceinline__ F2 f2_add(F2 x, F2 y) {
  F2 s = two_sum(x.hi, y.hi);
  return fast_two_sum(s.hi, __fadd_rn(s.lo, __fadd_rn(x.lo, y.lo)));
}
__device__ __forceinline__ F2 f2_mul(F2 x, F2 y) {
  F2 p = two_prod(x.hi, y.hi);
  const float c = __fmaf_rn(x.hi, y.lo, __fmul_rn(x.lo, y.hi));
  return fast_two_sum(p.hi, __fadd_rn(p.lo, c));
}
// n / d from an approximate reciprocal r of d.hi (relative error e ~ 2^-23):
// q1 = n.hi r is off by ~e, the remainder n - q1 d is formed exactly enough
// (~2^-48 of n), and its quotient by the same r corrects q1 to a relative
// error of order e^2 -- one Newton step on the quotient.
__device__ __forceinline__ F2 f2_div(F2 n, F2 d) {
  const float r = rcp_approx(d.hi);
  const float q1 = __fmul_rn(n.hi, r);
  const F2 qd = f2_mul({q1, 0.0f}, d);           // q1 d
  const F2 rem = f2_add(n, {-qd.hi, -qd.lo});     // n - q1 d
  return fast_two_sum(q1, __fmul_rn(rem.hi, r));
}
// acc += x (x an FP32 value)
__device__ __forceinline__ void f2_acc(F2 &acc, float x) {
  const F2 s = two_sum(acc.hi, x);
  acc = fast_two_sum(s.hi, __fadd_rn(s.lo, acc.lo));
}

// ------------------------------------------- macroscopic / reduction kernel
// Rows blockIdx.y, blockIdx.y + gridDim.y, ...: each thread adds the terms
// of its nodes (some 27 at 4096^2) one by one in FP32 pairs and takes part
// in one FP64 block reduction at the end (FP64 arithmetic is slow on this
// GPU: a reduction tree per node cost six times the per-node work, and FP64
// per-node sums 0.48 ms at 4096^2).  The squares are exact products, the
// velocity differences of the residual exact sums; a thread's pair sums
// are good to ~2^-44 relative.
// Four resident blocks a SM (64 registers a thread; 2 at the compiler's own
// 116): 0.37 -> 0.28 ms a lbmp_permeability call at 4096^2.
template <class S>
__global__ void __launch_bounds__(kMacroBX, 4)
    macro_kernel(const StepArgs a, const typename S::T *__restrict__ fin,
                 const float2 *__restrict__ med, const MacroOut o) {
  const int x = blockIdx.x * kMacroBX + threadIdx.x;
  const long long n = (long long)a.nx * a.ny;
  F2 sux = {0.0f, 0.0f}, suy = {0.0f, 0.0f}, sdr = {0.0f, 0.0f}, su2 = {0.0f, 0.0f},
     sdu = {0.0f, 0.0f};
  unsigned nonfinite = 0;
  for (int y = blockIdx.y; y < a.ny && x < a.nx; y += gridDim.y) {
    const bool wall = a.walls && (y == 0 || y == a.ny - 1);
    const long long j = (long long)y * a.nx + x;
    if (wall) {
      if (o.rho) o.rho[j] = 0.0;
      if (o.ux) o.ux[j] = 0.0;
      if (o.uy) o.uy[j] = 0.0;
      if (o.pops)
        for (int i = 0; i < 9; ++i) o.pops[i * n + j] = 0.0;
      continue;
    }
    float d[9];
    const long long jp = (long long)y * a.pitch + x;
    const float2 m = med[jp];
    pull_node<S>(fin, a, x, y, d);
    const bool col = a.pressure && (x == 0 || x == a.nx - 1);
    NodeState s;
    if (a.kn0) {  // dynamic Kn
      if (col) pressure_node<S, true>(fin, med, a, x, y, m.x, d);
      s = node_state<true>(d, m.x, m.y, a, a.kn0[jp]);
    } else {
      if (col) pressure_node<S, false>(fin, med, a, x, y, m.x, d);
      s = node_state<false>(d, m.x, m.y, a);
    }
    const float drho = s.drho_s * a.inv_scale;
    if (o.rho) o.rho[j] = (double)s.rho;
    if (o.ux) o.ux[j] = (double)s.ux;
    if (o.uy) o.uy[j] = (double)s.uy;
    if (o.pops) {
      const double r0 = (double)a.rho0;
      const double w[9] = {4.0 / 9.0,  1.0 / 9.0,  1.0 / 9.0,  1.0 / 9.0, 1.0 / 9.0,
                           1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0};
      const double is = (double)a.inv_scale;
      for (int i = 0; i < 9; ++i) o.pops[i * n + j] = w[i] * r0 + (double)d[i] * is;
    }
    if (o.partials) {
      const bool finite = isfinite(s.ux) && isfinite(s.uy) && isfinite(s.rho);
      if (finite) {
        f2_acc(sux, s.ux);
        f2_acc(suy, s.uy);
        f2_acc(sdr, drho);
        su2 = f2_add(su2, f2_add(two_prod(s.ux, s.ux), two_prod(s.uy, s.uy)));
      } else {
        ++nonfinite;
      }
      if (o.uprev) {
        const float2 up = o.uprev[jp];
        if (finite) {
          const F2 dx = two_sum(s.ux, -up.x), dy = two_sum(s.uy, -up.y);
          sdu = f2_add(sdu, f2_add(f2_mul(dx, dx), f2_mul(dy, dy)));
        }
        if (o.update_prev) o.uprev[jp] = make_float2(s.ux, s.uy);
      }
    }
  }
  if (o.partials) {
    double v[kNQ] = {(double)sux.hi + (double)sux.lo, (double)suy.hi + (double)suy.lo,
                     (double)sdr.hi + (double)sdr.lo, (double)su2.hi + (double)su2.lo,
                     (double)sdu.hi + (double)sdu.lo, (double)nonfinite};
    block_reduce_store<kMacroBX>(v, o.partials);
  }
}

// Up to 16 blocks of 256 threads on each of 152 SMs.
constexpr int kMacroMaxBlocks = 16 * 152;

static dim3 macro_grid(const StepArgs &a) {
  const int gx = (a.nx + kMacroBX - 1) / kMacroBX;
  const int gy = std::max(1, std::min(a.ny, kMacroMaxBlocks / gx));
  return dim3(gx, gy);
}

int macro_blocks(const StepArgs &a) {
  const dim3 g = macro_grid(a);
  return (int)(g.x * g.y);
}

int hist_blocks(const StepArgs &a) { return ((a.nx + kMacroBX - 1) / kMacroBX) * a.ny; }

cudaError_t launch_macro(int storage, const StepArgs &a, const void *fin,
                         const float2 *med, const MacroOut &o, cudaStream_t s) {
  const dim3 block(kMacroBX), grid = macro_grid(a);
  if (storage == 0)
    macro_kernel<StoreF32><<<grid, block, 0, s>>>(a, (const float *)fin, med, o);
  else
    macro_kernel<StoreF16><<<grid, block, 0, s>>>(a, (const __half *)fin, med, o);
  return cudaGetLastError();
}

// ------------------------------------------------------------- finalize
constexpr int kFinBX = 256;

__global__ void __launch_bounds__(kFinBX)
    finalize_kernel(const double *__restrict__ partials, int nblocks, int nq,
                    double *__restrict__ out, unsigned max_mask) {
  __shared__ double sh[kFinBX];
  for (int q = 0; q < nq; ++q) {
    const bool mx = (max_mask >> q) & 1u;
    double t = 0.0;
    for (int b = threadIdx.x; b < nblocks; b += kFinBX) {
      const double v = partials[(long long)b * nq + q];
      t = mx ? fmax(t, v) : t + v;
    }
    sh[threadIdx.x] = t;
    __syncthreads();
    for (int w = kFinBX / 2; w > 0; w >>= 1) {
      if (threadIdx.x < w)
        sh[threadIdx.x] = mx ? fmax(sh[threadIdx.x], sh[threadIdx.x + w])
                             : sh[threadIdx.x] + sh[threadIdx.x + w];
      __syncthreads();
    }
    if (threadIdx.x == 0) out[q] = sh[0];
    __syncthreads();
  }
}

cudaError_t launch_finalize(const double *partials, int nblocks, int nq, double *out,
                            cudaStream_t s, unsigned max_mask) {
  finalize_kernel<<<1, kFinBX, 0, s>>>(partials, nblocks, nq, out, max_mask);
  return cudaGetLastError();
}

// ------------------------------------------- normalised-velocity histogram
// |u| of node (x, y) in FP64 from the FP32 velocity of node_state (as the
// macroscopic kernel reports it), every operation rounded separately so
// that the bin decisions can be replayed exactly on the host.
template <class S, bool DYN>
__device__ __forceinline__ double node_speed(const typename S::T *__restrict__ fin,
                                             const float2 *__restrict__ med, const StepArgs &a,
                                             int x, int y) {
  float d[9];
  const long long jp = (long long)y * a.pitch + x;
  const float2 m = med[jp];
  pull_node<S>(fin, a, x, y, d);
  if (a.pressure && (x == 0 || x == a.nx - 1)) pressure_node<S, DYN>(fin, med, a, x, y, m.x, d);
  const NodeState s = node_state<DYN>(d, m.x, m.y, a, DYN ? a.kn0[jp] : 0.0f);
  const double ux = s.ux, uy = s.uy;
  return __dsqrt_rn(__dadd_rn(__dmul_rn(ux, ux), __dmul_rn(uy, uy)));
}

// Pass 1: block maxima of |u| over the fluid rows into partials[block].
template <class S, bool DYN>
__global__ void __launch_bounds__(kMacroBX)
    speed_max_kernel(const StepArgs a, const typename S::T *__restrict__ fin,
                     const float2 *__restrict__ med, double *__restrict__ partials) {
  const int y = blockIdx.y;
  const int x = blockIdx.x * kMacroBX + threadIdx.x;
  double v = 0.0;
  if (x < a.nx && !(a.walls && (y == 0 || y == a.ny - 1))) v = node_speed<S, DYN>(fin, med, a, x, y);
  if (!(v >= 0.0)) v = INFINITY;  // a non-finite speed poisons the maximum
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) v = fmax(v, __shfl_down_sync(0xffffffffu, v, off));
  __shared__ double red[kMacroBX / 32];
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < kMacroBX / 32; ++w) t = fmax(t, red[w]);
    partials[(long long)blockIdx.y * gridDim.x + blockIdx.x] = t;
  }
}

// Pass 2: bin k = min(floor(|u| / umax * nbins), nbins - 1) (0 if umax is
// 0), counted per block in shared memory, then added to counts.
template <class S, bool DYN>
__global__ void __launch_bounds__(kMacroBX)
    histogram_kernel(const StepArgs a, const typename S::T *__restrict__ fin,
                     const float2 *__restrict__ med, double umax, int nbins,
                     unsigned long long *__restrict__ counts) {
  __shared__ unsigned sh[kMaxHistBins];
  for (int k = threadIdx.x; k < nbins; k += kMacroBX) sh[k] = 0u;
  __syncthreads();
  const int y = blockIdx.y;
  const int x = blockIdx.x * kMacroBX + threadIdx.x;
  if (x < a.nx && !(a.walls && (y == 0 || y == a.ny - 1))) {
    int k = 0;
    if (umax > 0.0) {
      const double u0 = __ddiv_rn(node_speed<S, DYN>(fin, med, a, x, y), umax);
      const double f = floor(__dmul_rn(u0, (double)nbins));
      k = f >= (double)(nbins - 1) ? nbins - 1 : (int)f;
    }
    atomicAdd(&sh[k], 1u);
  }
  __syncthreads();
  for (int k = threadIdx.x; k < nbins; k += kMacroBX)
    if (sh[k]) atomicAdd(counts + k, (unsigned long long)sh[k]);
}

cudaError_t launch_speed_max(int storage, const StepArgs &a, const void *fin, const float2 *med,
                             double *partials, cudaStream_t s) {
  dim3 block(kMacroBX);
  dim3 grid((a.nx + kMacroBX - 1) / kMacroBX, a.ny);
  const bool dyn = a.kn0 != nullptr;
  if (storage == 0) {
    if (dyn) speed_max_kernel<StoreF32, true><<<grid, block, 0, s>>>(a, (const float *)fin, med, partials);
    else speed_max_kernel<StoreF32, false><<<grid, block, 0, s>>>(a, (const float *)fin, med, partials);
  } else {
    if (dyn) speed_max_kernel<StoreF16, true><<<grid, block, 0, s>>>(a, (const __half *)fin, med, partials);
    else speed_max_kernel<StoreF16, false><<<grid, block, 0, s>>>(a, (const __half *)fin, med, partials);
  }
  return cudaGetLastError();
}

cudaError_t launch_histogram(int storage, const StepArgs &a, const void *fin, const float2 *med,
                             double umax, int nbins, unsigned long long *counts, cudaStream_t s) {
  dim3 block(kMacroBX);
  dim3 grid((a.nx + kMacroBX - 1) / kMacroBX, a.ny);
  const bool dyn = a.kn0 != nullptr;
  if (storage == 0) {
    if (dyn)
      histogram_kernel<StoreF32, true><<<grid, block, 0, s>>>(a, (const float *)fin, med, umax, nbins, counts);
    else
      histogram_kernel<StoreF32, false><<<grid, block, 0, s>>>(a, (const float *)fin, med, umax, nbins, counts);
  } else {
    if (dyn)
      histogram_kernel<StoreF16, true><<<grid, block, 0, s>>>(a, (const __half *)fin, med, umax, nbins, counts);
    else
      histogram_kernel<StoreF16, false><<<grid, block, 0, s>>>(a, (const __half *)fin, med, umax, nbins, counts);
  }
  return cudaGetLastError();
}

// ---------------------------------------------------------------- medium
// The largest k_a of a dynamic-Kn medium (it only sets the FP16 scale) takes
// fc_f32 of the lattice header.

// 1 / k_a = 1 / (k_i f_c(Kn)) of Eq. 3 in FP64 with a single division.
// Eq. 6-7 (b = -1) as one fraction: with t = Kn^-0.4348 and a = 1 + 0.17 t,
//   1 + alpha Kn = (a + 1.358 Kn) / a,   1 + 4 Kn / (1 + Kn) = (1 + 5 Kn) / (1 + Kn),
//   1 / k_a = a (1 + Kn) / (k_i (a + 1.358 Kn) (1 + 5 Kn)).
// Only t comes from FP32 (log2f, exp2f: ~3e-7 relative); it enters through
// a in both numerator and denominator, whose sensitivities nearly cancel:
// d ln(1/k_a) / d ln t = 0.17 t 1.358 Kn / (a (a + 1.358 Kn)) <= 0.08, so
// the FP32 1/k_a stored is within ~0.1 ulp of the FP64 value before its
// final rounding.  FP64 runs at a small fraction of the FP32 rate on this
// GPU: the FP64 power of Kn made the precompute 50 times slower than its
// memory traffic.  Kn = 0 gives f_c = 1 exactly.
__device__ __forceinline__ double inv_ka(double k, double K, int model) {
  if (model == 1) return 1.0 / (k * fma(4.0, K, 1.0));
  if (K == 0.0) return 1.0 / k;
  const double t = (double)exp2f(-0.4348f * log2f((float)K));
  const double a = fma(0.17, t, 1.0);
  return (a * (1.0 + K)) / (k * fma(1.358, K, a) * fma(5.0, K, 1.0));
}

// ---- the same fraction in FP32-pair arithmetic (the F2 helpers above) ----
// FP64 instructions are the bottleneck of the precompute on this GPU, so
// for the usual ranges of k_i and Kn the fraction is evaluated with FP32
// pairs.  Beside the FP32 power of Kn (as in inv_ka) the result differs from
// the FP64 one by ~2^-40 before its final rounding to FP32.
// A double in [2^-60, 2^60] (not 0) as hi + lo with integer operations only: hi
// keeps the leading 24 bits, lo the next 29 (rounded to 24; the pair then
// carries d to a relative 2^-48).
__device__ __forceinline__ F2 f2_from_double(double d) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(d);
  const int e = (int)((b >> 52) & 0x7ff) - 1023;             // unbiased exponent
  const unsigned hib = (unsigned)((b >> 32) & 0x80000000u) |  // sign
                       ((unsigned)(e + 127) << 23) | (unsigned)((b >> 29) & 0x7fffffu);
  const float lo_int = (float)(unsigned)(b & 0x1fffffffull);  // the low 29 mantissa bits
  const float scale = __uint_as_float((unsigned)(e - 52 + 127) << 23);  // 2^(e - 52)
  return {__uint_as_float(hib), (b >> 63) ? -lo_int * scale : lo_int * scale};
}

// 1 / k_a of inv_ka() for k_i and Kn in the ranges FP32 pairs hold
// comfortably (k_i in [1e-16, 1e12], Kn in [1e-12, 1e6] or 0; the others
// take the FP64 fraction): FP32 to within the FP32 power's error.  k > 0
// and K >= 0 (or -0) on entry, so the range tests compare bit patterns: the
// bits of non-negative doubles order as their values (FP64 compares are
// as slow as the rest of FP64 on this GPU).
__device__ __forceinline__ float inv_ka_pair(double k, double K, int model) {
  const unsigned long long kb = (unsigned long long)__double_as_longlong(k);
  const unsigned long long Kb = (unsigned long long)__double_as_longlong(K) << 1;  // sign dropped
  const bool K0 = Kb == 0;
  const bool k_ok = kb >= 0x3c9cd2b297d889bcull && kb <= 0x426d1a94a2000000ull;  // [1e-16, 1e12]
  const bool K_ok = K0 || (Kb >= (0x3d719799812dea11ull << 1) &&
                           Kb <= (0x412e848000000000ull << 1));                  // [1e-12, 1e6]
  if (!k_ok || !K_ok) return (float)inv_ka(k, K, model);
  const F2 kk = f2_from_double(k);
  const F2 one = {1.0f, 0.0f};
  if (K0) {  // f_c = 1 in both models
    const F2 q = f2_div(one, kk);
    return __fadd_rn(q.hi, q.lo);
  }
  if (model == 1) {  // 1 / (k (1 + 4 Kn))
    const F2 KK = f2_from_double(K);
    const F2 den = f2_mul(kk, f2_add(one, f2_mul({4.0f, 0.0f}, KK)));
    const F2 q = f2_div(one, den);
    return __fadd_rn(q.hi, q.lo);
  }
  const F2 KK = f2_from_double(K);
  const float t = kn_power(KK.hi);  // Kn^-0.4348
  const F2 c017 = {0.17f, (float)(0.17 - (double)0.17f)};
  const F2 c1358 = {1.358f, (float)(1.358 - (double)1.358f)};
  const F2 a = f2_add(one, f2_mul(c017, {t, 0.0f}));  // 1 + 0.17 t
  const F2 num = f2_mul(a, f2_add(one, KK));
  const F2 den = f2_mul(f2_mul(kk, f2_add(a, f2_mul(c1358, KK))),
                        f2_add(one, f2_mul({5.0f, 0.0f}, KK)));
  const F2 q = f2_div(num, den);
  return __fadd_rn(q.hi, q.lo);
}

// A double in [2^-126, 1] rounded to the nearest FP32 (ties to even) with
// integer operations; the rest (0, and values too small for a normal FP32)
// by the FP64 conversion.
__device__ __forceinline__ float unit_to_float(double d) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(d);
  const int e = (int)((b >> 52) & 0x7ff) - 1023;
  if (e < -126) return (float)d;
  const unsigned rest = (unsigned)(b & 0x1fffffffull);  // the 29 bits dropped
  unsigned f = ((unsigned)(e + 127) << 23) | (unsigned)((b >> 29) & 0x7fffffu);
  if (rest > 0x10000000u || (rest == 0x10000000u && (f & 1u))) ++f;  // carries into the exponent
  return __uint_as_float(f);
}

// Range checks on the bits of an FP64 value (integer comparisons; NaN
// fails all of them).  0 <= e <= 1: the bits of a non-negative double order
// as the value; -0 counts as 0.
__device__ __forceinline__ bool in_unit_interval(double e) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(e);
  return b <= 0x3ff0000000000000ull || b == 0x8000000000000000ull;
}
// k > 0 (finite or +inf)
__device__ __forceinline__ bool positive_or_inf(double k) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(k);
  return b >= 1ull && b <= 0x7ff0000000000000ull;
}
// K >= 0 and finite
__device__ __forceinline__ bool nonneg_finite(double K) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(K);
  return b < 0x7ff0000000000000ull || b == 0x8000000000000000ull;
}

// One block per row up to 5 resident blocks of 256 threads on each of 152
// SMs (the launch bound keeps all of them resident); wider grids only add
// partials.
constexpr int kMediumMaxBlocks = 5 * 152;

// Grid-stride over rows: block b takes rows b, b + gridDim.x, ..., its
// threads x, x + 256, ...  Each thread accumulates its nodes' partial sums
// (one FP64 add per node: sum eps) and reduces them once at the end.
__global__ void __launch_bounds__(kMediumBX, kMediumMaxBlocks / 152)
    medium_kernel(const double *__restrict__ eps, const double *__restrict__ k_i,
                  const double *__restrict__ kn, int nx, int ny, int pitch, int y_lo,
                  int y_hi, int kn_model, float *__restrict__ kn0, float kn_scale_max,
                  float2 *__restrict__ med, unsigned *bad, double *__restrict__ partials) {
  F2 se = {0.0f, 0.0f};  // sum of eps: FP32 pairs (~44 bits) without FP64 arithmetic
  double se_small = 0.0;  // and the few eps below 2^-60
  unsigned nodes = 0, open = 0, flags = 0;
  float ka_max = 0.0f;         // dynamic Kn: the largest finite k_a
  float inv_min = INFINITY;    // static Kn: the smallest positive 1/k_a
  for (int y = blockIdx.x; y < ny; y += gridDim.x) {
    const bool fluid_row = y >= y_lo && y < y_hi;
    for (int x = threadIdx.x; x < nx; x += kMediumBX) {
      const long long j = (long long)y * nx + x;
      const long long jp = (long long)y * pitch + x;
      float2 out = make_float2(0.0f, 0.0f);
      float kn_out = 0.0f;
      if (fluid_row) {
        const double e = eps[j], k = k_i[j], K = kn[j];
        unsigned f = 0;
        if (!in_unit_interval(e)) f |= 1u;
        if (!positive_or_inf(k)) f |= 2u;
        if (!nonneg_finite(K)) f |= 4u;
        const float ef = unit_to_float(e);
        float inv_k = 0.0f, ka = 0.0f;
        if (!f) {
          if (kn0) {  // dynamic Kn: 1/k_i stored, k_a formed at every step
            const float kf = (float)k, Kf = (float)K;
            if (!(kf >= 1e-15f)) f |= 8u;
            inv_k = 1.0f / kf;                                    // 0 for k_i = inf
            ka = kf * fc_f32(Kf * kn_scale_max, kn_model);     // at the lowest pressure
            kn_out = Kf;
          } else {
            inv_k = inv_ka_pair(k, K, kn_model);                 // Eq. 3 with Eq. 6-7 or 4-5
            if (!(inv_k <= 1e15f)) f |= 8u;                       // k_a >= 1e-15 (FP32 math)
          }
        }
        flags |= f;
        out = make_float2(ef, inv_k);
        const unsigned long long eb = (unsigned long long)__double_as_longlong(e);
        if (eb >= (963ull << 52) && eb <= 0x3ff0000000000000ull)  // 2^-60 <= e <= 1
          se = f2_add(se, f2_from_double(e));
        else
          se_small += e;  // below 2^-60, -0, and values the flags reject
        ++nodes;
        if (!f && ef > 0.0f) {
          if (inv_k > 0.0f) {  // finite k_a
            if (kn0) ka_max = fmaxf(ka_max, ka);
            else inv_min = fminf(inv_min, inv_k);
          } else {
            ++open;  // open pores (k_a = inf)
          }
        }
      }
      med[jp] = out;
      if (kn0) kn0[jp] = kn_out;
    }
  }
  if (flags) atomicOr(bad, flags);
  // the correctly rounded 1 / x does not increase with x: the largest of the
  // nodes' 1 / inv_k is 1 / (their smallest inv_k)
  if (inv_min < INFINITY) ka_max = fmaxf(ka_max, 1.0f / inv_min);
  double v[kNQ] = {(double)se.hi + (double)se.lo + se_small, (double)nodes, (double)ka_max,
                   (double)open, 0.0, 0.0};
  block_reduce_store<kMediumBX>(v, partials, kMediumMaxMask);
}

int medium_blocks(int nx, int ny) {
  (void)nx;
  return ny < kMediumMaxBlocks ? ny : kMediumMaxBlocks;
}

cudaError_t launch_medium(const double *eps, const double *k_i, const double *kn,
                          int nx, int ny, int pitch, int y_lo, int y_hi, int kn_model,
                          float *kn0, double kn_scale_max, float2 *med, unsigned *bad,
                          double *partials, cudaStream_t s) {
  medium_kernel<<<medium_blocks(nx, ny), kMediumBX, 0, s>>>(
      eps, k_i, kn, nx, ny, pitch, y_lo, y_hi, kn_model, kn0, (float)kn_scale_max, med, bad,
      partials);
  return cudaGetLastError();
}

// ------------------------------------------------- apparent permeability
// k_a of every node of the fluid rows as the step sees it: 1 / (stored
// 1/k_a), or with a dynamic Kn 1 / ((1/k_i) / f_c(Kn0)) at the pressure
// p0 (q = 1) with the step's own FP32 f_c.  Plate rows read 0.
__global__ void __launch_bounds__(kMediumBX)
    ka_kernel(const float2 *__restrict__ med, const float *__restrict__ kn0, int nx, int ny,
              int pitch, int y_lo, int y_hi, int kn_model, double *__restrict__ ka) {
  const int y = blockIdx.y;
  const int x = blockIdx.x * kMediumBX + threadIdx.x;
  if (x >= nx) return;
  double v = 0.0;
  if (y >= y_lo && y < y_hi) {
    const long long jp = (long long)y * pitch + x;
    float inv = med[jp].y;
    if (kn0) inv = inv_ka_dynamic(inv, kn0[jp], kn_model);  // the step's form at p = p0
    v = 1.0 / (double)inv;  // inf for an open pore (1/k_a = 0)
  }
  ka[(long long)y * nx + x] = v;
}

cudaError_t launch_ka(const float2 *med, const float *kn0, int nx, int ny, int pitch, int y_lo,
                      int y_hi, int kn_model, double *ka, cudaStream_t s) {
  dim3 grid((nx + kMediumBX - 1) / kMediumBX, ny);
  ka_kernel<<<grid, kMediumBX, 0, s>>>(med, kn0, nx, ny, pitch, y_lo, y_hi, kn_model, ka);
  return cudaGetLastError();
}

// ----------------------------------------------------- population loading
// B_j(z) = f_j(z + e_j) when z + e_j is a fluid node (wrapped), f_opp(j)(z)
// when it lies in a plate row, and 0 (unused) beyond a pressure column.
template <class S>
__global__ void __launch_bounds__(kMacroBX)
    load_pops_kernel(const StepArgs a, const double *__restrict__ f,
                     typename S::T *__restrict__ buf) {
  const int y = a.y0 + blockIdx.y;
  const int x = blockIdx.x * kMacroBX + threadIdx.x;
  if (x >= a.nx) return;
  const int ex[9] = {0, 1, 0, -1, 0, 1, -1, -1, 1};
  const int ey[9] = {0, 0, 1, 0, -1, 1, 1, -1, -1};
  const int opp[9] = {0, 3, 4, 1, 2, 7, 8, 5, 6};
  const double w[9] = {4.0 / 9.0,  1.0 / 9.0,  1.0 / 9.0,  1.0 / 9.0, 1.0 / 9.0,
                       1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0};
  const long long n = (long long)a.nx * a.ny;
  const double r0 = (double)a.rho0;
  for (int j = 0; j < 9; ++j) {
    int tx = x + ex[j], ty = y + ey[j];
    double val;
    if (a.walls && (ty == 0 || ty == a.ny - 1)) {
      val = f[opp[j] * n + (long long)y * a.nx + x];
    } else {
      ty = (ty + a.ny) % a.ny;
      if (tx < 0 || tx >= a.nx) {
        if (a.pressure) {
          val = w[j] * r0;
        } else {
          tx = (tx + a.nx) % a.nx;
          val = f[j * n + (long long)ty * a.nx + tx];
        }
      } else {
        val = f[j * n + (long long)ty * a.nx + tx];
      }
    }
    S::st1(buf + j * a.plane + (long long)y * a.pitch + x,
           (float)((val - w[j] * r0) * (double)a.scale));
  }
}

cudaError_t launch_load_pops(int storage, const StepArgs &a, int rows, const double *f,
                             void *buf, cudaStream_t s) {
  dim3 block(kMacroBX);
  dim3 grid((a.nx + kMacroBX - 1) / kMacroBX, rows);
  if (storage == 0)
    load_pops_kernel<StoreF32><<<grid, block, 0, s>>>(a, f, (float *)buf);
  else
    load_pops_kernel<StoreF16><<<grid, block, 0, s>>>(a, f, (__half *)buf);
  return cudaGetLastError();
}

}  // namespace lbmp
