// Host-side launchers of the lbmp kernels (internal to the library).
#pragma once

#include <cuda_runtime.h>

#include "lattice.cuh"
#include "lbmp.h"

namespace lbmp {

// Number of FP64 quantities a reduction block writes:
// sum u_x, sum u_y, sum (rho - rho0), sum |u|^2, sum |u - u_prev|^2,
// count of non-finite nodes.
constexpr int kNQ = 6;

struct MacroOut {
  double *rho;       // [ny][nx] or NULL
  double *ux;        // [ny][nx] or NULL
  double *uy;        // [ny][nx] or NULL
  double *pops;      // [9][ny][nx] or NULL
  float2 *uprev;     // [ny][pitch] velocity snapshot, or NULL
  int update_prev;   // overwrite uprev with u after reading it
  double *partials;  // [blocks][kNQ] or NULL (no reduction)
};

// Beskok-Karniadakis-Civan factor (Eq. 6-7, b = -1); f_c(0) = 1.
__host__ __device__ inline double fc_bkc(double kn) {
  if (kn == 0.0) return 1.0;
  const double slip_b = -1.0;
  const double alpha = 1.358 / (1.0 + 0.170 * pow(kn, -0.4348));
  return (1.0 + alpha * kn) * (1.0 + 4.0 * kn / (1.0 - slip_b * kn));
}

// f_c of the selected correlation: 0 Eq. 6-7, 1 Klinkenberg's first-order
// Eq. 4-5 (f_c = 1 + 4 c Kn, c = 1).
__host__ __device__ inline double fc_model(double kn, int model) {
  return model == 1 ? 1.0 + 4.0 * kn : fc_bkc(kn);
}

// Row pitch (elements) of the device planes of a lattice nx wide: nx
// rounded up to kPitchAlign, plus kPitchSkew when that is a multiple of
// kPitchSkewEvery.  Row strides that are multiples of large powers of two
// (4096 FP16 nodes = 8 KiB) make the concurrent tile copies of the staged
// kernel alias in the DRAM channels: 89 GLUPS at 4096^2 FP16 against 124
// with the skew (and 86 -> 107 at 2048^2, 90 -> 128 at 6144^2).
constexpr int kPitchAlign = 64;
constexpr int kPitchSkewEvery = 512;
constexpr int kPitchSkew = 64;
inline int row_pitch(int nx) {
  int p = ((nx + kPitchAlign - 1) / kPitchAlign) * kPitchAlign;
  if (p % kPitchSkewEvery == 0) p += kPitchSkew;
  return p;
}

// One time step over rows [a.y0, a.y0 + rows).  sr: FP16 stochastic
// rounding with the bits of time level *tctr + k.
cudaError_t launch_step(int storage, bool sr, const StepArgs &a, int rows, const void *fin,
                        void *fout, const float2 *med, const unsigned long long *tctr, int k,
                        cudaStream_t s);
// The FP32 direct step (static Kn, no stochastic rounding) that also
// stores every updated node's post-stream moments: rho - rho0, m_x, m_y in
// three [ny][pitch] float planes at mom, a.plane apart (adjoint recompute).
cudaError_t launch_step_moments(const StepArgs &a, int rows, const float *fin, float *fout,
                                const float2 *med, float *mom, cudaStream_t s);
// Vectorised FP16 variant of the same step (four nodes per thread).
cudaError_t launch_wide(bool sr, const StepArgs &a, int rows, const void *fin, void *fout,
                        const float2 *med, const unsigned long long *tctr, int k,
                        cudaStream_t s);
// Staged variant of the same step (asynchronous bulk copies into a shared-
// memory ring, persistent grid of at most nsm CTAs); a bounded wait that
// gives up sets *err.  prepare_staged() raises the shared-memory limit of
// the kernels once per process.
cudaError_t prepare_staged();
cudaError_t launch_staged(int storage, bool sr, const StepArgs &a, int rows, const void *fin,
                          void *fout, const float2 *med, const unsigned long long *tctr, int k,
                          unsigned *err, int nsm, cudaStream_t s);
// Store msg as the calling thread's lbmp_last_error() text.
void set_last_error(const char *msg);

// Check the parameters of lbmp_create (and normalise J = 0, rho0 = 0 to 1);
// EINVAL with a message when invalid.  Touches no device.
lbmp_status validate_params(::lbmp_params *p);

// *tctr += n (one thread).
cudaError_t launch_bump(unsigned long long *tctr, int n, cudaStream_t s);

// Blocks a macroscopic/reduction launch over all ny rows uses.
int macro_blocks(const StepArgs &a);
// Blocks (partials) of the histogram's first pass (one block per 256 nodes
// of a row).
int hist_blocks(const StepArgs &a);
cudaError_t launch_macro(int storage, const StepArgs &a, const void *fin,
                         const float2 *med, const MacroOut &o, cudaStream_t s);

// Reduce [nblocks][nq] partials in a fixed order into out[0..nq): by sum,
// or by max for the quantities whose bit is set in max_mask.
cudaError_t launch_finalize(const double *partials, int nblocks, int nq, double *out,
                            cudaStream_t s, unsigned max_mask = 0u);

// Medium precompute: (eps, k_i, Kn) -> float2 (eps, 1/k_a) with f_c of
// kn_model; with kn0 != NULL (dynamic Kn) float2 (eps, 1/k_i) and kn0 = Kn.
// Flags invalid values in *bad; FP64 block partials over rows [y_lo, y_hi):
// sum eps, fluid nodes, max finite k_a (max-reduced, kMediumMaxMask; with a
// dynamic Kn at Kn * kn_scale_max), open-pore count.
constexpr unsigned kMediumMaxMask = 1u << 2;
int medium_blocks(int nx, int ny);
cudaError_t launch_medium(const double *eps, const double *k_i, const double *kn,
                          int nx, int ny, int pitch, int y_lo, int y_hi, int kn_model,
                          float *kn0, double kn_scale_max, float2 *med, unsigned *bad,
                          double *partials, cudaStream_t s);

// k_a per node as the step uses it ([ny][nx] float64; plate rows 0, open
// pores +inf); with kn0 != NULL the k_a at the reference pressure.
cudaError_t launch_ka(const float2 *med, const float *kn0, int nx, int ny, int pitch, int y_lo,
                      int y_hi, int kn_model, double *ka, cudaStream_t s);

// Normalised-velocity histogram: pass 1 writes the maximum of |u| over the
// fluid rows of each block (hist_blocks(a) doubles, a.y0 ignored);
// pass 2 adds the counts of bins min(floor(|u| / umax * nbins), nbins - 1)
// to counts[0..nbins).  nbins <= kMaxHistBins.
constexpr int kMaxHistBins = 64;
cudaError_t launch_speed_max(int storage, const StepArgs &a, const void *fin, const float2 *med,
                             double *partials, cudaStream_t s);
cudaError_t launch_histogram(int storage, const StepArgs &a, const void *fin, const float2 *med,
                             double umax, int nbins, unsigned long long *counts, cudaStream_t s);

// Inverse of the pull: write a post-collision buffer whose pull gives the
// post-stream populations f ([9][ny][nx] float64).
cudaError_t launch_load_pops(int storage, const StepArgs &a, int rows, const double *f,
                             void *buf, cudaStream_t s);

}  // namespace lbmp
