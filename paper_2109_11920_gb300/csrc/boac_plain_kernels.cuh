// boac_plain_kernels.cuh -- the unfused kernels of boac_plain.cu, declared
// for reuse by the gradient path (boac_grad.cu).  All are batched over
// candidates (grid z or y) and documented at their definitions.
#pragma once

#include <cuda_runtime.h>

#include "boac_internal.h"

namespace boac {

constexpr int kRayThreads = 128;   // ray kernels: one thread per (candidate, view, bin)
constexpr int kPixThreads = 256;   // pixel kernels: one thread per (candidate, pixel)

__global__ void attenuation_table_kernel(int n, int V, float dx, const float* __restrict__ mu,
                                         float* __restrict__ tab);
__global__ void project_otf_kernel(int n, int V, float dx, const float* __restrict__ mu,
                                   const float* __restrict__ F, float* __restrict__ q);
__global__ void project_table_kernel(int n, int V, float dx, const float* __restrict__ tab,
                                     const float* __restrict__ F, float* __restrict__ q);
__global__ void backproject_gather_kernel(int n, int V, float scale, const float* __restrict__ tab,
                                          const float* __restrict__ y, float* __restrict__ out,
                                          int accumulate);
__global__ void ratio_kernel(int count, const float* __restrict__ S, const float* __restrict__ q,
                             float* __restrict__ r);
__global__ void update_kernel(int count, float* __restrict__ F, const float* __restrict__ bp,
                              const float* __restrict__ sens);
// status (nullable): set to BOAC_ENONFINITE (unless already non-zero) when
// a candidate's score is -inf (q = 0 on a bin with S > 0).
__global__ void loglik_kernel(int nbin, const float* __restrict__ q, const float* __restrict__ S,
                              long long s_stride, int include_lgamma, double* __restrict__ L,
                              const double* __restrict__ lgS, int* status = nullptr);
// sum_i lgamma(S_i + 1) of one sinogram S[nbin] into scratch[0]
// (scratch: kLgammaScratchDoubles doubles, 8-byte aligned); returns scratch.
constexpr int kLgammaScratchDoubles = 31;
const double* lgamma_sum(int nbin, const float* S, double* scratch, cudaStream_t st);
// r = S / q over B candidates (0 where q <= 0), S rows s_stride apart (boac_grad.cu).
__global__ void ratio_batched_kernel(int B, int nbin, const float* __restrict__ S, long long s_stride,
                                     const float* __restrict__ q, float* __restrict__ r);

dim3 ray_grid(const boac_geom* g, int B);
int grid_1d(long long count, int threads);

// out[cand] (+)= scale * sum_v B_v^T (tab_v * y_v) for B candidates from an
// attenuation table [B][V][n][n] (boac_bpgroup.cu): grouped shared-memory
// scatter with per-grid partial images in `partial` (bp_partial_floats(g, B)
// floats), or the per-pixel gather where the geometry has no grouped kernel
// (then `partial` may be null).
size_t bp_partial_floats(const boac_geom* g, int B);
// q[cand][v][bin] = dx * sum_k tab_v[k][bin] F(sample (k, bin) of view v) for
// B candidates (boac_bpgroup.cu): one CTA per candidate and sample grid with
// F in shared memory, or one thread per ray where no grouped kernel exists.
int project_table(const boac_geom* g, int B, const float* tab, const float* F, float dx, float* q,
                  cudaStream_t st);
int backproject_table(const boac_geom* g, int B, const float* tab, const float* y, float scale, float* out,
                      int accumulate, float* partial, cudaStream_t st);

}  // namespace boac
