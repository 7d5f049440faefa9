// boac_fused.h -- declarations shared by the two fused MLEM kernels: the
// one-CTA-per-candidate kernel (boac_fused.cu, images up to 128 x 128 held
// in one SM's shared memory) and the cluster kernel (boac_band.cu, 256 x 256
// images split into bands of rows over the CTAs of a thread-block cluster).
#pragma once

#include <cuda_runtime.h>
#include <math.h>

#include "boac_internal.h"

namespace boac {

struct RaggedDesc {
    long long mu_off, S_off, F_off;  // float offsets into the caller's pools
    int K;                           // MLEM iterations of this candidate
    int out;                         // index of its score in L
};

struct FusedArgs {
    const float* mu;
    const float* S;
    long long s_stride;
    float* F;
    double* L;
    int include_lgamma;
    // Uniform batch with one shared sinogram: sum_i lgamma(S_i + 1), computed
    // once and subtracted from each score (nullptr: the term per bin).
    const double* lgS;
    int B, V, K;
    float dx;
    // Per-CTA slots, written and read by the same CTA within one launch:
    // read with plain (coherent) loads, never through the read-only path.
    float* tab;   // [slots][tab_floats]: attenuation exponents
    float* sens;  // [slots][n][n] (cluster kernel: [CTAs][band rows][n])
    // Images above 128 x 128 do not fit shared memory: their F, accumulator
    // and sample buffer live in a per-slot region of the workspace instead
    // (same layout), read through L1 and written through to L2.
    float* img;   // [slots][2 IMG + n WP] or unused
    // Ragged batches: per-candidate records (device), sorted by the host;
    // nullptr: uniform batch, candidate b at b * n^2 / b * s_stride, K = K.
    const RaggedDesc* desc;
    // Work split.  The batch's iterations are laid end to end, candidate
    // after candidate (candidate j occupies units [job_start[j],
    // job_start[j+1]), max(K, 1) units each; job_start == nullptr for a
    // uniform batch), and CTA (or cluster) m runs units [m cap, (m+1) cap) with
    // cap >= the longest candidate (McNaughton's wrap-around rule: every CTA
    // gets the same share, a candidate is cut between at most two CTAs).
    // A CTA takes its candidates in descending order, so the first part of
    // a cut candidate runs first on CTA m and its second part last on CTA
    // m+1; ready[j] tells the second part that the first has written F
    // (always long before it is needed, since cap >= the candidate length).
    const long long* job_start;
    long long cap;
    int* ready;    // [B] zeroed before the launch
    int* status;   // 0, or BOAC_ETIMEOUT if a bounded wait ran out
    // Cycles the second part of a cut candidate waits for the first part's
    // flag before giving up (boac_set_wait_cycles; default kWaitCycles).
    long long wait_cycles;
    // Candidate whose first part does not release its flag (-1: none).  Set
    // only by boac_test_mlem_handover, to make the bounded wait run out.
    int withhold;
    // One-CTA kernel, images up to 128 x 128: the scatter schedule of every
    // (grid, class) (nullptr: natural class order).
    const unsigned short* sched;
    // Cluster kernel only: the ray-run records of every (band, grid), and a
    // flag the record kernel sets if a run exceeds the kernel's buffers.
    const int* geo;
    int* geo_bad;
};

// Default number of cycles a CTA waits for the first part of a cut candidate
// before giving up (about 2 s at 2 GHz; the schedule leaves the wait a whole
// candidate's worth of slack, so it ends immediately in practice).
constexpr long long kWaitCycles = 1LL << 32;
// The process-wide wait limit in force (boac_set_wait_cycles).
long long wait_cycles();

// 2^x with the hardware approximation (relative error about 2^-22).
__device__ __forceinline__ float ex2(float x) {
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// 4-byte asynchronous copy global -> shared (no register staging); the
// copies a thread issued are complete after copy_async_wait_all().
__device__ __forceinline__ void copy_async4(float* dst_smem, const float* src) {
    const unsigned d = (unsigned)__cvta_generic_to_shared(dst_smem);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(d), "l"(src) : "memory");
}
__device__ __forceinline__ void copy_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void copy_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }

// Ask L2 to fetch the 128-byte line holding p (no register result).
// Exponent planes keep four consecutive samples of a thread's run
// together: element (k, b) of a plane walked by thread b along k (or (b, k)
// of a transposed plane walked by thread k along b) at ((k / 4) n + b) 4 +
// k % 4, so one 16-byte load gives a thread its next four samples and a
// warp's load covers 512 contiguous bytes.
__host__ __device__ constexpr int tab_ix(int n, int k, int lb) { return (((k >> 2) * n + lb) << 2) | (k & 3); }

__device__ __forceinline__ void prefetch_l2(const void* p) {
    asm volatile("prefetch.global.L2 [%0];" ::"l"(p));
}

__device__ __forceinline__ double loglik_term(double s, double q, int include_lgamma) {
    double t;
    if (s > 0.0) t = q > 0.0 ? s * log(q) - q : -INFINITY;
    else t = -q;
    if (include_lgamma) t -= lgamma(s + 1.0);
    return t;
}

// ---- fused score gradient (boac_gradfused.cu): one CTA or a cluster of G
// CTAs per candidate, 64 / 96 / 128 images, V % 4 == 0.
struct GradFusedArgs {
    const float* mu;  // [B][n][n] AREA map
    const float* S;
    long long s_stride;
    int B, V, K, ckpt;
    float dx;
    int include_lgamma;
    const double* lgS;  // shared sinogram: sum of ln S! (or nullptr)
    float* tab;         // per CTA: exponent planes of its grids
    float* sens;        // per CTA: n^2 (its rows)
    float* ck;          // per candidate: [nseg][n^2] F^{j ckpt}
    float* segF;        // per candidate: [ckpt + 1][n^2] iterates of a segment
    float* segz;        // per candidate: [ckpt][n^2] z^n = A^T r^n
    float* segq;        // per candidate: [ckpt][V / 4][4][n] q^n in grid coordinates
    float* segB;        // per candidate: [ckpt][V / 4][n][n] sample (k, b) of F^n at [b][k]
    float* Fbar;        // per candidate: [n^2]
    float* sensbar;     // per candidate: [n^2]
    float* abar;        // per candidate: [V / 4][n][n] adjoint of the mu samples of each grid
    float* mubar;       // per candidate: [n^2] adjoint of the pixels of mu
    double* L;
    float* F_out;       // [B][n][n] or nullptr
    const unsigned short* sched;
};

bool grad_fused_supported(const boac_geom* g);
// Cluster size G (1: one CTA per candidate) and the clusters to launch for B
// candidates; 0 if the fused gradient does not apply.
int grad_fused_plan(const boac_geom* g, int B, int* holders);
// Floats of one CTA's exponent slot for cluster size G.
size_t grad_fused_tab_floats(const boac_geom* g, int G);
// The scatter schedule of the geometry (cached on the device, else built
// into a.sched), then the kernel.
int grad_fused_launch(const boac_geom* g, const GradFusedArgs& a, int G, int clusters, cudaStream_t st);

// ---- cluster kernel (boac_band.cu): images of side n split into bands of
// rows over a cluster of nb CTAs per candidate, V % 4 == 0; instantiated for
// n = 256 with nb in {5, 6, 8} and n = 128 and 64 with nb in {2, 4, 8}.
bool band_supported(int n, int V, int nb);
size_t band_smem_bytes(int n, int nb);
size_t band_tab_floats(int n, int nb, int V);  // attenuation exponents, per CTA
size_t band_sens_floats(int n, int nb);        // sensitivity rows, per CTA
size_t band_geo_bytes(int n, int nb, int V);   // per-band ray-run records
// Largest number of clusters of nb CTAs resident at once (cached per device;
// 0 if the device cannot run them).
int band_max_clusters(int n, int nb);
// Launch the record kernel and the cluster kernel with `clusters` clusters.
int band_launch(int n, int nb, const FusedArgs& a, int clusters, cudaStream_t st);

}  // namespace boac
