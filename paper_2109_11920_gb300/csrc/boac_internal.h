// boac_internal.h -- host-side helpers shared by the library's .cu files.
#pragma once

#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>
#include <stddef.h>
#include <stdint.h>

#include "../../include/boac.h"

namespace boac {

// Largest supported image side and view count.
constexpr int kMaxN = 256;
constexpr int kMaxViews = 720;
// Largest number of size classes in one ragged batch.
constexpr int kMaxRaggedClasses = 8;

// Geometry checks shared by every entry point: n in [8, kMaxN], n_bins == n,
// bin_cm == pixel_cm > 0, n_views in [1, kMaxViews].
bool geom_ok(const boac_geom* g);

// Number of SMs of the current device (cached per device).
int sm_count();

// cudaStream_t from the ABI's void*.
inline cudaStream_t as_stream(void* s) { return reinterpret_cast<cudaStream_t>(s); }

// Map the last CUDA error to a status code (clears it).
int launch_status();

// NVTX range over a scope of host code (a no-op unless a profiler such as
// Nsight Systems is attached): entry points and their phases -- set-up,
// iterations, score -- show up by name on the host timeline next to the
// kernels they enqueue.
struct NvtxRange {
    explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange&) = delete;
    NvtxRange& operator=(const NvtxRange&) = delete;
};
// Consecutive phases of one scope: next() closes the current range and
// opens the following one.
struct NvtxPhases {
    explicit NvtxPhases(const char* name) { nvtxRangePushA(name); }
    void next(const char* name) {
        nvtxRangePop();
        nvtxRangePushA(name);
    }
    ~NvtxPhases() { nvtxRangePop(); }
    NvtxPhases(const NvtxPhases&) = delete;
    NvtxPhases& operator=(const NvtxPhases&) = delete;
};
#define BOAC_NVTX_CAT2(a, b) a##b
#define BOAC_NVTX_CAT(a, b) BOAC_NVTX_CAT2(a, b)
#define BOAC_RANGE(name) ::boac::NvtxRange BOAC_NVTX_CAT(boac_nvtx_, __LINE__)(name)

#ifdef BOAC_CHECKED
// Checked builds: the bounds-fault counters of the translation units whose
// kernels gather and scatter through the checked helpers (count, or -1 if
// the read failed; reset clears the counter).
int bounds_faults_fused(int reset);
int bounds_faults_bpgroup(int reset);
int bounds_faults_gradfused(int reset);
int bounds_faults_grad(int reset);
int bounds_faults_plain(int reset);
int bounds_faults_unfused(int reset);
int bounds_faults_sysmat(int reset);
int bounds_faults_band(int reset);
int bounds_faults_raster(int reset);
#endif

// Round up to a multiple of 256 bytes.
inline size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

// Plain path: workspace for one candidate (table, sens, bp, q, r).
size_t plain_candidate_bytes(const boac_geom* g);
size_t backproject_candidate_bytes(const boac_geom* g);

// boac_mlem: workspace for geometry g and B candidates (the fused kernel's,
// or the unfused path's for the small batches boac_mlem runs there).
size_t fused_workspace_bytes(const boac_geom* g, int B);

// Batched unfused MLEM (boac_unfused.cu): workspace and the call itself.
size_t unfused_workspace_bytes(const boac_geom* g, int B);
int mlem_unfused(const boac_geom* g, const float* mu, const float* S, long long s_stride, float* F, int K,
                 int B, double* L, int include_lgamma, void* ws, size_t ws_bytes, cudaStream_t st);

// Entries per candidate of the 9-parameter model (c_0..c_5, mu_b, mu_c, dR).
constexpr int kParams = 9;

// Eq. 3-4 for B candidates: coefficients p[cand * pstride + 0..5]; pstride
// 6 takes the tissue values from t, pstride kParams from p (t unused).
int rasterize_launch(const boac_geom* g, const boac_tissue* t, const float* p, int pstride, int B,
                     int mode, float* mu, cudaStream_t st);
// The pixel geometry of the n x n grid: pg[0][pix] = r, pg[k][pix] =
// P_k(cos theta), k = 1..5 (6 n^2 doubles).
int pixel_geom_launch(int n, double dx, double* pg, cudaStream_t st);

}  // namespace boac
