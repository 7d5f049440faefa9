// boac_common.cu -- status strings, argument checks, device queries and
// workspace sizes shared by every entry point.
#include <cuda_runtime.h>

#include "boac_internal.h"
#include "boac_plain_kernels.cuh"

namespace boac {

bool geom_ok(const boac_geom* g) {
    if (!g) return false;
    if (g->n < 8 || g->n > kMaxN) return false;
    if (g->n_bins != g->n) return false;
    if (!(g->pixel_cm > 0.0f) || g->bin_cm != g->pixel_cm) return false;
    if (g->n_views < 1 || g->n_views > kMaxViews) return false;
    return true;
}

int sm_count() {
    constexpr int kDev = 16;
    static int cached[kDev];
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    if (dev >= 0 && dev < kDev && cached[dev]) return cached[dev];
    int n = 0;
    if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    if (dev >= 0 && dev < kDev) cached[dev] = n;
    return n;
}

int launch_status() {
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? BOAC_OK : BOAC_ECUDA;
}

// Plain path workspace for one candidate at a time: attenuation table, then
// sens, bp (n^2 each), q, r (n_views * n each) and the back-projection's
// per-grid partial images.
size_t plain_candidate_bytes(const boac_geom* g) {
    size_t nn = (size_t)g->n * g->n, vb = (size_t)g->n_views * g->n_bins;
    return align256(sizeof(float) * vb * g->n) + 2 * align256(sizeof(float) * nn) +
           2 * align256(sizeof(float) * vb) + align256(sizeof(float) * bp_partial_floats(g, 1));
}

// boac_backproject: per candidate, its table and its partial images.
size_t backproject_candidate_bytes(const boac_geom* g) {
    return sizeof(float) * ((size_t)g->n_views * g->n * g->n + bp_partial_floats(g, 1));
}

}  // namespace boac

using namespace boac;

extern "C" const char* boac_status_string(int status) {
    switch (status) {
        case BOAC_OK: return "ok";
        case BOAC_EINVAL: return "invalid argument";
        case BOAC_ECUDA: return "CUDA error";
        case BOAC_EWORKSPACE: return "workspace missing or too small";
        case BOAC_EUNSUPPORTED: return "geometry not supported by the library";
        case BOAC_ETIMEOUT: return "a bounded wait on the device ran out";
        case BOAC_ENONFINITE: return "a score is -inf (zero expected counts on a bin with counts)";
        default: return "unknown status";
    }
}

extern "C" int boac_abi_version(void) { return 1; }

extern "C" int boac_bounds_faults(int* faults, int reset) {
#ifdef BOAC_CHECKED
    if (!faults) return BOAC_EINVAL;
    // one counter per translation unit that uses the checked helpers
    int (*const readers[])(int) = {bounds_faults_fused,   bounds_faults_bpgroup, bounds_faults_gradfused,
                                   bounds_faults_grad,    bounds_faults_plain,   bounds_faults_unfused,
                                   bounds_faults_sysmat,  bounds_faults_band,    bounds_faults_raster};
    int total = 0;
    for (int (*r)(int) : readers) {
        const int v = r(reset);
        if (v < 0) return BOAC_ECUDA;
        total += v;
    }
    *faults = total;
    return BOAC_OK;
#else
    (void)faults;
    (void)reset;
    return BOAC_EUNSUPPORTED;
#endif
}

extern "C" size_t boac_workspace_bytes(const boac_geom* g, int B, int op) {
    if (!geom_ok(g) || B < 1) return 0;
    size_t vb = (size_t)g->n_views * g->n_bins;
    switch (op) {
        case BOAC_OP_PROJECT: return 0;
        case BOAC_OP_BACKPROJECT: return 2 * 256 + backproject_candidate_bytes(g) * (size_t)B;
        case BOAC_OP_MLEM: return fused_workspace_bytes(g, B);
        case BOAC_OP_MLEM_PLAIN: return plain_candidate_bytes(g);
        case BOAC_OP_SCORE: return align256(sizeof(float) * (size_t)B * vb);
        case BOAC_OP_MLEM_UNFUSED: return unfused_workspace_bytes(g, B);
        default: return 0;
    }
}
