// boac_unfused.cu -- MLEM for a batch of candidates with one launch per step
// of the iteration (attenuation table once; per iteration q = A F, r = S / q,
// z = A^T r, F <- F z / sens), every launch covering the whole batch.  Where
// the batch is too small to fill the GPU with the fused kernel's one CTA (or
// one cluster) per candidate, these kernels spread one candidate over many
// CTAs (one per sample grid in the projector and the back-projector) and
// finish sooner; boac_mlem takes this path there.
#include <cuda_runtime.h>

#include "boac_device.cuh"
#include "boac_internal.h"
#include "boac_plain_kernels.cuh"

namespace boac {

namespace {

struct UnfusedLayout {
    size_t status, tab, sens, z, q, r, partial, total;
};

UnfusedLayout unfused_layout(const boac_geom* g, int B) {
    const size_t nn = (size_t)g->n * g->n, vb = (size_t)g->n_views * g->n_bins, Bs = (size_t)B;
    UnfusedLayout l{};
    size_t off = 0;
    auto take = [&](size_t floats) {
        const size_t at = off;
        off += align256(sizeof(float) * floats);
        return at;
    };
    l.status = take(1);
    l.tab = take(Bs * (size_t)g->n_views * nn);
    l.sens = take(Bs * nn);
    l.z = take(Bs * nn);
    l.q = take(Bs * vb);
    l.r = take(Bs * vb);
    l.partial = take(bp_partial_floats(g, B));
    l.total = off;
    return l;
}

}  // namespace

size_t unfused_workspace_bytes(const boac_geom* g, int B) {
    if (!geom_ok(g) || B < 1) return 0;
    return unfused_layout(g, B).total;
}

int mlem_unfused(const boac_geom* g, const float* mu, const float* S, long long s_stride, float* F, int K,
                 int B, double* L, int include_lgamma, void* ws, size_t ws_bytes, cudaStream_t st) {
    const UnfusedLayout l = unfused_layout(g, B);
    if (!ws || ws_bytes < l.total) return BOAC_EWORKSPACE;
    char* base = static_cast<char*>(ws);
    auto P = [&](size_t off) { return reinterpret_cast<float*>(base + off); };
    float *tab = P(l.tab), *sens = P(l.sens), *z = P(l.z), *q = P(l.q), *r = P(l.r), *partial = P(l.partial);
    const float dx = g->pixel_cm;
    const size_t nn = (size_t)g->n * g->n, vb = (size_t)g->n_views * g->n_bins;
    const long long cnt_pix = (long long)B * nn, cnt_bin = (long long)B * vb;
    // the status word boac_workspace_status reads: this path has no waits
    cudaMemsetAsync(base + l.status, 0, sizeof(int), st);
    BOAC_RANGE("set-up: attenuation tables, sensitivity");
    attenuation_table_kernel<<<ray_grid(g, B), kRayThreads, 0, st>>>(g->n, g->n_views, dx, mu, tab);
    int s = backproject_table(g, B, tab, nullptr, dx, sens, 0, partial, st);
    if (s != BOAC_OK) return s;
    for (int it = 0; it < K; ++it) {
        BOAC_RANGE("MLEM iteration");
        s = project_table(g, B, tab, F, dx, q, st);
        if (s != BOAC_OK) return s;
        ratio_batched_kernel<<<grid_1d(cnt_bin, 256), 256, 0, st>>>(B, (int)vb, S, s_stride, q, r);
        s = backproject_table(g, B, tab, r, dx, z, 0, partial, st);
        if (s != BOAC_OK) return s;
        update_kernel<<<grid_1d(cnt_pix, 256), 256, 0, st>>>((int)cnt_pix, F, z, sens);
    }
    if (L) {
        BOAC_RANGE("score (Eq. 5)");
        s = project_table(g, B, tab, F, dx, q, st);
        if (s != BOAC_OK) return s;
        // one shared sinogram: its ln S! sum once, in the status slot's spare bytes
        const double* lgS = include_lgamma && s_stride == 0
                                ? lgamma_sum((int)vb, S, reinterpret_cast<double*>(base + l.status + 8), st)
                                : nullptr;
        loglik_kernel<<<B, 256, 0, st>>>((int)vb, q, S, s_stride, include_lgamma, L, lgS,
                                         reinterpret_cast<int*>(base + l.status));
    }
    return launch_status();
}

}  // namespace boac

using namespace boac;

extern "C" int boac_mlem_unfused(const boac_geom* g, const float* mu, const float* S, long long s_stride,
                                 float* F, int K, int B, double* L, int include_lgamma, void* ws,
                                 size_t ws_bytes, void* stream) {
    BOAC_RANGE("boac_mlem_unfused");
    if (!geom_ok(g) || !mu || !S || !F || B < 1 || B > 65535 || K < 0 || s_stride < 0) return BOAC_EINVAL;
    if ((long long)B * g->n * g->n > 0x7fffffffLL) return BOAC_EINVAL;
    return mlem_unfused(g, mu, S, s_stride, F, K, B, L, include_lgamma, ws, ws_bytes, as_stream(stream));
}

#ifdef BOAC_CHECKED
namespace boac {
BOAC_FAULT_READER(bounds_faults_unfused)
}  // namespace boac
#endif
