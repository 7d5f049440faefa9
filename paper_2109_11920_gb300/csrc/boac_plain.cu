// boac_plain.cu -- the unfused operators: forward projection (Eq. 1-2), its
// exact adjoint, the launch-per-step MLEM loop used as the comparison
// baseline, and the float64 log-likelihood reduction (Eq. 5).
//
// Ray kernels run one thread per (candidate, view, bin) and walk the ray from
// the detector side (k = n-1) inwards, so the attenuation suffix sum of
// Eq. 1's inner integral is a running register sum.  The back-projector is a
// per-pixel gather over the <= 3 x 3 ray samples whose bilinear footprint
// contains the pixel, with the weights recomputed exactly as the projector
// computes them (sample_uw + pixel_weight), so no atomics are needed and the
// result is deterministic.
#include <cuda_runtime.h>
#include <math.h>

#include "boac_device.cuh"
#include "boac_internal.h"
#include "boac_plain_kernels.cuh"

namespace boac {

// attenuation factor of every ray sample: tab[cand][v][k][b]
__global__ void attenuation_table_kernel(int n, int V, float dx, const float* __restrict__ mu,
                                         float* __restrict__ tab) {
    const int b = blockIdx.x * blockDim.x + threadIdx.x, v = blockIdx.y, cand = blockIdx.z;
    if (b >= n) return;
    const size_t nn = (size_t)n * n;
    const float* m_img = mu + cand * nn;
    float* t = tab + ((size_t)cand * V + v) * nn;
    float cs, sn;
    view_cos_sin(v, V, &cs, &sn);
    const float c = 0.5f * (float)(n - 1);
    float suffix = 0.0f;
    for (int k = n - 1; k >= 0; --k) {
        float u, w;
        sample_uw(k, b, cs, sn, c, &u, &w);
        const float m = bilerp_global(m_img, n, u, w);
        t[(size_t)k * n + b] = expf(-dx * (0.5f * m + suffix));
        suffix += m;
    }
}

// q[cand][v][b] = dx sum_k a_k F_k with the attenuation integrated on the fly
__global__ void project_otf_kernel(int n, int V, float dx, const float* __restrict__ mu,
                                   const float* __restrict__ F, float* __restrict__ q) {
    const int b = blockIdx.x * blockDim.x + threadIdx.x, v = blockIdx.y, cand = blockIdx.z;
    if (b >= n) return;
    const size_t nn = (size_t)n * n;
    const float* m_img = mu + cand * nn;
    const float* f_img = F + cand * nn;
    float cs, sn;
    view_cos_sin(v, V, &cs, &sn);
    const float c = 0.5f * (float)(n - 1);
    float suffix = 0.0f, acc = 0.0f;
    for (int k = n - 1; k >= 0; --k) {
        float u, w;
        sample_uw(k, b, cs, sn, c, &u, &w);
        const float m = bilerp_global(m_img, n, u, w);
        const float a = expf(-dx * (0.5f * m + suffix));
        suffix += m;
        acc = fmaf(a, bilerp_global(f_img, n, u, w), acc);
    }
    q[((size_t)cand * V + v) * n + b] = dx * acc;
}

// q = A F with a precomputed attenuation table
__global__ void project_table_kernel(int n, int V, float dx, const float* __restrict__ tab,
                                     const float* __restrict__ F, float* __restrict__ q) {
    const int b = blockIdx.x * blockDim.x + threadIdx.x, v = blockIdx.y, cand = blockIdx.z;
    if (b >= n) return;
    const size_t nn = (size_t)n * n;
    const float* t = tab + ((size_t)cand * V + v) * nn;
    const float* f_img = F + cand * nn;
    float cs, sn;
    view_cos_sin(v, V, &cs, &sn);
    const float c = 0.5f * (float)(n - 1);
    float acc = 0.0f;
    for (int k = n - 1; k >= 0; --k) {
        float u, w;
        sample_uw(k, b, cs, sn, c, &u, &w);
        acc = fmaf(__ldg(t + (size_t)k * n + b), bilerp_global(f_img, n, u, w), acc);
    }
    q[((size_t)cand * V + v) * n + b] = dx * acc;
}

// out[cand] (+)= scale * sum_v B_v^T (tab_v * y_v) (y == nullptr: y = 1), as
// a per-pixel gather: with tab = attenuation and scale = dx this is A^T y.
__global__ void backproject_gather_kernel(int n, int V, float scale, const float* __restrict__ tab,
                                          const float* __restrict__ y, float* __restrict__ out,
                                          int accumulate) {
    extern __shared__ float csn[];  // [V][2]
    for (int v = threadIdx.x; v < V; v += blockDim.x) view_cos_sin(v, V, &csn[2 * v], &csn[2 * v + 1]);
    __syncthreads();
    const int cand = blockIdx.y;
    const int pix = blockIdx.x * blockDim.x + threadIdx.x;
    if (pix >= n * n) return;
    const int i = pix / n, j = pix % n;
    const size_t nn = (size_t)n * n;
    const float c = 0.5f * (float)(n - 1);
    const float jc = (float)j - c, ic = (float)i - c;
    const float* yc = y ? y + (size_t)cand * V * n : nullptr;
    float acc = 0.0f;
    for (int v = 0; v < V; ++v) {
        const float cs = csn[2 * v], sn = csn[2 * v + 1];
        const float* t = tab + ((size_t)cand * V + v) * nn;
        // continuous (k', b') of the pixel centre on this view's sample grid
        const float bp = c + jc * cs + ic * sn;
        const float kp = c - jc * sn + ic * cs;
        int kmin = (int)floorf(kp - 1.4143f) + 1, kmax = (int)floorf(kp + 1.4143f);
        int bmin = (int)floorf(bp - 1.4143f) + 1, bmax = (int)floorf(bp + 1.4143f);
        kmin = max(kmin, 0);
        bmin = max(bmin, 0);
        kmax = min(kmax, n - 1);
        bmax = min(bmax, n - 1);
        float vacc = 0.0f;
        for (int b = bmin; b <= bmax; ++b) {
            float bacc = 0.0f;
            for (int k = kmin; k <= kmax; ++k) {
                float u, w;
                sample_uw(k, b, cs, sn, c, &u, &w);
                const float wt = pixel_weight(u, w, i, j, n);
                if (wt != 0.0f) bacc = fmaf(wt, __ldg(t + (size_t)k * n + b), bacc);
            }
            vacc = fmaf(bacc, yc ? __ldg(yc + (size_t)v * n + b) : 1.0f, vacc);
        }
        acc += vacc;
    }
    float* o = out + (size_t)cand * nn + pix;
    *o = accumulate ? *o + scale * acc : scale * acc;
}

__global__ void ratio_kernel(int count, const float* __restrict__ S, const float* __restrict__ q,
                             float* __restrict__ r) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < count; i += gridDim.x * blockDim.x) {
        const float qi = q[i];
        r[i] = qi > 0.0f ? __ldg(S + i) / qi : 0.0f;
    }
}

__global__ void update_kernel(int count, float* __restrict__ F, const float* __restrict__ bp,
                              const float* __restrict__ sens) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < count; i += gridDim.x * blockDim.x) {
        const float s = sens[i];
        F[i] = s > 0.0f ? F[i] * bp[i] / s : 0.0f;
    }
}

// L[cand] = sum_i S_i ln q_i - q_i [- lgamma(S_i + 1)] in float64.  Fixed
// per-thread strides and a fixed reduction tree: deterministic.  With lgS
// (candidates sharing one sinogram) the ln S! term is its precomputed sum,
// subtracted once, instead of a term per bin.
__global__ void loglik_kernel(int nbin, const float* __restrict__ q, const float* __restrict__ S,
                              long long s_stride, int include_lgamma, double* __restrict__ L,
                              const double* __restrict__ lgS, int* status) {
    __shared__ double part[32];
    const int cand = blockIdx.x;
    const float* qc = q + (size_t)cand * nbin;
    const float* Sc = S + (size_t)cand * s_stride;
    double acc = 0.0;
    for (int i = threadIdx.x; i < nbin; i += blockDim.x) {
        const double s = (double)__ldg(Sc + i), qi = (double)__ldg(qc + i);
        double term;
        if (s > 0.0) term = qi > 0.0 ? s * log(qi) - qi : -INFINITY;
        else term = -qi;
        if (include_lgamma && !lgS) term -= lgamma(s + 1.0);
        acc += term;
    }
    for (int off = 16; off > 0; off >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, off);
    if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += part[w];
        L[cand] = include_lgamma && lgS ? t - *lgS : t;
        if (status && t == -INFINITY) atomicCAS(status, BOAC_OK, BOAC_ENONFINITE);
    }
}

// sum_i lgamma(S_i + 1) over one sinogram (the ln S! term of Eq. 5, equal
// for every candidate that shares the sinogram), float64: block b adds bins
// b * blockDim + t, b * blockDim + t + G blockDim, ... into part[b] with a
// fixed reduction tree; one thread then adds part[0..G) in order.
__global__ void lgamma_partial_kernel(int nbin, const float* __restrict__ S, double* __restrict__ part) {
    __shared__ double red[32];
    double acc = 0.0;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < nbin; i += gridDim.x * blockDim.x)
        acc += lgamma((double)__ldg(S + i) + 1.0);
    for (int off = 16; off > 0; off >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, off);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
        part[blockIdx.x] = t;
    }
}

__global__ void lgamma_final_kernel(int nparts, const double* __restrict__ part, double* __restrict__ out) {
    double t = 0.0;
    for (int i = 0; i < nparts; ++i) t += part[i];
    *out = t;
}

const double* lgamma_sum(int nbin, const float* S, double* scratch, cudaStream_t st) {
    int parts = (nbin + 255) / 256;
    if (parts > kLgammaScratchDoubles - 1) parts = kLgammaScratchDoubles - 1;
    if (parts < 1) parts = 1;
    lgamma_partial_kernel<<<parts, 256, 0, st>>>(nbin, S, scratch + 1);
    lgamma_final_kernel<<<1, 1, 0, st>>>(parts, scratch + 1, scratch);
    return scratch;
}

dim3 ray_grid(const boac_geom* g, int B) {
    return dim3((g->n + kRayThreads - 1) / kRayThreads, g->n_views, B);
}

int grid_1d(long long count, int threads) {
    long long b = (count + threads - 1) / threads;
    long long cap = 16LL * (sm_count() > 0 ? sm_count() : 1);
    return (int)(b < cap ? b : cap);
}

}  // namespace boac

using namespace boac;

extern "C" int boac_project(const boac_geom* g, const float* mu, const float* F, int B, float* q,
                            void* stream) {
    BOAC_RANGE("boac_project");
    if (!geom_ok(g) || !mu || !F || !q || B < 1 || B > 65535) return BOAC_EINVAL;
    project_otf_kernel<<<ray_grid(g, B), kRayThreads, 0, as_stream(stream)>>>(
        g->n, g->n_views, g->pixel_cm, mu, F, q);
    return launch_status();
}

extern "C" int boac_backproject(const boac_geom* g, const float* mu, const float* y, int B,
                                float* out, void* ws, size_t ws_bytes, void* stream) {
    BOAC_RANGE("boac_backproject");
    if (!geom_ok(g) || !mu || !out || B < 1 || B > 65535) return BOAC_EINVAL;
    const size_t nn = (size_t)g->n * g->n;
    const size_t per = backproject_candidate_bytes(g);  // one candidate's table + partials
    if (!ws || ws_bytes < per + 2 * 256) return BOAC_EWORKSPACE;
    const size_t fit = (ws_bytes - 2 * 256) / per;
    const int chunk = (int)(fit < (size_t)B ? fit : (size_t)B);
    cudaStream_t st = as_stream(stream);
    char* base = static_cast<char*>(ws);
    float* tab = reinterpret_cast<float*>(base);
    float* partial = reinterpret_cast<float*>(
        base + align256(sizeof(float) * (size_t)chunk * g->n_views * nn));
    for (int c0 = 0; c0 < B; c0 += chunk) {
        const int cb = (B - c0) < chunk ? (B - c0) : chunk;
        attenuation_table_kernel<<<ray_grid(g, cb), kRayThreads, 0, st>>>(
            g->n, g->n_views, g->pixel_cm, mu + c0 * nn, tab);
        int s = launch_status();
        if (s != BOAC_OK) return s;
        s = backproject_table(g, cb, tab, y ? y + (size_t)c0 * g->n_views * g->n_bins : nullptr,
                              g->pixel_cm, out + c0 * nn, 0, partial, st);
        if (s != BOAC_OK) return s;
    }
    return BOAC_OK;
}

extern "C" int boac_loglik(const boac_geom* g, const float* q, const float* S, long long s_stride,
                           int B, int include_lgamma, double* L, void* stream) {
    BOAC_RANGE("boac_loglik");
    if (!geom_ok(g) || !q || !S || !L || B < 1 || s_stride < 0) return BOAC_EINVAL;
    loglik_kernel<<<B, 256, 0, as_stream(stream)>>>(g->n_views * g->n_bins, q, S, s_stride,
                                                     include_lgamma, L, nullptr);
    return launch_status();
}

extern "C" int boac_score(const boac_geom* g, const float* mu, const float* S, long long s_stride,
                          const float* F, int B, int include_lgamma, double* L, void* ws,
                          size_t ws_bytes, void* stream) {
    BOAC_RANGE("boac_score");
    if (!geom_ok(g) || !mu || !S || !F || !L || B < 1 || B > 65535 || s_stride < 0)
        return BOAC_EINVAL;
    const size_t vb = (size_t)g->n_views * g->n_bins;
    if (!ws || ws_bytes < sizeof(float) * vb * B) return BOAC_EWORKSPACE;
    float* q = static_cast<float*>(ws);
    int s = boac_project(g, mu, F, B, q, stream);
    if (s != BOAC_OK) return s;
    return boac_loglik(g, q, S, s_stride, B, include_lgamma, L, stream);
}

extern "C" int boac_mlem_plain(const boac_geom* g, const float* mu, const float* S,
                               long long s_stride, float* F, int K, int B, double* L,
                               int include_lgamma, void* ws, size_t ws_bytes, void* stream) {
    BOAC_RANGE("boac_mlem_plain");
    if (!geom_ok(g) || !mu || !S || !F || B < 1 || K < 0 || s_stride < 0) return BOAC_EINVAL;
    if (!ws || ws_bytes < plain_candidate_bytes(g)) return BOAC_EWORKSPACE;
    const size_t nn = (size_t)g->n * g->n, vb = (size_t)g->n_views * g->n_bins;
    char* base = static_cast<char*>(ws);
    float* tab = reinterpret_cast<float*>(base);
    base += align256(sizeof(float) * vb * g->n);
    float* sens = reinterpret_cast<float*>(base);
    base += align256(sizeof(float) * nn);
    float* bp = reinterpret_cast<float*>(base);
    base += align256(sizeof(float) * nn);
    float* q = reinterpret_cast<float*>(base);
    base += align256(sizeof(float) * vb);
    float* r = reinterpret_cast<float*>(base);
    base += align256(sizeof(float) * vb);
    float* partial = reinterpret_cast<float*>(base);
    cudaStream_t st = as_stream(stream);
    const int V = g->n_views, n = g->n;
    const float dx = g->pixel_cm;
    for (int cand = 0; cand < B; ++cand) {
        const float* m_c = mu + cand * nn;
        const float* S_c = S + (size_t)cand * s_stride;
        float* F_c = F + cand * nn;
        attenuation_table_kernel<<<ray_grid(g, 1), kRayThreads, 0, st>>>(n, V, dx, m_c, tab);
        int s = backproject_table(g, 1, tab, nullptr, dx, sens, 0, partial, st);
        if (s != BOAC_OK) return s;
        for (int it = 0; it < K; ++it) {
            project_table(g, 1, tab, F_c, dx, q, st);
            ratio_kernel<<<grid_1d((long long)vb, 256), 256, 0, st>>>((int)vb, S_c, q, r);
            backproject_table(g, 1, tab, r, dx, bp, 0, partial, st);
            update_kernel<<<grid_1d((long long)nn, 256), 256, 0, st>>>((int)nn, F_c, bp, sens);
        }
        if (L) {
            project_table(g, 1, tab, F_c, dx, q, st);
            loglik_kernel<<<1, 256, 0, st>>>((int)vb, q, S_c, 0, include_lgamma, L + cand, nullptr);
        }
        s = launch_status();
        if (s != BOAC_OK) return s;
    }
    return BOAC_OK;
}

#ifdef BOAC_CHECKED
namespace boac {
BOAC_FAULT_READER(bounds_faults_plain)
}  // namespace boac
#endif
