// boac_bpgroup.cu -- grouped projection and back-projection (Eq. 2 and its
// adjoint) for the unfused paths -- boac_backproject, the launch-per-step
// MLEM and the gradient -- from a table of attenuation factors
// tab[cand][v][k][b]:
//
//   q[cand][v][b] = dx * sum_k tab_v[k][b] F(sample (k, b) of view v)
//   out[cand] (+)= scale * sum_v B_v^T (tab_v * y_v)      (y = 1 if null)
//
// One CTA per (candidate, sample grid): the 4 views phi + j pi/2 (or the 2
// views phi, phi + pi when the view count is not a multiple of 4) share one
// grid of ray samples.  The projector samples F (held in shared memory) on
// the grid and sums along the grid's columns (views phi, phi + pi) and rows
// (the other two).  The back-projector sums the views' weights
// G = scale * sum a_v y_v on the grid in shared memory and scatters them once
// into a shared-memory image with the race-free class scatter; each CTA
// writes its image to its own slice of a workspace and a second kernel sums
// the slices in grid order, so the result is deterministic.  Image sides
// other than 64, 96 and 128 (and odd view counts) use the per-ray and
// per-pixel kernels of boac_plain.cu instead.
#include <cuda_runtime.h>

#include "boac_device.cuh"
#include "boac_internal.h"
#include "boac_plain_kernels.cuh"

namespace boac {

template <int N, int NT, bool QUAD>
__global__ void __launch_bounds__(NT, 1)
    bp_group_kernel(int V, float scale, const float* __restrict__ tab, const float* __restrict__ y,
                    float* __restrict__ partial) {
    constexpr int P = N + 1, IMG = (N + 1) * (N + 2) + 1, WP = N + 1;
    constexpr int NSEG = NT / N, SEG = N / NSEG;
    static_assert(NT % N == 0 && N % NSEG == 0, "segmentation");
    extern __shared__ __align__(16) float smem[];
    float* acc = smem;     // padded image, pixel (i, j) at (i+1) P + (j+1)
    float* W = acc + IMG;  // [N][WP] grid weights G
    const int gi = blockIdx.x, cand = blockIdx.y;
    const int ngrid = QUAD ? V / 4 : V / 2;
    const int tid = threadIdx.x, lb = tid % N, seg = tid / N, k0 = seg * SEG;
    const size_t nn = (size_t)N * N;
    const float* tb = tab + (size_t)cand * V * nn;
    const float* yc = y ? y + (size_t)cand * V * N : nullptr;
    float cs, sn;
    view_cos_sin(gi, V, &cs, &sn);
    const float c = 0.5f * (float)(N - 1);
    for (int i = tid; i < IMG; i += NT) acc[i] = 0.0f;
    // views phi (sample (k, b)) and phi + pi (its sample (n-1-k, n-1-b)):
    // column-parallel, coalesced along b
    {
        const int v1 = gi, v2 = gi + V / 2;
        const float y1 = yc ? __ldg(yc + (size_t)v1 * N + lb) : 1.0f;
        const float y2 = yc ? __ldg(yc + (size_t)v2 * N + (N - 1 - lb)) : 1.0f;
        const float* t1 = tb + (size_t)v1 * nn;
        const float* t2 = tb + (size_t)v2 * nn;
        for (int s = 0; s < SEG; ++s) {
            const int k = k0 + s;
            W[k * WP + lb] = scale * fmaf(__ldg(t1 + (size_t)k * N + lb), y1,
                                          __ldg(t2 + (size_t)(N - 1 - k) * N + (N - 1 - lb)) * y2);
        }
    }
    if (QUAD) {
        // views phi + pi/2 (its sample (n-1-b, k)) and phi + 3pi/2 (its
        // sample (b, n-1-k)): row-parallel, coalesced along k
        __syncthreads();
        const int v3 = gi + V / 4, v4 = gi + 3 * V / 4;
        const int k = lb;
        const float y3 = yc ? __ldg(yc + (size_t)v3 * N + k) : 1.0f;
        const float y4 = yc ? __ldg(yc + (size_t)v4 * N + (N - 1 - k)) : 1.0f;
        const float* t3 = tb + (size_t)v3 * nn;
        const float* t4 = tb + (size_t)v4 * nn;
        for (int s = 0; s < SEG; ++s) {
            const int b = k0 + s;
            W[k * WP + b] += scale * fmaf(__ldg(t3 + (size_t)(N - 1 - b) * N + k), y3,
                                          __ldg(t4 + (size_t)b * N + (N - 1 - k)) * y4);
        }
    }
    __syncthreads();
    scatter_classes<N, NT, P, WP>(W, acc, cs, sn, c);
    float* out = partial + ((size_t)cand * ngrid + gi) * nn;
    for (int i = tid; i < (int)nn; i += NT) out[i] = acc[(i / N + 1) * P + (i % N) + 1];
}

// q for the grid's views from the padded image of F in shared memory:
// column pass (thread: column lb, samples k in its segment) for views phi
// and phi + pi, row pass (thread: row lb, samples b in its segment) for
// phi + pi/2 (sample (n-1-b, k) of that view) and phi + 3pi/2 (sample
// (b, n-1-k)); segment sums reduced in segment order.
template <int N, int NT, bool QUAD>
__global__ void __launch_bounds__(NT) project_group_kernel(int V, float dx, const float* __restrict__ tab,
                                                          const float* __restrict__ F, float* __restrict__ q) {
    constexpr int P = N + 1, IMG = (N + 1) * (N + 2) + 1;
    constexpr int NSEG = NT / N, SEG = N / NSEG;
    static_assert(NT % N == 0 && N % NSEG == 0, "segmentation");
    extern __shared__ __align__(16) float smem[];
    float* img = smem;      // padded F, pixel (i, j) at (i+1) P + (j+1)
    float* red = img + IMG;  // [4][NSEG][N] segment sums
    const int gi = blockIdx.x, cand = blockIdx.y;
    const int tid = threadIdx.x, lb = tid % N, seg = tid / N, k0 = seg * SEG;
    const size_t nn = (size_t)N * N;
    const float* tb = tab + (size_t)cand * V * nn;
    const float* f = F + (size_t)cand * nn;
    for (int i = tid; i < IMG; i += NT) img[i] = 0.0f;
    __syncthreads();
    for (int i = tid; i < (int)nn; i += NT) img[(i / N + 1) * P + (i % N) + 1] = __ldg(f + i);
    __syncthreads();
    float cs, sn;
    view_cos_sin(gi, V, &cs, &sn);
    const float c = 0.5f * (float)(N - 1);
    const int v1 = gi, v2 = gi + V / 2, v3 = gi + V / 4, v4 = gi + 3 * V / 4;
    {
        const float* t1 = tb + (size_t)v1 * nn;
        const float* t2 = tb + (size_t)v2 * nn;
        float a1 = 0.0f, a2 = 0.0f;
        for (int s = 0; s < SEG; ++s) {
            const int k = k0 + s;
            float u, w;
            sample_uw(k, lb, cs, sn, c, &u, &w);
            const float fv = bilerp_padded(img, P, N, u, w);
            a1 = fmaf(__ldg(t1 + (size_t)k * N + lb), fv, a1);
            a2 = fmaf(__ldg(t2 + (size_t)(N - 1 - k) * N + (N - 1 - lb)), fv, a2);
        }
        red[seg * N + lb] = a1;
        red[(NSEG + seg) * N + lb] = a2;
    }
    if (QUAD) {
        const float* t3 = tb + (size_t)v3 * nn;
        const float* t4 = tb + (size_t)v4 * nn;
        const int k = lb;
        float a3 = 0.0f, a4 = 0.0f;
        for (int s = 0; s < SEG; ++s) {
            const int b = k0 + s;
            float u, w;
            sample_uw(k, b, cs, sn, c, &u, &w);
            const float fv = bilerp_padded(img, P, N, u, w);
            a3 = fmaf(__ldg(t3 + (size_t)(N - 1 - b) * N + k), fv, a3);
            a4 = fmaf(__ldg(t4 + (size_t)b * N + (N - 1 - k)), fv, a4);
        }
        red[(2 * NSEG + seg) * N + lb] = a3;
        red[(3 * NSEG + seg) * N + lb] = a4;
    }
    __syncthreads();
    for (int t = tid; t < (QUAD ? 4 : 2) * N; t += NT) {
        const int vi = t / N, j = t % N;
        float sum = 0.0f;
#pragma unroll
        for (int s2 = 0; s2 < NSEG; ++s2) sum += red[(vi * NSEG + s2) * N + j];
        const int v = vi == 0 ? v1 : vi == 1 ? v2 : vi == 2 ? v3 : v4;
        q[((size_t)cand * V + v) * N + ((vi & 1) ? N - 1 - j : j)] = dx * sum;
    }
}

// out[cand][pix] (+)= sum over grids of partial[cand][grid][pix], grid order.
__global__ void sum_grids_kernel(int B, int ngrid, int nn, const float* __restrict__ partial,
                                 float* __restrict__ out, int accumulate) {
    const long long total = (long long)B * nn;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
         i += (long long)gridDim.x * blockDim.x) {
        const long long cand = i / nn, pix = i % nn;
        const float* p = partial + cand * ngrid * (long long)nn + pix;
        float s = 0.0f;
        for (int g = 0; g < ngrid; ++g) s += p[(long long)g * nn];
        out[i] = accumulate ? out[i] + s : s;
    }
}

template <int N, int NT, bool QUAD>
static int bp_group_launch(int V, int B, float scale, const float* tab, const float* y, float* partial,
                           cudaStream_t st) {
    constexpr size_t smem = sizeof(float) * ((size_t)(N + 1) * (N + 2) + 1 + (size_t)N * (N + 1));
    constexpr int kDev = 64;
    static bool attr_set[kDev];
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kDev) return launch_status();
    if (!attr_set[dev]) {
        if (cudaFuncSetAttribute(bp_group_kernel<N, NT, QUAD>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)smem) != cudaSuccess)
            return launch_status();
        attr_set[dev] = true;
    }
    const int ngrid = QUAD ? V / 4 : V / 2;
    bp_group_kernel<N, NT, QUAD><<<dim3(ngrid, B), NT, smem, st>>>(V, scale, tab, y, partial);
    return launch_status();
}

template <int N, int NT, bool QUAD>
static int project_group_launch(int V, int B, float dx, const float* tab, const float* F, float* q,
                                cudaStream_t st) {
    constexpr size_t smem = sizeof(float) * ((size_t)(N + 1) * (N + 2) + 1 + 4 * (size_t)N * (NT / N));
    constexpr int kDev = 64;
    static bool attr_set[kDev];
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kDev) return launch_status();
    if (!attr_set[dev]) {
        if (cudaFuncSetAttribute(project_group_kernel<N, NT, QUAD>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)smem) != cudaSuccess)
            return launch_status();
        attr_set[dev] = true;
    }
    const int ngrid = QUAD ? V / 4 : V / 2;
    project_group_kernel<N, NT, QUAD><<<dim3(ngrid, B), NT, smem, st>>>(V, dx, tab, F, q);
    return launch_status();
}

// Whether the grouped kernels handle this geometry.
static bool bp_grouped(const boac_geom* g) {
    return (g->n == 64 || g->n == 96 || g->n == 128) && g->n_views % 2 == 0;
}

size_t bp_partial_floats(const boac_geom* g, int B) {
    if (!bp_grouped(g)) return 0;
    const int ngrid = g->n_views % 4 == 0 ? g->n_views / 4 : g->n_views / 2;
    return (size_t)B * ngrid * g->n * g->n;
}

int backproject_table(const boac_geom* g, int B, const float* tab, const float* y, float scale, float* out,
                      int accumulate, float* partial, cudaStream_t st) {
    const int n = g->n, V = g->n_views;
    if (!bp_grouped(g) || !partial) {
        const dim3 pg((unsigned)(((size_t)n * n + kPixThreads - 1) / kPixThreads), B);
        backproject_gather_kernel<<<pg, kPixThreads, sizeof(float) * 2 * V, st>>>(n, V, scale, tab, y, out,
                                                                                 accumulate);
        return launch_status();
    }
    const bool quad = V % 4 == 0;
    int s = BOAC_EUNSUPPORTED;
#define X(NV, TV)                                                                       \
    if (n == NV)                                                                        \
        s = quad ? bp_group_launch<NV, TV, true>(V, B, scale, tab, y, partial, st)      \
                 : bp_group_launch<NV, TV, false>(V, B, scale, tab, y, partial, st);
    X(64, 256) X(96, 768) X(128, 1024)
#undef X
    if (s != BOAC_OK) return s;
    const int ngrid = quad ? V / 4 : V / 2;
    const long long total = (long long)B * n * n;
    sum_grids_kernel<<<grid_1d(total, 256), 256, 0, st>>>(B, ngrid, n * n, partial, out, accumulate);
    return launch_status();
}

int project_table(const boac_geom* g, int B, const float* tab, const float* F, float dx, float* q,
                  cudaStream_t st) {
    const int n = g->n, V = g->n_views;
    if (!bp_grouped(g)) {
        project_table_kernel<<<ray_grid(g, B), kRayThreads, 0, st>>>(n, V, dx, tab, F, q);
        return launch_status();
    }
    const bool quad = V % 4 == 0;
    int s = BOAC_EUNSUPPORTED;
#define X(NV, TV)                                                                \
    if (n == NV)                                                                 \
        s = quad ? project_group_launch<NV, TV, true>(V, B, dx, tab, F, q, st)   \
                 : project_group_launch<NV, TV, false>(V, B, dx, tab, F, q, st);
    X(64, 256) X(96, 384) X(128, 512)
#undef X
    return s;
}

#ifdef BOAC_CHECKED
BOAC_FAULT_READER(bounds_faults_bpgroup)
#endif

}  // namespace boac
