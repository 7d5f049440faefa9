// boac_fused.cu -- batched MLEM in one persistent fused kernel (Sec. III,
// step 3: "a fixed number of MLEM iterations ... for each candidate set c_k",
// with the system matrix, forward- and back-projection on the GPU, Sec. III
// last paragraph).
//
// One CTA owns one candidate at a time and keeps its whole state on chip:
//   img0  F (padded n+2 rows x n+3 floats, zero ring)   -- mu during set-up
//   img1  back-projection accumulator (same layout)
//   W     n x n ray-sample buffer (attenuation sums, then G = dx a r)
// The candidate's "system matrix" -- the attenuation factor of every ray
// sample -- is built once per candidate into a per-CTA slot of the workspace
// and read back (coalesced, from L2/HBM) in every iteration.
//
// Views phi and phi + pi share one sample grid: sample (k, b) of view
// v + V/2 is sample (n-1-k, n-1-b) of view v, so one bilinear sampling of F
// serves two views, the two attenuation factors differ only in the scan
// direction (suffix vs prefix along k), and the two views' back-projection
// weights G = dx (a_v r_v + a_{v+V/2} r_{v+V/2}) are summed on the grid
// before ONE transposed-bilinear scatter.
//
// The scatter is race-free and deterministic without atomics: the samples
// are split into 9 classes by (k mod 3, b mod 3); two samples of one class
// are >= 3 lattice steps apart, i.e. >= 3/sqrt(2) > 2 pixels apart along
// some image axis, so their 2x2 pixel footprints are disjoint.
#include <cuda_runtime.h>
#include <math.h>

#include "boac_device.cuh"
#include "boac_internal.h"

namespace boac {

struct FusedArgs {
    const float* mu;
    const float* S;
    long long s_stride;
    float* F;
    double* L;
    int include_lgamma;
    int B, V, K;
    float dx;
    // Per-CTA slots, written and read by the same CTA within one launch:
    // read with plain (coherent) loads, never through the read-only path.
    float* tab;   // [slots][V][n][n]: pair p -> planes 2p (view p), 2p+1 (view p+V/2)
    float* sens;  // [slots][n][n]
};

template <int N>
struct FusedShape {
    static constexpr int P = N + 3;          // padded row pitch (odd)
    static constexpr int IMG = (N + 2) * P;  // floats per padded image
    static constexpr int NN = N * N;
};

template <int N, int NT>
__host__ __device__ constexpr size_t fused_smem_bytes(int V) {
    return sizeof(float) * (2 * FusedShape<N>::IMG + FusedShape<N>::NN + (NT / N) * 2 * N + 2 * N +
                            2 * ((V + 1) / 2) * 2) +
           sizeof(double) * 32;
}

// Scatter G (W, n x n) into the padded accumulator img1 with the bilinear
// weights of grid (cs, sn), class by class (see the file comment).
template <int N, int NT>
__device__ __forceinline__ void scatter_classes(const float* __restrict__ W, float* img1, float cs,
                                                float sn, float c) {
    constexpr int P = FusedShape<N>::P;
#pragma unroll
    for (int cls = 0; cls < 9; ++cls) {
        const int pk = cls / 3, pb = cls % 3;
        const int nkc = (N - pk + 2) / 3, nbc = (N - pb + 2) / 3;
        for (int t = threadIdx.x; t < nkc * nbc; t += NT) {
            const int k = pk + 3 * (t / nbc), b = pb + 3 * (t % nbc);
            const float g = W[k * N + b];
            float u, w;
            sample_uw(k, b, cs, sn, c, &u, &w);
            scatter_padded(img1, P, N, u, w, g);
        }
        __syncthreads();
    }
}

// CTAs per SM the register allocation is sized for (shared memory allows
// about four 64x64 CTAs per SM, one of the larger sizes).
template <int N>
constexpr int fused_min_blocks() { return N <= 64 ? 4 : 1; }

template <int N, int NT>
__global__ void __launch_bounds__(NT, fused_min_blocks<N>()) mlem_fused_kernel(FusedArgs a) {
    constexpr int P = FusedShape<N>::P, IMG = FusedShape<N>::IMG, NN = FusedShape<N>::NN;
    constexpr int NSEG = NT / N, SEG = N / NSEG;
    static_assert(NT % N == 0 && N % NSEG == 0, "column segmentation");

    extern __shared__ __align__(16) float smem[];
    float* img0 = smem;
    float* img1 = img0 + IMG;
    float* W = img1 + IMG;
    float* red = W + NN;            // [NSEG][2][N]
    float* r1 = red + NSEG * 2 * N; // [N]
    float* r2 = r1 + N;             // [N]
    float* csn = r2 + N;            // [V][2]
    double* dred = reinterpret_cast<double*>(csn + 2 * ((a.V + 1) / 2) * 2);

    const int tid = threadIdx.x;
    const int V = a.V, half = V / 2;
    const float c = 0.5f * (float)(N - 1);
    const float dx = a.dx;
    const int bcol = tid % N, seg = tid / N;
    const int k0 = seg * SEG;

    for (int v = tid; v < V; v += NT) view_cos_sin(v, V, &csn[2 * v], &csn[2 * v + 1]);

    float* tab = a.tab + (size_t)blockIdx.x * V * NN;
    float* sens = a.sens + (size_t)blockIdx.x * NN;

    for (int cand = blockIdx.x; cand < a.B; cand += gridDim.x) {
        const float* __restrict__ S = a.S + (size_t)cand * a.s_stride;
        const float* __restrict__ mu = a.mu + (size_t)cand * NN;

        // ---- set-up: mu -> img0 (zero ring), img1 = 0
        for (int i = tid; i < IMG; i += NT) {
            img0[i] = 0.0f;
            img1[i] = 0.0f;
        }
        __syncthreads();
        for (int i = tid; i < NN; i += NT) img0[(i / N + 1) * P + (i % N) + 1] = __ldg(mu + i);
        __syncthreads();

        // ---- system matrix (attenuation factors) + sensitivity A^T 1
        for (int p = 0; p < half; ++p) {
            const float cs = csn[2 * p], sn = csn[2 * p + 1];
            float* t1 = tab + (size_t)(2 * p) * NN;      // view p: suffix along k
            float* t2 = tab + (size_t)(2 * p + 1) * NN;  // view p+V/2: prefix along k
            float ssum = 0.0f;
            for (int s = 0; s < SEG; ++s) {
                float u, w;
                sample_uw(k0 + s, bcol, cs, sn, c, &u, &w);
                float m = bilerp_padded(img0, P, N, u, w);
                W[(k0 + s) * N + bcol] = m;
                ssum += m;
            }
            red[seg * N + bcol] = ssum;
            __syncthreads();
            float before = 0.0f, after = 0.0f;
#pragma unroll
            for (int s2 = 0; s2 < NSEG; ++s2) {
                float v = red[s2 * N + bcol];
                if (s2 < seg) before += v;
                if (s2 > seg) after += v;
            }
            float pre = before;
            for (int s = 0; s < SEG; ++s) {
                const int k = k0 + s;
                float m = W[k * N + bcol];
                t2[k * N + bcol] = expf(-dx * (0.5f * m + pre));
                pre += m;
            }
            float suf = after;
            for (int s = SEG - 1; s >= 0; --s) {
                const int k = k0 + s;
                float m = W[k * N + bcol];
                float a1 = expf(-dx * (0.5f * m + suf));
                suf += m;
                t1[k * N + bcol] = a1;
                W[k * N + bcol] = dx * (a1 + t2[k * N + bcol]);
            }
            __syncthreads();
            scatter_classes<N, NT>(W, img1, cs, sn, c);
        }
        for (int i = tid; i < NN; i += NT) {
            const int pi = (i / N + 1) * P + (i % N) + 1;
            sens[i] = img1[pi];
            img0[pi] = a.F[(size_t)cand * NN + i];
        }
        __syncthreads();
        for (int i = tid; i < IMG; i += NT) img1[i] = 0.0f;
        __syncthreads();

        // ---- MLEM iterations
        for (int it = 0; it < a.K; ++it) {
            for (int p = 0; p < half; ++p) {
                const float cs = csn[2 * p], sn = csn[2 * p + 1];
                const float* t1 = tab + (size_t)(2 * p) * NN;
                const float* t2 = tab + (size_t)(2 * p + 1) * NN;
                // forward: sample F on the grid and reduce both views' columns
                float acc1 = 0.0f, acc2 = 0.0f;
                for (int s = 0; s < SEG; ++s) {
                    const int k = k0 + s;
                    float u, w;
                    sample_uw(k, bcol, cs, sn, c, &u, &w);
                    float f = bilerp_padded(img0, P, N, u, w);
                    acc1 = fmaf(t1[k * N + bcol], f, acc1);
                    acc2 = fmaf(t2[k * N + bcol], f, acc2);
                }
                red[(seg * 2 + 0) * N + bcol] = acc1;
                red[(seg * 2 + 1) * N + bcol] = acc2;
                __syncthreads();
                if (tid < N) {
                    float q1 = 0.0f, q2 = 0.0f;
#pragma unroll
                    for (int s2 = 0; s2 < NSEG; ++s2) {
                        q1 += red[(s2 * 2 + 0) * N + tid];
                        q2 += red[(s2 * 2 + 1) * N + tid];
                    }
                    q1 *= dx;
                    q2 *= dx;
                    const float S1 = __ldg(S + (size_t)p * N + tid);
                    const float S2 = __ldg(S + (size_t)(p + half) * N + (N - 1 - tid));
                    r1[tid] = q1 > 0.0f ? S1 / q1 : 0.0f;
                    r2[tid] = q2 > 0.0f ? S2 / q2 : 0.0f;
                }
                __syncthreads();
                // back-projection weights of both views on the shared grid
                const float rr1 = dx * r1[bcol], rr2 = dx * r2[bcol];
                for (int s = 0; s < SEG; ++s) {
                    const int k = k0 + s;
                    W[k * N + bcol] = fmaf(t1[k * N + bcol], rr1, t2[k * N + bcol] * rr2);
                }
                __syncthreads();
                scatter_classes<N, NT>(W, img1, cs, sn, c);
            }
            // multiplicative update; clears the accumulator for the next pass
            for (int i = tid; i < IMG; i += NT) {
                const int row = i / P, col = i % P;
                if (row >= 1 && row <= N && col >= 1 && col <= N) {
                    const float sv = sens[(row - 1) * N + (col - 1)];
                    img0[i] = sv > 0.0f ? img0[i] * img1[i] / sv : 0.0f;
                }
                img1[i] = 0.0f;
            }
            __syncthreads();
        }

        // ---- Eq. 5 score of F^K (float32 projection, float64 reduction)
        if (a.L) {
            double lacc = 0.0;
            for (int p = 0; p < half; ++p) {
                const float cs = csn[2 * p], sn = csn[2 * p + 1];
                const float* t1 = tab + (size_t)(2 * p) * NN;
                const float* t2 = tab + (size_t)(2 * p + 1) * NN;
                float acc1 = 0.0f, acc2 = 0.0f;
                for (int s = 0; s < SEG; ++s) {
                    const int k = k0 + s;
                    float u, w;
                    sample_uw(k, bcol, cs, sn, c, &u, &w);
                    float f = bilerp_padded(img0, P, N, u, w);
                    acc1 = fmaf(t1[k * N + bcol], f, acc1);
                    acc2 = fmaf(t2[k * N + bcol], f, acc2);
                }
                red[(seg * 2 + 0) * N + bcol] = acc1;
                red[(seg * 2 + 1) * N + bcol] = acc2;
                __syncthreads();
                if (tid < N) {
                    float q1 = 0.0f, q2 = 0.0f;
#pragma unroll
                    for (int s2 = 0; s2 < NSEG; ++s2) {
                        q1 += red[(s2 * 2 + 0) * N + tid];
                        q2 += red[(s2 * 2 + 1) * N + tid];
                    }
                    q1 *= dx;
                    q2 *= dx;
                    const double S1 = __ldg(S + (size_t)p * N + tid);
                    const double S2 = __ldg(S + (size_t)(p + half) * N + (N - 1 - tid));
                    const double qq[2] = {(double)q1, (double)q2}, ss[2] = {S1, S2};
#pragma unroll
                    for (int e = 0; e < 2; ++e) {
                        double term;
                        if (ss[e] > 0.0) term = qq[e] > 0.0 ? ss[e] * log(qq[e]) - qq[e] : -INFINITY;
                        else term = -qq[e];
                        if (a.include_lgamma) term -= lgamma(ss[e] + 1.0);
                        lacc += term;
                    }
                }
                __syncthreads();
            }
            // deterministic block reduction (threads >= N hold 0)
            for (int off = 16; off > 0; off >>= 1) lacc += __shfl_down_sync(0xffffffffu, lacc, off);
            if ((tid & 31) == 0) dred[tid >> 5] = lacc;
            __syncthreads();
            if (tid == 0) {
                double t = 0.0;
                for (int wi = 0; wi < NT / 32; ++wi) t += dred[wi];
                a.L[cand] = t;
            }
        }

        // ---- F^K out
        for (int i = tid; i < NN; i += NT) a.F[(size_t)cand * NN + i] = img0[(i / N + 1) * P + (i % N) + 1];
        __syncthreads();
    }
}

// ---------------------------------------------------------------- host side
template <int N, int NT>
static int fused_occupancy(int V) {
    constexpr int kDev = 16;
    static int cached[kDev][kMaxViews + 1];  // 0 = not yet computed
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0) { cudaGetLastError(); return 0; }
    if (V < 0 || V > kMaxViews) return 0;
    if (dev < kDev && cached[dev][V]) return cached[dev][V];
    size_t smem = fused_smem_bytes<N, NT>(V);
    if (cudaFuncSetAttribute(mlem_fused_kernel<N, NT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)smem) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    int nb = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, mlem_fused_kernel<N, NT>, NT, smem) !=
        cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    if (dev < kDev) cached[dev][V] = nb;
    return nb;
}

template <int N, int NT>
static int fused_launch(const FusedArgs& a, int slots, cudaStream_t st) {
    size_t smem = fused_smem_bytes<N, NT>(a.V);
    if (cudaFuncSetAttribute(mlem_fused_kernel<N, NT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)smem) != cudaSuccess)
        return launch_status();
    mlem_fused_kernel<N, NT><<<slots, NT, smem, st>>>(a);
    return launch_status();
}

// Dispatch on the image side: (N, threads per CTA).
#define BOAC_FUSED_SIZES(X) X(64, 256) X(96, 768) X(128, 1024)

int fused_slots(const boac_geom* g, int B) {
    int per_sm = 0;
#define X(NV, TV) \
    if (g->n == NV) per_sm = fused_occupancy<NV, TV>(g->n_views);
    BOAC_FUSED_SIZES(X)
#undef X
    if (per_sm <= 0) return 0;
    long long slots = (long long)per_sm * sm_count();
    return (int)(slots < B ? slots : B);
}

size_t fused_workspace_bytes(const boac_geom* g, int B) {
    int slots = fused_slots(g, B);
    if (slots <= 0) return 0;
    size_t nn = (size_t)g->n * g->n;
    return align256(sizeof(float) * (size_t)slots * nn * g->n_views) +
           align256(sizeof(float) * (size_t)slots * nn);
}

}  // namespace boac

using namespace boac;

extern "C" int boac_mlem(const boac_geom* g, const float* mu, const float* S, long long s_stride,
                         float* F, int K, int B, double* L, int include_lgamma, void* ws,
                         size_t ws_bytes, void* stream) {
    if (!geom_ok(g) || !mu || !S || !F || B < 1 || K < 0 || s_stride < 0) return BOAC_EINVAL;
    if (g->n_views % 2) return BOAC_EINVAL;
    bool have = false;
#define X(NV, TV) have |= (g->n == NV);
    BOAC_FUSED_SIZES(X)
#undef X
    if (!have) return BOAC_EUNSUPPORTED;
    int slots = fused_slots(g, B);
    if (slots <= 0) return BOAC_ECUDA;
    size_t need = fused_workspace_bytes(g, B);
    if (!ws || ws_bytes < need) return BOAC_EWORKSPACE;
    size_t nn = (size_t)g->n * g->n;
    FusedArgs a;
    a.mu = mu;
    a.S = S;
    a.s_stride = s_stride;
    a.F = F;
    a.L = L;
    a.include_lgamma = include_lgamma;
    a.B = B;
    a.V = g->n_views;
    a.K = K;
    a.dx = g->pixel_cm;
    a.tab = static_cast<float*>(ws);
    a.sens = reinterpret_cast<float*>(static_cast<char*>(ws) +
                                      align256(sizeof(float) * (size_t)slots * nn * g->n_views));
    cudaStream_t st = as_stream(stream);
#define X(NV, TV) \
    if (g->n == NV) return fused_launch<NV, TV>(a, slots, st);
    BOAC_FUSED_SIZES(X)
#undef X
    return BOAC_EUNSUPPORTED;
}

// ---------------------------------------------------------------------------
// Allocation-free variant of boac_mlem.
//
// Some callers cannot allocate device memory at the moment they want a
// reconstruction: code running inside another framework's memory pool or
// allocator lock, a callback that must not call cudaMalloc (which can
// synchronise the device), or a host process that has no allocator of its
// own to hand the library a workspace.  boac_mlem_noalloc takes the fused
// kernel's scratch (per-CTA attenuation tables and sensitivity images) from
// a fixed array compiled into this library instead of from a caller
// workspace.  The array lives in device memory on every GPU that loads the
// library, for as long as the process runs.
namespace boac {

// Size of the built-in scratch: 64 MiB.
constexpr size_t kNoAllocScratchBytes = size_t(64) << 20;
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

// Device address of g_noalloc_scratch, looked up once per device.  In host
// code the array's name stands for a host-side shadow, not device memory,
// so the kernel must be given the address cudaGetSymbolAddress returns.
static void* noalloc_scratch_ptr() {
    constexpr int kDev = 64;
    static void* cached[kDev];
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kDev) {
        cudaGetLastError();
        return nullptr;
    }
    if (!cached[dev]) {
        void* p = nullptr;
        if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) {
            cudaGetLastError();
            return nullptr;
        }
        cached[dev] = p;
    }
    return cached[dev];
}

// Largest number of resident CTA slots whose tables and sensitivity images
// fit the built-in scratch (0 if not even one does).
static int noalloc_slots(const boac_geom* g, int B) {
    int slots = fused_slots(g, B);
    const size_t nn = (size_t)g->n * g->n;
    while (slots > 0 && align256(sizeof(float) * (size_t)slots * nn * g->n_views) +
                                align256(sizeof(float) * (size_t)slots * nn) >
                            kNoAllocScratchBytes)
        --slots;
    return slots;
}

}  // namespace boac

extern "C" int boac_mlem_noalloc(const boac_geom* g, const float* mu, const float* S,
                                 long long s_stride, float* F, int K, int B, double* L,
                                 int include_lgamma, void* stream) {
    if (!geom_ok(g) || !mu || !S || !F || B < 1 || K < 0 || s_stride < 0) return BOAC_EINVAL;
    if (g->n_views % 2) return BOAC_EINVAL;
    bool have = false;
#define X(NV, TV) have |= (g->n == NV);
    BOAC_FUSED_SIZES(X)
#undef X
    if (!have) return BOAC_EUNSUPPORTED;
    if (fused_slots(g, B) <= 0) return BOAC_ECUDA;
    const int slots = noalloc_slots(g, B);
    if (slots <= 0) return BOAC_EWORKSPACE;  // one candidate's scratch exceeds 64 MiB
    void* scratch = noalloc_scratch_ptr();
    if (!scratch) return BOAC_ECUDA;
    const size_t nn = (size_t)g->n * g->n;
    FusedArgs a;
    a.mu = mu;
    a.S = S;
    a.s_stride = s_stride;
    a.F = F;
    a.L = L;
    a.include_lgamma = include_lgamma;
    a.B = B;
    a.V = g->n_views;
    a.K = K;
    a.dx = g->pixel_cm;
    // The kernel writes every table entry and sensitivity pixel of a slot
    // before reading it, so the scratch needs no clearing between calls.
    a.tab = static_cast<float*>(scratch);
    a.sens = reinterpret_cast<float*>(static_cast<char*>(scratch) +
                                      align256(sizeof(float) * (size_t)slots * nn * g->n_views));
    cudaStream_t st = as_stream(stream);
#define X(NV, TV) \
    if (g->n == NV) return fused_launch<NV, TV>(a, slots, st);
    BOAC_FUSED_SIZES(X)
#undef X
    return BOAC_EUNSUPPORTED;
}
