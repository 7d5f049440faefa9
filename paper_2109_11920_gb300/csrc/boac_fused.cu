// boac_fused.cu -- batched MLEM in one persistent fused kernel (Sec. III,
// step 3: "a fixed number of MLEM iterations ... for each candidate set c_k",
// with the system matrix, forward- and back-projection on the GPU, Sec. III
// last paragraph).
//
// One CTA owns one candidate at a time and keeps its whole state on chip:
//   img0  F (padded n+2 rows x n+1 floats, zero ring)   -- mu during set-up
//   img1  back-projection accumulator (same layout)
//   W     n x (n+1) ray-sample buffer (F samples, then G = dx a r)
// The candidate's "system matrix" -- the attenuation of every ray sample --
// is built once per candidate into a per-CTA slot of the workspace (as
// exp2 exponents) and read back, coalesced, in every iteration.
//
// Four views share one sample grid: with bins and ray samples on the pixel
// pitch, the grids of phi, phi + pi/2, phi + pi and phi + 3pi/2 are the same
// set of points (a quarter turn maps the lattice onto itself), so sample
// (k, b) of view phi + pi is sample (n-1-k, n-1-b) of view phi, and the rays
// of phi + pi/2 and phi + 3pi/2 are the grid's rows.  One bilinear sampling of
// F serves four views (column sums for phi, phi + pi; row sums for the other
// two), and the four views' back-projection weights
//   G = dx (a_phi r_phi + a_{phi+pi} r_{phi+pi} + a_{phi+pi/2} r + a_{phi+3pi/2} r)
// are summed on the grid before ONE transposed-bilinear scatter.  View counts
// that are not a multiple of 4 use pairs (phi, phi + pi) the same way.
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
    float* tab;   // [slots][tab_floats]: attenuation exponents, see below
    float* sens;  // [slots][n][n]
};

// Shared-memory and work layout of one CTA (image side N, NT threads).
template <int N, int NT>
struct FusedShape {
    // Padded image: pixel (i, j), i, j in [-1, n], at (i+1) P + (j+1) with
    // P = n + 1, so the right padding column of row i and the left padding
    // column of row i+1 are the same zero cell; P = 1 (mod 32) for n a
    // multiple of 32 spreads rotated rows of samples over the banks.
    static constexpr int P = N + 1;
    static constexpr int IMG = (N + 1) * (N + 2) + 1;
    static constexpr int NN = N * N;
    static constexpr int WP = N + 1;         // sample-buffer pitch (odd)
    static constexpr int NSEG = NT / N;      // segments per column / row
    static constexpr int SEG = N / NSEG;     // samples per segment
    static_assert(NT % N == 0 && N % NSEG == 0, "segmentation");
};

// Views that share one sample grid: 4 (phi + j pi/2, needs V % 4 == 0) or 2
// (phi, phi + pi).  Attenuation exponents stored per grid, already scaled by
// -dx log2(e) so that a = exp2(y):
//   Xc[k][b] = view phi        (detector at k -> +inf, suffix along k)
//   Uc[b]    = whole-column sum: the view phi + pi exponent is Uc - Xc
//   XrT[b][k] = view phi + pi/2 (detector at b -> -inf, prefix along b),
//               stored transposed for row-parallel access
//   Ur[k]    = whole-row sum: the view phi + 3pi/2 exponent is Ur - XrT
// because for one ray the half-cell sums towards both ends add up to the
// ray's total: a_phi * a_{phi+pi} = exp(-dx sum_k mu_k).
__host__ __device__ constexpr size_t fused_group_floats(int n, bool quad) {
    return quad ? 2 * (size_t)n * n + 2 * (size_t)n : (size_t)n * n + (size_t)n;
}
__host__ __device__ constexpr size_t fused_tab_floats(int n, int V) {
    // V/4 groups of 4 views or V/2 groups of 2: the same total
    return (size_t)(V / 2) * ((size_t)n * n + (size_t)n);
}

template <int N, int NT>
__host__ __device__ constexpr size_t fused_smem_bytes(int V) {
    using L = FusedShape<N, NT>;
    return sizeof(float) * (2 * L::IMG + N * L::WP + 4 * L::NSEG * N + 4 * N + 2 * ((V + 1) / 2) * 2) +
           sizeof(double) * 32;
}

// Scatter G (W, pitch WP) into the padded accumulator img1 with the bilinear
// weights of grid (cs, sn), class by class (see the file comment).
template <int N, int NT>
__device__ __forceinline__ void scatter_classes(const float* __restrict__ W, float* img1, float cs,
                                                float sn, float c) {
    constexpr int P = FusedShape<N, NT>::P, WP = FusedShape<N, NT>::WP;
#pragma unroll
    for (int cls = 0; cls < 9; ++cls) {
        const int pk = cls / 3, pb = cls % 3;
        const int nkc = (N - pk + 2) / 3, nbc = (N - pb + 2) / 3;
        for (int t = threadIdx.x; t < nkc * nbc; t += NT) {
            const int k = pk + 3 * (t / nbc), b = pb + 3 * (t % nbc);
            const float g = W[k * WP + b];
            float u, w;
            sample_uw(k, b, cs, sn, c, &u, &w);
            scatter_padded(img1, P, N, u, w, g);
        }
        __syncthreads();
    }
}

// 2^x with the hardware approximation (relative error about 2^-22).
__device__ __forceinline__ float ex2(float x) {
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

__device__ __forceinline__ double loglik_term(double s, double q, int include_lgamma) {
    double t;
    if (s > 0.0) t = q > 0.0 ? s * log(q) - q : -INFINITY;
    else t = -q;
    if (include_lgamma) t -= lgamma(s + 1.0);
    return t;
}

// CTAs per SM the register allocation is sized for (shared memory allows
// three 64x64 CTAs per SM, one of the larger sizes).
template <int N>
constexpr int fused_min_blocks() { return N <= 64 ? 3 : 1; }

template <int N, int NT, bool QUAD>
__global__ void __launch_bounds__(NT, fused_min_blocks<N>()) mlem_fused_kernel(FusedArgs a) {
    using Lay = FusedShape<N, NT>;
    constexpr int P = Lay::P, IMG = Lay::IMG, NN = Lay::NN, WP = Lay::WP;
    constexpr int NSEG = Lay::NSEG, SEG = Lay::SEG;
    constexpr float kLog2e = 1.44269504088896340736f;
    static_assert(!QUAD || NT >= 2 * N, "row views need 2N threads in the ratio step");

    extern __shared__ __align__(16) float smem[];
    float* img0 = smem;                 // F (mu during set-up), padded
    float* img1 = img0 + IMG;           // back-projection accumulator, padded
    float* W = img1 + IMG;              // [N][WP] grid samples / weights
    float* redc = W + N * WP;           // [2][NSEG][N] column partial sums
    float* redr = redc + 2 * NSEG * N;  // [2][NSEG][N] row partial sums
    float* rr = redr + 2 * NSEG * N;    // [4][N] ratios r = S / q per view
    float* csn = rr + 4 * N;            // [V][2]
    double* dred = reinterpret_cast<double*>(csn + 2 * ((a.V + 1) / 2) * 2);

    const int tid = threadIdx.x;
    const int V = a.V;
    const int ngrid = QUAD ? V / 4 : V / 2;
    const float c = 0.5f * (float)(N - 1);
    const float dx = a.dx;
    const float ndl = -dx * kLog2e;
    // column mapping: thread owns column `lb`, samples k in [k0, k0 + SEG);
    // row mapping: thread owns row `lb`, samples b in [k0, k0 + SEG)
    const int lb = tid % N, seg = tid / N;
    const int k0 = seg * SEG;
    const size_t gstride = fused_group_floats(N, QUAD);

    for (int v = tid; v < V; v += NT) view_cos_sin(v, V, &csn[2 * v], &csn[2 * v + 1]);

    float* tab = a.tab + (size_t)blockIdx.x * fused_tab_floats(N, V);
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

        // ---- system matrix (attenuation exponents) + sensitivity A^T 1
        for (int gi = 0; gi < ngrid; ++gi) {
            const float cs = csn[2 * gi], sn = csn[2 * gi + 1];
            float* Xc = tab + gi * gstride;
            float* XrT = Xc + NN;
            float* Uc = QUAD ? Xc + 2 * NN : Xc + NN;
            float* Ur = Uc + N;
            float ps = 0.0f;
            for (int s = 0; s < SEG; ++s) {
                float u, w;
                sample_uw(k0 + s, lb, cs, sn, c, &u, &w);
                const float m = bilerp_padded(img0, P, N, u, w);
                W[(k0 + s) * WP + lb] = m;
                ps += m;
            }
            redc[seg * N + lb] = ps;
            __syncthreads();
            {   // columns: suffix sums towards k = N-1
                float after = 0.0f, total = 0.0f;
#pragma unroll
                for (int s2 = 0; s2 < NSEG; ++s2) {
                    const float v = redc[s2 * N + lb];
                    total += v;
                    if (s2 > seg) after += v;
                }
                float suf = after;
                for (int s = SEG - 1; s >= 0; --s) {
                    const int k = k0 + s;
                    const float m = W[k * WP + lb];
                    Xc[k * N + lb] = ndl * (0.5f * m + suf);
                    suf += m;
                }
                if (seg == 0) Uc[lb] = ndl * total;
            }
            if (QUAD) {  // rows: prefix sums from b = 0
                float pr = 0.0f;
                for (int s = 0; s < SEG; ++s) pr += W[lb * WP + k0 + s];
                redr[seg * N + lb] = pr;
                __syncthreads();
                float before = 0.0f, total = 0.0f;
#pragma unroll
                for (int s2 = 0; s2 < NSEG; ++s2) {
                    const float v = redr[s2 * N + lb];
                    total += v;
                    if (s2 < seg) before += v;
                }
                float pre = before;
                for (int s = 0; s < SEG; ++s) {
                    const int b = k0 + s;
                    const float m = W[lb * WP + b];
                    XrT[b * N + lb] = ndl * (0.5f * m + pre);
                    pre += m;
                }
                if (seg == 0) Ur[lb] = ndl * total;
            }
            __syncthreads();
            {   // G = dx (sum of the grid's views' attenuation factors)
                const float uc = Uc[lb];
                for (int s = 0; s < SEG; ++s) {
                    const int k = k0 + s;
                    const float y = Xc[k * N + lb];
                    W[k * WP + lb] = dx * (ex2(y) + ex2(uc - y));
                }
            }
            if (QUAD) {
                __syncthreads();
                const float ur = Ur[lb];
                for (int s = 0; s < SEG; ++s) {
                    const int b = k0 + s;
                    const float y = XrT[b * N + lb];
                    W[lb * WP + b] += dx * (ex2(y) + ex2(ur - y));
                }
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

        // ---- MLEM iterations, then one more forward pass for the score
        double lacc = 0.0;
        for (int it = 0; it <= a.K; ++it) {
            const bool scoring = (it == a.K);
            if (scoring && !a.L) break;
            for (int gi = 0; gi < ngrid; ++gi) {
                const float cs = csn[2 * gi], sn = csn[2 * gi + 1];
                const float* Xc = tab + gi * gstride;
                const float* XrT = Xc + NN;
                const float* Uc = QUAD ? Xc + 2 * NN : Xc + NN;
                const float* Ur = Uc + N;
                const int vc1 = gi, vc2 = gi + V / 2;           // column views
                const int vr1 = gi + V / 4, vr2 = gi + 3 * V / 4;  // row views (QUAD)
                // forward, column views: sample F on the grid
                {
                    const float uc = Uc[lb];
                    float acc1 = 0.0f, acc2 = 0.0f;
                    for (int s = 0; s < SEG; ++s) {
                        const int k = k0 + s;
                        float u, w;
                        sample_uw(k, lb, cs, sn, c, &u, &w);
                        const float f = bilerp_padded(img0, P, N, u, w);
                        if (QUAD) W[k * WP + lb] = f;
                        const float y = Xc[k * N + lb];
                        acc1 = fmaf(ex2(y), f, acc1);
                        acc2 = fmaf(ex2(uc - y), f, acc2);
                    }
                    redc[seg * N + lb] = acc1;
                    redc[(NSEG + seg) * N + lb] = acc2;
                }
                if (QUAD) {  // forward, row views: the samples back from W
                    __syncthreads();
                    const float ur = Ur[lb];
                    float acc3 = 0.0f, acc4 = 0.0f;
                    for (int s = 0; s < SEG; ++s) {
                        const int b = k0 + s;
                        const float f = W[lb * WP + b];
                        const float y = XrT[b * N + lb];
                        acc3 = fmaf(ex2(y), f, acc3);
                        acc4 = fmaf(ex2(ur - y), f, acc4);
                    }
                    redr[seg * N + lb] = acc3;
                    redr[(NSEG + seg) * N + lb] = acc4;
                }
                __syncthreads();
                // q, then r = S / q (or the Eq. 5 terms when scoring)
                if (tid < (QUAD ? 2 * N : N)) {
                    const int j = tid % N;
                    const bool row = tid >= N;
                    const float* rp = row ? redr : redc;
                    float q1 = 0.0f, q2 = 0.0f;
#pragma unroll
                    for (int s2 = 0; s2 < NSEG; ++s2) {
                        q1 += rp[s2 * N + j];
                        q2 += rp[(NSEG + s2) * N + j];
                    }
                    q1 *= dx;
                    q2 *= dx;
                    const int v1 = row ? vr1 : vc1, v2 = row ? vr2 : vc2;
                    const float S1 = __ldg(S + (size_t)v1 * N + j);
                    const float S2 = __ldg(S + (size_t)v2 * N + (N - 1 - j));
                    if (scoring) {
                        lacc += loglik_term(S1, q1, a.include_lgamma) + loglik_term(S2, q2, a.include_lgamma);
                    } else {
                        rr[(row ? 2 : 0) * N + j] = q1 > 0.0f ? S1 / q1 : 0.0f;
                        rr[(row ? 3 : 1) * N + j] = q2 > 0.0f ? S2 / q2 : 0.0f;
                    }
                }
                __syncthreads();
                if (scoring) continue;
                // back-projection weights of the grid's views
                {
                    const float uc = Uc[lb];
                    const float r1 = dx * rr[lb], r2 = dx * rr[N + lb];
                    for (int s = 0; s < SEG; ++s) {
                        const int k = k0 + s;
                        const float y = Xc[k * N + lb];
                        W[k * WP + lb] = fmaf(ex2(y), r1, ex2(uc - y) * r2);
                    }
                }
                if (QUAD) {
                    __syncthreads();
                    const float ur = Ur[lb];
                    const float r3 = dx * rr[2 * N + lb], r4 = dx * rr[3 * N + lb];
                    for (int s = 0; s < SEG; ++s) {
                        const int b = k0 + s;
                        const float y = XrT[b * N + lb];
                        W[lb * WP + b] += fmaf(ex2(y), r3, ex2(ur - y) * r4);
                    }
                }
                __syncthreads();
                scatter_classes<N, NT>(W, img1, cs, sn, c);
            }
            if (scoring) break;
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

        // ---- Eq. 5: deterministic block reduction of the float64 terms
        if (a.L) {
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
template <int N, int NT, bool QUAD>
static int fused_occupancy(int V) {
    constexpr int kDev = 16;
    static int cached[kDev][kMaxViews + 1];  // 0 = not yet computed
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0) { cudaGetLastError(); return 0; }
    if (V < 0 || V > kMaxViews) return 0;
    if (dev < kDev && cached[dev][V]) return cached[dev][V];
    size_t smem = fused_smem_bytes<N, NT>(V);
    if (cudaFuncSetAttribute(mlem_fused_kernel<N, NT, QUAD>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)smem) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    int nb = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, mlem_fused_kernel<N, NT, QUAD>, NT, smem) !=
        cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    if (dev < kDev) cached[dev][V] = nb;
    return nb;
}

template <int N, int NT, bool QUAD>
static int fused_launch_t(const FusedArgs& a, int slots, cudaStream_t st) {
    size_t smem = fused_smem_bytes<N, NT>(a.V);
    if (cudaFuncSetAttribute(mlem_fused_kernel<N, NT, QUAD>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)smem) != cudaSuccess)
        return launch_status();
    mlem_fused_kernel<N, NT, QUAD><<<slots, NT, smem, st>>>(a);
    return launch_status();
}

// Four views per sample grid when the view count allows it, else two.
template <int N, int NT>
static int fused_launch(const FusedArgs& a, int slots, cudaStream_t st) {
    return (a.V % 4 == 0) ? fused_launch_t<N, NT, true>(a, slots, st)
                          : fused_launch_t<N, NT, false>(a, slots, st);
}

// Dispatch on the image side: (N, threads per CTA).
#define BOAC_FUSED_SIZES(X) X(64, 256) X(96, 768) X(128, 1024)

// Workspace for `slots` CTA slots: the attenuation-exponent tables, then the
// sensitivity images.  Returns the total bytes; *sens_off the offset of the
// sensitivity images.
static size_t fused_slot_layout(const boac_geom* g, int slots, size_t* sens_off = nullptr) {
    const size_t tab = align256(sizeof(float) * (size_t)slots * fused_tab_floats(g->n, g->n_views));
    if (sens_off) *sens_off = tab;
    return tab + align256(sizeof(float) * (size_t)slots * g->n * g->n);
}

int fused_slots(const boac_geom* g, int B) {
    int per_sm = 0;
#define X(NV, TV)                                                                   \
    if (g->n == NV)                                                                 \
        per_sm = (g->n_views % 4 == 0) ? fused_occupancy<NV, TV, true>(g->n_views) \
                                       : fused_occupancy<NV, TV, false>(g->n_views);
    BOAC_FUSED_SIZES(X)
#undef X
    if (per_sm <= 0) return 0;
    long long slots = (long long)per_sm * sm_count();
    return (int)(slots < B ? slots : B);
}

size_t fused_workspace_bytes(const boac_geom* g, int B) {
    int slots = fused_slots(g, B);
    if (slots <= 0) return 0;
    return fused_slot_layout(g, slots);
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
    size_t sens_off = 0;
    fused_slot_layout(g, slots, &sens_off);
    a.tab = static_cast<float*>(ws);
    a.sens = reinterpret_cast<float*>(static_cast<char*>(ws) + sens_off);
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
    while (slots > 0 && fused_slot_layout(g, slots) > kNoAllocScratchBytes) --slots;
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
    size_t sens_off = 0;
    fused_slot_layout(g, slots, &sens_off);
    a.tab = static_cast<float*>(scratch);
    a.sens = reinterpret_cast<float*>(static_cast<char*>(scratch) + sens_off);
    cudaStream_t st = as_stream(stream);
#define X(NV, TV) \
    if (g->n == NV) return fused_launch<NV, TV>(a, slots, st);
    BOAC_FUSED_SIZES(X)
#undef X
    return BOAC_EUNSUPPORTED;
}
