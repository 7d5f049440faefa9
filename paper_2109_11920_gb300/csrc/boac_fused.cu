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

#include <algorithm>
#include <atomic>
#include <vector>

#include <cooperative_groups.h>

#include "boac_device.cuh"
#include "boac_fused.h"
#include "boac_internal.h"
#include "boac_plain_kernels.cuh"
#include "boac_sched.cuh"

namespace cg = cooperative_groups;

namespace boac {

// Shared-memory and work layout of one CTA (image side N, NT threads).
template <int N, int NT>
struct FusedShape {
    // Padded image: pixel (i, j), i, j in [-1, n], at (i+1) P + (j+1) with
    // P = n + 1, so the right padding column of row i and the left padding
    // column of row i+1 are the same zero cell; P = 1 (mod 32) for n a
    // multiple of 32 spreads rotated rows of samples over the banks.
    static constexpr int P = N + 1;
    static constexpr int IMG = (N + 1) * (N + 2) + 1;
    static constexpr int IMGA = (IMG + 3) & ~3;  // an image's floats, rounded to 16 bytes
    static constexpr int NN = N * N;
    // Sample-buffer pitch: rows start 16 bytes apart in whole groups, and a
    // quarter-warp's 16-byte row accesses (threads on consecutive rows) fall
    // on 8 different 16-byte bank groups since (N + 4) / 4 is odd.
    static constexpr int WP = N + 4;
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
// (the planes in the interleaved order of tab_ix below)
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
// The attenuation exponents one CTA keeps: all grids (G = 1), or in cluster
// mode the grids of one of G ranks, at most ceil(grids / G).
__host__ __device__ constexpr size_t fused_tab_floats(int n, int V, bool quad, int G) {
    return G <= 1 ? fused_tab_floats(n, V)
                  : (size_t)(((quad ? V / 4 : V / 2) + G - 1) / G) * fused_group_floats(n, quad);
}

// Whether the images of an n x n candidate live in global memory.
__host__ __device__ constexpr bool fused_global_images(int n) { return n > 128; }

template <int N, int NT>
__host__ __device__ constexpr size_t fused_image_floats() {
    using L = FusedShape<N, NT>;
    return 2 * (size_t)L::IMGA + (size_t)N * L::WP;
}

template <int N, int NT>
__host__ __device__ constexpr size_t fused_smem_bytes(int V) {
    using L = FusedShape<N, NT>;
    return sizeof(float) * ((fused_global_images(N) ? 0 : fused_image_floats<N, NT>()) +
                            4 * L::NSEG * N + 8 * N + 2 * ((V + 1) / 2) * 2) +
           sizeof(double) * 33;
}

// CTAs per SM the register allocation is sized for: as many as shared memory
// allows (three 64x64 CTAs, one of the larger sizes), but no fewer than 64
// registers per thread.
template <int N, int NT>
constexpr int fused_min_blocks() {
    return (N <= 64 ? 3 : 1) < 1024 / NT ? (N <= 64 ? 3 : 1) : (1024 / NT > 0 ? 1024 / NT : 1);
}

// The scatter schedule of grid gi (images up to 128 x 128 only).
template <int N>
__device__ __forceinline__ const unsigned short* grid_sched(const FusedArgs& a, int gi) {
    return a.sched + (size_t)gi * 9 * SchedShape<(N <= 128 ? N : 128)>::CLS_ENTRIES;
}

// G = 1: one CTA per candidate at a time (the batch's iterations split over
// the CTAs).  G > 1 (cluster mode, for batches too small to fill the GPU one
// CTA per candidate): a thread-block cluster of G CTAs per candidate, CTA
// rank r working on the sample grids [r V' / G, (r + 1) V' / G) (V' grids)
// with its own copy of F and its own accumulator; after every iteration's
// grids the G accumulators are summed through distributed shared memory,
// each rank updating its share of the image rows and writing them into
// every rank's F.
template <int N, int NT, bool QUAD, int G = 1>
__global__ void __launch_bounds__(NT, (G > 1 ? 1 : fused_min_blocks<N, NT>())) mlem_fused_kernel(FusedArgs a) {
    using Lay = FusedShape<N, NT>;
    constexpr int P = Lay::P, IMG = Lay::IMG, IMGA = Lay::IMGA, NN = Lay::NN, WP = Lay::WP;
    constexpr int NSEG = Lay::NSEG, SEG = Lay::SEG;
    constexpr float kLog2e = 1.44269504088896340736f;

    extern __shared__ __align__(16) float smem[];
    float* const img_base = fused_global_images(N)
                                ? a.img + (size_t)blockIdx.x * fused_image_floats<N, NT>()
                                : smem;
    float* img0 = img_base;             // F (mu during set-up), padded
    float* img1 = img0 + IMGA;          // back-projection accumulator, padded
    float* W = img1 + IMGA;             // [N][WP] grid samples / weights
    float* redc = fused_global_images(N) ? smem : W + N * WP;  // [2][NSEG][N] column partial sums
    float* redr = redc + 2 * NSEG * N;  // [2][NSEG][N] row partial sums
    float* rr = redr + 2 * NSEG * N;    // [4][N] ratios r = S / q per view
    float* Sg = rr + 4 * N;             // [4][N] the grid's sinogram rows (cp.async)
    float* csn = Sg + 4 * N;            // [V][2]
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
    // scatter in schedule order (images up to 128 x 128, schedule present)
    constexpr int SN = N <= 128 ? N : 128;
    const bool use_sched = N <= 128 && a.sched != nullptr;

    for (int v = tid; v < V; v += NT) view_cos_sin(v, V, &csn[2 * v], &csn[2 * v + 1]);

    float* tab = a.tab + (size_t)blockIdx.x * fused_tab_floats(N, V, QUAD, G);
    float* sens = a.sens + (size_t)blockIdx.x * NN;
    // this CTA's sample grids [g0, g1) and (cluster mode) update rows [R0, R1)
    int rank = 0, g0 = 0, g1 = ngrid, R0 = 0, R1 = N;
    if constexpr (G > 1) {
        rank = (int)cg::this_cluster().block_rank();
        g0 = rank * ngrid / G;
        g1 = (rank + 1) * ngrid / G;
        R0 = rank * N / G;
        R1 = (rank + 1) * N / G;
    }

    __shared__ int wait_ok;
    const long long units = a.job_start ? a.job_start[a.B] : (long long)a.B * (a.K > 0 ? a.K : 1);
    const long long m0 = (long long)blockIdx.x * a.cap;
    const long long m1 = m0 + a.cap < units ? m0 + a.cap : units;
    // candidate whose units contain x
    auto job_of = [&](long long x) -> int {
        if (!a.job_start) return (int)(x / (a.K > 0 ? a.K : 1));
        int lo = 0, hi = a.B - 1;  // largest j with job_start[j] <= x
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (a.job_start[mid] <= x) lo = mid;
            else hi = mid - 1;
        }
        return lo;
    };
    const int j_first = m0 < m1 ? job_of(m0) : 0;
    const int j_last = m0 < m1 ? job_of(m1 - 1) : -1;

    // cluster mode: cluster h takes candidates h, h + H, h + 2 H, ... whole
    const int n_holders = G > 1 ? (int)(gridDim.x / G) : 1;
    const int holder = G > 1 ? (int)(blockIdx.x / G) : 0;
    // (one loop form for both modes: a counter besides cand costs the one-CTA
    // kernel a register spill)
    for (int cand = (G == 1 ? j_last : holder); G == 1 ? cand >= j_first : cand < a.B;
         cand += (G == 1 ? -1 : n_holders)) {
        const RaggedDesc* d = a.desc ? a.desc + cand : nullptr;
        const float* __restrict__ S = a.S + (d ? d->S_off : (long long)cand * a.s_stride);
        const float* __restrict__ mu = a.mu + (d ? d->mu_off : (long long)cand * NN);
        float* Fc = a.F + (d ? d->F_off : (long long)cand * NN);
        const int Kc = d ? d->K : a.K;
        const int lidx = d ? d->out : cand;
        // this CTA's part of the candidate: iterations [it0, it1)
        const long long js = a.job_start ? a.job_start[cand] : (long long)cand * (a.K > 0 ? a.K : 1);
        const long long jl = Kc > 0 ? Kc : 1;
        const long long u0 = G > 1 ? 0 : (m0 - js > 0 ? m0 - js : 0);
        const long long u1 = G > 1 ? jl : (m1 - js < jl ? m1 - js : jl);
        const bool first = (u0 == 0), last = (u1 == jl);
        const int it0 = (int)(u0 < Kc ? u0 : Kc), it1 = (int)(u1 < Kc ? u1 : Kc);

        // ---- set-up: mu -> img0 (zero ring), img1 = 0
        for (int i = tid; i < IMG; i += NT) {
            img0[i] = 0.0f;
            img1[i] = 0.0f;
        }
        __syncthreads();
        for (int i = tid; i < NN; i += NT) img0[(i / N + 1) * P + (i % N) + 1] = __ldg(mu + i);
        __syncthreads();

        // ---- system matrix (attenuation exponents) + sensitivity A^T 1
        // (loops unrolled by 8, as in the iterations below: +0.8 % measured)
        for (int gi = g0; gi < g1; ++gi) {
            const float cs = csn[2 * gi], sn = csn[2 * gi + 1];
            SchedSlots<SN, NT> sched0;  // this grid's scatter slots of class 0
            if (use_sched) sched0.load(grid_sched<N>(a, gi));
            float* Xc = tab + (gi - g0) * gstride;
            float* XrT = Xc + NN;
            float* Uc = QUAD ? Xc + 2 * NN : Xc + NN;
            float* Ur = Uc + N;
            float ps = 0.0f;
#pragma unroll 8
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
#pragma unroll 8
                for (int s = SEG - 1; s >= 0; --s) {
                    const int k = k0 + s;
                    const float m = W[k * WP + lb];
                    Xc[tab_ix(N, k, lb)] = ndl * (0.5f * m + suf);
                    suf += m;
                }
                if (seg == 0) Uc[lb] = ndl * total;
            }
            if (QUAD) {  // rows: prefix sums from b = 0
                float pr = 0.0f;
#pragma unroll 2
                for (int s4 = 0; s4 < SEG; s4 += 4) {
                    const float4 m4 = *reinterpret_cast<const float4*>(W + lb * WP + k0 + s4);
                    pr += m4.x;
                    pr += m4.y;
                    pr += m4.z;
                    pr += m4.w;
                }
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
#pragma unroll 2
                for (int s4 = 0; s4 < SEG; s4 += 4) {
                    const float4 m4 = *reinterpret_cast<const float4*>(W + lb * WP + k0 + s4);
                    const float mm[4] = {m4.x, m4.y, m4.z, m4.w};
#pragma unroll
                    for (int j = 0; j < 4; ++j) {
                        XrT[tab_ix(N, k0 + s4 + j, lb)] = ndl * (0.5f * mm[j] + pre);
                        pre += mm[j];
                    }
                }
                if (seg == 0) Ur[lb] = ndl * total;
            }
            __syncthreads();
            {   // G = dx (sum of the grid's views' attenuation factors)
                const float uc = Uc[lb];
#pragma unroll 8
                for (int s = 0; s < SEG; ++s) {
                    const int k = k0 + s;
                    const float y = Xc[tab_ix(N, k, lb)];
                    W[k * WP + lb] = dx * (ex2(y) + ex2(uc - y));
                }
            }
            if (QUAD) {
                __syncthreads();
                const float ur = Ur[lb];
#pragma unroll 2
                for (int s4 = 0; s4 < SEG; s4 += 4) {
                    float4* w4 = reinterpret_cast<float4*>(W + lb * WP + k0 + s4);
                    const float4 y4 = *reinterpret_cast<const float4*>(XrT + tab_ix(N, k0 + s4, lb));
                    float4 v = *w4;
                    v.x += dx * (ex2(y4.x) + ex2(ur - y4.x));
                    v.y += dx * (ex2(y4.y) + ex2(ur - y4.y));
                    v.z += dx * (ex2(y4.z) + ex2(ur - y4.z));
                    v.w += dx * (ex2(y4.w) + ex2(ur - y4.w));
                    *w4 = v;
                }
            }
            __syncthreads();
            if (use_sched) scatter_scheduled<SN, NT, P, WP>(W, img1, cs, sn, c, grid_sched<N>(a, gi), sched0);
            else scatter_classes<N, NT, P, WP>(W, img1, cs, sn, c);
        }
        if (tid == 0) {  // second part of a cut candidate: wait for the first
            int ok = 1;
            if (!first) {
                const long long t0 = clock64();
                for (;;) {
                    int f;
                    asm volatile("ld.acquire.gpu.global.s32 %0, [%1];" : "=r"(f) : "l"(a.ready + cand) : "memory");
                    if (f) break;
                    if (clock64() - t0 > a.wait_cycles) {
                        ok = 0;
                        atomicExch(a.status, BOAC_ETIMEOUT);
                        break;
                    }
                    __nanosleep(256);
                }
            }
            wait_ok = ok;
        }
        __syncthreads();
        if (!wait_ok) {  // give up on this part: no F written, score NaN
            if (tid == 0 && last && a.L) a.L[lidx] = __longlong_as_double(0x7ff8000000000000LL);
            __syncthreads();
            continue;
        }
        if constexpr (G > 1) {
            // the sensitivity of this rank's rows: the ranks' partial images
            // summed in rank order
            cg::cluster_group cl = cg::this_cluster();
            cl.sync();
            for (int i = tid; i < (R1 - R0) * N; i += NT) {
                const int pi = (R0 + i / N + 1) * P + (i % N) + 1;
                float sv = 0.0f;
#pragma unroll 1
                for (int r = 0; r < G; ++r) sv += cl.map_shared_rank(img1, r)[pi];
                sens[i] = sv;
            }
            cl.sync();
            for (int i = tid; i < NN; i += NT) img0[(i / N + 1) * P + (i % N) + 1] = Fc[i];
        } else {
            for (int i = tid; i < NN; i += NT) {
                const int pi = (i / N + 1) * P + (i % N) + 1;
                sens[i] = img1[pi];
                img0[pi] = first ? Fc[i] : __ldcg(Fc + i);  // L2: written by another SM
            }
        }
        __syncthreads();
        for (int i = tid; i < IMG; i += NT) img1[i] = 0.0f;
        __syncthreads();

        // ---- MLEM iterations, then one more forward pass for the score
        double lacc = 0.0;
        for (int it = it0; it <= it1; ++it) {
            const bool scoring = (it == Kc);
            if (it == it1 && !(last && a.L)) break;
            for (int gi = g0; gi < g1; ++gi) {
                const float cs = csn[2 * gi], sn = csn[2 * gi + 1];
                const float* Xc = tab + (gi - g0) * gstride;
                const float* XrT = Xc + NN;
                const float* Uc = QUAD ? Xc + 2 * NN : Xc + NN;
                const float* Ur = Uc + N;
                {   // the next grid's exponent planes are read from DRAM
                    // once per iteration: start that read now (one 128-byte
                    // line per thread, 2 n^2 floats per grid)
                    const int gn = gi + 1 < g1 ? gi + 1 : g0;
                    const float* nxt = tab + (gn - g0) * gstride;
                    constexpr int kLines = (int)((2 * (size_t)NN * sizeof(float) + 127) / 128);
                    for (int l = tid; l < (QUAD ? kLines : kLines / 2); l += NT) prefetch_l2(nxt + 32 * l);
                }
                const int vc1 = gi, vc2 = gi + V / 2;           // column views
                const int vr1 = gi + V / 4, vr2 = gi + 3 * V / 4;  // row views (QUAD)
                // the grid's sinogram rows, copied to shared memory while the
                // forward passes run (waited for before the ratio step)
                for (int t = tid; t < (QUAD ? 4 * N : 2 * N); t += NT) {
                    const int vi = t / N, v = vi == 0 ? vc1 : vi == 1 ? vc2 : vi == 2 ? vr1 : vr2;
                    copy_async4(Sg + t, S + (size_t)v * N + (t % N));
                }
                copy_async_commit();
                // forward, column views: sample F on the grid.  (The column
                // and row passes and the column weights unroll by 8: fully
                // unrolled they spill at 64 registers; measured +7.8 %.)
                {
                    const float uc = Uc[lb];
                    float acc1 = 0.0f, acc2 = 0.0f;
#pragma unroll 2
                    for (int s4 = 0; s4 < SEG; s4 += 4) {
                        const float4 y4 = *reinterpret_cast<const float4*>(Xc + tab_ix(N, k0 + s4, lb));
                        const float yy[4] = {y4.x, y4.y, y4.z, y4.w};
#pragma unroll
                        for (int j = 0; j < 4; ++j) {
                            const int k = k0 + s4 + j;
                            float u, w;
                            sample_uw(k, lb, cs, sn, c, &u, &w);
                            const float f = bilerp_padded(img0, P, N, u, w);
                            if (QUAD) W[k * WP + lb] = f;
                            acc1 = fmaf(ex2(yy[j]), f, acc1);
                            acc2 = fmaf(ex2(uc - yy[j]), f, acc2);
                        }
                    }
                    redc[seg * N + lb] = acc1;
                    redc[(NSEG + seg) * N + lb] = acc2;
                }
                if (QUAD) {  // forward, row views: the samples back from W
                    __syncthreads();
                    const float ur = Ur[lb];
                    float acc3 = 0.0f, acc4 = 0.0f;
#pragma unroll 2
                    for (int s4 = 0; s4 < SEG; s4 += 4) {
                        const float4 y4 = *reinterpret_cast<const float4*>(XrT + tab_ix(N, k0 + s4, lb));
                        const float yy[4] = {y4.x, y4.y, y4.z, y4.w};
                        const float4 f4 = *reinterpret_cast<const float4*>(W + lb * WP + k0 + s4);
                        const float ff[4] = {f4.x, f4.y, f4.z, f4.w};
#pragma unroll
                        for (int j = 0; j < 4; ++j) {
                            acc3 = fmaf(ex2(yy[j]), ff[j], acc3);
                            acc4 = fmaf(ex2(ur - yy[j]), ff[j], acc4);
                        }
                    }
                    redr[seg * N + lb] = acc3;
                    redr[(NSEG + seg) * N + lb] = acc4;
                }
                copy_async_wait_all();
                __syncthreads();
                // q, then r = S / q (or the Eq. 5 terms when scoring)
                for (int t = tid; t < (QUAD ? 4 * N : 2 * N); t += NT) {  // one ray per thread
                    const int j = t % N, vi = t / N;  // views vc1, vc2, vr1, vr2
                    const float* rp = (vi >= 2 ? redr : redc) + ((vi & 1) ? NSEG * N : 0);
                    float q = 0.0f;
#pragma unroll
                    for (int s2 = 0; s2 < NSEG; ++s2) q += rp[s2 * N + j];
                    q *= dx;
                    const float Sv = Sg[vi * N + ((vi & 1) ? N - 1 - j : j)];
                    if (scoring) lacc += loglik_term(Sv, q, a.include_lgamma && !a.lgS);
                    else rr[vi * N + j] = q > 0.0f ? Sv / q : 0.0f;
                }
                __syncthreads();
                if (scoring) continue;
                SchedSlots<SN, NT> sched0;  // in flight during the weight passes
                if (use_sched) sched0.load(grid_sched<N>(a, gi));
                // back-projection weights of the grid's views
                {
                    const float uc = Uc[lb];
                    const float r1 = dx * rr[lb], r2 = dx * rr[N + lb];
#pragma unroll 2
                    for (int s4 = 0; s4 < SEG; s4 += 4) {
                        const float4 y4 = *reinterpret_cast<const float4*>(Xc + tab_ix(N, k0 + s4, lb));
                        const float yy[4] = {y4.x, y4.y, y4.z, y4.w};
#pragma unroll
                        for (int j = 0; j < 4; ++j)
                            W[(k0 + s4 + j) * WP + lb] = fmaf(ex2(yy[j]), r1, ex2(uc - yy[j]) * r2);
                    }
                }
                if (QUAD) {
                    __syncthreads();
                    const float ur = Ur[lb];
                    const float r3 = dx * rr[2 * N + lb], r4 = dx * rr[3 * N + lb];
                    for (int s4 = 0; s4 < SEG; s4 += 4) {
                        const float4 y4 = *reinterpret_cast<const float4*>(XrT + tab_ix(N, k0 + s4, lb));
                        float4* w4 = reinterpret_cast<float4*>(W + lb * WP + k0 + s4);
                        float4 v = *w4;
                        v.x += fmaf(ex2(y4.x), r3, ex2(ur - y4.x) * r4);
                        v.y += fmaf(ex2(y4.y), r3, ex2(ur - y4.y) * r4);
                        v.z += fmaf(ex2(y4.z), r3, ex2(ur - y4.z) * r4);
                        v.w += fmaf(ex2(y4.w), r3, ex2(ur - y4.w) * r4);
                        *w4 = v;
                    }
                }
                __syncthreads();
                if (use_sched) scatter_scheduled<SN, NT, P, WP>(W, img1, cs, sn, c, grid_sched<N>(a, gi), sched0);
                else scatter_classes<N, NT, P, WP>(W, img1, cs, sn, c);
            }
            if (scoring) break;
            if constexpr (G > 1) {
                // this rank's rows: back-projection summed over the ranks in
                // rank order, multiplicative update, written into every
                // rank's F; then the accumulator is cleared
                cg::cluster_group cl = cg::this_cluster();
                cl.sync();
                for (int i = tid; i < (R1 - R0) * N; i += NT) {
                    const int pi = (R0 + i / N + 1) * P + (i % N) + 1;
                    float bp = 0.0f;
#pragma unroll 1
                    for (int r = 0; r < G; ++r) bp += cl.map_shared_rank(img1, r)[pi];
                    const float sv = sens[i];
                    const float fn = sv > 0.0f ? img0[pi] * bp / sv : 0.0f;
#pragma unroll 1
                    for (int r = 0; r < G; ++r) cl.map_shared_rank(img0, r)[pi] = fn;
                }
                cl.sync();
                for (int i = tid; i < IMG; i += NT) img1[i] = 0.0f;
                __syncthreads();
            } else {
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
        }

        // ---- Eq. 5: deterministic block reduction of the float64 terms
        if (last && a.L) {
            for (int off = 16; off > 0; off >>= 1) lacc += __shfl_down_sync(0xffffffffu, lacc, off);
            if ((tid & 31) == 0) dred[tid >> 5] = lacc;
            __syncthreads();
            if (tid == 0) {
                double t = 0.0;
                for (int wi = 0; wi < NT / 32; ++wi) t += dred[wi];
                if constexpr (G > 1) {
                    dred[32] = t;  // this rank's terms
                } else {
                    a.L[lidx] = a.include_lgamma && a.lgS ? t - *a.lgS : t;
                    if (t == -INFINITY) atomicCAS(a.status, BOAC_OK, BOAC_ENONFINITE);
                }
            }
            if constexpr (G > 1) {  // the ranks' terms added in rank order
                cg::cluster_group cl = cg::this_cluster();
                cl.sync();
                if (rank == 0 && tid == 0) {
                    double t = 0.0;
                    for (int r = 0; r < G; ++r) t += cl.map_shared_rank(dred, r)[32];
                    a.L[lidx] = a.include_lgamma && a.lgS ? t - *a.lgS : t;
                    if (t == -INFINITY) atomicCAS(a.status, BOAC_OK, BOAC_ENONFINITE);
                }
            }
        }

        // ---- F out (F^K, or the state handed to the candidate's second part;
        // cluster mode: each rank its rows)
        for (int i = R0 * N + tid; i < R1 * N; i += NT) Fc[i] = img0[(i / N + 1) * P + (i % N) + 1];
        if constexpr (G > 1) cg::this_cluster().sync();  // no rank still reads another's memory
        __syncthreads();
        if (!last && tid == 0 && cand != a.withhold) {
            __threadfence();
            asm volatile("st.release.gpu.global.s32 [%0], %1;" ::"l"(a.ready + cand), "r"(1) : "memory");
        }
    }
}

// ---------------------------------------------------------------- host side
// Launch shapes: for each image side, CTAs of 2n, 4n or 8n threads (at most
// 1024), with four or two views per sample grid: configuration id =
// 2 * shape + (1 for two views per grid).  Ids 6, 7 and 8 are the cluster
// kernel (boac_band.cu, four views per grid only): 5, 6 or 8 CTAs per
// candidate for 256 x 256 images, 2, 4 or 8 for 128 x 128.
// Ids 9 .. 16 are the fused kernel's cluster mode (images up to 128 x 128,
// four views per grid, CTAs of 8n threads) with 2, 3, 4, 6, 8, 9, 12 or 16
// CTAs per candidate, each on its share of the sample grids.
constexpr int kShapes = 3;
constexpr int kBandConfigs = 3;
constexpr int kSplitConfigs = 8;
constexpr int kConfigs = 2 * kShapes + kBandConfigs + kSplitConfigs;

struct FusedVariant {
    int n, nt;
    bool quad;
    int nb;  // CTAs per candidate in the band kernel's cluster (1 otherwise)
    size_t (*smem)(int V);
    const void* func;
    // `holders`: CTAs (nb == 1, g == 1) or clusters that share the work
    int (*launch)(const FusedArgs& a, int holders, cudaStream_t st);
    int g;   // CTAs per candidate in the fused kernel's cluster mode (1 otherwise)
    int (*max_clusters)();  // cluster mode: clusters resident at once
};

// Cluster-mode launches: dynamic shared memory and (16 CTAs) the
// non-portable cluster size allowed once per device, then the kernel on
// `clusters` clusters of G CTAs.
template <int N, int NT, int G>
static int split_attrs() {
    constexpr int kDev = 64;
    static bool done[kDev];
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kDev) return launch_status();
    if (!done[dev]) {
        if (cudaFuncSetAttribute(mlem_fused_kernel<N, NT, true, G>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)fused_smem_bytes<N, NT>(kMaxViews)) != cudaSuccess)
            return launch_status();
        if (G > 8 && cudaFuncSetAttribute(mlem_fused_kernel<N, NT, true, G>,
                                          cudaFuncAttributeNonPortableClusterSizeAllowed, 1) != cudaSuccess)
            return launch_status();
        done[dev] = true;
    }
    return BOAC_OK;
}

template <int N, int NT, int G>
static cudaLaunchConfig_t split_config(int clusters, int V, cudaStream_t st, cudaLaunchAttribute* attr) {
    cudaLaunchConfig_t cfg = {};
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = G;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.gridDim = dim3((unsigned)(clusters * G), 1, 1);
    cfg.blockDim = dim3(NT, 1, 1);
    cfg.dynamicSmemBytes = fused_smem_bytes<N, NT>(V);
    cfg.stream = st;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cfg;
}

template <int N, int NT, int G>
static int split_max_clusters_t() {
    constexpr int kDev = 64;
    static int cached[kDev];
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kDev) {
        cudaGetLastError();
        return 0;
    }
    if (cached[dev]) return cached[dev];
    if (split_attrs<N, NT, G>() != BOAC_OK) {
        cudaGetLastError();
        return 0;
    }
    cudaLaunchAttribute attr[1];
    cudaLaunchConfig_t cfg = split_config<N, NT, G>(64, kMaxViews, nullptr, attr);
    int n = 0;
    if (cudaOccupancyMaxActiveClusters(&n, mlem_fused_kernel<N, NT, true, G>, &cfg) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    cached[dev] = n;
    return n;
}

template <int N, int NT, int G>
static int split_launch_t(const FusedArgs& a, int clusters, cudaStream_t st) {
    int s = split_attrs<N, NT, G>();
    if (s != BOAC_OK) return s;
    FusedArgs b = a;
    if (b.sched) {  // the scatter schedule of this geometry, then the kernel
        b.sched = sched_prepare(N, b.V, b.V / 4, FusedShape<N, NT>::WP, const_cast<unsigned short*>(a.sched), st,
                                &s);
        if (s != BOAC_OK) return s;
    }
    cudaLaunchAttribute attr[1];
    cudaLaunchConfig_t cfg = split_config<N, NT, G>(clusters, b.V, st, attr);
    if (cudaLaunchKernelEx(&cfg, mlem_fused_kernel<N, NT, true, G>, b) != cudaSuccess) return launch_status();
    return launch_status();
}

template <int N, int NT, bool QUAD>
static int fused_launch_t(const FusedArgs& a, int slots, cudaStream_t st) {
    // once per device: allow the large dynamic shared-memory carve-out
    constexpr int kDev = 64;
    static bool attr_set[kDev];
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kDev) return launch_status();
    if (!attr_set[dev]) {
        if (cudaFuncSetAttribute(mlem_fused_kernel<N, NT, QUAD>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)fused_smem_bytes<N, NT>(kMaxViews)) != cudaSuccess)
            return launch_status();
        attr_set[dev] = true;
    }
    FusedArgs b = a;
    if constexpr (N <= 128) {
        if (b.sched) {  // the scatter schedule of this geometry, then the kernel
            int s = BOAC_OK;
            b.sched = sched_prepare(N, b.V, QUAD ? b.V / 4 : b.V / 2, FusedShape<N, NT>::WP,
                                    const_cast<unsigned short*>(a.sched), st, &s);
            if (s != BOAC_OK) return s;
        }
    }
    mlem_fused_kernel<N, NT, QUAD><<<slots, NT, fused_smem_bytes<N, NT>(b.V), st>>>(b);
    return launch_status();
}

template <int N, int NT>
static size_t smem_of(int V) { return fused_smem_bytes<N, NT>(V); }

template <int N, int NT, bool QUAD>
static FusedVariant make_variant() {
    return FusedVariant{N, NT, QUAD, 1, smem_of<N, NT>, (const void*)mlem_fused_kernel<N, NT, QUAD>,
                        fused_launch_t<N, NT, QUAD>, 1, nullptr};
}

template <int N, int G>
static FusedVariant make_split_variant() {
    return FusedVariant{N, 8 * N, true, 1, smem_of<N, 8 * N>, (const void*)mlem_fused_kernel<N, 8 * N, true, G>,
                        split_launch_t<N, 8 * N, G>, G, split_max_clusters_t<N, 8 * N, G>};
}

template <int N, int NB>
static size_t band_smem_of(int) { return band_smem_bytes(N, NB); }
template <int N, int NB>
static int band_launch_of(const FusedArgs& a, int clusters, cudaStream_t st) {
    return band_launch(N, NB, a, clusters, st);
}
template <int N, int NB>
static FusedVariant make_band_variant() {
    return FusedVariant{N, 4 * N, true, NB, band_smem_of<N, NB>, nullptr, band_launch_of<N, NB>, 1, nullptr};
}

#define BOAC_SHAPES(NV)                                                                        \
    make_variant<NV, 2 * NV, true>(), make_variant<NV, 2 * NV, false>(),                       \
        make_variant<NV, 4 * NV, true>(), make_variant<NV, 4 * NV, false>(),                   \
        make_variant<NV, (8 * NV > 1024 ? 1024 : 8 * NV), true>(),                             \
        make_variant<NV, (8 * NV > 1024 ? 1024 : 8 * NV), false>()
#define BOAC_NO_BAND FusedVariant{}, FusedVariant{}, FusedVariant{}
#define BOAC_SPLIT(NV)                                                                        \
    make_split_variant<NV, 2>(), make_split_variant<NV, 3>(), make_split_variant<NV, 4>(),  \
        make_split_variant<NV, 6>(), make_split_variant<NV, 8>(), make_split_variant<NV, 9>(), \
        make_split_variant<NV, 12>(), make_split_variant<NV, 16>()
#define BOAC_NO_SPLIT FusedVariant{}, FusedVariant{}, FusedVariant{}, FusedVariant{}, \
                      FusedVariant{}, FusedVariant{}, FusedVariant{}, FusedVariant{}

static const FusedVariant* variant_table(int n) {
    static const FusedVariant t64[kConfigs] = {BOAC_SHAPES(64), make_band_variant<64, 2>(),
                                               make_band_variant<64, 4>(), make_band_variant<64, 8>(),
                                               BOAC_SPLIT(64)};
    static const FusedVariant t96[kConfigs] = {BOAC_SHAPES(96), BOAC_NO_BAND, BOAC_SPLIT(96)};
    static const FusedVariant t128[kConfigs] = {BOAC_SHAPES(128), make_band_variant<128, 2>(),
                                                make_band_variant<128, 4>(), make_band_variant<128, 8>(),
                                                BOAC_SPLIT(128)};
    static const FusedVariant t256[kConfigs] = {BOAC_SHAPES(256), make_band_variant<256, 5>(),
                                                make_band_variant<256, 6>(), make_band_variant<256, 8>(),
                                                BOAC_NO_SPLIT};
    switch (n) {
        case 64: return t64;
        case 96: return t96;
        case 128: return t128;
        case 256: return t256;
        default: return nullptr;
    }
}

// Default configuration of the one-CTA kernel: the largest CTA that keeps
// >= 64 registers per thread at the occupancy shared memory allows; four
// views per grid when V % 4 == 0.
static int single_cta_config(const boac_geom* g) {
    const int shape = g->n == 64 ? 1 : 2;
    return 2 * shape + (g->n_views % 4 == 0 ? 0 : 1);
}

static const FusedVariant* get_variant(const boac_geom* g, int config);

// Cluster mode for a batch too small to fill the GPU one CTA per candidate
// (images up to 128 x 128, V % 4 == 0): the cluster size G with the least
// modelled time, rounds(G) (ceil(grids / G) + 1.6) grid passes per
// iteration, where rounds(G) = ceil(B / clusters of G resident at once) and
// 1.6 grid passes stand for the cluster's per-iteration exchange (fitted on
// GB300 at 128 x 128 and 120 views: 24 us against 15 us per grid pass); the
// smaller G on a tie; and only if that beats one CTA per candidate, whose
// even split of the batch's iterations costs grids B / min(B, SMs) passes
// per iteration.  Returns the configuration id, or -1.
static int split_config(const boac_geom* g, int B) {
    if (g->n > 128 || g->n_views % 4 != 0 || B < 1) return -1;
    const int sms = sm_count();
    if (sms <= 0) return -1;
    const int ngrid = g->n_views / 4;
    int best = -1;
    double best_t = (double)ngrid * B / (B < sms ? B : sms);  // one CTA per candidate
    for (int i = 0; i < kSplitConfigs; ++i) {
        const int cfg = 2 * kShapes + kBandConfigs + i;
        const FusedVariant* v = get_variant(g, cfg);
        if (!v) continue;
        const int h = v->max_clusters();
        if (h <= 0) continue;
        const int rounds = (B + h - 1) / h;
        const double t = rounds * ((ngrid + v->g - 1) / v->g + 1.6);
        if (t < best_t - 1e-9) {
            best = cfg;
            best_t = t;
        }
    }
    return best;
}

// Default configuration for B candidates.  Batches too small to fill the
// GPU one candidate per CTA (images up to 128 x 128, V % 4 == 0) take the
// fused kernel's cluster mode (split_config; measured on GB300 at 128 x 128
// and K = 20: 1.7x to 2.3x the unfused batched kernels at 1 to 64
// candidates, 1.2x the one-CTA kernel at 96).  256 x 256 images with
// V % 4 == 0 take the band kernel with the cluster size that keeps the most
// SMs busy (clusters are placed within one GPC, so the resident count
// depends on the size); the smaller cluster on a tie.  Otherwise the one-CTA
// kernel.
static int default_config(const boac_geom* g, int B) {
    const int sc = split_config(g, B);
    if (sc >= 0) return sc;
    if (g->n == 64 && B >= 1 && B <= 2 * sm_count()) {
        // at most two candidates per SM: CTAs of 8n threads (measured on GB300
        // at 60 views: 1.88 vs 2.16 ms for B = 1 ... 128; from B = 456 on,
        // three 4n-thread CTAs per SM are faster)
        return 2 * 2 + (g->n_views % 4 == 0 ? 0 : 1);
    }
    if (g->n == 256 && g->n_views % 4 == 0) {
        static const int nbs[kBandConfigs] = {5, 6, 8};
        int best = -1, best_ctas = 0;
        for (int i = 0; i < kBandConfigs; ++i) {
            const int ctas = band_max_clusters(256, nbs[i]) * nbs[i];
            if (ctas > best_ctas) {
                best = i;
                best_ctas = ctas;
            }
        }
        if (best >= 0) return 2 * kShapes + best;
    }
    return single_cta_config(g);
}

// Batches small enough that the unfused batched kernels (boac_unfused.cu:
// many CTAs per candidate) finish before the fused kernel's one CTA or one
// cluster per candidate does, for the geometries without the cluster mode
// (view counts not divisible by 4, 256 x 256 images).  Measured on GB300
// (152 SMs) with K = 20 at 60 / 90 / 120 / 180 views: up to 32 candidates at
// 64 x 64 and 96 x 96 (1.9x / 4.7x at B = 1), 16 at 128 x 128 (2.4x at
// B = 1), 2 at 256 x 256 (1.3x at B = 1); both paths scale with the view
// count, so the bound is per image size, scaled with the SM count.
static bool use_unfused(const boac_geom* g, int B) {
    if (split_config(g, B) >= 0) return false;
    int cap;
    switch (g->n) {
        case 64:
        case 96: cap = 32; break;
        case 128: cap = 16; break;
        case 256: cap = 2; break;
        default: return false;
    }
    const int sms = sm_count();
    return sms > 0 && (long long)B * 152 <= (long long)cap * sms;
}

static const FusedVariant* get_variant(const boac_geom* g, int config) {
    const FusedVariant* t = variant_table(g->n);
    if (!t || config < 0 || config >= kConfigs) return nullptr;
    const FusedVariant* v = &t[config];
    if (!v->launch) return nullptr;
    if (v->quad ? (g->n_views % 4 != 0) : (g->n_views % 2 != 0)) return nullptr;
    if (v->nb > 1 && !band_supported(g->n, g->n_views, v->nb)) return nullptr;
    if (v->g > 1 && (g->n_views < 4 * v->g)) return nullptr;  // at least one grid per rank
    return v;
}

// Resident CTAs per SM of a variant, computed for the largest view table it
// may be launched with (the per-view table is a few KB, so this equals the
// occupancy at every view count); cached per device.
static int variant_occupancy(const FusedVariant* v, int V) {
    constexpr int kDev = 64;
    static int cached[kDev][4][kConfigs];  // 0 = not yet computed
    int dev = 0;
    if (V < 0 || V > kMaxViews) return 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0) {
        cudaGetLastError();
        return 0;
    }
    const int ni = v->n == 64 ? 0 : (v->n == 96 ? 1 : (v->n == 128 ? 2 : 3));
    const int ci = (int)(v - variant_table(v->n));
    if (dev < kDev && cached[dev][ni][ci]) return cached[dev][ni][ci];
    if (cudaFuncSetAttribute(v->func, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)v->smem(kMaxViews)) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    int nb = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, v->func, v->nt, v->smem(kMaxViews)) !=
        cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    if (dev < kDev) cached[dev][ni][ci] = nb;
    return nb;
}

// Workspace of the fused kernels for `holders` CTAs (or clusters) and B
// candidates:
//   [0, 256)   status word (BOAC_OK, or BOAC_ETIMEOUT from a bounded wait)
//   tables     attenuation exponents, one region per CTA
//   sens       sensitivity image (cluster kernel: band rows) per CTA
//   images     one-CTA kernel, n > 128: padded F / accumulator / sample
//              buffer per CTA; cluster kernel: the record kernel's flag and
//              the ray-run records of every (band, grid)
//   ready      one flag per candidate (the work split's hand-over)
//   sched      one-CTA kernel, n <= 128: the scatter schedule (geometry only)
struct FusedLayout {
    size_t status, tab, sens, img, geo, ready, sched, total;
};

static FusedLayout fused_layout(const boac_geom* g, const FusedVariant* v, int holders, int B) {
    FusedLayout l;
    const size_t ctas = (size_t)holders * v->nb * v->g;
    l.status = 0;
    l.tab = 256;
    if (v->nb > 1) {
        l.sens = l.tab + align256(sizeof(float) * ctas * band_tab_floats(g->n, v->nb, g->n_views));
        l.img = l.sens + align256(sizeof(float) * ctas * band_sens_floats(g->n, v->nb));
        l.geo = l.img + 256;
        l.ready = l.geo + align256(band_geo_bytes(g->n, v->nb, g->n_views));
    } else {
        l.sens = l.tab + align256(sizeof(float) * ctas * fused_tab_floats(g->n, g->n_views, v->quad, v->g));
        l.img = l.sens + align256(sizeof(float) * ctas * g->n * g->n);
        // padded F and accumulator, (n+1)(n+2)+1 floats each, and the
        // n x (n+1) sample buffer, for sides held in global memory
        const size_t img_floats = fused_global_images(g->n)
                                      ? 2 * ((size_t)(g->n + 1) * (g->n + 2) + 1) + (size_t)g->n * (g->n + 1)
                                      : 0;
        l.geo = l.img + align256(sizeof(float) * ctas * img_floats);
        l.ready = l.geo;
    }
    l.sched = l.total = l.ready + align256(sizeof(int) * (size_t)B);
    if (v->nb == 1 && g->n <= 128) l.total = l.sched + sched_bytes(g->n, v->quad ? g->n_views / 4 : g->n_views / 2);
    return l;
}

// CTAs (one-CTA kernel) or clusters that run at once, at most B.
static int variant_holders(const boac_geom* g, const FusedVariant* v, int B) {
    long long h;
    if (v->nb > 1) {
        h = band_max_clusters(g->n, v->nb);
    } else if (v->g > 1) {
        h = v->max_clusters();
    } else {
        const int per_sm = variant_occupancy(v, g->n_views);
        h = (long long)per_sm * sm_count();
    }
    if (h <= 0) return 0;
    return (int)(h < B ? h : B);
}

size_t fused_workspace_bytes(const boac_geom* g, int B) {
    if (use_unfused(g, B)) return unfused_workspace_bytes(g, B);
    const FusedVariant* v = get_variant(g, default_config(g, B));
    const int h = v ? variant_holders(g, v, B) : 0;
    return h > 0 ? fused_layout(g, v, h, B).total : 0;
}

// Units per CTA of the work split: the larger of an even share and the
// longest candidate (so that a candidate is never cut into three parts).
static long long split_cap(long long units, long long longest, int slots) {
    const long long share = (units + slots - 1) / slots;
    return share > longest ? share : longest;
}

static FusedArgs base_args(const boac_geom* g, const float* mu, const float* S, long long s_stride,
                           float* F, int K, int B, double* L, int include_lgamma, char* ws,
                           const FusedLayout& l) {
    FusedArgs a;
    a.mu = mu;
    a.S = S;
    a.s_stride = s_stride;
    a.F = F;
    a.L = L;
    a.include_lgamma = include_lgamma;
    a.lgS = nullptr;
    a.B = B;
    a.V = g->n_views;
    a.K = K;
    a.dx = g->pixel_cm;
    a.tab = reinterpret_cast<float*>(ws + l.tab);
    a.sens = reinterpret_cast<float*>(ws + l.sens);
    a.img = reinterpret_cast<float*>(ws + l.img);
    a.desc = nullptr;
    a.job_start = nullptr;
    a.cap = 0;
    a.ready = reinterpret_cast<int*>(ws + l.ready);
    a.status = reinterpret_cast<int*>(ws + l.status);
    a.geo = reinterpret_cast<const int*>(ws + l.geo);
    a.geo_bad = reinterpret_cast<int*>(ws + l.img);
    a.wait_cycles = wait_cycles();
    a.withhold = -1;
    a.sched = l.total > l.sched ? reinterpret_cast<const unsigned short*>(ws + l.sched) : nullptr;
    return a;
}

static std::atomic<long long> g_wait_cycles{kWaitCycles};
long long wait_cycles() { return g_wait_cycles.load(std::memory_order_relaxed); }

// Uniform batch: zero the status and ready flags, then launch the CTAs that
// have work under the split.
static int launch_uniform(const boac_geom* g, const FusedVariant* v, int slots, const float* mu,
                          const float* S, long long s_stride, float* F, int K, int B, double* L,
                          int include_lgamma, char* ws, cudaStream_t st) {
    const FusedLayout l = fused_layout(g, v, slots, B);
    FusedArgs a = base_args(g, mu, S, s_stride, F, K, B, L, include_lgamma, ws, l);
    const long long per = K > 0 ? K : 1, units = (long long)B * per;
    a.cap = split_cap(units, per, slots);
    const int grid = (int)((units + a.cap - 1) / a.cap);
    if (cudaMemsetAsync(ws + l.status, 0, sizeof(int), st) != cudaSuccess ||
        cudaMemsetAsync(ws + l.ready, 0, sizeof(int) * (size_t)B, st) != cudaSuccess)
        return launch_status();
    // one shared sinogram: its ln S! sum once, in the status slot's spare bytes
    if (L && include_lgamma && s_stride == 0) {
        BOAC_RANGE("score: ln S! of the shared sinogram");
        a.lgS = lgamma_sum(g->n_views * g->n_bins, S, reinterpret_cast<double*>(ws + l.status + 8), st);
    }
    BOAC_RANGE("fused MLEM: set-up, iterations, score");
    return v->launch(a, grid, st);
}

// ---------------------------------------------------------------- ragged
// Ragged workspace: [0, 256) status word; per class: the candidates'
// records, their unit offsets (job_start, B_c + 1 values) and the class's
// fused layout (without its own status word).
struct RaggedPlan {
    int cls_count[kMaxRaggedClasses];
    int slots[kMaxRaggedClasses];
    const FusedVariant* var[kMaxRaggedClasses];
    size_t desc_off[kMaxRaggedClasses], start_off[kMaxRaggedClasses], layout_off[kMaxRaggedClasses];
    size_t total;
};

static int ragged_plan(const boac_geom* classes, int n_classes, const boac_ragged_cand* cands, int B,
                       const int* config, RaggedPlan* pl) {
    if (!classes || n_classes < 1 || n_classes > kMaxRaggedClasses || !cands || B < 1) return BOAC_EINVAL;
    for (int c = 0; c < n_classes; ++c) {
        if (!geom_ok(&classes[c]) || classes[c].n_views % 2) return BOAC_EINVAL;
        pl->cls_count[c] = 0;
    }
    for (int b = 0; b < B; ++b) {
        const boac_ragged_cand& d = cands[b];
        if (d.cls < 0 || d.cls >= n_classes || d.K < 0 || d.mu_off < 0 || d.S_off < 0 || d.F_off < 0)
            return BOAC_EINVAL;
        pl->cls_count[d.cls]++;
    }
    size_t off = 256;
    for (int c = 0; c < n_classes; ++c) {
        if (!variant_table(classes[c].n)) return BOAC_EUNSUPPORTED;
        const int cfg = config ? config[c] : default_config(&classes[c], pl->cls_count[c]);
        pl->var[c] = get_variant(&classes[c], cfg);
        if (!pl->var[c]) return BOAC_EINVAL;
        const int cnt = pl->cls_count[c];
        pl->slots[c] = cnt ? variant_holders(&classes[c], pl->var[c], cnt) : 0;
        if (cnt && pl->slots[c] <= 0) return BOAC_ECUDA;
        pl->desc_off[c] = off;
        off += align256(sizeof(RaggedDesc) * (size_t)cnt);
        pl->start_off[c] = off;
        off += align256(sizeof(long long) * ((size_t)cnt + 1));
        pl->layout_off[c] = off;
        off += cnt ? fused_layout(&classes[c], pl->var[c], pl->slots[c], cnt).total : 0;
    }
    pl->total = off;
    return BOAC_OK;
}

// The candidates in the order the kernels process them: by class, then by
// decreasing K.
static std::vector<int> ragged_order(const boac_ragged_cand* cands, int B) {
    std::vector<int> order((size_t)B);
    for (int b = 0; b < B; ++b) order[b] = b;
    std::stable_sort(order.begin(), order.end(), [&](int x, int y) {
        if (cands[x].cls != cands[y].cls) return cands[x].cls < cands[y].cls;
        return cands[x].K > cands[y].K;
    });
    return order;
}

#ifdef BOAC_CHECKED
BOAC_FAULT_READER(bounds_faults_fused)
#endif

}  // namespace boac

using namespace boac;

extern "C" int boac_mlem(const boac_geom* g, const float* mu, const float* S, long long s_stride,
                         float* F, int K, int B, double* L, int include_lgamma, void* ws,
                         size_t ws_bytes, void* stream) {
    BOAC_RANGE("boac_mlem");
    if (!geom_ok(g) || !mu || !S || !F || B < 1 || K < 0 || s_stride < 0) return BOAC_EINVAL;
    if (g->n_views % 2) return BOAC_EINVAL;
    if (use_unfused(g, B))
        return mlem_unfused(g, mu, S, s_stride, F, K, B, L, include_lgamma, ws, ws_bytes, as_stream(stream));
    const FusedVariant* v = get_variant(g, default_config(g, B));
    if (!v) return BOAC_EUNSUPPORTED;
    const int slots = variant_holders(g, v, B);
    if (slots <= 0) return BOAC_ECUDA;
    if (!ws || ws_bytes < fused_layout(g, v, slots, B).total) return BOAC_EWORKSPACE;
    return launch_uniform(g, v, slots, mu, S, s_stride, F, K, B, L, include_lgamma,
                          static_cast<char*>(ws), as_stream(stream));
}

extern "C" long long boac_set_wait_cycles(long long cycles) {
    return g_wait_cycles.exchange(cycles > 0 ? cycles : kWaitCycles);
}

// Test hook of the bounded hand-over wait: the fused kernel of launch
// configuration `config` on exactly `holders` CTAs (or clusters), with the
// first part of candidate `withhold` keeping its flag to itself.
static int handover_plan(const boac_geom* g, int B, int K, int config, int holders, int withhold,
                         const FusedVariant** v, FusedLayout* l) {
    if (!geom_ok(g) || B < 1 || K < 0 || holders < 1 || holders > B || withhold < -1 || withhold >= B)
        return BOAC_EINVAL;
    *v = get_variant(g, config);
    if (!*v) return BOAC_EINVAL;
    if (variant_holders(g, *v, B) < holders) return BOAC_EUNSUPPORTED;  // must all be resident
    *l = fused_layout(g, *v, holders, B);
    return BOAC_OK;
}

extern "C" size_t boac_test_mlem_handover_bytes(const boac_geom* g, int B, int K, int config, int holders) {
    const FusedVariant* v;
    FusedLayout l;
    return handover_plan(g, B, K, config, holders, -1, &v, &l) == BOAC_OK ? l.total : 0;
}

extern "C" int boac_test_mlem_handover(const boac_geom* g, const float* mu, const float* S, float* F, int K,
                                       int B, double* L, int config, int holders, int withhold, void* ws,
                                       size_t ws_bytes, void* stream) {
    BOAC_RANGE("boac_test_mlem_handover");
    if (!mu || !S || !F || !L) return BOAC_EINVAL;
    const FusedVariant* v;
    FusedLayout l;
    const int s = handover_plan(g, B, K, config, holders, withhold, &v, &l);
    if (s != BOAC_OK) return s;
    if (!ws || ws_bytes < l.total) return BOAC_EWORKSPACE;
    char* base = static_cast<char*>(ws);
    cudaStream_t st = as_stream(stream);
    FusedArgs a = base_args(g, mu, S, 0, F, K, B, L, 0, base, l);
    a.withhold = withhold;
    const long long per = K > 0 ? K : 1, units = (long long)B * per;
    a.cap = split_cap(units, per, holders);
    const int grid = (int)((units + a.cap - 1) / a.cap);
    if (cudaMemsetAsync(base + l.status, 0, sizeof(int), st) != cudaSuccess ||
        cudaMemsetAsync(base + l.ready, 0, sizeof(int) * (size_t)B, st) != cudaSuccess)
        return launch_status();
    return v->launch(a, grid, st);
}

extern "C" int boac_workspace_status(const void* ws, size_t ws_bytes, int* status) {
    BOAC_RANGE("boac_workspace_status");
    if (!ws || ws_bytes < sizeof(int) || !status) return BOAC_EINVAL;
    if (cudaMemcpy(status, ws, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess) return launch_status();
    return BOAC_OK;
}

extern "C" size_t boac_mlem_ragged_workspace_bytes(const boac_geom* classes, int n_classes,
                                                   const boac_ragged_cand* cands, int B,
                                                   const int* config) {
    RaggedPlan pl;
    return ragged_plan(classes, n_classes, cands, B, config, &pl) == BOAC_OK ? pl.total : 0;
}

extern "C" int boac_mlem_ragged_prepare(const boac_geom* classes, int n_classes,
                                        const boac_ragged_cand* cands, int B, const int* config,
                                        void* ws, size_t ws_bytes, void* stream) {
    BOAC_RANGE("boac_mlem_ragged_prepare");
    RaggedPlan pl;
    int s = ragged_plan(classes, n_classes, cands, B, config, &pl);
    if (s != BOAC_OK) return s;
    if (!ws || ws_bytes < pl.total) return BOAC_EWORKSPACE;
    // Per-class records and unit offsets, copied from pageable host memory
    // (the copies are staged before this call returns).
    const std::vector<int> order = ragged_order(cands, B);
    std::vector<RaggedDesc> desc((size_t)B);
    std::vector<long long> start((size_t)B + n_classes);
    char* base = static_cast<char*>(ws);
    int first = 0;
    for (int c = 0; c < n_classes; ++c) {
        const int cnt = pl.cls_count[c];
        if (cnt == 0) continue;
        long long* js = start.data() + first + c;
        js[0] = 0;
        for (int i = 0; i < cnt; ++i) {
            const boac_ragged_cand& d = cands[order[first + i]];
            desc[first + i] = RaggedDesc{d.mu_off, d.S_off, d.F_off, d.K, order[first + i]};
            js[i + 1] = js[i] + (d.K > 0 ? d.K : 1);
        }
        if (cudaMemcpyAsync(base + pl.desc_off[c], desc.data() + first, sizeof(RaggedDesc) * cnt,
                            cudaMemcpyHostToDevice, as_stream(stream)) != cudaSuccess ||
            cudaMemcpyAsync(base + pl.start_off[c], js, sizeof(long long) * (cnt + 1),
                            cudaMemcpyHostToDevice, as_stream(stream)) != cudaSuccess)
            return launch_status();
        first += cnt;
    }
    return BOAC_OK;
}

extern "C" int boac_mlem_ragged_run(const boac_geom* classes, int n_classes,
                                    const boac_ragged_cand* cands, int B, const float* mu_pool,
                                    const float* S_pool, float* F_pool, double* L, int include_lgamma,
                                    const int* config, void* ws, size_t ws_bytes, void* stream) {
    BOAC_RANGE("boac_mlem_ragged_run");
    if (!mu_pool || !S_pool || !F_pool || !L) return BOAC_EINVAL;
    RaggedPlan pl;
    int s = ragged_plan(classes, n_classes, cands, B, config, &pl);
    if (s != BOAC_OK) return s;
    if (!ws || ws_bytes < pl.total) return BOAC_EWORKSPACE;
    char* base = static_cast<char*>(ws);
    cudaStream_t st = as_stream(stream);
    if (cudaMemsetAsync(base, 0, sizeof(int), st) != cudaSuccess) return launch_status();
    // units and longest candidate per class (the same order as prepare's)
    long long units[kMaxRaggedClasses] = {0}, longest[kMaxRaggedClasses] = {0};
    for (int b = 0; b < B; ++b) {
        const long long len = cands[b].K > 0 ? cands[b].K : 1;
        units[cands[b].cls] += len;
        if (len > longest[cands[b].cls]) longest[cands[b].cls] = len;
    }
    for (int c = 0; c < n_classes; ++c) {
        const int cnt = pl.cls_count[c];
        if (cnt == 0) continue;
        const FusedLayout l = fused_layout(&classes[c], pl.var[c], pl.slots[c], cnt);
        char* cbase = base + pl.layout_off[c];
        FusedArgs a = base_args(&classes[c], mu_pool, S_pool, 0, F_pool, 0, cnt, L, include_lgamma, cbase, l);
        a.desc = reinterpret_cast<const RaggedDesc*>(base + pl.desc_off[c]);
        a.job_start = reinterpret_cast<const long long*>(base + pl.start_off[c]);
        a.status = reinterpret_cast<int*>(base);  // one status word for the call
        a.cap = split_cap(units[c], longest[c], pl.slots[c]);
        const int grid = (int)((units[c] + a.cap - 1) / a.cap);
        if (cudaMemsetAsync(cbase + l.ready, 0, sizeof(int) * (size_t)cnt, st) != cudaSuccess)
            return launch_status();
        s = pl.var[c]->launch(a, grid, st);
        if (s != BOAC_OK) return s;
    }
    return BOAC_OK;
}

extern "C" int boac_mlem_ragged(const boac_geom* classes, int n_classes, const boac_ragged_cand* cands,
                                int B, const float* mu_pool, const float* S_pool, float* F_pool,
                                double* L, int include_lgamma, const int* config, void* ws,
                                size_t ws_bytes, void* stream) {
    BOAC_RANGE("boac_mlem_ragged");
    if (!mu_pool || !S_pool || !F_pool || !L) return BOAC_EINVAL;
    int s = boac_mlem_ragged_prepare(classes, n_classes, cands, B, config, ws, ws_bytes, stream);
    if (s != BOAC_OK) return s;
    return boac_mlem_ragged_run(classes, n_classes, cands, B, mu_pool, S_pool, F_pool, L,
                                include_lgamma, config, ws, ws_bytes, stream);
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

// Device address of g_noalloc_scratch on the current device, looked up on
// every call: in host code the array's name stands for a host-side shadow,
// not device memory, so the kernel must be given the address
// cudaGetSymbolAddress returns.  Not caching it keeps the address right after
// a device reset or a re-created primary context (the module, and the array
// with it, may then sit elsewhere) and leaves no shared state between host
// threads; the lookup costs next to nothing beside an MLEM launch.
static void* noalloc_scratch_ptr() {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) {
        cudaGetLastError();
        return nullptr;
    }
    return p;
}

// Largest number of resident CTA slots whose tables, sensitivity images and
// the candidates' hand-over flags fit the built-in scratch (0 if not even
// one slot does).
static int noalloc_slots(const boac_geom* g, const FusedVariant* v, int B) {
    int slots = variant_holders(g, v, B);
    while (slots > 0 && fused_layout(g, v, slots, B).total > kNoAllocScratchBytes) --slots;
    return slots;
}

}  // namespace boac

extern "C" int boac_mlem_noalloc(const boac_geom* g, const float* mu, const float* S,
                                 long long s_stride, float* F, int K, int B, double* L,
                                 int include_lgamma, void* stream) {
    BOAC_RANGE("boac_mlem_noalloc");
    // L is required: the status word of the bounded hand-over wait lives in
    // the built-in array, out of the caller's reach, so a candidate that gave
    // up shows only as a NaN score.
    if (!geom_ok(g) || !mu || !S || !F || !L || B < 1 || K < 0 || s_stride < 0) return BOAC_EINVAL;
    if (g->n_views % 2) return BOAC_EINVAL;
    // the one-CTA kernel: its per-CTA scratch is the smallest
    const FusedVariant* v = get_variant(g, single_cta_config(g));
    if (!v) return BOAC_EUNSUPPORTED;
    if (variant_holders(g, v, B) <= 0) return BOAC_ECUDA;
    const int slots = noalloc_slots(g, v, B);
    if (slots <= 0) return BOAC_EWORKSPACE;  // one candidate's scratch exceeds 64 MiB
    void* scratch = noalloc_scratch_ptr();
    if (!scratch) return BOAC_ECUDA;
    // The kernel writes every table entry and sensitivity pixel of a slot
    // before reading it; the status word and the candidates' hand-over flags
    // must start at zero and are cleared here, on the caller's stream.
    return launch_uniform(g, v, slots, mu, S, s_stride, F, K, B, L, include_lgamma,
                          static_cast<char*>(scratch), as_stream(stream));
}
