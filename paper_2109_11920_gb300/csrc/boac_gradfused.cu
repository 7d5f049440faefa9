// boac_gradfused.cu -- the score gradient of boac_score_grad (reverse mode
// through the K MLEM iterations of Sec. III step 3, the Eq. 5 score and the
// AREA rasterisation of Eq. 4) in one persistent kernel per batch, for
// 64 x 64, 96 x 96 and 128 x 128 images with a view count divisible by 4.
//
// A candidate is owned by a thread-block cluster of G CTAs (G = 1: one CTA)
// with the on-chip layout of the fused MLEM kernel (boac_fused.cu): the
// image being sampled and the back-projection accumulator as padded
// shared-memory images, the sample buffer W, and the candidate's attenuation
// exponents for the rank's share of the sample grids in a per-CTA slot of
// the workspace.  Per candidate the kernel runs
//   1. set-up: exponents of the rank's grids, sensitivity sens = A^T 1;
//   2. K MLEM iterations from F = 1, storing F every ckpt iterations;
//   3. the score at F^K (Eq. 5) and its adjoint: qbar = S/q - 1 (0 where
//      q = 0 < S, -1 where S = 0), Fbar = A^T qbar, and the adjoint of every
//      attenuation factor, abar += dx qbar (B F^K);
//   4. the reverse sweep, one checkpoint segment at a time (last first):
//      recompute the segment's iterates F^n, q^n, z^n = A^T r^n (the last
//      segment keeps them from the forward pass), then for
//      n from the segment's end down to its start
//        zbar = Fbar F^n / sens,  sensbar -= Fbar F^{n+1} / sens,
//        rbar = A zbar,  qbar' = -rbar S / (q^n)^2 (0 where q^n = 0),
//        abar += dx (r^n (B zbar) + qbar' (B F^n)),
//        Fbar <- Fbar z^n / sens + A^T qbar';
//   5. the sensitivity's share, abar += dx (B sensbar);
//   6. mubar, the adjoint of the pixels of mu: the transposed sampling of
//      the mu samples' adjoint of every grid.
// No abar is stored: each step turns its abar into the adjoint of the mu
// samples on chip (a scan along each ray, the four views of a grid summed)
// and adds that, one value per sample of each grid, into a per-candidate
// buffer.  The float64 reduction of mubar to d/dc runs as a small batched
// kernel after this one (boac_grad.cu).
//
// In cluster mode (G > 1) rank r walks the grids [r V'/G, (r+1) V'/G) of the
// V' = V/4 sample grids with its own copies of the sampled images; every
// pixel-wise step is done by the rank owning the pixel's row, which sums
// the ranks' accumulators through distributed shared memory in rank order
// and writes its rows into every rank's image (F, zbar, sensbar) or into
// the candidate's buffers in global memory (checkpoints, segment iterates,
// Fbar, sensbar).
#include <cooperative_groups.h>
#include <cuda_runtime.h>
#include <math.h>

#include "boac_device.cuh"
#include "boac_fused.h"
#include "boac_internal.h"
#include "boac_plain_kernels.cuh"
#include "boac_sched.cuh"

namespace cg = cooperative_groups;

namespace boac {

// x += v at L2, the old value not returned (a reduction, not a load and a
// store).  Every element of the mu-sample adjoint is updated by one thread
// per pass, and one thread's updates of an address are applied in program
// order, so the sums are those of a read-modify-write, bit for bit.
__device__ __forceinline__ void red_add(float* p, float v) { atomicAdd(p, v); }

template <int N>
struct GradShape {
    static constexpr int NT = 8 * N;
    static constexpr int P = N + 1, WP = N + 1, NN = N * N;
    static constexpr int IMG = (N + 1) * (N + 2) + 1;
    static constexpr int NSEG = 8, SEG = N / 8;
    static constexpr size_t GSTRIDE = 2 * (size_t)NN + 2 * (size_t)N;  // one grid's exponent planes
};

template <int N>
__host__ __device__ constexpr size_t grad_fused_smem_bytes(int V) {
    using S = GradShape<N>;
    return sizeof(float) * (2 * (size_t)S::IMG + (size_t)N * S::WP + 4 * S::NSEG * N + 16 * N + 2 * (size_t)V) +
           sizeof(double) * 33;
}

template <int N, int G>
__global__ void __launch_bounds__(8 * N, 1) grad_fused_kernel(GradFusedArgs a) {
    using Sh = GradShape<N>;
    constexpr int NT = Sh::NT, P = Sh::P, WP = Sh::WP, NN = Sh::NN, IMG = Sh::IMG;
    constexpr int NSEG = Sh::NSEG, SEG = Sh::SEG;
    constexpr float kLog2e = 1.44269504088896340736f;
    constexpr int CE = SchedShape<N>::CLS_ENTRIES;

    extern __shared__ __align__(16) float smem[];
    float* img0 = smem;             // the image being sampled (F, mu, zbar, sensbar), padded
    float* img1 = img0 + IMG;       // back-projection accumulator, padded
    float* W = img1 + IMG;          // [N][WP] grid samples / weights
    float* redc = W + N * WP;       // [2][NSEG][N]
    float* redr = redc + 2 * NSEG * N;
    float* qv = redr + 2 * NSEG * N;  // [4][N] per-ray values of the grid (grid coordinates)
    float* c1 = qv + 4 * N;           // [4][N]
    float* c2 = c1 + 4 * N;           // [4][N]
    float* Sg = c2 + 4 * N;           // [4][N] the grid's sinogram rows by grid coordinate
    float* csn = Sg + 4 * N;          // [V][2]
    double* dred = reinterpret_cast<double*>(csn + 2 * a.V);

    const int tid = threadIdx.x, V = a.V;
    const int ngrid = V / 4;
    const float c = 0.5f * (float)(N - 1);
    const float dx = a.dx;
    const float ndl = -dx * kLog2e;
    const int lb = tid % N, seg = tid / N, k0 = seg * SEG;
    constexpr size_t gstride = Sh::GSTRIDE;
    for (int v = tid; v < V; v += NT) view_cos_sin(v, V, &csn[2 * v], &csn[2 * v + 1]);

    int rank = 0, g0 = 0, g1 = ngrid, R0 = 0, R1 = N;
    if constexpr (G > 1) {
        rank = (int)cg::this_cluster().block_rank();
        g0 = rank * ngrid / G;
        g1 = (rank + 1) * ngrid / G;
        R0 = rank * N / G;
        R1 = (rank + 1) * N / G;
    }
    float* tab = a.tab + (size_t)blockIdx.x * ((ngrid + G - 1) / G) * gstride;
    float* sens = a.sens + (size_t)blockIdx.x * NN;
    const int nseg = (a.K + a.ckpt - 1) / a.ckpt;
    const int holder = (int)(blockIdx.x / G), n_holders = (int)(gridDim.x / G);

    auto cluster_sync = [&]() {
        if constexpr (G > 1) cg::this_cluster().sync();
        else __syncthreads();
    };
    // the accumulators of all ranks at padded index pi, summed in rank order
    auto acc_sum = [&](int pi) -> float {
        if constexpr (G > 1) {
            cg::cluster_group cl = cg::this_cluster();
            float s = 0.0f;
#pragma unroll 1
            for (int r = 0; r < G; ++r) s += cl.map_shared_rank(img1, r)[pi];
            return s;
        } else {
            return img1[pi];
        }
    };
    // value v of padded index pi into every rank's img0
    auto put_all = [&](int pi, float v) {
        if constexpr (G > 1) {
            cg::cluster_group cl = cg::this_cluster();
#pragma unroll 1
            for (int r = 0; r < G; ++r) cl.map_shared_rank(img0, r)[pi] = v;
        } else {
            img0[pi] = v;
        }
    };
    auto pad = [&](int i) { return (i / N + 1) * P + (i % N) + 1; };
    auto clear_acc = [&]() {
        for (int i = tid; i < IMG; i += NT) img1[i] = 0.0f;
    };

    // ---- per-grid passes (the fused MLEM kernel's, with the grid's
    // exponent planes Xc (view phi, suffix), Uc, XrT (view phi + pi/2,
    // prefix, transposed), Ur; a = exp2(exponent))
    // Forward projection of img0 on grid gi: W <- the samples, qv <- dx sum a
    // sample for views phi, phi + pi (columns) and phi +- pi/2 (rows), in grid
    // coordinates.  Also stages the grid's sinogram rows into Sg (by grid
    // coordinate: S of view phi + pi and phi + 3pi/2 reversed).
    auto project_grid = [&](int gi, const float* S, float* bf) {
        const float cs = csn[2 * gi], sn = csn[2 * gi + 1];
        const float* Xc = tab + (gi - g0) * gstride;
        {   // the next grid's exponent planes: start their read from DRAM now
            const int gn = gi + 1 < g1 ? gi + 1 : g0;
            const float* nxt = tab + (gn - g0) * gstride;
            constexpr int kLines = (int)((2 * (size_t)NN * sizeof(float) + 127) / 128);
            for (int l = tid; l < kLines; l += NT) prefetch_l2(nxt + 32 * l);
        }
        const float* XrT = Xc + NN;
        const float* Uc = Xc + 2 * NN;
        const float* Ur = Uc + N;
        for (int t = tid; t < 4 * N; t += NT) {
            const int vi = t / N, j = t % N;
            const int v = vi == 0 ? gi : vi == 1 ? gi + V / 2 : vi == 2 ? gi + V / 4 : gi + 3 * V / 4;
            Sg[t] = __ldg(S + (size_t)v * N + ((vi & 1) ? N - 1 - j : j));
        }
        {
            const float uc = Uc[lb];
            float acc1 = 0.0f, acc2 = 0.0f;
            float fq[4];
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
                    W[k * WP + lb] = f;
                    fq[j] = f;  // bf: sample (k, b) at b n + k, four k per store, read once
                    acc1 = fmaf(ex2(yy[j]), f, acc1);
                    acc2 = fmaf(ex2(uc - yy[j]), f, acc2);
                }
                if (bf) __stcs(reinterpret_cast<float4*>(bf + lb * N + k0 + s4), make_float4(fq[0], fq[1], fq[2], fq[3]));
            }
            redc[seg * N + lb] = acc1;
            redc[(NSEG + seg) * N + lb] = acc2;
        }
        __syncthreads();
        {
            const float ur = Ur[lb];
            float acc3 = 0.0f, acc4 = 0.0f;
#pragma unroll 2
            for (int s4 = 0; s4 < SEG; s4 += 4) {
                const float4 y4 = *reinterpret_cast<const float4*>(XrT + tab_ix(N, k0 + s4, lb));
                const float yy[4] = {y4.x, y4.y, y4.z, y4.w};
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    const float f = W[lb * WP + k0 + s4 + j];
                    acc3 = fmaf(ex2(yy[j]), f, acc3);
                    acc4 = fmaf(ex2(ur - yy[j]), f, acc4);
                }
            }
            redr[seg * N + lb] = acc3;
            redr[(NSEG + seg) * N + lb] = acc4;
        }
        __syncthreads();
        for (int t = tid; t < 4 * N; t += NT) {
            const int vi = t / N, j = t % N;
            const float* rp = (vi >= 2 ? redr : redc) + ((vi & 1) ? NSEG * N : 0);
            float q = 0.0f;
#pragma unroll
            for (int s2 = 0; s2 < NSEG; ++s2) q += rp[s2 * N + j];
            qv[t] = q * dx;
        }
        __syncthreads();
    };
    // The adjoint of the mu samples of grid gi, added into Mg ([k][b], grid
    // coordinates) for one step.  Per view v the adjoint of the factor at
    // sample s is abar_v(s) = a_v(s) dx (k1_v x(s) + k2_v y(s)), x the
    // samples in W, y those stored by an earlier project_grid of another
    // image (sample (k, b) at Yc[b n + k]; nullptr: none),
    // k1 / k2 per ray in grid coordinates.  A factor's exponent sums the mu
    // samples between its sample and the detector (half its own), so the
    // sample's adjoint is -dx (abar/2 + the abar of the samples farther from
    // the detector): a prefix along k for view phi, a suffix for phi + pi, a
    // suffix along b for phi + pi/2 and a prefix for phi + 3pi/2.  The four
    // views of a grid share its samples, so one sum per sample is added.
    // Each thread scans its SEG samples of a ray; the other segments enter
    // as a constant per (ray, segment) from the segment totals.  The column
    // views' part within the segment goes out at once; the row pass leaves
    // its part in W, and the rest (row part and both constants) goes out as
    // a second reduction per sample, lanes along b in both.
    auto mubar_grid = [&](int gi, float* Mg, const float* k1, const float* k2, const float* Yc) {
        const bool Y = Yc != nullptr;
        const float* Xc = tab + (gi - g0) * gstride;
        const float* XrT = Xc + NN;
        const float* Uc = Xc + 2 * NN;
        const float* Ur = Uc + N;
        {   // views phi, phi + pi: thread on column lb
            const float uc = Uc[lb];
            const float w11 = dx * k1[lb], w12 = dx * k1[N + lb];
            const float w21 = Y ? dx * k2[lb] : 0.0f, w22 = Y ? dx * k2[N + lb] : 0.0f;
            float p1 = 0.0f, q2 = 0.0f;
#pragma unroll 1
            for (int s4 = 0; s4 < SEG; s4 += 4) {
                const float4 y4 = Y ? __ldcg(reinterpret_cast<const float4*>(Yc + lb * N + k0 + s4))
                                    : make_float4(0.0f, 0.0f, 0.0f, 0.0f);
                const float yy[4] = {y4.x, y4.y, y4.z, y4.w};
                const float4 e4 = *reinterpret_cast<const float4*>(Xc + tab_ix(N, k0 + s4, lb));
                const float ee[4] = {e4.x, e4.y, e4.z, e4.w};
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    const int k = k0 + s4 + j;
                    const float x = W[k * WP + lb];
                    const float ye = ee[j];
                    const float a1 = ex2(ye) * fmaf(w21, yy[j], w11 * x);
                    const float a2 = ex2(uc - ye) * fmaf(w22, yy[j], w12 * x);
                    q2 += a2;
                    red_add(Mg + k * N + lb, -dx * fmaf(0.5f, a1 + a2, p1 - q2));  // + a2 of the segment
                    p1 += a1;
                }
            }
            redc[seg * N + lb] = p1;
            redc[(NSEG + seg) * N + lb] = q2;
        }
        __syncthreads();
        {   // views phi + pi/2, phi + 3pi/2: thread on row lb
            const int k = lb;
            const float ur = Ur[k];
            const float w13 = dx * k1[2 * N + k], w14 = dx * k1[3 * N + k];
            const float w23 = Y ? dx * k2[2 * N + k] : 0.0f, w24 = Y ? dx * k2[3 * N + k] : 0.0f;
            float q3 = 0.0f, p4 = 0.0f;
#pragma unroll 1
            for (int s4 = 0; s4 < SEG; s4 += 4) {
                const float4 e4 = *reinterpret_cast<const float4*>(XrT + tab_ix(N, k0 + s4, k));
                const float ee[4] = {e4.x, e4.y, e4.z, e4.w};
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    const int b = k0 + s4 + j;
                    const float x = W[k * WP + b];
                    const float yv = Y ? __ldcg(Yc + b * N + k) : 0.0f;
                    const float ye = ee[j];
                    const float a3 = ex2(ye) * fmaf(w23, yv, w13 * x);
                    const float a4 = ex2(ur - ye) * fmaf(w24, yv, w14 * x);
                    q3 += a3;
                    W[k * WP + b] = fmaf(0.5f, a3 + a4, p4 - q3);  // + a3 of the segment
                    p4 += a4;
                }
            }
            redr[seg * N + k] = q3;
            redr[(NSEG + seg) * N + k] = p4;
        }
        __syncthreads();
        // constants of this thread's segment: column lb (a1 of the earlier
        // segments, a2 of this and the later ones), row lb (a3 of this and
        // the later segments, a4 of the earlier ones)
        float cc = 0.0f, cr = 0.0f;
#pragma unroll
        for (int s2 = 0; s2 < NSEG; ++s2) {
            cc += s2 < seg ? redc[s2 * N + lb] : redc[(NSEG + s2) * N + lb];
            cr += s2 >= seg ? redr[s2 * N + lb] : redr[(NSEG + s2) * N + lb];
        }
        __syncthreads();
        redr[seg * N + lb] = cr;
        __syncthreads();
        const float* crow = redr + (lb / SEG) * N;  // row constants of column lb's segment
#pragma unroll
        for (int s = 0; s < SEG; ++s) {
            const int k = k0 + s;
            red_add(Mg + k * N + lb, -dx * (W[k * WP + lb] + crow[k] + cc));
        }
        __syncthreads();
    };
    // Back-projection of per-ray coefficients kc (grid coordinates) on grid
    // gi into img1: W <- dx sum_v a_v kc_v, then the scheduled scatter.
    auto backproject_grid = [&](int gi, const float* kc) {
        const float cs = csn[2 * gi], sn = csn[2 * gi + 1];
        const float* Xc = tab + (gi - g0) * gstride;
        const float* XrT = Xc + NN;
        const float* Uc = Xc + 2 * NN;
        const float* Ur = Uc + N;
        const unsigned short* gs = a.sched + (size_t)gi * 9 * CE;
        SchedSlots<N, NT> sched0;
        sched0.load(gs);
        {
            const float uc = Uc[lb];
            const float r1 = dx * kc[lb], r2 = dx * kc[N + lb];
#pragma unroll 2
            for (int s4 = 0; s4 < SEG; s4 += 4) {
                const float4 y4 = *reinterpret_cast<const float4*>(Xc + tab_ix(N, k0 + s4, lb));
                const float yy[4] = {y4.x, y4.y, y4.z, y4.w};
#pragma unroll
                for (int j = 0; j < 4; ++j) W[(k0 + s4 + j) * WP + lb] = fmaf(ex2(yy[j]), r1, ex2(uc - yy[j]) * r2);
            }
        }
        __syncthreads();
        {
            const float ur = Ur[lb];
            const float r3 = dx * kc[2 * N + lb], r4 = dx * kc[3 * N + lb];
            for (int s4 = 0; s4 < SEG; s4 += 4) {
                const float4 y4 = *reinterpret_cast<const float4*>(XrT + tab_ix(N, k0 + s4, lb));
                const float yy[4] = {y4.x, y4.y, y4.z, y4.w};
#pragma unroll
                for (int j = 0; j < 4; ++j) W[lb * WP + k0 + s4 + j] += fmaf(ex2(yy[j]), r3, ex2(ur - yy[j]) * r4);
            }
        }
        __syncthreads();
        scatter_scheduled<N, NT, P, WP>(W, img1, cs, sn, c, gs, sched0);
    };

    for (int cand = holder; cand < a.B; cand += n_holders) {
        const float* __restrict__ S = a.S + (long long)cand * a.s_stride;
        const float* __restrict__ mu = a.mu + (size_t)cand * NN;
        float* ck = a.ck + (size_t)cand * (nseg > 0 ? nseg : 1) * NN;
        float* segF = a.segF + (size_t)cand * (a.ckpt + 1) * NN;
        float* segz = a.segz + (size_t)cand * a.ckpt * NN;
        float* segq = a.segq + (size_t)cand * a.ckpt * V * N;
        float* Fbar = a.Fbar + (size_t)cand * NN;
        float* sensbar = a.sensbar + (size_t)cand * NN;
        float* Ms = a.abar + (size_t)cand * ngrid * NN;
        float* segB = a.segB + (size_t)cand * a.ckpt * ngrid * NN;

        // ---- 1. set-up: mu -> img0, exponents of this rank's grids, sens
        for (int i = tid; i < IMG; i += NT) {
            img0[i] = 0.0f;
            img1[i] = 0.0f;
        }
        __syncthreads();
        for (int i = tid; i < NN; i += NT) img0[pad(i)] = __ldg(mu + i);
        // the mu-sample adjoint of this rank's grids starts at 0; sensbar
        // (this rank's rows) too
        for (size_t i = (size_t)g0 * NN + tid; i < (size_t)g1 * NN; i += NT) Ms[i] = 0.0f;
        for (int i = R0 * N + tid; i < R1 * N; i += NT) sensbar[i] = 0.0f;
        __syncthreads();
        for (int gi = g0; gi < g1; ++gi) {
            const float cs = csn[2 * gi], sn = csn[2 * gi + 1];
            float* Xc = tab + (gi - g0) * gstride;
            float* XrT = Xc + NN;
            float* Uc = Xc + 2 * NN;
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
            {
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
            {
                float pr = 0.0f;
#pragma unroll 8
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
#pragma unroll 8
                for (int s = 0; s < SEG; ++s) {
                    const int b = k0 + s;
                    const float m = W[lb * WP + b];
                    XrT[tab_ix(N, b, lb)] = ndl * (0.5f * m + pre);
                    pre += m;
                }
                if (seg == 0) Ur[lb] = ndl * total;
            }
            __syncthreads();
            for (int t = tid; t < 4 * N; t += NT) c1[t] = 1.0f;
            __syncthreads();
            backproject_grid(gi, c1);  // sens: a_v summed on the grid, scattered
        }
        cluster_sync();
        for (int i = R0 * N + tid; i < R1 * N; i += NT) sens[i - R0 * N] = acc_sum(pad(i));
        cluster_sync();
        // F^0 = 1 in every rank's img0 (interior); accumulator cleared
        for (int i = tid; i < NN; i += NT) img0[pad(i)] = 1.0f;
        clear_acc();
        __syncthreads();

        // one MLEM iteration of img0 (F) on this rank's grids, then the
        // update of the rows of this rank; with `rec`, F^n, q^n and z^n into
        // the segment buffers at position t
        auto mlem_iteration = [&](bool rec, int t) {
            if (rec)
                for (int i = R0 * N + tid; i < R1 * N; i += NT) segF[(size_t)t * NN + i] = img0[pad(i)];
            for (int gi = g0; gi < g1; ++gi) {
                // (rec: the samples of F^n too, for the reverse step's abar)
                project_grid(gi, S, rec ? segB + ((size_t)t * ngrid + gi) * NN : nullptr);
                for (int u = tid; u < 4 * N; u += NT) {
                    const float q = qv[u];
                    if (rec) segq[((size_t)t * ngrid + gi) * 4 * N + u] = q;
                    c1[u] = q > 0.0f ? Sg[u] / q : 0.0f;
                }
                __syncthreads();
                backproject_grid(gi, c1);
            }
            cluster_sync();
            for (int i = R0 * N + tid; i < R1 * N; i += NT) {
                const int pi = pad(i);
                const float z = acc_sum(pi), sv = sens[i - R0 * N];
                if (rec) segz[(size_t)t * NN + i] = z;
                put_all(pi, sv > 0.0f ? img0[pi] * z / sv : 0.0f);
            }
            cluster_sync();
            clear_acc();
            __syncthreads();
        };

        // ---- 2. forward with checkpoints; the iterations of the last
        // segment keep their data for the reverse sweep as they run, so that
        // segment is not recomputed
        const int n_last = nseg > 0 ? (nseg - 1) * a.ckpt : 0;
        for (int it = 0; it < a.K; ++it) {
            if (it % a.ckpt == 0)
                for (int i = R0 * N + tid; i < R1 * N; i += NT) ck[(size_t)(it / a.ckpt) * NN + i] = img0[pad(i)];
            mlem_iteration(it >= n_last, it - n_last);
        }

        // ---- 3. score at F^K and its adjoint
        double lacc = 0.0;
        for (int gi = g0; gi < g1; ++gi) {
            project_grid(gi, S, nullptr);
            for (int u = tid; u < 4 * N; u += NT) {
                const float s = Sg[u], q = qv[u];
                lacc += loglik_term(s, q, a.include_lgamma && !a.lgS);
                c1[u] = s > 0.0f ? (q > 0.0f ? s / q - 1.0f : 0.0f) : -1.0f;
            }
            __syncthreads();
            mubar_grid(gi, Ms + (size_t)gi * NN, c1, nullptr, nullptr);  // W holds B F^K
            backproject_grid(gi, c1);
        }
        for (int off = 16; off > 0; off >>= 1) lacc += __shfl_down_sync(0xffffffffu, lacc, off);
        if ((tid & 31) == 0) dred[tid >> 5] = lacc;
        if (a.F_out)
            for (int i = R0 * N + tid; i < R1 * N; i += NT) a.F_out[(size_t)cand * NN + i] = img0[pad(i)];
        __syncthreads();
        if (tid == 0) {
            double t = 0.0;
            for (int wi = 0; wi < NT / 32; ++wi) t += dred[wi];
            dred[32] = t;
        }
        cluster_sync();
        if (rank == 0 && tid == 0) {
            double t = 0.0;
            if constexpr (G > 1) {
                cg::cluster_group cl = cg::this_cluster();
                for (int r = 0; r < G; ++r) t += cl.map_shared_rank(dred, r)[32];
            } else {
                t = dred[32];
            }
            a.L[cand] = a.include_lgamma && a.lgS ? t - *a.lgS : t;
        }
        for (int i = R0 * N + tid; i < R1 * N; i += NT) Fbar[i] = acc_sum(pad(i));
        cluster_sync();
        clear_acc();
        __syncthreads();

        // ---- 4. reverse sweep, one checkpoint segment at a time
        for (int j = nseg - 1; j >= 0; --j) {
            const int n0 = j * a.ckpt;
            const int len = a.K - n0 < a.ckpt ? a.K - n0 : a.ckpt;
            if (j < nseg - 1) {  // recompute: F^{n0} from its checkpoint into every rank's img0
                for (int i = R0 * N + tid; i < R1 * N; i += NT) put_all(pad(i), __ldcg(ck + (size_t)j * NN + i));
                cluster_sync();
                for (int t = 0; t < len; ++t) mlem_iteration(true, t);
            }
            // F^{n0 + len} (the last segment: F^K, still in img0)
            for (int i = R0 * N + tid; i < R1 * N; i += NT) segF[(size_t)len * NN + i] = img0[pad(i)];
            cluster_sync();
            for (int t = len - 1; t >= 0; --t) {
                const float* Fn = segF + (size_t)t * NN;
                const float* Fn1 = segF + (size_t)(t + 1) * NN;
                const float* zn = segz + (size_t)t * NN;
                // zbar into every rank's img0; sensbar; the kept part of Fbar
                for (int i = R0 * N + tid; i < R1 * N; i += NT) {
                    const float sv = sens[i - R0 * N];
                    float zb = 0.0f, keep = 0.0f;
                    if (sv > 0.0f) {
                        const float fb = __ldcg(Fbar + i) / sv;
                        zb = fb * __ldcg(Fn + i);
                        sensbar[i] = __ldcg(sensbar + i) - fb * __ldcg(Fn1 + i);
                        keep = fb * __ldcg(zn + i);
                    }
                    put_all(pad(i), zb);
                    Fbar[i] = keep;
                }
                cluster_sync();
                for (int gi = g0; gi < g1; ++gi) {
                    {   // this grid's B F^n samples, read by mubar_grid below
                        const float* yb = segB + ((size_t)t * ngrid + gi) * NN;
                        constexpr int kLinesY = (int)(((size_t)NN * sizeof(float) + 127) / 128);
                        for (int l = tid; l < kLinesY; l += NT) prefetch_l2(yb + 32 * l);
                    }
                    project_grid(gi, S, nullptr);  // W <- B zbar, qv <- A zbar (rbar)
                    for (int u = tid; u < 4 * N; u += NT) {
                        const float q = __ldcg(segq + ((size_t)t * ngrid + gi) * 4 * N + u), s = Sg[u];
                        c1[u] = q > 0.0f ? s / q : 0.0f;                       // r^n
                        c2[u] = q > 0.0f ? -qv[u] * (s / (q * q)) : 0.0f;      // qbar'
                    }
                    __syncthreads();
                    mubar_grid(gi, Ms + (size_t)gi * NN, c1, c2, segB + ((size_t)t * ngrid + gi) * NN);  // y = B F^n
                    backproject_grid(gi, c2);
                }
                cluster_sync();
                for (int i = R0 * N + tid; i < R1 * N; i += NT) Fbar[i] = __ldcg(Fbar + i) + acc_sum(pad(i));
                cluster_sync();
                clear_acc();
                __syncthreads();
            }
        }

        // ---- 5. the sensitivity's share: abar += dx (B sensbar)
        for (int i = R0 * N + tid; i < R1 * N; i += NT) put_all(pad(i), __ldcg(sensbar + i));
        cluster_sync();
        for (int t = tid; t < 4 * N; t += NT) c1[t] = 1.0f;
        __syncthreads();
        for (int gi = g0; gi < g1; ++gi) {
            project_grid(gi, S, nullptr);  // W <- B sensbar
            mubar_grid(gi, Ms + (size_t)gi * NN, c1, nullptr, nullptr);
        }

        // ---- 6. the mu samples' adjoint to the pixels: mubar = sum over
        // grids of the transposed sampling of Ms (img1 is clear here)
        for (int gi = g0; gi < g1; ++gi) {
            const unsigned short* gs = a.sched + (size_t)gi * 9 * CE;
            SchedSlots<N, NT> sched0;
            sched0.load(gs);
            const float* Mg = Ms + (size_t)gi * NN;
#pragma unroll 4
            for (int s = 0; s < SEG; ++s) W[(k0 + s) * WP + lb] = __ldcg(Mg + (k0 + s) * N + lb);
            __syncthreads();
            scatter_scheduled<N, NT, P, WP>(W, img1, csn[2 * gi], csn[2 * gi + 1], c, gs, sched0);
        }
        cluster_sync();
        for (int i = R0 * N + tid; i < R1 * N; i += NT) a.mubar[(size_t)cand * NN + i] = acc_sum(pad(i));
        cluster_sync();  // no rank still reads another's memory
        clear_acc();
    }
}

// ---------------------------------------------------------------- host side
constexpr int kGradSizes[] = {1, 2, 4, 8};
constexpr int kGradSizeCount = 4;

template <int N, int G>
static cudaLaunchConfig_t grad_config(int clusters, int V, cudaStream_t st, cudaLaunchAttribute* attr) {
    cudaLaunchConfig_t cfg = {};
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = G;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.gridDim = dim3((unsigned)(clusters * G), 1, 1);
    cfg.blockDim = dim3(8 * N, 1, 1);
    cfg.dynamicSmemBytes = grad_fused_smem_bytes<N>(V);
    cfg.stream = st;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cfg;
}

template <int N, int G>
static int grad_attrs() {
    constexpr int kDev = 64;
    static bool done[kDev];
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kDev) return launch_status();
    if (!done[dev]) {
        if (cudaFuncSetAttribute(grad_fused_kernel<N, G>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)grad_fused_smem_bytes<N>(kMaxViews)) != cudaSuccess)
            return launch_status();
        done[dev] = true;
    }
    return BOAC_OK;
}

// Clusters of G CTAs (G = 1: CTAs) resident at once; cached per device.
template <int N, int G>
static int grad_holders_t() {
    constexpr int kDev = 64;
    static int cached[kDev];
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kDev) {
        cudaGetLastError();
        return 0;
    }
    if (cached[dev]) return cached[dev];
    if (grad_attrs<N, G>() != BOAC_OK) {
        cudaGetLastError();
        return 0;
    }
    int h = 0;
    if (G == 1) {
        int per = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, grad_fused_kernel<N, G>, 8 * N,
                                                          grad_fused_smem_bytes<N>(kMaxViews)) != cudaSuccess) {
            cudaGetLastError();
            return 0;
        }
        h = per * sm_count();
    } else {
        cudaLaunchAttribute attr[1];
        cudaLaunchConfig_t cfg = grad_config<N, G>(64, kMaxViews, nullptr, attr);
        if (cudaOccupancyMaxActiveClusters(&h, grad_fused_kernel<N, G>, &cfg) != cudaSuccess) {
            cudaGetLastError();
            return 0;
        }
    }
    cached[dev] = h;
    return h;
}

static int grad_holders(int n, int G) {
#define X(NV)                                                  \
    if (n == NV) {                                             \
        switch (G) {                                           \
            case 1: return grad_holders_t<NV, 1>();            \
            case 2: return grad_holders_t<NV, 2>();            \
            case 4: return grad_holders_t<NV, 4>();            \
            case 8: return grad_holders_t<NV, 8>();            \
        }                                                      \
    }
    X(64) X(96) X(128)
#undef X
    return 0;
}

bool grad_fused_supported(const boac_geom* g) {
    return (g->n == 64 || g->n == 96 || g->n == 128) && g->n_views % 4 == 0;
}

// The cluster size for B candidates: the least modelled time, rounds(G)
// (ceil(grids / G) + 1.6) grid passes per step, rounds = ceil(B / resident
// clusters of G) (the fused MLEM kernel's model; one CTA is G = 1); returns
// G and the clusters to launch, or 0.
int grad_fused_plan(const boac_geom* g, int B, int* holders) {
    if (!grad_fused_supported(g) || B < 1) return 0;
    const int ngrid = g->n_views / 4;
    int best = 0, best_h = 0;
    double best_t = 0.0;
    for (int i = 0; i < kGradSizeCount; ++i) {
        const int G = kGradSizes[i];
        if (ngrid < G) continue;
        const int h = grad_holders(g->n, G);
        if (h <= 0) continue;
        const int rounds = (B + h - 1) / h;
        const double t = rounds * ((ngrid + G - 1) / G + (G > 1 ? 1.6 : 0.0));
        if (best == 0 || t < best_t - 1e-9) {
            best = G;
            best_h = h < B ? h : B;
            best_t = t;
        }
    }
    *holders = best_h;
    return best;
}

size_t grad_fused_tab_floats(const boac_geom* g, int G) {
    return (size_t)((g->n_views / 4 + G - 1) / G) * (2 * (size_t)g->n * g->n + 2 * (size_t)g->n);
}

template <int N, int G>
static int grad_launch_t(const GradFusedArgs& a, int clusters, cudaStream_t st) {
    int s = grad_attrs<N, G>();
    if (s != BOAC_OK) return s;
    cudaLaunchAttribute attr[1];
    cudaLaunchConfig_t cfg = grad_config<N, G>(clusters, a.V, st, attr);
    if (G == 1) {
        grad_fused_kernel<N, G><<<clusters, 8 * N, grad_fused_smem_bytes<N>(a.V), st>>>(a);
        return launch_status();
    }
    if (cudaLaunchKernelEx(&cfg, grad_fused_kernel<N, G>, a) != cudaSuccess) return launch_status();
    return launch_status();
}

int grad_fused_launch(const boac_geom* g, const GradFusedArgs& args, int G, int clusters, cudaStream_t st) {
    if (clusters < 1) return BOAC_EINVAL;
    GradFusedArgs a = args;
    int s = BOAC_OK;
    a.sched = sched_prepare(g->n, g->n_views, g->n_views / 4, g->n + 1 /* GradShape<N>::WP */,
                            const_cast<unsigned short*>(args.sched), st, &s);
    if (s != BOAC_OK) return s;
#define X(NV)                                                           \
    if (g->n == NV) {                                                   \
        switch (G) {                                                    \
            case 1: return grad_launch_t<NV, 1>(a, clusters, st);       \
            case 2: return grad_launch_t<NV, 2>(a, clusters, st);       \
            case 4: return grad_launch_t<NV, 4>(a, clusters, st);       \
            case 8: return grad_launch_t<NV, 8>(a, clusters, st);       \
        }                                                               \
    }
    X(64) X(96) X(128)
#undef X
    return BOAC_EUNSUPPORTED;
}

}  // namespace boac

#ifdef BOAC_CHECKED
namespace boac {
BOAC_FAULT_READER(bounds_faults_gradfused)
}  // namespace boac
#endif
