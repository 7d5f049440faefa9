// boac_grad.cu -- d ln P / d c_k: the derivative of the Eq. 5 score after K
// MLEM iterations (Sec. III step 3) with respect to the Legendre coefficients
// of Eq. 3, through the AREA rasterisation of Eq. 4.  The paper's optimiser
// is gradient-free; this gives the Bayesian optimiser gradients it can use
// alongside its surrogate.
//
// Exact reverse mode of the discretised pipeline, batched over candidates:
//   forward:  mu = raster(c); a = attenuation table; sens = A^T 1;
//             F^{n+1} = F^n (A^T (S / A F^n)) / sens, F^0 = 1;
//             L = sum S ln q - q [- ln S!], q = A F^K
//   reverse:  qbar = S/q - 1;  Fbar = A^T qbar;  abar += dx qbar (B F^K)
//             for n = K-1 .. 0 (F^n recomputed segment by segment from
//             checkpoints stored every `ckpt_every` iterations):
//               zbar = Fbar F^n / sens;  sensbar -= Fbar F^{n+1} / sens;
//               Fbar <- Fbar z^n / sens + A^T qbar',
//               with rbar = A zbar, qbar' = -rbar S / q^2,
//               abar += dx (r^n (B zbar) + qbar' (B F^n))
//             abar += dx (B sensbar)                       (sens = A^T 1)
//             mbar_k = -dx (abar_k a_k / 2 + sum_{k'<k} abar_k' a_k')
//             mubar = sum_v B_v^T mbar_v
//             dL/dc_k = sum_pixels mubar dmu/dR P_k(cos theta)   (float64)
// where B_v is bilinear sampling on view v's ray grid and abar the adjoint of
// the attenuation factor of every ray sample.  Float32 throughout except the
// score and the final sum over pixels, which are float64.
#include <cuda_runtime.h>
#include <math.h>

#include "boac_device.cuh"
#include "boac_fused.h"
#include "boac_internal.h"
#include "boac_plain_kernels.cuh"
#include "boac_sched.cuh"

namespace boac {

// abar[cand][v][k][b] += dx (y1[v][b] (B_v X1)(k, b) + y2[v][b] (B_v X2)(k, b))
// (y == nullptr: 1; X2 == nullptr: no second term).  One thread per ray.
__global__ void abar_accum_kernel(int n, int V, float dx, const float* __restrict__ y1,
                                  const float* __restrict__ X1, const float* __restrict__ y2,
                                  const float* __restrict__ X2, float* __restrict__ abar) {
    const int b = blockIdx.x * blockDim.x + threadIdx.x, v = blockIdx.y, cand = blockIdx.z;
    if (b >= n) return;
    const size_t nn = (size_t)n * n, vb = (size_t)V * n;
    const float w1 = dx * (y1 ? __ldg(y1 + cand * vb + (size_t)v * n + b) : 1.0f);
    const float w2 = X2 ? dx * (y2 ? __ldg(y2 + cand * vb + (size_t)v * n + b) : 1.0f) : 0.0f;
    if (w1 == 0.0f && w2 == 0.0f) return;
    const float* x1 = X1 + cand * nn;
    const float* x2 = X2 ? X2 + cand * nn : nullptr;
    float* ab = abar + ((size_t)cand * V + v) * nn;
    float cs, sn;
    view_cos_sin(v, V, &cs, &sn);
    const float c = 0.5f * (float)(n - 1);
    for (int k = 0; k < n; ++k) {
        float u, w;
        sample_uw(k, b, cs, sn, c, &u, &w);
        float add = w1 * bilerp_global(x1, n, u, w);
        if (x2) add = fmaf(w2, bilerp_global(x2, n, u, w), add);
        ab[(size_t)k * n + b] += add;
    }
}

// The same accumulation, one CTA per (candidate, sample grid), X1 and X2
// sampled through L1 as in the per-ray kernel but once per grid point for
// the grid's views: a column pass for views phi (table entry (k, b)) and
// phi + pi ((n-1-k, n-1-b)), a row pass for phi + pi/2 ((n-1-b, k)) and
// phi + 3pi/2 ((b, n-1-k)), every table access coalesced.
template <int N, int NT, bool QUAD>
__global__ void __launch_bounds__(NT) abar_grid_kernel(int V, float dx, const float* __restrict__ y1,
                                                      const float* __restrict__ X1, const float* __restrict__ y2,
                                                      const float* __restrict__ X2, float* __restrict__ abar) {
    constexpr int NSEG = NT / N, SEG = N / NSEG;
    static_assert(NT % N == 0 && N % NSEG == 0, "segmentation");
    const int gi = blockIdx.x, cand = blockIdx.y;
    const int tid = threadIdx.x, lb = tid % N, k0 = (tid / N) * SEG;
    const size_t nn = (size_t)N * N, vb = (size_t)V * N;
    const float* x1 = X1 + cand * nn;
    const float* x2 = X2 ? X2 + cand * nn : nullptr;
    float cs, sn;
    view_cos_sin(gi, V, &cs, &sn);
    const float c = 0.5f * (float)(N - 1);
    auto wt = [&](const float* y, int v, int bin) {
        return dx * (y ? __ldg(y + cand * vb + (size_t)v * N + bin) : 1.0f);
    };
    float* ab = abar + (size_t)cand * V * nn;
    {   // columns: views phi and phi + pi
        const int v1 = gi, v2 = gi + V / 2;
        const float w11 = wt(y1, v1, lb), w12 = wt(y1, v2, N - 1 - lb);
        const float w21 = x2 ? wt(y2, v1, lb) : 0.0f, w22 = x2 ? wt(y2, v2, N - 1 - lb) : 0.0f;
        float* a1 = ab + (size_t)v1 * nn;
        float* a2 = ab + (size_t)v2 * nn;
        for (int s = 0; s < SEG; ++s) {
            const int k = k0 + s;
            float u, w;
            sample_uw(k, lb, cs, sn, c, &u, &w);
            const float f1 = bilerp_global(x1, N, u, w);
            const float f2 = x2 ? bilerp_global(x2, N, u, w) : 0.0f;
            a1[(size_t)k * N + lb] += fmaf(w21, f2, w11 * f1);
            a2[(size_t)(N - 1 - k) * N + (N - 1 - lb)] += fmaf(w22, f2, w12 * f1);
        }
    }
    if (QUAD) {  // rows: views phi + pi/2 and phi + 3pi/2
        const int v3 = gi + V / 4, v4 = gi + 3 * V / 4, k = lb;
        const float w13 = wt(y1, v3, k), w14 = wt(y1, v4, N - 1 - k);
        const float w23 = x2 ? wt(y2, v3, k) : 0.0f, w24 = x2 ? wt(y2, v4, N - 1 - k) : 0.0f;
        float* a3 = ab + (size_t)v3 * nn;
        float* a4 = ab + (size_t)v4 * nn;
        for (int s = 0; s < SEG; ++s) {
            const int b = k0 + s;
            float u, w;
            sample_uw(k, b, cs, sn, c, &u, &w);
            const float f1 = bilerp_global(x1, N, u, w);
            const float f2 = x2 ? bilerp_global(x2, N, u, w) : 0.0f;
            a3[(size_t)(N - 1 - b) * N + k] += fmaf(w23, f2, w13 * f1);
            a4[(size_t)b * N + (N - 1 - k)] += fmaf(w24, f2, w14 * f1);
        }
    }
}

// abar += dx (y1 (B X1) + y2 (B X2)) for B candidates: per grid for image
// sides 64, 96, 128 and even view counts, else one thread per ray.
static int abar_accum(const boac_geom* g, int B, float dx, const float* y1, const float* X1, const float* y2,
                      const float* X2, float* abar, cudaStream_t st) {
    const int n = g->n, V = g->n_views;
    if (!((n == 64 || n == 96 || n == 128) && V % 2 == 0)) {
        abar_accum_kernel<<<ray_grid(g, B), kRayThreads, 0, st>>>(n, V, dx, y1, X1, y2, X2, abar);
        return launch_status();
    }
    const bool quad = V % 4 == 0;
    const dim3 grid(quad ? V / 4 : V / 2, B);
#define X(NV, TV)                                                                                   \
    if (n == NV) {                                                                                  \
        if (quad) abar_grid_kernel<NV, TV, true><<<grid, TV, 0, st>>>(V, dx, y1, X1, y2, X2, abar);  \
        else abar_grid_kernel<NV, TV, false><<<grid, TV, 0, st>>>(V, dx, y1, X1, y2, X2, abar);      \
    }
    X(64, 256) X(96, 384) X(128, 512)
#undef X
    return launch_status();
}

// In place: abar -> mbar_k = -dx (abar_k a_k / 2 + sum_{k' < k} abar_k' a_k')
// (derivative of a_k = exp(-dx (m_k/2 + sum_{k'>k} m_k')) w.r.t. the mu
// samples m of the ray).  One thread per ray.
__global__ void mbar_kernel(int n, int V, float dx, const float* __restrict__ tab,
                            float* __restrict__ abar) {
    const int b = blockIdx.x * blockDim.x + threadIdx.x, v = blockIdx.y, cand = blockIdx.z;
    if (b >= n) return;
    const size_t nn = (size_t)n * n;
    const float* t = tab + ((size_t)cand * V + v) * nn;
    float* ab = abar + ((size_t)cand * V + v) * nn;
    float prefix = 0.0f;
    for (int k = 0; k < n; ++k) {
        const float aa = ab[(size_t)k * n + b] * __ldg(t + (size_t)k * n + b);
        ab[(size_t)k * n + b] = -dx * (0.5f * aa + prefix);
        prefix += aa;
    }
}


__global__ void fill_ones_kernel(long long count, float* __restrict__ x) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < count;
         i += (long long)gridDim.x * blockDim.x)
        x[i] = 1.0f;
}

// r = S / q over B candidates (0 where q <= 0); S rows s_stride apart.
__global__ void ratio_batched_kernel(int B, int nbin, const float* __restrict__ S, long long s_stride,
                                     const float* __restrict__ q, float* __restrict__ r) {
    const long long total = (long long)B * nbin;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
         i += (long long)gridDim.x * blockDim.x) {
        const int cand = (int)(i / nbin), j = (int)(i % nbin);
        const float qi = q[i];
        r[i] = qi > 0.0f ? __ldg(S + cand * s_stride + j) / qi : 0.0f;
    }
}

// d L / d q^K: S/q - 1 (S > 0, q > 0), -1 (S == 0), 0 where L = -inf.
__global__ void qbar_final_kernel(int B, int nbin, const float* __restrict__ S, long long s_stride,
                                  const float* __restrict__ q, float* __restrict__ qbar) {
    const long long total = (long long)B * nbin;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
         i += (long long)gridDim.x * blockDim.x) {
        const int cand = (int)(i / nbin), j = (int)(i % nbin);
        const float s = __ldg(S + cand * s_stride + j), qi = q[i];
        qbar[i] = s > 0.0f ? (qi > 0.0f ? s / qi - 1.0f : 0.0f) : -1.0f;
    }
}

// qbar = -rbar S / q^2 where q > 0 (r = S / q), else 0.
__global__ void qbar_step_kernel(int B, int nbin, const float* __restrict__ S, long long s_stride,
                                 const float* __restrict__ q, const float* __restrict__ rbar,
                                 float* __restrict__ qbar) {
    const long long total = (long long)B * nbin;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
         i += (long long)gridDim.x * blockDim.x) {
        const int cand = (int)(i / nbin), j = (int)(i % nbin);
        const float qi = q[i];
        qbar[i] = qi > 0.0f ? -rbar[i] * (__ldg(S + cand * s_stride + j) / (qi * qi)) : 0.0f;
    }
}

// Adjoint of F^{n+1} = F^n z / sens for one step (per pixel):
//   zbar = Fbar F^n / sens; sensbar -= Fbar F^{n+1} / sens; Fnew = Fbar z / sens.
__global__ void mlem_step_adjoint_kernel(long long count, const float* __restrict__ Fbar,
                                         const float* __restrict__ Fn, const float* __restrict__ Fn1,
                                         const float* __restrict__ z, const float* __restrict__ sens,
                                         float* __restrict__ zbar, float* __restrict__ sensbar,
                                         float* __restrict__ Fnew) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < count;
         i += (long long)gridDim.x * blockDim.x) {
        const float s = sens[i];
        if (s > 0.0f) {
            const float fb = Fbar[i] / s;
            zbar[i] = fb * Fn[i];
            sensbar[i] -= fb * Fn1[i];
            Fnew[i] = fb * z[i];
        } else {
            zbar[i] = 0.0f;
            Fnew[i] = 0.0f;
        }
    }
}

// dL/dc_k = sum_pixels mubar dmu/dR P_k(z) for the AREA map
//   mu = (mu_b - mu_c) f(R) + mu_c f(R + dR), f(R') = clamp(1/2 + (R'-r)/dx, 0, 1),
//   R = max(0, sum c_k P_k(z)):  dmu/dR = ((mu_b - mu_c) f'(R) + mu_c f'(R+dR)) [R > 0],
// and with NP = 9 (per-candidate tissue values after the coefficients) also
//   dL/dmu_b = sum mubar f(R),  dL/dmu_c = sum mubar (f(R + dR) - f(R)),
//   dL/ddR = sum mubar mu_c f'(R + dR) [dR > 0],
// accumulated in float64 with a fixed reduction tree: block (cand, h) sums
// the pixels of part h of kCoefParts (a fixed split, so a candidate's
// gradient does not depend on the batch) into part_out[cand][h][NP], and
// grad_coef_sum_kernel adds the parts in order.
constexpr int kCoefParts = 8;
// pg: the pixel geometry (r, P_1..P_5 per pixel, pixel_geom_launch).
template <int NP>
__global__ void grad_coef_kernel(int n, double dx, double mu_b0, double mu_c0, double dR0,
                                 const float* __restrict__ coef, const float* __restrict__ mubar,
                                 const double* __restrict__ pg, double* __restrict__ part_out) {
    __shared__ double part[32][NP];
    const int cand = blockIdx.x, h = blockIdx.y;
    const int chunk = (n * n + kCoefParts - 1) / kCoefParts;
    const int p0 = h * chunk, p1 = p0 + chunk < n * n ? p0 + chunk : n * n;
    double c6[6];
#pragma unroll
    for (int k = 0; k < 6; ++k) c6[k] = (double)__ldg(coef + cand * NP + k);
    double mu_b = mu_b0, mu_c = mu_c0, dR = dR0;
    if (NP == kParams) {
        mu_b = (double)__ldg(coef + cand * NP + 6);
        mu_c = (double)__ldg(coef + cand * NP + 7);
        const double d = (double)__ldg(coef + cand * NP + 8);
        dR = d > 0.0 ? d : 0.0;
    }
    double acc[NP];
#pragma unroll
    for (int k = 0; k < NP; ++k) acc[k] = 0.0;
    const float* mb = mubar + (size_t)cand * n * n;
    const size_t nn = (size_t)n * n;
    for (int pix = p0 + threadIdx.x; pix < p1; pix += blockDim.x) {
        const double r = __ldg(pg + pix);
        double P[6];
        P[0] = 1.0;
#pragma unroll
        for (int k = 1; k < 6; ++k) P[k] = __ldg(pg + k * nn + pix);
        double R = 0.0;
#pragma unroll
        for (int k = 0; k < 6; ++k) R += c6[k] * P[k];
        if (NP == kParams) {
            const double m = (double)mb[pix];
            const double Rc = R > 0.0 ? R : 0.0;
            const double ein = 0.5 + (Rc - r) / dx, eout = 0.5 + (Rc + dR - r) / dx;
            const double fin = fmin(fmax(ein, 0.0), 1.0), fout = fmin(fmax(eout, 0.0), 1.0);
            acc[6] += m * fin;
            acc[7] += m * (fout - fin);
            if (dR > 0.0 && eout > 0.0 && eout < 1.0) acc[8] += m * mu_c / dx;
        }
        if (!(R > 0.0)) continue;
        const double ein = 0.5 + (R - r) / dx, eout = 0.5 + (R + dR - r) / dx;
        const double din = (ein > 0.0 && ein < 1.0) ? 1.0 / dx : 0.0;
        const double dout = (eout > 0.0 && eout < 1.0) ? 1.0 / dx : 0.0;
        const double dmu = (mu_b - mu_c) * din + mu_c * dout;
        if (dmu == 0.0) continue;
        const double s = (double)mb[pix] * dmu;
#pragma unroll
        for (int k = 0; k < 6; ++k) acc[k] += s * P[k];
    }
#pragma unroll
    for (int k = 0; k < NP; ++k)
        for (int off = 16; off > 0; off >>= 1) acc[k] += __shfl_down_sync(0xffffffffu, acc[k], off);
    if ((threadIdx.x & 31) == 0)
#pragma unroll
        for (int k = 0; k < NP; ++k) part[threadIdx.x >> 5][k] = acc[k];
    __syncthreads();
    if (threadIdx.x < NP) {
        double t = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += part[w][threadIdx.x];
        part_out[((size_t)cand * kCoefParts + h) * NP + threadIdx.x] = t;
    }
}

template <int NP>
__global__ void grad_coef_sum_kernel(int B, const double* __restrict__ part, double* __restrict__ grad) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= B * NP) return;
    const int cand = i / NP, k = i % NP;
    double t = 0.0;
    for (int h = 0; h < kCoefParts; ++h) t += part[((size_t)cand * kCoefParts + h) * NP + k];
    grad[i] = t;
}

// Doubles of coef_launch's scratch: the pixel geometry, then the parts.
static size_t coef_scratch_doubles(const boac_geom* g, int B) {
    return 6 * (size_t)g->n * g->n + (size_t)B * kCoefParts * kParams;
}

// mubar -> dL/dc (t != nullptr: c[B][6] with t's tissue values) or dL/dp
// (t == nullptr: p[B][9]); scratch: coef_scratch_doubles(g, B) doubles.
static int coef_launch(const boac_geom* g, const boac_tissue* t, const float* c, const float* mubar, int B,
                       double* scratch, double* dL_dc, cudaStream_t st) {
    const int n = g->n;
    const double dx = (double)g->pixel_cm;
    double* pg = scratch;
    double* part = scratch + 6 * (size_t)n * n;
    const int s = pixel_geom_launch(n, dx, pg, st);
    if (s != BOAC_OK) return s;
    const dim3 grid((unsigned)B, kCoefParts);
    if (t) {
        grad_coef_kernel<6><<<grid, 256, 0, st>>>(n, dx, (double)t->mu_b, (double)t->mu_c, (double)t->dR, c, mubar,
                                                  pg, part);
        grad_coef_sum_kernel<6><<<(B * 6 + 255) / 256, 256, 0, st>>>(B, part, dL_dc);
    } else {
        grad_coef_kernel<kParams><<<grid, 256, 0, st>>>(n, dx, 0.0, 0.0, 0.0, c, mubar, pg, part);
        grad_coef_sum_kernel<kParams><<<(B * kParams + 255) / 256, 256, 0, st>>>(B, part, dL_dc);
    }
    return launch_status();
}

// ------------------------------------------------------------- workspace
struct GradLayout {
    size_t mu, tab, abar, sens, sensbar, Fbar, Fnew, zbar, mubar, Fk, ck, Fseg, zseg, qseg, rseg, qK,
        qbar, rbar, partial, lg, coefp, total;
};

static GradLayout grad_layout(const boac_geom* g, int B, int K, int ckpt) {
    const size_t nn = (size_t)g->n * g->n, vb = (size_t)g->n_views * g->n_bins;
    const size_t Bs = (size_t)B;
    const int nseg = (K + ckpt - 1) / ckpt;
    GradLayout L{};
    size_t off = 0;
    auto take = [&](size_t floats) {
        size_t o = off;
        off += align256(floats * sizeof(float));
        return o;
    };
    L.mu = take(Bs * nn);
    L.tab = take(Bs * g->n_views * nn);
    L.abar = take(Bs * g->n_views * nn);
    L.sens = take(Bs * nn);
    L.sensbar = take(Bs * nn);
    L.Fbar = take(Bs * nn);
    L.Fnew = take(Bs * nn);
    L.zbar = take(Bs * nn);
    L.mubar = take(Bs * nn);
    L.Fk = take(Bs * nn);
    L.ck = take(Bs * (size_t)(nseg > 0 ? nseg : 1) * nn);
    L.Fseg = take(Bs * (size_t)(ckpt + 1) * nn);
    L.zseg = take(Bs * (size_t)ckpt * nn);
    L.qseg = take(Bs * (size_t)ckpt * vb);
    L.rseg = take(Bs * (size_t)ckpt * vb);
    L.qK = take(Bs * vb);
    L.qbar = take(Bs * vb);
    L.rbar = take(Bs * vb);
    L.partial = take(bp_partial_floats(g, B));
    L.lg = take(2 * kLgammaScratchDoubles);  // the ln S! sum of a shared sinogram
    L.coefp = take(2 * coef_scratch_doubles(g, B));  // doubles
    L.total = off;
    return L;
}

// Workspace of the fused gradient (boac_gradfused.cu) with cluster size G on
// `holders` clusters: per CTA its exponent slot and sensitivity rows; per
// candidate the AREA map, checkpoints, segment iterates (with their samples
// on every grid), Fbar, sensbar, the adjoint of the mu samples of every grid
// and mubar; the ln S! scratch, the coefficient reduction's partial sums and
// the scatter schedule.
struct GradFusedLayout {
    size_t mu, tab, sens, ck, segF, segz, segq, segB, Fbar, sensbar, abar, mubar, lg, coefp, sched, total;
};

static GradFusedLayout grad_fused_layout(const boac_geom* g, int B, int K, int ckpt, int G, int holders) {
    const size_t nn = (size_t)g->n * g->n, vb = (size_t)g->n_views * g->n_bins;
    const size_t Bs = (size_t)B, ctas = (size_t)holders * G;
    const int nseg = (K + ckpt - 1) / ckpt;
    GradFusedLayout L{};
    size_t off = 0;
    auto take = [&](size_t floats) {
        size_t o = off;
        off += align256(floats * sizeof(float));
        return o;
    };
    L.mu = take(Bs * nn);
    L.tab = take(ctas * grad_fused_tab_floats(g, G));
    L.sens = take(ctas * nn);
    L.ck = take(Bs * (size_t)(nseg > 0 ? nseg : 1) * nn);
    L.segF = take(Bs * (size_t)(ckpt + 1) * nn);
    L.segz = take(Bs * (size_t)ckpt * nn);
    L.segq = take(Bs * (size_t)ckpt * vb);
    L.segB = take(Bs * (size_t)ckpt * (g->n_views / 4) * nn);
    L.Fbar = take(Bs * nn);
    L.sensbar = take(Bs * nn);
    L.abar = take(Bs * (size_t)(g->n_views / 4) * nn);
    L.mubar = take(Bs * nn);
    L.lg = take(2 * kLgammaScratchDoubles);
    L.coefp = take(2 * coef_scratch_doubles(g, B));  // doubles
    L.sched = off;
    off += sched_bytes(g->n, g->n_views / 4);
    L.total = off;
    return L;
}

// The fused path: rasterise (AREA), the fused kernel (through mubar), then
// the coefficients.
static int score_grad_fused_run(const boac_geom* g, const boac_tissue* t, const float* c, const float* S,
                                long long s_stride, int K, int ckpt, int B, int include_lgamma, double* L,
                                double* dL_dc, float* F_out, void* ws, size_t ws_bytes, cudaStream_t st, int G,
                                int holders) {
    const GradFusedLayout lay = grad_fused_layout(g, B, K, ckpt, G, holders);
    if (!ws || ws_bytes < lay.total) return BOAC_EWORKSPACE;
    char* base = static_cast<char*>(ws);
    auto P = [&](size_t off) { return reinterpret_cast<float*>(base + off); };
    const int V = g->n_views;
    const float dx = g->pixel_cm;
    const size_t vb = (size_t)V * g->n_bins;
    NvtxPhases phase("gradient (fused): rasterise");
    int s = rasterize_launch(g, t, c, t ? 6 : kParams, B, BOAC_RASTER_AREA, P(lay.mu), st);
    if (s != BOAC_OK) return s;
    GradFusedArgs a;
    a.mu = P(lay.mu);
    a.S = S;
    a.s_stride = s_stride;
    a.B = B;
    a.V = V;
    a.K = K;
    a.ckpt = ckpt;
    a.dx = dx;
    a.include_lgamma = include_lgamma;
    a.lgS = include_lgamma && s_stride == 0
                ? lgamma_sum((int)vb, S, reinterpret_cast<double*>(base + lay.lg), st)
                : nullptr;
    a.tab = P(lay.tab);
    a.sens = P(lay.sens);
    a.ck = P(lay.ck);
    a.segF = P(lay.segF);
    a.segz = P(lay.segz);
    a.segq = P(lay.segq);
    a.segB = P(lay.segB);
    a.Fbar = P(lay.Fbar);
    a.sensbar = P(lay.sensbar);
    a.abar = P(lay.abar);
    a.mubar = P(lay.mubar);
    a.L = L;
    a.F_out = F_out;
    a.sched = reinterpret_cast<const unsigned short*>(base + lay.sched);
    phase.next("gradient (fused): forward, score, reverse sweep");
    s = grad_fused_launch(g, a, G, holders, st);
    if (s != BOAC_OK) return s;
    phase.next("gradient (fused): pixels -> coefficients");
    return coef_launch(g, t, c, P(lay.mubar), B, reinterpret_cast<double*>(base + lay.coefp), dL_dc, st);
}

// The path boac_score_grad takes: the fused kernel where it applies (G > 0).
static int grad_plan(const boac_geom* g, int B, int* holders) {
    *holders = 0;
    return grad_fused_plan(g, B, holders);
}

}  // namespace boac

using namespace boac;

extern "C" size_t boac_score_grad_workspace_bytes(const boac_geom* g, int B, int K, int ckpt_every) {
    if (!geom_ok(g) || B < 1 || B > 65535 || K < 0 || ckpt_every < 1) return 0;
    int holders = 0;
    const int G = grad_plan(g, B, &holders);
    const size_t fused = G > 0 ? grad_fused_layout(g, B, K, ckpt_every, G, holders).total : 0;
    const size_t unfused = grad_layout(g, B, K, ckpt_every).total;
    return fused > unfused ? fused : unfused;
}

// Score and gradient of B candidates: t != nullptr takes c[B][6] with the
// tissue values of t and writes dL_dc[B][6]; t == nullptr takes the
// 9-parameter form c[B][9] and writes dL_dc[B][9].
static int score_grad_run(const boac_geom* g, const boac_tissue* t, const float* c,
                          const float* S, long long s_stride, int K, int ckpt_every, int B,
                          int include_lgamma, double* L, double* dL_dc, float* F_out, void* ws,
                          size_t ws_bytes, void* stream, bool allow_fused = true) {
    if (allow_fused) {
        int holders = 0;
        const int G = grad_plan(g, B, &holders);
        if (G > 0)
            return score_grad_fused_run(g, t, c, S, s_stride, K, ckpt_every, B, include_lgamma, L, dL_dc, F_out,
                                        ws, ws_bytes, as_stream(stream), G, holders);
    }
    const GradLayout lay = grad_layout(g, B, K, ckpt_every);
    if (!ws || ws_bytes < lay.total) return BOAC_EWORKSPACE;
    char* base = static_cast<char*>(ws);
    auto P = [&](size_t off) { return reinterpret_cast<float*>(base + off); };
    float *mu = P(lay.mu), *tab = P(lay.tab), *abar = P(lay.abar), *sens = P(lay.sens),
          *sensbar = P(lay.sensbar), *Fbar = P(lay.Fbar), *Fnew = P(lay.Fnew), *zbar = P(lay.zbar),
          *mubar = P(lay.mubar), *Fk = P(lay.Fk), *ck = P(lay.ck), *Fseg = P(lay.Fseg),
          *zseg = P(lay.zseg), *qseg = P(lay.qseg), *rseg = P(lay.rseg), *qK = P(lay.qK),
          *qbar = P(lay.qbar), *rbar = P(lay.rbar), *partial = P(lay.partial);
    cudaStream_t st = as_stream(stream);
    const int n = g->n, V = g->n_views;
    const float dx = g->pixel_cm;
    const size_t nn = (size_t)n * n, vb = (size_t)V * g->n_bins;
    const long long cnt_pix = (long long)B * nn, cnt_bin = (long long)B * vb;
    const dim3 rg = ray_grid(g, B);
    const int g1p = grid_1d(cnt_pix, 256), g1b = grid_1d(cnt_bin, 256);

    // one MLEM step F_in -> F_out, leaving q, r and z = A^T r behind
    auto mlem_step = [&](const float* F_in, float* F_o, float* q, float* r, float* z) {
        project_table(g, B, tab, F_in, dx, q, st);
        ratio_batched_kernel<<<g1b, 256, 0, st>>>(B, (int)vb, S, s_stride, q, r);
        backproject_table(g, B, tab, r, dx, z, 0, partial, st);
        cudaMemcpyAsync(F_o, F_in, sizeof(float) * cnt_pix, cudaMemcpyDeviceToDevice, st);
        update_kernel<<<g1p, 256, 0, st>>>((int)cnt_pix, F_o, z, sens);
    };
    // ---- forward
    NvtxPhases phase("gradient: forward MLEM with checkpoints");
    int s = rasterize_launch(g, t, c, t ? 6 : kParams, B, BOAC_RASTER_AREA, mu, st);
    if (s != BOAC_OK) return s;
    attenuation_table_kernel<<<rg, kRayThreads, 0, st>>>(n, V, dx, mu, tab);
    backproject_table(g, B, tab, nullptr, dx, sens, 0, partial, st);
    cudaMemsetAsync(abar, 0, sizeof(float) * (size_t)B * V * nn, st);
    cudaMemsetAsync(sensbar, 0, sizeof(float) * cnt_pix, st);
    // F^0 = 1 into checkpoint 0; F^{j ckpt} into checkpoint j; F^K into Fk.
    // Iterates in between alternate between two temporaries (Fbar and Fnew
    // are not yet in use).
    fill_ones_kernel<<<g1p, 256, 0, st>>>(cnt_pix, ck);
    {
        const float* cur = ck;
        float* temps[2] = {Fnew, Fbar};
        int next_temp = 0;
        for (int it = 0; it < K; ++it) {
            float* nxt;
            if (it + 1 == K) nxt = Fk;
            else if ((it + 1) % ckpt_every == 0) nxt = ck + (size_t)((it + 1) / ckpt_every) * B * nn;
            else {
                nxt = temps[next_temp];
                next_temp ^= 1;
            }
            mlem_step(cur, nxt, qseg, rseg, zseg);
            cur = nxt;
        }
        if (K == 0) cudaMemcpyAsync(Fk, ck, sizeof(float) * cnt_pix, cudaMemcpyDeviceToDevice, st);
    }
    // ---- score and d L / d q^K
    phase.next("gradient: score and its adjoint");
    project_table(g, B, tab, Fk, dx, qK, st);
    const double* lgS = include_lgamma && s_stride == 0
                            ? lgamma_sum((int)vb, S, reinterpret_cast<double*>(base + lay.lg), st)
                            : nullptr;
    loglik_kernel<<<B, 256, 0, st>>>((int)vb, qK, S, s_stride, include_lgamma, L, lgS);
    if (F_out) cudaMemcpyAsync(F_out, Fk, sizeof(float) * cnt_pix, cudaMemcpyDeviceToDevice, st);
    qbar_final_kernel<<<g1b, 256, 0, st>>>(B, (int)vb, S, s_stride, qK, qbar);
    backproject_table(g, B, tab, qbar, dx, Fbar, 0, partial, st);
    abar_accum(g, B, dx, qbar, Fk, nullptr, nullptr, abar, st);

    // ---- reverse through the iterations, one checkpoint segment at a time
    phase.next("gradient: reverse sweep");
    const int nseg = (K + ckpt_every - 1) / ckpt_every;
    for (int j = nseg - 1; j >= 0; --j) {
        const int n0 = j * ckpt_every;
        const int len = (K - n0) < ckpt_every ? (K - n0) : ckpt_every;
        cudaMemcpyAsync(Fseg, ck + (size_t)j * B * nn, sizeof(float) * cnt_pix, cudaMemcpyDeviceToDevice, st);
        for (int tt = 0; tt < len; ++tt)
            mlem_step(Fseg + (size_t)tt * B * nn, Fseg + (size_t)(tt + 1) * B * nn, qseg + (size_t)tt * B * vb,
                      rseg + (size_t)tt * B * vb, zseg + (size_t)tt * B * nn);
        for (int tt = len - 1; tt >= 0; --tt) {
            const float* Fn = Fseg + (size_t)tt * B * nn;
            const float* Fn1 = Fseg + (size_t)(tt + 1) * B * nn;
            const float* q = qseg + (size_t)tt * B * vb;
            const float* r = rseg + (size_t)tt * B * vb;
            const float* z = zseg + (size_t)tt * B * nn;
            mlem_step_adjoint_kernel<<<g1p, 256, 0, st>>>(cnt_pix, Fbar, Fn, Fn1, z, sens, zbar, sensbar, Fnew);
            project_table(g, B, tab, zbar, dx, rbar, st);
            qbar_step_kernel<<<g1b, 256, 0, st>>>(B, (int)vb, S, s_stride, q, rbar, qbar);
            backproject_table(g, B, tab, qbar, dx, Fnew, 1, partial, st);
            abar_accum(g, B, dx, r, zbar, qbar, Fn, abar, st);
            float* tmp = Fbar;
            Fbar = Fnew;
            Fnew = tmp;
        }
    }
    // sens = A^T 1
    abar_accum(g, B, dx, nullptr, sensbar, nullptr, nullptr, abar, st);
    // attenuation -> mu samples -> pixels -> coefficients
    mbar_kernel<<<rg, kRayThreads, 0, st>>>(n, V, dx, tab, abar);
    backproject_table(g, B, abar, nullptr, 1.0f, mubar, 0, partial, st);
    return coef_launch(g, t, c, mubar, B, reinterpret_cast<double*>(base + lay.coefp), dL_dc, st);
}

extern "C" int boac_score_grad(const boac_geom* g, const boac_tissue* t, const float* c,
                               const float* S, long long s_stride, int K, int ckpt_every, int B,
                               int include_lgamma, double* L, double* dL_dc, float* F_out, void* ws,
                               size_t ws_bytes, void* stream) {
    BOAC_RANGE("boac_score_grad");
    if (!geom_ok(g) || !t || !c || !S || !L || !dL_dc || B < 1 || B > 65535 || K < 0 ||
        ckpt_every < 1 || s_stride < 0 || !(t->dR >= 0.0f))
        return BOAC_EINVAL;
    return score_grad_run(g, t, c, S, s_stride, K, ckpt_every, B, include_lgamma, L, dL_dc, F_out,
                          ws, ws_bytes, stream);
}

extern "C" int boac_score_grad_unfused(const boac_geom* g, const boac_tissue* t, const float* c,
                                       const float* S, long long s_stride, int K, int ckpt_every, int B,
                                       int include_lgamma, double* L, double* dL_dc, float* F_out, void* ws,
                                       size_t ws_bytes, void* stream) {
    BOAC_RANGE("boac_score_grad_unfused");
    if (!geom_ok(g) || !t || !c || !S || !L || !dL_dc || B < 1 || B > 65535 || K < 0 ||
        ckpt_every < 1 || s_stride < 0 || !(t->dR >= 0.0f))
        return BOAC_EINVAL;
    return score_grad_run(g, t, c, S, s_stride, K, ckpt_every, B, include_lgamma, L, dL_dc, F_out,
                          ws, ws_bytes, stream, false);
}

extern "C" int boac_score_grad_params(const boac_geom* g, const float* p, const float* S,
                                      long long s_stride, int K, int ckpt_every, int B,
                                      int include_lgamma, double* L, double* dL_dp, float* F_out,
                                      void* ws, size_t ws_bytes, void* stream) {
    BOAC_RANGE("boac_score_grad_params");
    if (!geom_ok(g) || !p || !S || !L || !dL_dp || B < 1 || B > 65535 || K < 0 ||
        ckpt_every < 1 || s_stride < 0)
        return BOAC_EINVAL;
    return score_grad_run(g, nullptr, p, S, s_stride, K, ckpt_every, B, include_lgamma, L, dL_dp,
                          F_out, ws, ws_bytes, stream);
}

#ifdef BOAC_CHECKED
namespace boac {
BOAC_FAULT_READER(bounds_faults_grad)
}  // namespace boac
#endif
