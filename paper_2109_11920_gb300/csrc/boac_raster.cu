// boac_raster.cu -- Eq. 3 (Legendre head boundary) and Eq. 4 (model
// attenuation map) on the pixel grid, evaluated in float64 so that the class
// of a pixel is decided as exactly as the definition allows.  A thread takes
// one pixel for a group of kRasterGroup candidates: the pixel's radius and
// Legendre values (a square root and five divisions, the costly part at the
// GPU's float64 rate) are computed once for the group.
#include <cuda_runtime.h>
#include <math.h>

#include "boac_device.cuh"
#include "boac_internal.h"

namespace boac {

constexpr int kRasterGroup = 8;

// The Legendre polynomials P_0..P_5 at z = cos theta by Bonnet's recursion
// (k+1) P_{k+1} = (2k+1) z P_k - k P_{k-1}.
__device__ __forceinline__ void legendre_values(double z, double* P) {
    P[0] = 1.0;
    P[1] = z;
#pragma unroll
    for (int k = 1; k < 5; ++k)
        P[k + 1] = __ddiv_rn(__dsub_rn(__dmul_rn((double)(2 * k + 1), __dmul_rn(z, P[k])),
                                       __dmul_rn((double)k, P[k - 1])),
                             (double)(k + 1));
}

// R(theta) before clamping: sum_{k=0..5} c_k P_k(z), in order of k.
__device__ __forceinline__ double legendre_series(const double* c, const double* P) {
    double R = 0.0;
#pragma unroll
    for (int k = 0; k < 6; ++k) R = __dadd_rn(R, __dmul_rn(c[k], P[k]));
    return R;
}

// Fraction of the pixel inside radius Rp: one-pixel radial ramp.
__device__ __forceinline__ double ramp(double Rp, double r, double dx) {
    double f = __dadd_rn(0.5, __ddiv_rn(__dsub_rn(Rp, r), dx));
    return fmin(fmax(f, 0.0), 1.0);
}

// Candidate cand's coefficients are coef[cand * pstride + 0..5]; with
// pstride = 9 its tissue values follow them (mu_b, mu_c, dR; a negative or
// NaN dR is taken as 0), with pstride = 6 every candidate uses the arguments.
// Item idx is pixel idx % n^2 of candidate group idx / n^2.
__global__ void rasterize_kernel(int n, double dx, double mu_b0, double mu_c0, double dR0,
                                 const float* __restrict__ coef, int pstride, int B, int mode,
                                 float* __restrict__ mu) {
    const long long nn = (long long)n * n;
    const long long total = (long long)((B + kRasterGroup - 1) / kRasterGroup) * nn;
    for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < total;
         idx += (long long)gridDim.x * blockDim.x) {
        const int grp = (int)(idx / nn);
        const int pix = (int)(idx % nn);
        const int i = pix / n, j = pix % n;
        const double cc = 0.5 * (double)(n - 1);
        const double x = __dmul_rn((double)j - cc, dx), y = __dmul_rn((double)i - cc, dx);
        const double r = __dsqrt_rn(__dadd_rn(__dmul_rn(x, x), __dmul_rn(y, y)));
        const double z = r > 0.0 ? __ddiv_rn(x, r) : 1.0;  // cos(atan2(y, x))
        double P[6];
        legendre_values(z, P);
        const int c0 = grp * kRasterGroup, c1 = c0 + kRasterGroup < B ? c0 + kRasterGroup : B;
        for (int cand = c0; cand < c1; ++cand) {
            double c6[6];
#pragma unroll
            for (int k = 0; k < 6; ++k) c6[k] = (double)__ldg(coef + (long long)cand * pstride + k);
            double mu_b = mu_b0, mu_c = mu_c0, dR = dR0;
            if (pstride == kParams) {
                const float* t = coef + (long long)cand * kParams + 6;
                mu_b = (double)__ldg(t);
                mu_c = (double)__ldg(t + 1);
                const double d = (double)__ldg(t + 2);
                dR = d > 0.0 ? d : 0.0;
            }
            double R = legendre_series(c6, P);
            if (!(R > 0.0)) R = 0.0;
            double m;
            if (mode == BOAC_RASTER_CENTER) {
                m = r < R ? mu_b : (r < __dadd_rn(R, dR) ? mu_c : 0.0);
            } else {
                const double fin = ramp(R, r, dx), fout = ramp(__dadd_rn(R, dR), r, dx);
                m = __dadd_rn(__dmul_rn(mu_b, fin), __dmul_rn(mu_c, __dsub_rn(fout, fin)));
            }
            mu[(long long)cand * nn + pix] = (float)m;
        }
    }
}

// The pixel geometry of the n x n grid for the gradient's coefficient
// reduction: pg[0][pix] = r, pg[k][pix] = P_k(cos theta) for k = 1..5, with
// the operations of rasterize_kernel (so both see the same R).
__global__ void pixel_geom_kernel(int n, double dx, double* __restrict__ pg) {
    const int nn = n * n;
    const int pix = blockIdx.x * blockDim.x + threadIdx.x;
    if (pix >= nn) return;
    const int i = pix / n, j = pix % n;
    const double cc = 0.5 * (double)(n - 1);
    const double x = __dmul_rn((double)j - cc, dx), y = __dmul_rn((double)i - cc, dx);
    const double r = __dsqrt_rn(__dadd_rn(__dmul_rn(x, x), __dmul_rn(y, y)));
    const double z = r > 0.0 ? __ddiv_rn(x, r) : 1.0;
    double P[6];
    legendre_values(z, P);
    pg[pix] = r;
#pragma unroll
    for (int k = 1; k < 6; ++k) pg[(size_t)k * nn + pix] = P[k];
}

}  // namespace boac

using namespace boac;

namespace boac {

int pixel_geom_launch(int n, double dx, double* pg, cudaStream_t st) {
    pixel_geom_kernel<<<(n * n + 255) / 256, 256, 0, st>>>(n, dx, pg);
    return launch_status();
}

int rasterize_launch(const boac_geom* g, const boac_tissue* t, const float* p, int pstride, int B,
                     int mode, float* mu, cudaStream_t st) {
    long long total = (long long)((B + kRasterGroup - 1) / kRasterGroup) * g->n * g->n;
    int threads = 256;
    long long blocks = (total + threads - 1) / threads;
    long long cap = 64LL * (sm_count() > 0 ? sm_count() : 1);
    if (blocks > cap) blocks = cap;
    const double mu_b = t ? (double)t->mu_b : 0.0, mu_c = t ? (double)t->mu_c : 0.0,
                 dR = t ? (double)t->dR : 0.0;
    rasterize_kernel<<<(int)blocks, threads, 0, st>>>(g->n, (double)g->pixel_cm, mu_b, mu_c, dR, p,
                                                      pstride, B, mode, mu);
    return launch_status();
}

}  // namespace boac

extern "C" int boac_rasterize_mu(const boac_geom* g, const boac_tissue* t, const float* c, int B,
                                 int mode, float* mu, void* stream) {
    BOAC_RANGE("boac_rasterize_mu");
    if (!geom_ok(g) || !t || !c || !mu || B < 1) return BOAC_EINVAL;
    if (mode != BOAC_RASTER_CENTER && mode != BOAC_RASTER_AREA) return BOAC_EINVAL;
    if (!(t->dR >= 0.0f)) return BOAC_EINVAL;
    return rasterize_launch(g, t, c, 6, B, mode, mu, as_stream(stream));
}

extern "C" int boac_rasterize_mu_params(const boac_geom* g, const float* p, int B, int mode,
                                        float* mu, void* stream) {
    BOAC_RANGE("boac_rasterize_mu_params");
    if (!geom_ok(g) || !p || !mu || B < 1) return BOAC_EINVAL;
    if (mode != BOAC_RASTER_CENTER && mode != BOAC_RASTER_AREA) return BOAC_EINVAL;
    return rasterize_launch(g, nullptr, p, kParams, B, mode, mu, as_stream(stream));
}

#ifdef BOAC_CHECKED
namespace boac {
BOAC_FAULT_READER(bounds_faults_raster)
}  // namespace boac
#endif
