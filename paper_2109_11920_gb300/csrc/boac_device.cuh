// boac_device.cuh -- device helpers shared by every kernel of the library:
// view angles, ray-sample coordinates, bilinear sampling and its transpose.
//
// Every kernel computes the continuous pixel coordinates (u, w) of ray sample
// (k, b) with sample_uw(), so the forward projector, the back-projector and
// the gradient all use bit-identical bilinear weights (the back-projector is
// the exact transpose of the projector in float32 up to summation order).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/boac.h"

namespace boac {

// Checked builds (-DBOAC_CHECKED, libboac_checked.so): the shared-memory
// index of every bilinear gather and scatter, and every scatter-schedule
// entry, is checked before use; an index out of range is counted in this
// translation unit's fault counter and the access is skipped (never a trap
// or a fault), so a checked run reports the fault count instead of
// corrupting memory.  Normal builds compile the checks away.
#ifdef BOAC_CHECKED
static __device__ int g_bounds_faults;
__device__ __forceinline__ bool index_ok(long long i, long long n) {
    if (i >= 0 && i < n) return true;
    atomicAdd(&g_bounds_faults, 1);
    return false;
}
// Host side, one per translation unit: read (and optionally clear) the count.
#define BOAC_FAULT_READER(name)                                                              \
    int name(int reset) {                                                                    \
        int v = 0;                                                                           \
        if (cudaMemcpyFromSymbol(&v, g_bounds_faults, sizeof(int)) != cudaSuccess) return -1; \
        if (reset) {                                                                         \
            const int z = 0;                                                                 \
            if (cudaMemcpyToSymbol(g_bounds_faults, &z, sizeof(int)) != cudaSuccess) return -1; \
        }                                                                                    \
        return v;                                                                            \
    }
#else
__device__ __forceinline__ constexpr bool index_ok(long long, long long) { return true; }
#endif

// cos/sin of phi_v = 2 pi v / V (Sec. V: views uniformly spaced over the full
// angular range).  The quadrant is taken exactly, so views a quarter turn
// apart are exact rotations of each other; the in-quadrant angle is
// evaluated in float64 and rounded once to float32.
__device__ __forceinline__ void view_cos_sin(int v, int V, float* cs, float* sn) {
    long long four_v = 4LL * (long long)v;
    int quadrant = (int)((four_v / V) % 4);
    long long rem = four_v % V;
    double th = 1.5707963267948966192 * (double)rem / (double)V;
    double s, c;
    sincos(th, &s, &c);
    float fc = (float)c, fs = (float)s;
    switch (quadrant) {
        case 0: *cs = fc; *sn = fs; break;
        case 1: *cs = -fs; *sn = fc; break;
        case 2: *cs = -fc; *sn = -fs; break;
        default: *cs = fs; *sn = -fc; break;
    }
}

// Continuous (column u, row w) pixel index of ray sample k of bin b in the
// view with (cs, sn): p = s (cs, sn) + t (-sn, cs), s = (b - c) dx,
// t = (k - c) dx, c = (n - 1) / 2 (bins and samples share the pixel pitch).
// The bin term is innermost so that loops along a ray can hoist it.
__device__ __forceinline__ void sample_uw(int k, int b, float cs, float sn, float c,
                                          float* u, float* w) {
    float bc = (float)b - c;
    float kc = (float)k - c;
    *u = fmaf(-kc, sn, fmaf(bc, cs, c));
    *w = fmaf(kc, cs, fmaf(bc, sn, c));
}

__device__ __forceinline__ bool inside_open(float u, float w, int n) {
    return u > -1.0f && u < (float)n && w > -1.0f && w < (float)n;
}

// Bilinear sample of a zero-padded shared-memory image.  `img` points at
// padded element (0, 0) = pixel (-1, -1); rows are P floats apart; the pad
// ring (pixels -1 and n) holds zeros.  Samples outside (-1, n)^2 are 0.
__device__ __forceinline__ float bilerp_padded(const float* img, int P, int n, float u, float w) {
    if (!inside_open(u, w, n)) return 0.0f;
    float fj = floorf(u), fi = floorf(w);
    float au = u - fj, aw = w - fi;
    const int idx = ((int)fi + 1) * P + ((int)fj + 1);
    if (!index_ok(idx, (long long)P * (n + 1))) return 0.0f;  // idx + P + 1 < P (n + 2) + 1
    const float* p = img + idx;
    float v00 = p[0], v01 = p[1], v10 = p[P], v11 = p[P + 1];
    float top = fmaf(au, v01 - v00, v00);
    float bot = fmaf(au, v11 - v10, v10);
    return fmaf(aw, bot - top, top);
}

// Transpose of bilerp_padded: add g times each bilinear weight to the four
// neighbours (non-atomic read-modify-write; callers guarantee that no two
// threads touch the same pixel concurrently).
__device__ __forceinline__ void scatter_padded(float* img, int P, int n, float u, float w, float g) {
    if (!inside_open(u, w, n)) return;
    float fj = floorf(u), fi = floorf(w);
    float au = u - fj, aw = w - fi;
    const int idx = ((int)fi + 1) * P + ((int)fj + 1);
    if (!index_ok(idx, (long long)P * (n + 1))) return;
    float* p = img + idx;
    float g1 = g * aw, g0 = g - g1;          // row weights (1 - aw), aw
    float g01 = g0 * au, g00 = g0 - g01;     // (1-aw)(1-au), (1-aw) au
    float g11 = g1 * au, g10 = g1 - g11;     // aw (1-au), aw au
    p[0] += g00;
    p[1] += g01;
    p[P] += g10;
    p[P + 1] += g11;
}

// Bilinear sample of an unpadded global-memory image with per-neighbour
// bounds checks (plain kernels).
__device__ __forceinline__ float bilerp_global(const float* __restrict__ img, int n, float u, float w) {
    if (!inside_open(u, w, n)) return 0.0f;
    float fj = floorf(u), fi = floorf(w);
    float au = u - fj, aw = w - fi;
    int j0 = (int)fj, i0 = (int)fi;
    float v00 = 0.f, v01 = 0.f, v10 = 0.f, v11 = 0.f;
    bool jl = j0 >= 0, jh = j0 + 1 < n, il = i0 >= 0, ih = i0 + 1 < n;
    if (il && jl) v00 = __ldg(img + i0 * n + j0);
    if (il && jh) v01 = __ldg(img + i0 * n + j0 + 1);
    if (ih && jl) v10 = __ldg(img + (i0 + 1) * n + j0);
    if (ih && jh) v11 = __ldg(img + (i0 + 1) * n + j0 + 1);
    float top = fmaf(au, v01 - v00, v00);
    float bot = fmaf(au, v11 - v10, v10);
    return fmaf(aw, bot - top, top);
}

// Bilinear weight with which ray sample (u, w) reads pixel (i, j): the same
// products as scatter_padded (exact transpose of the forward weights).
__device__ __forceinline__ float pixel_weight(float u, float w, int i, int j, int n) {
    if (!inside_open(u, w, n)) return 0.0f;
    float fj = floorf(u), fi = floorf(w);
    int j0 = (int)fj, i0 = (int)fi;
    int dj = j - j0, di = i - i0;
    if ((unsigned)dj > 1u || (unsigned)di > 1u) return 0.0f;
    float au = u - fj, aw = w - fi;
    float r = di ? aw : 1.0f - aw;
    float cw = dj ? au : 1.0f - au;
    return r * cw;
}

// Transposed bilinear scatter of a whole sample grid, race-free without
// atomics: G (n x n samples, row pitch WP) is added into the padded
// accumulator img1 (row pitch P) with the weights of grid (cs, sn).  Samples
// are split into 9 classes by (k mod 3, b mod 3); two samples of one class
// are >= 3 lattice steps apart, i.e. more than 2 pixels apart along some
// image axis, so their 2x2 footprints are disjoint and a class is a plain
// read-modify-write pass.  Classes run in a fixed order (deterministic).
// Called by all NT threads of the CTA; ends with a barrier.
template <int N, int NT, int P, int WP>
__device__ __forceinline__ void scatter_classes(const float* __restrict__ W, float* img1, float cs,
                                                float sn, float c) {
#pragma unroll
    for (int cls = 0; cls < 9; ++cls) {
        const int pk = cls / 3, pb = cls % 3;
        const int nkc = (N - pk + 2) / 3, nbc = (N - pb + 2) / 3;
        for (int t = threadIdx.x; t < nkc * nbc; t += NT) {
            const int k = pk + 3 * (t / nbc), b = pb + 3 * (t % nbc);
            if (!index_ok(k * WP + b, (long long)N * WP)) continue;
            const float g = W[k * WP + b];
            float u, w;
            sample_uw(k, b, cs, sn, c, &u, &w);
            scatter_padded(img1, P, N, u, w, g);
        }
        __syncthreads();
    }
}

}  // namespace boac
