// boac_sysmat.cu -- the system matrix A^mu of Sec. III written out as a sparse
// matrix, and MLEM on it: the explicit-matrix counterpart of the matrix-free
// fused path.
//
// A row is one detector bin (v, b); its entries are the pixels read by the
// bilinear samples of that ray, A[(v,b)][p] = dx sum_k a_k w_k(p) (Eq. 1-2
// with the library's discretisation).  Which pixels a ray reads depends on
// the geometry only, so the sparsity pattern (CSR of A and of A^T) is built
// once per geometry and shared by every candidate; each candidate holds only
// its values, once in the order of A and once in the order of A^T, so that
// both products stream their values contiguously.  Every entry also records
// the run of samples k0 .. k0 + cnt - 1 that read its pixel (consecutive:
// the samples lie one pixel apart on a line and a pixel is read by the
// samples inside an open 2 x 2 square around it), which the value fill sums
// in a fixed order.
#include <cuda_runtime.h>
#include <limits.h>
#include <stdlib.h>

#include "boac_device.cuh"
#include "boac_internal.h"
#include "boac_plain_kernels.cuh"

struct boac_sysmat {
    boac_geom g;
    int R;             // rows: n_views * n_bins
    long long nnz;
    int* row_ptr;      // [R + 1]
    int* col;          // [nnz] pixel i * n + j, ascending within a row
    int* contrib;      // [nnz] k0 | cnt << 16
    int* colT_ptr;     // [n * n + 1]
    int* rowT;         // [nnz] row of each entry of A^T, ascending within a pixel
    int* posT;         // [nnz] position of entry e of A in the order of A^T
};

namespace boac {
namespace {

constexpr int kBuildThreads = 256;     // row and column build kernels
constexpr int kColSortCap = 4096;      // longest column segment the sort handles
constexpr int kWarpsPerBlock = 8;      // value fill and products: one warp per row / pixel
constexpr int kCandGroup = 8;          // candidates per warp in the products

// Flag bits of the build's consistency checks.
constexpr int kFlagRun = 1, kFlagCount = 2, kFlagColumn = 4;

__device__ __forceinline__ int next_pow2(int x) {
    int p = 1;
    while (p < x) p <<= 1;
    return p;
}

// Exclusive prefix sum over the block (blockDim.x a multiple of 32, <= 1024);
// returns the prefix of x and writes the block total to *total.
__device__ int block_exclusive_scan(int x, int* sh32, int* total) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    int incl = x;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, incl, off);
        if (lane >= off) incl += y;
    }
    if (lane == 31) sh32[warp] = incl;
    __syncthreads();
    if (warp == 0) {
        int s = lane < nw ? sh32[lane] : 0;
#pragma unroll
        for (int off = 1; off < 32; off <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, s, off);
            if (lane >= off) s += y;
        }
        sh32[lane] = s;  // inclusive scan of the warp totals
    }
    __syncthreads();
    const int before = warp > 0 ? sh32[warp - 1] : 0;
    *total = sh32[nw - 1];
    __syncthreads();
    return before + incl - x;
}

// Ascending bitonic sort of key[0..P) (P a power of two) carrying val along
// (val may be null).  Called by the whole block; ends with a barrier.
__device__ void block_sort(int* key, int* val, int P) {
    for (int k = 2; k <= P; k <<= 1)
        for (int j = k >> 1; j > 0; j >>= 1) {
            for (int i = threadIdx.x; i < P; i += blockDim.x) {
                const int l = i ^ j;
                if (l > i) {
                    const bool up = (i & k) == 0;
                    const int a = key[i], b = key[l];
                    if ((a > b) == up) {
                        key[i] = b;
                        key[l] = a;
                        if (val) {
                            const int t = val[i];
                            val[i] = val[l];
                            val[l] = t;
                        }
                    }
                }
            }
            __syncthreads();
        }
}

// The (pixel, sample) pairs of row (v, b), sorted: key = pixel * n + k for
// every in-grid bilinear neighbour of every sample inside (-1, n)^2, INT_MAX
// for the rest.  Returns the number of valid keys (they come first).
__device__ int row_pairs(int n, int V, int row, int* key, int P, int* sh32) {
    const int v = row / n, b = row % n;
    float cs, sn;
    view_cos_sin(v, V, &cs, &sn);
    const float c = 0.5f * (float)(n - 1);
    int valid = 0;
    for (int t = threadIdx.x; t < P; t += blockDim.x) {
        int kk = INT_MAX;
        if (t < 4 * n) {
            const int k = t >> 2, corner = t & 3;
            float u, w;
            sample_uw(k, b, cs, sn, c, &u, &w);
            if (inside_open(u, w, n)) {
                const int i = (int)floorf(w) + (corner >> 1), j = (int)floorf(u) + (corner & 1);
                if (i >= 0 && i < n && j >= 0 && j < n) kk = (i * n + j) * n + k;
            }
        }
        key[t] = kk;
        valid += kk != INT_MAX;
    }
    __syncthreads();
    block_sort(key, nullptr, P);
    int total;
    block_exclusive_scan(valid, sh32, &total);
    return total;
}

__global__ void __launch_bounds__(kBuildThreads)
row_count_kernel(int n, int V, int* __restrict__ rowcnt) {
    __shared__ int key[1024];
    __shared__ int sh32[32];
    const int row = blockIdx.x;
    const int P = next_pow2(4 * n);
    const int nvalid = row_pairs(n, V, row, key, P, sh32);
    int starts = 0;
    for (int t = threadIdx.x; t < nvalid; t += blockDim.x)
        starts += t == 0 || key[t] / n != key[t - 1] / n;
    int total;
    block_exclusive_scan(starts, sh32, &total);
    if (threadIdx.x == 0) rowcnt[row] = total;
}

__global__ void __launch_bounds__(kBuildThreads)
row_fill_kernel(int n, int V, const int* __restrict__ row_ptr, int* __restrict__ col,
                int* __restrict__ contrib, int* __restrict__ flag) {
    __shared__ int key[1024];
    __shared__ int start_pos[1024];
    __shared__ int sh32[32];
    const int row = blockIdx.x;
    const int P = next_pow2(4 * n);
    const int nvalid = row_pairs(n, V, row, key, P, sh32);
    // each thread owns a contiguous slice of the sorted keys
    const int per = (P + blockDim.x - 1) / blockDim.x;
    const int t0 = threadIdx.x * per;
    int starts = 0;
    for (int t = t0; t < t0 + per && t < nvalid; ++t) starts += t == 0 || key[t] / n != key[t - 1] / n;
    int nruns;
    int rank = block_exclusive_scan(starts, sh32, &nruns);
    for (int t = t0; t < t0 + per && t < nvalid; ++t)
        if (t == 0 || key[t] / n != key[t - 1] / n) start_pos[rank++] = t;
    __syncthreads();
    const int base = row_ptr[row];
    if (nruns != row_ptr[row + 1] - base) {
        if (threadIdx.x == 0) atomicOr(flag, kFlagCount);
        return;
    }
    for (int r = threadIdx.x; r < nruns; r += blockDim.x) {
        const int t = start_pos[r];
        const int end = r + 1 < nruns ? start_pos[r + 1] : nvalid;
        const int cnt = end - t;
        const int k0 = key[t] % n;
        if (key[end - 1] % n != k0 + cnt - 1) atomicOr(flag, kFlagRun);
        col[base + r] = key[t] / n;
        contrib[base + r] = k0 | (cnt << 16);
    }
}

// out[0..count] = exclusive prefix sums of in[0..count) (out[count] = total);
// one block of 1024 threads, each scanning a contiguous slice.
__global__ void __launch_bounds__(1024)
scan_kernel(const int* __restrict__ in, int count, int* __restrict__ out) {
    __shared__ int sh32[32];
    const int per = (count + blockDim.x - 1) / blockDim.x;
    const int t0 = threadIdx.x * per;
    int s = 0;
    for (int t = t0; t < t0 + per && t < count; ++t) s += in[t];
    int total;
    int run = block_exclusive_scan(s, sh32, &total);
    for (int t = t0; t < t0 + per && t < count; ++t) {
        out[t] = run;
        run += in[t];
    }
    if (threadIdx.x == 0) out[count] = total;
}

__global__ void col_count_kernel(long long nnz, int nn, const int* __restrict__ col,
                                 int* __restrict__ colcnt) {
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < nnz;
         e += (long long)gridDim.x * blockDim.x) {
        const int p = col[e];
        if ((unsigned)p < (unsigned)nn) atomicAdd(colcnt + p, 1);
    }
}

// Entries of A into their pixel's segment of A^T, in arrival order (sorted
// afterwards): one block per row.
__global__ void transpose_scatter_kernel(const int* __restrict__ row_ptr, const int* __restrict__ col,
                                         const int* __restrict__ colT_ptr, int* __restrict__ cursor,
                                         int* __restrict__ rowT, int* __restrict__ tmpE) {
    const int row = blockIdx.x;
    for (int e = row_ptr[row] + threadIdx.x; e < row_ptr[row + 1]; e += blockDim.x) {
        const int p = col[e];
        const int pos = colT_ptr[p] + atomicAdd(cursor + p, 1);
        rowT[pos] = row;
        tmpE[pos] = e;
    }
}

// Sort each pixel's segment of A^T by row (rows are distinct within a
// segment, so the result does not depend on the arrival order) and record
// where every entry of A went.
__global__ void __launch_bounds__(kBuildThreads)
col_sort_kernel(const int* __restrict__ colT_ptr, int* __restrict__ rowT, const int* __restrict__ tmpE,
                int* __restrict__ posT, int* __restrict__ flag) {
    __shared__ int key[kColSortCap];
    __shared__ int val[kColSortCap];
    const int p = blockIdx.x;
    const int s0 = colT_ptr[p], len = colT_ptr[p + 1] - s0;
    if (len > kColSortCap) {
        if (threadIdx.x == 0) atomicOr(flag, kFlagColumn);
        return;
    }
    const int P = next_pow2(len > 0 ? len : 1);
    for (int t = threadIdx.x; t < P; t += blockDim.x) {
        key[t] = t < len ? rowT[s0 + t] : INT_MAX;
        val[t] = t < len ? tmpE[s0 + t] : -1;
    }
    __syncthreads();
    block_sort(key, val, P);
    for (int t = threadIdx.x; t < len; t += blockDim.x) {
        rowT[s0 + t] = key[t];
        posT[val[t]] = s0 + t;
    }
}

// Per-candidate arrays are interleaved by groups of kCandGroup candidates:
// element x of candidate cand sits at [cand / kCandGroup][x][cand % kCandGroup],
// so one entry's values, or one pixel's (one bin's) operands, of a whole
// group fill one 32-byte sector and a warp's reads along a row are one
// contiguous stream.  vals: [groups][2][nnz][kCandGroup] (A's order, then
// A^T's); F, sens: [groups][n*n][kCandGroup]; r: [groups][R][kCandGroup].
struct alignas(32) Group8 {
    float4 lo, hi;
};
static_assert(kCandGroup == 8, "Group8 carries one group");

__device__ __forceinline__ Group8 load8(const float* p) {
    const float4* q = reinterpret_cast<const float4*>(p);
    return Group8{__ldg(q), __ldg(q + 1)};
}
__device__ __forceinline__ Group8 load8_stream(const float* p) {
    const float4* q = reinterpret_cast<const float4*>(p);
    return Group8{__ldcs(q), __ldcs(q + 1)};
}
__device__ __forceinline__ void fma8(float* acc, const Group8& a, const Group8& b) {
    acc[0] = fmaf(a.lo.x, b.lo.x, acc[0]);
    acc[1] = fmaf(a.lo.y, b.lo.y, acc[1]);
    acc[2] = fmaf(a.lo.z, b.lo.z, acc[2]);
    acc[3] = fmaf(a.lo.w, b.lo.w, acc[3]);
    acc[4] = fmaf(a.hi.x, b.hi.x, acc[4]);
    acc[5] = fmaf(a.hi.y, b.hi.y, acc[5]);
    acc[6] = fmaf(a.hi.z, b.hi.z, acc[6]);
    acc[7] = fmaf(a.hi.w, b.hi.w, acc[7]);
}

__device__ __forceinline__ float warp_sum(float x) {
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) x += __shfl_xor_sync(0xffffffffu, x, off);
    return x;
}

// The eight warp sums of acc[]; lane c (< 8) returns the sum of acc[c].
__device__ __forceinline__ float warp_sums8(const float* acc, int lane) {
    float mine = 0.0f;
#pragma unroll
    for (int cc = 0; cc < kCandGroup; ++cc) {
        const float s = warp_sum(acc[cc]);
        if (cc == lane) mine = s;
    }
    return mine;
}

constexpr int kFillWarps = 4;  // value fill: one warp per row, a group of candidates

// Values of the candidate group blockIdx.y: one warp per row.  For each
// candidate of the group the attenuation factors of the row's samples,
// a_k = exp(-dx (mu_k / 2 + sum_{k' > k} mu_k')) with mu_k the bilinear
// sample of mu, go to shared memory; each entry then sums dx a_k w_k(p) over
// its run of samples, for the eight candidates at once, and is written in
// A's order and, at posT[e], in A^T's.  Candidates >= B get zeros.
__global__ void __launch_bounds__(kFillWarps * 32)
values_kernel(int n, int V, float dx, int R, long long nnz, int B, const int* __restrict__ row_ptr,
              const int* __restrict__ col, const int* __restrict__ contrib, const int* __restrict__ posT,
              const float* __restrict__ mu, float* __restrict__ vals) {
    __shared__ float sh_a[kFillWarps][kCandGroup][kMaxN];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int row = blockIdx.x * kFillWarps + warp, grp = blockIdx.y;
    if (row >= R) return;  // whole warps leave; only warp-level synchronisation follows
    const int v = row / n, b = row % n;
    float cs, sn;
    view_cos_sin(v, V, &cs, &sn);
    const float c = 0.5f * (float)(n - 1);
    const int per = (n + 31) >> 5;  // <= 8 samples per lane
    const int k_lo = lane * per;
    for (int cc = 0; cc < kCandGroup; ++cc) {
        const int cand = grp * kCandGroup + cc;
        float* a = sh_a[warp][cc];
        if (cand >= B) {
            for (int k = lane; k < n; k += 32) a[k] = 0.0f;
            continue;
        }
        const float* m_img = mu + (size_t)cand * n * n;
        float m_loc[kMaxN / 32];
        float tot = 0.0f;
#pragma unroll
        for (int q = 0; q < kMaxN / 32; ++q) {
            const int k = k_lo + q;
            float m = 0.0f;
            if (q < per && k < n) {
                float u, w;
                sample_uw(k, b, cs, sn, c, &u, &w);
                m = bilerp_global(m_img, n, u, w);
            }
            m_loc[q] = m;
            tot += m;
        }
        float incl = tot;  // sum over lanes >= lane
#pragma unroll
        for (int off = 1; off < 32; off <<= 1) {
            const float o = __shfl_down_sync(0xffffffffu, incl, off);
            if (lane + off < 32) incl += o;
        }
        float suffix = incl - tot;
#pragma unroll
        for (int q = kMaxN / 32 - 1; q >= 0; --q) {
            const int k = k_lo + q;
            if (q < per && k < n) {
                a[k] = expf(-dx * (0.5f * m_loc[q] + suffix));
                suffix += m_loc[q];
            }
        }
    }
    __syncwarp();
    float* vA = vals + (size_t)grp * 2 * (size_t)nnz * kCandGroup;
    float* vT = vA + (size_t)nnz * kCandGroup;
    for (int e = row_ptr[row] + lane; e < row_ptr[row + 1]; e += 32) {
        const int p = col[e], cb = contrib[e];
        const int k0 = cb & 0xffff, k1 = min(n, k0 + (cb >> 16));
        const int i = p / n, j = p - i * n;
        float acc[kCandGroup];
#pragma unroll
        for (int cc = 0; cc < kCandGroup; ++cc) acc[cc] = 0.0f;
        for (int k = k0; k < k1; ++k) {
            float u, w;
            sample_uw(k, b, cs, sn, c, &u, &w);
            const float wt = pixel_weight(u, w, i, j, n);
#pragma unroll
            for (int cc = 0; cc < kCandGroup; ++cc) acc[cc] = fmaf(sh_a[warp][cc][k], wt, acc[cc]);
        }
        const float4 lo = make_float4(dx * acc[0], dx * acc[1], dx * acc[2], dx * acc[3]);
        const float4 hi = make_float4(dx * acc[4], dx * acc[5], dx * acc[6], dx * acc[7]);
        float4* dA = reinterpret_cast<float4*>(vA + (size_t)e * kCandGroup);
        float4* dT = reinterpret_cast<float4*>(vT + (size_t)posT[e] * kCandGroup);
        dA[0] = lo;
        dA[1] = hi;
        dT[0] = lo;
        dT[1] = hi;
    }
}

// sens = A^T 1 per candidate: one warp per pixel and group.
__global__ void __launch_bounds__(kWarpsPerBlock * 32)
sens_kernel(int nn, long long nnz, const int* __restrict__ colT_ptr, const float* __restrict__ vals,
            float* __restrict__ sens) {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int p = blockIdx.x * kWarpsPerBlock + warp, grp = blockIdx.y;
    if (p >= nn) return;
    const float* vT = vals + ((size_t)grp * 2 + 1) * (size_t)nnz * kCandGroup;
    float acc[kCandGroup];
#pragma unroll
    for (int cc = 0; cc < kCandGroup; ++cc) acc[cc] = 0.0f;
    const Group8 one{make_float4(1.f, 1.f, 1.f, 1.f), make_float4(1.f, 1.f, 1.f, 1.f)};
    for (int e = colT_ptr[p] + lane; e < colT_ptr[p + 1]; e += 32) fma8(acc, load8(vT + (size_t)e * kCandGroup), one);
    const float mine = warp_sums8(acc, lane);
    if (lane < kCandGroup) sens[((size_t)grp * nn + p) * kCandGroup + lane] = mine;
}

// F [B][n*n] <-> interleaved [groups][n*n][8] (zeros for candidates >= B).
__global__ void interleave_kernel(int nn, int B, const float* __restrict__ F, float* __restrict__ Fi) {
    const long long total = (long long)((B + kCandGroup - 1) / kCandGroup) * nn * kCandGroup;
    for (long long x = blockIdx.x * (long long)blockDim.x + threadIdx.x; x < total;
         x += (long long)gridDim.x * blockDim.x) {
        const int cc = (int)(x % kCandGroup);
        const long long gp = x / kCandGroup;
        const int p = (int)(gp % nn), grp = (int)(gp / nn);
        const int cand = grp * kCandGroup + cc;
        Fi[x] = cand < B ? F[(size_t)cand * nn + p] : 0.0f;
    }
}
__global__ void deinterleave_kernel(int nn, int B, const float* __restrict__ Fi, float* __restrict__ F) {
    const long long total = (long long)B * nn;
    for (long long x = blockIdx.x * (long long)blockDim.x + threadIdx.x; x < total;
         x += (long long)gridDim.x * blockDim.x) {
        const int cand = (int)(x / nn), p = (int)(x % nn);
        F[x] = Fi[((size_t)(cand / kCandGroup) * nn + p) * kCandGroup + cand % kCandGroup];
    }
}

// q = A F for the group blockIdx.y: one warp per row, each entry's column
// index and eight values loaded once.  FI: F is interleaved [groups][n*n][8]
// (else [B][n*n]).  RATIO: r = S / q (0 where q <= 0) goes to out
// [groups][R][8]; else q goes to out [B][R].
template <bool FI, bool RATIO>
__global__ void __launch_bounds__(kWarpsPerBlock * 32)
forward_kernel(int R, int nn, long long nnz, const int* __restrict__ row_ptr, const int* __restrict__ col,
               const float* __restrict__ vals, const float* __restrict__ F, int B, const float* __restrict__ S,
               long long s_stride, float* __restrict__ out) {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int row = blockIdx.x * kWarpsPerBlock + warp, grp = blockIdx.y;
    if (row >= R) return;
    const int c0 = grp * kCandGroup, nc = min(kCandGroup, B - c0);
    const float* vA = vals + (size_t)grp * 2 * (size_t)nnz * kCandGroup;
    float acc[kCandGroup];
#pragma unroll
    for (int cc = 0; cc < kCandGroup; ++cc) acc[cc] = 0.0f;
    const int e1 = row_ptr[row + 1];
    for (int e = row_ptr[row] + lane; e < e1; e += 32) {
        const int p = __ldg(col + e);
        const Group8 v = load8_stream(vA + (size_t)e * kCandGroup);
        if (FI) {
            fma8(acc, v, load8(F + ((size_t)grp * nn + p) * kCandGroup));
        } else {
            const float a[kCandGroup] = {v.lo.x, v.lo.y, v.lo.z, v.lo.w, v.hi.x, v.hi.y, v.hi.z, v.hi.w};
#pragma unroll
            for (int cc = 0; cc < kCandGroup; ++cc)
                if (cc < nc) acc[cc] = fmaf(a[cc], __ldg(F + (size_t)(c0 + cc) * nn + p), acc[cc]);
        }
    }
    const float q = warp_sums8(acc, lane);
    if (RATIO) {
        // the slots of candidates beyond B in the last group get 0
        if (lane < kCandGroup) {
            const float sv = lane < nc ? __ldg(S + (size_t)(c0 + lane) * s_stride + row) : 0.0f;
            out[((size_t)grp * R + row) * kCandGroup + lane] = q > 0.0f ? sv / q : 0.0f;
        }
    } else if (lane < nc) {
        out[(size_t)(c0 + lane) * R + row] = q;
    }
}

// z = A^T r, then F <- F z / sens (0 where sens = 0), for the group
// blockIdx.y: one warp per pixel; F, r and sens interleaved.
__global__ void __launch_bounds__(kWarpsPerBlock * 32)
backward_update_kernel(int nn, int R, long long nnz, const int* __restrict__ colT_ptr,
                       const int* __restrict__ rowT, const float* __restrict__ vals,
                       const float* __restrict__ r, const float* __restrict__ sens, float* __restrict__ F) {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int p = blockIdx.x * kWarpsPerBlock + warp, grp = blockIdx.y;
    if (p >= nn) return;
    const float* vT = vals + ((size_t)grp * 2 + 1) * (size_t)nnz * kCandGroup;
    const float* rg = r + (size_t)grp * R * kCandGroup;
    float acc[kCandGroup];
#pragma unroll
    for (int cc = 0; cc < kCandGroup; ++cc) acc[cc] = 0.0f;
    const int e1 = colT_ptr[p + 1];
    for (int e = colT_ptr[p] + lane; e < e1; e += 32) {
        const int row = __ldg(rowT + e);
        fma8(acc, load8_stream(vT + (size_t)e * kCandGroup), load8(rg + (size_t)row * kCandGroup));
    }
    const float z = warp_sums8(acc, lane);
    if (lane < kCandGroup) {
        const size_t i = ((size_t)grp * nn + p) * kCandGroup + lane;
        const float s = sens[i];
        F[i] = s > 0.0f ? F[i] * z / s : 0.0f;
    }
}

dim3 rows_grid(int count, int B) {
    return dim3((unsigned)((count + kWarpsPerBlock - 1) / kWarpsPerBlock),
                (unsigned)((B + kCandGroup - 1) / kCandGroup));
}

void free_sysmat(boac_sysmat* m) {
    if (!m) return;
    cudaFree(m->row_ptr);
    cudaFree(m->col);
    cudaFree(m->contrib);
    cudaFree(m->colT_ptr);
    cudaFree(m->rowT);
    cudaFree(m->posT);
    free(m);
}

}  // namespace
}  // namespace boac

using namespace boac;

extern "C" int boac_sysmat_create(const boac_geom* g, boac_sysmat** out, void* stream) {
    BOAC_RANGE("boac_sysmat_create");
    if (!out) return BOAC_EINVAL;
    *out = nullptr;
    if (!geom_ok(g)) return BOAC_EINVAL;
    cudaStream_t st = as_stream(stream);
    const int n = g->n, V = g->n_views, R = V * g->n_bins, nn = n * n;
    boac_sysmat* m = static_cast<boac_sysmat*>(calloc(1, sizeof(boac_sysmat)));
    if (!m) return BOAC_ECUDA;
    m->g = *g;
    m->R = R;
    int *rowcnt = nullptr, *colcnt = nullptr, *cursor = nullptr, *flag = nullptr, *tmpE = nullptr;
    int status = BOAC_ECUDA;
    int h_flag = 0, h_nnz = 0;
    auto fail = [&](int s) {
        cudaStreamSynchronize(st);
        cudaFree(rowcnt);
        cudaFree(colcnt);
        cudaFree(cursor);
        cudaFree(flag);
        cudaFree(tmpE);
        free_sysmat(m);
        cudaGetLastError();
        return s;
    };
    if (cudaMalloc(&rowcnt, sizeof(int) * R) != cudaSuccess ||
        cudaMalloc(&m->row_ptr, sizeof(int) * (R + 1)) != cudaSuccess ||
        cudaMalloc(&colcnt, sizeof(int) * nn) != cudaSuccess ||
        cudaMalloc(&cursor, sizeof(int) * nn) != cudaSuccess ||
        cudaMalloc(&m->colT_ptr, sizeof(int) * (nn + 1)) != cudaSuccess ||
        cudaMalloc(&flag, sizeof(int)) != cudaSuccess)
        return fail(BOAC_ECUDA);
    cudaMemsetAsync(flag, 0, sizeof(int), st);
    cudaMemsetAsync(colcnt, 0, sizeof(int) * nn, st);
    cudaMemsetAsync(cursor, 0, sizeof(int) * nn, st);
    // 1. entries per row, CSR row pointers, nnz
    row_count_kernel<<<R, kBuildThreads, 0, st>>>(n, V, rowcnt);
    scan_kernel<<<1, 1024, 0, st>>>(rowcnt, R, m->row_ptr);
    if (cudaMemcpyAsync(&h_nnz, m->row_ptr + R, sizeof(int), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
        return fail(BOAC_ECUDA);
    m->nnz = h_nnz;
    const size_t ne = (size_t)(h_nnz > 0 ? h_nnz : 1);
    if (cudaMalloc(&m->col, sizeof(int) * ne) != cudaSuccess ||
        cudaMalloc(&m->contrib, sizeof(int) * ne) != cudaSuccess ||
        cudaMalloc(&m->rowT, sizeof(int) * ne) != cudaSuccess ||
        cudaMalloc(&m->posT, sizeof(int) * ne) != cudaSuccess ||
        cudaMalloc(&tmpE, sizeof(int) * ne) != cudaSuccess)
        return fail(BOAC_ECUDA);
    // 2. column indices and sample runs; checked before anything indexes by them
    row_fill_kernel<<<R, kBuildThreads, 0, st>>>(n, V, m->row_ptr, m->col, m->contrib, flag);
    if (cudaMemcpyAsync(&h_flag, flag, sizeof(int), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
        return fail(BOAC_ECUDA);
    if (h_flag) return fail(BOAC_EUNSUPPORTED);
    // 3. the transposed pattern
    col_count_kernel<<<grid_1d(h_nnz, 256), 256, 0, st>>>(h_nnz, nn, m->col, colcnt);
    scan_kernel<<<1, 1024, 0, st>>>(colcnt, nn, m->colT_ptr);
    transpose_scatter_kernel<<<R, 128, 0, st>>>(m->row_ptr, m->col, m->colT_ptr, cursor, m->rowT, tmpE);
    col_sort_kernel<<<nn, kBuildThreads, 0, st>>>(m->colT_ptr, m->rowT, tmpE, m->posT, flag);
    if (cudaMemcpyAsync(&h_flag, flag, sizeof(int), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
        return fail(BOAC_ECUDA);
    if (h_flag) return fail(BOAC_EUNSUPPORTED);
    status = launch_status();
    if (status != BOAC_OK) return fail(status);
    cudaFree(rowcnt);
    cudaFree(colcnt);
    cudaFree(cursor);
    cudaFree(flag);
    cudaFree(tmpE);
    *out = m;
    return BOAC_OK;
}

extern "C" int boac_sysmat_destroy(boac_sysmat* m) {
    if (!m) return BOAC_EINVAL;
    free_sysmat(m);
    return BOAC_OK;
}

extern "C" long long boac_sysmat_nnz(const boac_sysmat* m) { return m ? m->nnz : -1; }

extern "C" int boac_sysmat_pattern(const boac_sysmat* m, int* row_ptr, int* col, int* colT_ptr, int* rowT,
                                   void* stream) {
    BOAC_RANGE("boac_sysmat_pattern");
    if (!m) return BOAC_EINVAL;
    cudaStream_t st = as_stream(stream);
    const size_t nn = (size_t)m->g.n * m->g.n, ne = (size_t)m->nnz;
    if (row_ptr) cudaMemcpyAsync(row_ptr, m->row_ptr, sizeof(int) * (m->R + 1), cudaMemcpyDeviceToDevice, st);
    if (col && ne) cudaMemcpyAsync(col, m->col, sizeof(int) * ne, cudaMemcpyDeviceToDevice, st);
    if (colT_ptr) cudaMemcpyAsync(colT_ptr, m->colT_ptr, sizeof(int) * (nn + 1), cudaMemcpyDeviceToDevice, st);
    if (rowT && ne) cudaMemcpyAsync(rowT, m->rowT, sizeof(int) * ne, cudaMemcpyDeviceToDevice, st);
    return launch_status();
}

static size_t groups_of(int B) { return (size_t)((B + kCandGroup - 1) / kCandGroup); }

extern "C" int boac_sysmat_values(const boac_sysmat* m, const float* mu, int B, float* vals, void* stream) {
    BOAC_RANGE("boac_sysmat_values");
    if (!m || !mu || !vals || B < 1 || B > 65535) return BOAC_EINVAL;
    if (m->nnz == 0) return BOAC_OK;
    const dim3 grid((unsigned)((m->R + kFillWarps - 1) / kFillWarps), (unsigned)groups_of(B));
    values_kernel<<<grid, kFillWarps * 32, 0, as_stream(stream)>>>(
        m->g.n, m->g.n_views, m->g.pixel_cm, m->R, m->nnz, B, m->row_ptr, m->col, m->contrib, m->posT, mu, vals);
    return launch_status();
}

extern "C" int boac_sysmat_project(const boac_sysmat* m, const float* vals, const float* F, int B, float* q,
                                   void* stream) {
    BOAC_RANGE("boac_sysmat_project");
    if (!m || !vals || !F || !q || B < 1 || B > 65535) return BOAC_EINVAL;
    const int nn = m->g.n * m->g.n;
    forward_kernel<false, false><<<rows_grid(m->R, B), kWarpsPerBlock * 32, 0, as_stream(stream)>>>(
        m->R, nn, m->nnz, m->row_ptr, m->col, vals, F, B, nullptr, 0, q);
    return launch_status();
}

// Workspace: F and sens interleaved [groups][n*n][8] each, r [groups][R][8]
// (the final q [B][R] reuses it), then the ln S! sum of a shared sinogram.
extern "C" size_t boac_sysmat_mlem_workspace_bytes(const boac_sysmat* m, int B) {
    if (!m || B < 1) return 0;
    return sizeof(float) * groups_of(B) * kCandGroup * (2 * (size_t)m->g.n * m->g.n + (size_t)m->R) +
           sizeof(double) * kLgammaScratchDoubles;
}

extern "C" int boac_sysmat_mlem(const boac_sysmat* m, const float* vals, const float* S, long long s_stride,
                                float* F, int K, int B, double* L, int include_lgamma, void* ws,
                                size_t ws_bytes, void* stream) {
    BOAC_RANGE("boac_sysmat_mlem");
    if (!m || !vals || !S || !F || K < 0 || B < 1 || B > 65535 || s_stride < 0) return BOAC_EINVAL;
    if (!ws || ws_bytes < boac_sysmat_mlem_workspace_bytes(m, B)) return BOAC_EWORKSPACE;
    cudaStream_t st = as_stream(stream);
    const int nn = m->g.n * m->g.n, R = m->R;
    const size_t G = groups_of(B);
    float* Fi = static_cast<float*>(ws);
    float* sens = Fi + G * nn * kCandGroup;
    float* r = sens + G * nn * kCandGroup;
    const int threads = kWarpsPerBlock * 32;
    interleave_kernel<<<grid_1d((long long)G * nn * kCandGroup, 256), 256, 0, st>>>(nn, B, F, Fi);
    sens_kernel<<<rows_grid(nn, B), threads, 0, st>>>(nn, m->nnz, m->colT_ptr, vals, sens);
    for (int it = 0; it < K; ++it) {
        forward_kernel<true, true><<<rows_grid(R, B), threads, 0, st>>>(R, nn, m->nnz, m->row_ptr, m->col, vals,
                                                                       Fi, B, S, s_stride, r);
        backward_update_kernel<<<rows_grid(nn, B), threads, 0, st>>>(nn, R, m->nnz, m->colT_ptr, m->rowT, vals,
                                                                      r, sens, Fi);
    }
    deinterleave_kernel<<<grid_1d((long long)B * nn, 256), 256, 0, st>>>(nn, B, Fi, F);
    if (L) {
        forward_kernel<true, false><<<rows_grid(R, B), threads, 0, st>>>(R, nn, m->nnz, m->row_ptr, m->col, vals,
                                                                        Fi, B, S, s_stride, r);
        double* scratch = reinterpret_cast<double*>(r + G * (size_t)R * kCandGroup);
        const double* lgS = include_lgamma && s_stride == 0 ? lgamma_sum(R, S, scratch, st) : nullptr;
        loglik_kernel<<<B, 256, 0, st>>>(R, r, S, s_stride, include_lgamma, L, lgS);
    }
    return launch_status();
}

#ifdef BOAC_CHECKED
namespace boac {
BOAC_FAULT_READER(bounds_faults_sysmat)
}  // namespace boac
#endif
