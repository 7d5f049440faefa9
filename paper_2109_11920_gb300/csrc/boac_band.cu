// boac_band.cu -- the fused batched MLEM of Sec. III (step 3, with the
// forward- and back-projection of Eq. 2 on the GPU) for 256 x 256 images,
// whose F, accumulator and sample buffer do not fit one SM's shared memory.
//
// A thread-block cluster of NB CTAs owns one candidate.  CTA r of the
// cluster holds band r of the image -- rows [r H, r H + H), H = ceil(n / NB)
// -- of F and of the back-projection accumulator in its shared memory, plus
// one row above and one below (the row below is the next band's first row:
// a copy of it in F, contributions to it in the accumulator).
//
// The sample grids are those of the one-CTA kernel (boac_fused.cu): four
// views phi + j pi/2 share one grid, with ray samples and bins on the pixel
// pitch.  Each grid is described with a base view whose angle lies in
// (-45, 45] degrees, so that its rays (the grid's columns, along k) run
// within 45 degrees of the image's row axis and cross every band in a short
// run.  A ray sample belongs to the band that holds the top row of its
// bilinear footprint, so every CTA gathers and scatters only in its own
// shared memory.  Within a band, the samples of a column form one run of
// consecutive k and those of a row (along b) one run of consecutive b; a
// small kernel records these runs for every (band, grid) before the main
// kernel starts (the same float arithmetic as the main kernel, so the
// records hold exactly the samples the main kernel would find).
//
// Per grid a CTA
//   1. gathers F at its samples (column runs), forms the column sums of the
//      two column views, and the row sums of the two row views from the
//      sample buffer (row runs);
//   2. publishes its partial sums; after a cluster barrier every CTA adds
//      the NB partials in rank order (distributed shared memory reads), so
//      all CTAs hold the same q and r = S / q;
//   3. forms the back-projection weights of the grid's four views on its
//      samples and scatters them into its accumulator band with the 9-class
//      race-free scatter.
// After the last grid, every CTA adds the contributions its upper neighbour
// made to its first row, applies the multiplicative update to its rows, and
// copies its lower neighbour's new first row.  The attenuation exponents are
// built once per candidate (suffix and prefix sums of the mu samples along
// each ray, across bands through the same published partial sums) and read
// back in the order the CTA's threads walk their runs.
#include <cooperative_groups.h>
#include <cuda_runtime.h>
#include <math.h>

#include "boac_device.cuh"
#include "boac_fused.h"
#include "boac_internal.h"

namespace cg = cooperative_groups;

namespace boac {

// First image row of band r (r = NB: n).  Equal bands leave the CTAs of the
// middle bands waiting less than the outer ones: near 45 degrees the
// rotated sample grid misses the image's corners, so the outer bands hold
// fewer samples.  For 5 bands the heights 52, 51, 49, 51, 53 lower the sum
// over the 180-view grids of the busiest band's samples by 5 % (sizes found
// by a local search of that sum); the other cluster sizes gain nothing
// within their shared-memory room and use equal heights.
template <int N, int NB>
__host__ __device__ constexpr int band_start(int r) {
    if (N == 256 && NB == 5)
        return r <= 0 ? 0 : r == 1 ? 52 : r == 2 ? 103 : r == 3 ? 152 : r == 4 ? 203 : 256;
    return r * ((N + NB - 1) / NB) < N ? r * ((N + NB - 1) / NB) : N;
}

template <int N, int NB>
__host__ __device__ constexpr int band_max_rows() {
    int h = 0;
    for (int r = 0; r < NB; ++r)
        h = band_start<N, NB>(r + 1) - band_start<N, NB>(r) > h ? band_start<N, NB>(r + 1) - band_start<N, NB>(r) : h;
    return h;
}

template <int N_, int NB>
struct BandShape {
    static constexpr int N = N_;
    static constexpr int NT = 4 * N_;
    static constexpr int H = band_max_rows<N_, NB>();  // rows of the tallest band
    // Padded band image: pixel (i, j), j in [-1, n], at local row i - R0 + 1,
    // column j + 1; the right padding column of a row and the left padding
    // column of the next are the same zero cell.
    static constexpr int P = N + 1;
    static constexpr int BIMG = (H + 2) * P + 1;  // band + the rows above and below
    static constexpr int WP = N + 1;              // sample-buffer pitch
    // Longest in-band run of a column: the band's H (+1 for the row above
    // band 0) rows crossed at up to 45 degrees, plus rounding slack.
    static constexpr int LC = ((H + 1) * 141422 + 99999) / 100000 + 2;
    static constexpr int TC = NT / N;             // threads per column
    static constexpr int SC = (LC + TC - 1) / TC; // column-run steps per thread
    static constexpr int SR = (LC + 1) / 2;       // row-run steps per thread (bound)
    static constexpr int REC = 8 + 4 * N;         // ints per (band, grid) record
    // table floats per grid: Xc and XrC (column-run order), XrT (row-run
    // order), Uc, Ur
    static constexpr size_t GSTRIDE = (size_t)(2 * SC + SR) * NT + 2 * N;
    static_assert(band_start<N_, NB>(NB - 1) < N && band_start<N_, NB>(NB) == N, "every band owns a row");
    static_assert(TC * N == NT && 4 * N == NT, "thread mapping");
};

// Record layout per (band, grid): [0] first active row kmin, [1] active rows
// R, [2] threads per row T, [3] column steps, [4] row steps, [5], [6] the
// base view's cos and sin (float bits), [7] the 5-class scatter lattice
// (beta, 0: none, see band_scatter5),
// then col_lo[n], col_len[n] (the run of column b: k in [lo, lo + len)),
// row_lo[n], row_len[n] (the run of row k: b in [lo, lo + len)).
enum { kRecKmin = 0, kRecRows = 1, kRecT = 2, kRecSc = 3, kRecSr = 4, kRecCos = 5, kRecSin = 6, kRecLat = 7,
       kRecHdr = 8 };

// Five-class alternative to the 9-class scatter: class cls holds the
// samples with k + beta b = cls (mod 5), beta in {2, 3}.  Two samples of one
// class differ by a lattice vector (m, n) with m + beta n = 0 (mod 5); their
// footprints are disjoint if the rotated vector (n cs - m sn, n sn + m cs) is
// at least 2 pixels long along an image axis.  Vectors with |m| or |n| > 2
// are at least 3 long (so more than 2 along some axis); those inside the box
// |m|, |n| <= 2 are tested, with a margin for the rounding of the sample
// coordinates.  Returns beta, or 0 where neither lattice qualifies (within
// about 0.05 degrees of the axes).
__host__ __device__ inline int scatter5_beta(float cs, float sn) {
    for (int beta = 3; beta >= 2; --beta) {
        bool good = true;
        for (int m = -2; m <= 2; ++m)
            for (int n = -2; n <= 2; ++n) {
                if ((m == 0 && n == 0) || (m + beta * n + 25) % 5 != 0) continue;
                const float du = fabsf((float)n * cs - (float)m * sn);
                const float dw = fabsf((float)n * sn + (float)m * cs);
                if (fmaxf(du, dw) < 2.001f) good = false;
            }
        if (good) return beta;
    }
    return 0;
}

// Base view of grid gi (views gi + j V/4): gi itself when its angle is at
// most 45 degrees, else gi - V/4 (= gi + 3V/4), whose angle is in (-45, 0).
__host__ __device__ __forceinline__ int band_base_view(int gi, int V) {
    return 8 * gi <= V ? gi : gi + 3 * V / 4;
}

// Band of a sample whose footprint's top row is fi (fi = -1: band 0).
template <int N, int NB>
__device__ __forceinline__ int band_of_row(int fi) {
    int r = 0;
#pragma unroll
    for (int q = 1; q < NB; ++q) r += fi >= band_start<N, NB>(q);
    return r;
}

// Bilinear sample / transposed scatter in a padded band image of BIMG
// floats whose local row 0 is image row R0 - 1; the sample is known to lie
// in the band (checked builds verify that the 2 x 2 footprint does).
template <int P, int BIMG>
__device__ __forceinline__ float bilerp_band(const float* img, int R0, float u, float w) {
    const float fj = floorf(u), fi = floorf(w);
    const float au = u - fj, aw = w - fi;
    const int idx = ((int)fi - R0 + 1) * P + ((int)fj + 1);
    if (!index_ok(idx, (long long)BIMG - P - 1)) return 0.0f;
    const float* p = img + idx;
    const float v00 = p[0], v01 = p[1], v10 = p[P], v11 = p[P + 1];
    const float top = fmaf(au, v01 - v00, v00);
    const float bot = fmaf(au, v11 - v10, v10);
    return fmaf(aw, bot - top, top);
}

template <int P, int BIMG>
__device__ __forceinline__ void scatter_band(float* img, int R0, float u, float w, float g) {
    const float fj = floorf(u), fi = floorf(w);
    const float au = u - fj, aw = w - fi;
    const int idx = ((int)fi - R0 + 1) * P + ((int)fj + 1);
    if (!index_ok(idx, (long long)BIMG - P - 1)) return;
    float* p = img + idx;
    const float g1 = g * aw, g0 = g - g1;
    const float g01 = g0 * au, g00 = g0 - g01;
    const float g11 = g1 * au, g10 = g1 - g11;
    p[0] += g00;
    p[1] += g01;
    p[P] += g10;
    p[P + 1] += g11;
}

// ---------------------------------------------------------------- records
// One CTA of n threads per (grid, band): thread b finds the run of column b
// by testing every k; thread k then finds the run of row k from the column
// runs.  A run that is not contiguous or exceeds the main kernel's buffers
// sets *bad (the main kernel then does nothing).
template <int N, int NB>
__global__ void __launch_bounds__(N) band_records_kernel(int V, int* geo, int* bad) {
    using S = BandShape<N, NB>;
    const int gi = blockIdx.x, r = blockIdx.y, ngrid = V / 4, t = threadIdx.x;
    int* rec = geo + ((size_t)r * ngrid + gi) * S::REC;
    __shared__ int s_lo[N], s_len[N];
    __shared__ int s_kmin, s_kmax, s_sc, s_sr, s_bad;
    if (t == 0) {
        s_kmin = N;
        s_kmax = -1;
        s_sc = 0;
        s_sr = 0;
        s_bad = 0;
    }
    float cs, sn;
    view_cos_sin(band_base_view(gi, V), V, &cs, &sn);
    const float c = 0.5f * (float)(N - 1);
    int lo = -1, hi = -1, cnt = 0;
    for (int k = 0; k < N; ++k) {
        float u, w;
        sample_uw(k, t, cs, sn, c, &u, &w);
        if (inside_open(u, w, N) && band_of_row<N, NB>((int)floorf(w)) == r) {
            if (lo < 0) lo = k;
            hi = k;
            ++cnt;
        }
    }
    bool ok = (cnt == 0 || hi - lo + 1 == cnt) && cnt <= S::LC && cs > 0.0f;
    if (cnt == 0) lo = 0;
    s_lo[t] = lo;
    s_len[t] = cnt;
    rec[kRecHdr + t] = lo;
    rec[kRecHdr + N + t] = cnt;
    __syncthreads();
    int blo = -1, bhi = -1, bcnt = 0;
    for (int b = 0; b < N; ++b) {
        if (t >= s_lo[b] && t < s_lo[b] + s_len[b]) {
            if (blo < 0) blo = b;
            bhi = b;
            ++bcnt;
        }
    }
    ok = ok && (bcnt == 0 || bhi - blo + 1 == bcnt);
    if (bcnt == 0) blo = 0;
    rec[kRecHdr + 2 * N + t] = blo;
    rec[kRecHdr + 3 * N + t] = bcnt;
    __syncthreads();
    if (bcnt > 0) {
        atomicMin(&s_kmin, t);
        atomicMax(&s_kmax, t);
    }
    atomicMax(&s_sc, (cnt + S::TC - 1) / S::TC);
    __syncthreads();
    const int R = s_kmax >= s_kmin ? s_kmax - s_kmin + 1 : 0;
    const int T = R > 0 ? S::NT / R : S::NT;
    if (R > 0 && (t < s_kmin || t > s_kmax) && bcnt > 0) ok = false;
    atomicMax(&s_sr, (bcnt + T - 1) / T);
    if (!ok) atomicExch(&s_bad, 1);
    __syncthreads();
    if (t == 0) {
        rec[kRecKmin] = R > 0 ? s_kmin : 0;
        rec[kRecRows] = R;
        rec[kRecT] = T;
        rec[kRecSc] = s_sc;
        rec[kRecSr] = s_sr;
        rec[kRecCos] = __float_as_int(cs);
        rec[kRecSin] = __float_as_int(sn);
        rec[kRecLat] = scatter5_beta(cs, sn);
        if (s_bad || s_sc > S::SC || s_sr > S::SR) atomicExch(bad, 1);
    }
}

// ---------------------------------------------------------------- kernel
// Shared-memory layout (bytes): 32 doubles for the score reduction, 16 ints
// of flags, then floats, then two slots holding a grid's record (copied
// from global memory with cp.async).
template <int N, int NB>
struct BandSmem {
    using S = BandShape<N, NB>;
    static constexpr int F0 = 0;                        // F band (mu during set-up)
    static constexpr int A0 = F0 + S::BIMG;             // accumulator band
    static constexpr int W0 = A0 + S::BIMG;             // [LC][WP] sample buffer
    static constexpr int PUB0 = W0 + S::LC * S::WP;     // [2][4][n] published partial sums
    static constexpr int CP0 = PUB0 + 8 * S::N;         // [2][TC][n] column-run partials
    static constexpr int RP0 = CP0 + 2 * S::TC * S::N;  // [2][NT] row-run partials
    static constexpr int RR0 = RP0 + 2 * S::NT;         // [4][n] dx r per view
    static constexpr int FLOATS = RR0 + 4 * S::N;
    static constexpr size_t HEAD = 32 * sizeof(double) + 16 * sizeof(int);
    static constexpr size_t RECS = (HEAD + sizeof(float) * (size_t)FLOATS + 15) / 16 * 16;
    static constexpr size_t BYTES = RECS + 2 * sizeof(int) * (size_t)S::REC;
    static_assert(S::REC % 4 == 0, "records are copied in 16-byte pieces");
    static_assert(BYTES <= 227 * 1024, "shared memory of one CTA");
};

// The 5-class scatter (beta from the grid's record): 4 threads per column
// walk the column run's samples of each class.  Ends with a barrier.
template <int N, int NB>
__device__ __forceinline__ void band_scatter5(const float* W, float* Ab, const int* colLo, const int* colLen,
                                              int R0, float cs, float sn, float c, int beta) {
    using S = BandShape<N, NB>;
    constexpr int NT = S::NT, WP = S::WP, P = S::P, M = NT / N;
    const int tid = threadIdx.x, b = tid % N, mm = tid / N;
    const int lo = colLo[b], len = colLen[b];
#pragma unroll
    for (int cls = 0; cls < 5; ++cls) {
        const int r5 = (cls + (5 - beta) * b) % 5;  // the class's k (mod 5) in column b
        const int k1 = lo + (r5 - lo % 5 + 5) % 5;
        for (int k = k1 + 5 * mm; k < lo + len; k += 5 * M) {
            const float g = W[(k - lo) * WP + b];
            float u, w;
            sample_uw(k, b, cs, sn, c, &u, &w);
            scatter_band<P, S::BIMG>(Ab, R0, u, w, g);
        }
        __syncthreads();
    }
}

// The 9-class race-free scatter of the sample buffer into the accumulator
// band (two samples of one class are >= 3 lattice steps apart, so their 2x2
// footprints are disjoint); columns b = pb (mod 3) get NT / #columns threads
// each, which walk the run's samples k = pk (mod 3).  Ends with a barrier.
template <int N, int NB>
__device__ __forceinline__ void band_scatter(const float* W, float* Ab, const int* colLo, const int* colLen,
                                             int R0, float cs, float sn, float c) {
    using S = BandShape<N, NB>;
    constexpr int NT = S::NT, WP = S::WP, P = S::P;
    const int tid = threadIdx.x;
#pragma unroll  // constant class offsets and column counts: +16 % measured
    for (int cls = 0; cls < 9; ++cls) {
        const int pk = cls / 3, pb = cls % 3;
        const int nbc = (N - pb + 2) / 3;
        const int M = NT / nbc;
        if (tid < nbc * M) {
            const int b = pb + 3 * (tid % nbc), mm = tid / nbc;
            const int lo = colLo[b], len = colLen[b];
            const int k1 = lo + (pk - lo % 3 + 3) % 3;  // first k >= lo with k = pk (mod 3)
            for (int k = k1 + 3 * mm; k < lo + len; k += 3 * M) {
                const float g = W[(k - lo) * WP + b];
                float u, w;
                sample_uw(k, b, cs, sn, c, &u, &w);
                scatter_band<P, S::BIMG>(Ab, R0, u, w, g);
            }
        }
        __syncthreads();
    }
}

template <int N, int NB>
__global__ void __launch_bounds__(4 * N, N == 64 ? 4 : (N == 128 && NB > 2) ? 2 : 1) mlem_band_kernel(FusedArgs a) {
    using S = BandShape<N, NB>;
    using L = BandSmem<N, NB>;
    constexpr int NT = S::NT, H = S::H, P = S::P, BIMG = S::BIMG, WP = S::WP, TC = S::TC;
    constexpr float kLog2e = 1.44269504088896340736f;
    if (*a.geo_bad) return;  // set before this launch: uniform over all CTAs

    cg::cluster_group cl = cg::this_cluster();
    const int r = (int)cl.block_rank();
    const int hold = blockIdx.x / NB;
    const int R0 = band_start<N, NB>(r);
    const int rows = band_start<N, NB>(r + 1) - R0;

    extern __shared__ __align__(16) unsigned char smem_raw[];
    double* dred = reinterpret_cast<double*>(smem_raw);
    int* flag = reinterpret_cast<int*>(smem_raw + 32 * sizeof(double));  // [0]: hand-over
    float* sm = reinterpret_cast<float*>(smem_raw + L::HEAD);
    int* recs = reinterpret_cast<int*>(smem_raw + L::RECS);  // [2][REC]
    float* Fb = sm + L::F0;
    float* Ab = sm + L::A0;
    float* W = sm + L::W0;
    float* pub = sm + L::PUB0;
    float* cpart = sm + L::CP0;
    float* rpart = sm + L::RP0;
    float* rr = sm + L::RR0;

    const int tid = threadIdx.x;
    const int V = a.V, ngrid = V / 4;
    const float c = 0.5f * (float)(N - 1);
    const float dx = a.dx;
    const float ndl = -dx * kLog2e;
    // column mapping: column cb, quarter cq of its run; row mapping per grid
    const int cb = tid % N, cq = tid / N;


    float* tab = a.tab + (size_t)blockIdx.x * ngrid * S::GSTRIDE;
    float* sens = a.sens + (size_t)blockIdx.x * H * N;
    const int* geo = a.geo + (size_t)r * ngrid * S::REC;

    const long long units = a.job_start ? a.job_start[a.B] : (long long)a.B * (a.K > 0 ? a.K : 1);
    const long long m0 = (long long)hold * a.cap;
    const long long m1 = m0 + a.cap < units ? m0 + a.cap : units;
    auto job_of = [&](long long x) -> int {
        if (!a.job_start) return (int)(x / (a.K > 0 ? a.K : 1));
        int lo = 0, hi = a.B - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (a.job_start[mid] <= x) lo = mid;
            else hi = mid - 1;
        }
        return lo;
    };
    const int j_first = m0 < m1 ? job_of(m0) : 0;
    const int j_last = m0 < m1 ? job_of(m1 - 1) : -1;

    // per-grid run bookkeeping of this thread (row runs: rcnt = 0 if none)
    struct Runs {
        int clo, ck0, ccnt;      // column run: k = clo + ck0 + s, s < ccnt
        int rk, rlo, rb0, rcnt;  // row run: row rk, b = rlo + rb0 + s, s < rcnt
    };
    // The runs of grid g are staged in shared-memory slot (step parity): the
    // next grid's record is loaded from global memory during a grid step and
    // stored into the other slot before that step's last barriers.
    int rb = 0;  // slot of the current grid step
    // Start copying grid g's record into slot `slot` (16 bytes per thread,
    // no registers held); complete with rec_wait() before a barrier.
    auto rec_copy = [&](int g, int slot) {
        if (tid < S::REC / 4) {
            const int* src = geo + (size_t)g * S::REC + 4 * tid;
            const unsigned dst = (unsigned)__cvta_generic_to_shared(recs + slot * S::REC + 4 * tid);
            asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(dst), "l"(src) : "memory");
        }
        asm volatile("cp.async.commit_group;" ::: "memory");
    };
    auto rec_wait = [&]() { asm volatile("cp.async.wait_all;" ::: "memory"); };
    // row mapping: thread tid < R T takes row kmin + tid / T, part tid % T
    auto runs_of = [&](int slot) -> Runs {
        Runs x;
        const int* h = recs + slot * S::REC;
        const int* rs = h + kRecHdr;
        const int lo = rs[cb], len = rs[N + cb];
        const int cS = (len + TC - 1) / TC;
        x.clo = lo;
        x.ck0 = cq * cS;
        x.ccnt = len - x.ck0 < cS ? len - x.ck0 : cS;
        if (x.ccnt < 0) x.ccnt = 0;
        const int kmin = h[kRecKmin], R = h[kRecRows], T = h[kRecT];
        const bool ract = R > 0 && tid < R * T;
        const int rq = ract ? tid % T : 0;
        x.rk = ract ? kmin + tid / T : 0;
        const int rl = ract ? rs[2 * N + x.rk] : 0;
        const int rn = ract ? rs[3 * N + x.rk] : 0;
        const int rS = ract ? (rn + T - 1) / T : 0;
        x.rlo = rl;
        x.rb0 = rq * rS;
        x.rcnt = rn - x.rb0 < rS ? rn - x.rb0 : rS;
        if (x.rcnt < 0) x.rcnt = 0;
        return x;
    };
    rec_copy(0, 0);
    rec_wait();  // read after the set-up's first barrier
    auto remote = [&](float* p, int rank) -> const float* { return cl.map_shared_rank(p, rank); };

    for (int cand = j_last; cand >= j_first; --cand) {
        const RaggedDesc* d = a.desc ? a.desc + cand : nullptr;
        const float* __restrict__ Sg = a.S + (d ? d->S_off : (long long)cand * a.s_stride);
        const float* __restrict__ mu = a.mu + (d ? d->mu_off : (long long)cand * N * N);
        float* Fc = a.F + (d ? d->F_off : (long long)cand * N * N);
        const int Kc = d ? d->K : a.K;
        const int lidx = d ? d->out : cand;
        const long long js = a.job_start ? a.job_start[cand] : (long long)cand * (a.K > 0 ? a.K : 1);
        const long long jl = Kc > 0 ? Kc : 1;
        const long long u0 = m0 - js > 0 ? m0 - js : 0, u1 = m1 - js < jl ? m1 - js : jl;
        const bool first = (u0 == 0), last = (u1 == jl);
        const int it0 = (int)(u0 < Kc ? u0 : Kc), it1 = (int)(u1 < Kc ? u1 : Kc);

        // ---- set-up: mu band -> Fb, accumulator cleared
        for (int i = tid; i < BIMG; i += NT) {
            Fb[i] = 0.0f;
            Ab[i] = 0.0f;
        }
        __syncthreads();
        for (int i = tid; i < (rows + 2) * N; i += NT) {
            const int l = i / N, j = i % N, gr = R0 - 1 + l;
            if (gr >= 0 && gr < N) Fb[l * P + j + 1] = __ldg(mu + (size_t)gr * N + j);
        }
        __syncthreads();

        int buf = 0;
        // ---- attenuation exponents of every grid, sensitivity A^T 1
        for (int gi = 0; gi < ngrid; ++gi) {
            const float cs = __int_as_float(recs[rb * S::REC + kRecCos]);
            const float sn = __int_as_float(recs[rb * S::REC + kRecSin]);
            const Runs x = runs_of(rb);
            const int* colLo = recs + rb * S::REC + kRecHdr;
            const int* colLen = colLo + N;
            float* Xc = tab + gi * S::GSTRIDE;
            float* XrC = Xc + S::SC * NT;
            float* XrT = XrC + S::SC * NT;
            float* Uc = XrT + S::SR * NT;
            float* Ur = Uc + N;
            float* pb_ = pub + buf * 4 * N;
            {
                float ps = 0.0f;
                for (int s = 0; s < x.ccnt; ++s) {
                    float u, w;
                    sample_uw(x.clo + x.ck0 + s, cb, cs, sn, c, &u, &w);
                    const float m = bilerp_band<P, S::BIMG>(Fb, R0, u, w);
                    W[(x.ck0 + s) * WP + cb] = m;
                    ps += m;
                }
                cpart[cq * N + cb] = ps;
            }
            __syncthreads();
            {
                float pr = 0.0f;
                for (int s = 0; s < x.rcnt; ++s) {
                    const int b = x.rlo + x.rb0 + s;
                    pr += W[(x.rk - colLo[b]) * WP + b];
                }
                rpart[tid] = pr;
            }
            __syncthreads();
            if (tid < N) {
                float tcol = 0.0f;
#pragma unroll
                for (int q2 = 0; q2 < TC; ++q2) tcol += cpart[q2 * N + tid];
                pb_[tid] = tcol;
            } else if (tid < 2 * N) {
                const int* h = recs + rb * S::REC;
                const int k = tid - N, kmin = h[kRecKmin], T = h[kRecT];
                float trow = 0.0f;
                if (k >= kmin && k < kmin + h[kRecRows])
                    for (int q2 = 0; q2 < T; ++q2) trow += rpart[(k - kmin) * T + q2];
                pb_[N + k] = trow;
            }
            cl.sync();
            rec_copy(gi + 1 < ngrid ? gi + 1 : 0, rb ^ 1);
            {   // columns: suffix along k; bands r' > r lie further along the ray
                float after = 0.0f, total = 0.0f;
                for (int q2 = 0; q2 < NB; ++q2) {
                    const float v = remote(pb_, q2)[cb];
                    total += v;
                    if (q2 > r) after += v;
                }
                for (int q2 = cq + 1; q2 < TC; ++q2) after += cpart[q2 * N + cb];
                float suf = after;
                for (int s = x.ccnt - 1; s >= 0; --s) {
                    const float m = W[(x.ck0 + s) * WP + cb];
                    Xc[s * NT + tid] = ndl * (0.5f * m + suf);
                    suf += m;
                }
                if (cq == 0) Uc[cb] = ndl * total;
            }
            if (x.rcnt > 0) {  // rows: prefix along b; the bands before lie on the side sn points away from
                const int* h = recs + rb * S::REC;
                const int T = h[kRecT], rq = tid % T, rbase = (x.rk - h[kRecKmin]) * T;
                float before = 0.0f, total = 0.0f;
                for (int q2 = 0; q2 < NB; ++q2) {
                    const float v = remote(pb_, q2)[N + x.rk];
                    total += v;
                    if (sn > 0.0f ? q2 < r : q2 > r) before += v;
                }
                for (int q2 = 0; q2 < rq; ++q2) before += rpart[rbase + q2];
                float pre = before;
                for (int s = 0; s < x.rcnt; ++s) {
                    const int b = x.rlo + x.rb0 + s;
                    const int j = x.rk - colLo[b];
                    const float m = W[j * WP + b];
                    const float y = ndl * (0.5f * m + pre);
                    XrT[s * NT + tid] = y;
                    // the same exponent at the sample's place in the column runs
                    const int cS = (colLen[b] + TC - 1) / TC, q3 = j / cS;
                    XrC[(j - q3 * cS) * NT + q3 * N + b] = y;
                    pre += m;
                }
                if (rq == 0) Ur[x.rk] = ndl * total;
            }
            buf ^= 1;
            rec_wait();
            rb ^= 1;
            __syncthreads();
            {   // G = dx (sum of the grid's four attenuation factors)
                const float uc = Uc[cb];
                for (int s = 0; s < x.ccnt; ++s) {
                    const float y = Xc[s * NT + tid];
                    W[(x.ck0 + s) * WP + cb] = dx * (ex2(y) + ex2(uc - y));
                }
            }
            __syncthreads();
            if (x.rcnt > 0) {
                const float ur = Ur[x.rk];
                for (int s = 0; s < x.rcnt; ++s) {
                    const int b = x.rlo + x.rb0 + s;
                    const float y = XrT[s * NT + tid];
                    W[(x.rk - colLo[b]) * WP + b] += dx * (ex2(y) + ex2(ur - y));
                }
            }
            __syncthreads();
            if (const int beta = colLo[kRecLat - kRecHdr])  // this grid's record
                band_scatter5<N, NB>(W, Ab, colLo, colLen, R0, cs, sn, c, beta);
            else
                band_scatter<N, NB>(W, Ab, colLo, colLen, R0, cs, sn, c);
        }
        cl.sync();  // every band's accumulator complete
        for (int i = tid; i < rows * N; i += NT) {
            const int l = i / N + 1, j = i % N;
            float v = Ab[l * P + j + 1];
            if (l == 1 && r > 0) v += remote(Ab, r - 1)[(R0 - band_start<N, NB>(r - 1) + 1) * P + j + 1];
            sens[i] = v;
        }
        // second part of a cut candidate: rank 0 waits for the first part,
        // the cluster shares the outcome (every CTA then takes the same path)
        if (r == 0 && tid == 0) {
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
            flag[0] = ok;
        }
        cl.sync();  // halo rows read; rank 0's flag visible
        const int wait_ok = *cl.map_shared_rank(flag, 0);
        if (!wait_ok) {  // give up on this part: no F written, score NaN
            if (r == 0 && tid == 0 && last && a.L) a.L[lidx] = __longlong_as_double(0x7ff8000000000000LL);
            cl.sync();
            continue;
        }
        // F rows R0 - 1 .. R0 + H (own rows and both neighbours)
        for (int i = tid; i < BIMG; i += NT) {
            Fb[i] = 0.0f;
            Ab[i] = 0.0f;
        }
        __syncthreads();
        for (int i = tid; i < (rows + 2) * N; i += NT) {
            const int l = i / N, j = i % N, gr = R0 - 1 + l;
            if (gr >= 0 && gr < N) Fb[l * P + j + 1] = first ? Fc[(size_t)gr * N + j] : __ldcg(Fc + (size_t)gr * N + j);
        }
        __syncthreads();

        // ---- MLEM iterations, then one more forward pass for the score
        double lacc = 0.0;
        for (int it = it0; it <= it1; ++it) {
            const bool scoring = (it == Kc);
            if (it == it1 && !(last && a.L)) break;
            for (int gi = 0; gi < ngrid; ++gi) {
                const float cs = __int_as_float(recs[rb * S::REC + kRecCos]);
                const float sn = __int_as_float(recs[rb * S::REC + kRecSin]);
                const Runs x = runs_of(rb);
                const int* colLo = recs + rb * S::REC + kRecHdr;
                const int* colLen = colLo + N;
                const float* Xc = tab + gi * S::GSTRIDE;
                const float* XrC = Xc + S::SC * NT;
                const float* XrT = XrC + S::SC * NT;
                const float* Uc = XrT + S::SR * NT;
                const float* Ur = Uc + N;
                float* pb_ = pub + buf * 4 * N;
                {   // the next grid's exponents are read from DRAM once per
                    // iteration: start that read now
                    const int gn = gi + 1 < ngrid ? gi + 1 : 0;
                    const float* nxt = tab + gn * S::GSTRIDE;
                    const int* rn = geo + (size_t)gn * S::REC;
                    const int lc = (__ldg(rn + kRecSc) * NT) / 32, lr = (__ldg(rn + kRecSr) * NT) / 32;
                    for (int l = tid; l < lc; l += NT) {
                        prefetch_l2(nxt + 32 * l);
                        prefetch_l2(nxt + S::SC * NT + 32 * l);
                    }
                    for (int l = tid; l < lr; l += NT) prefetch_l2(nxt + 2 * S::SC * NT + 32 * l);
                }
                const int v1 = band_base_view(gi, V), v2 = (v1 + V / 2) % V;
                const int v3 = (v1 + V / 4) % V, v4 = (v1 + 3 * V / 4) % V;
                {   // forward, column views: sample F on the band's column runs
                    const float uc = Uc[cb];
                    float acc1 = 0.0f, acc2 = 0.0f;
                    for (int s = 0; s < x.ccnt; ++s) {
                        float u, w;
                        sample_uw(x.clo + x.ck0 + s, cb, cs, sn, c, &u, &w);
                        const float f = bilerp_band<P, S::BIMG>(Fb, R0, u, w);
                        W[(x.ck0 + s) * WP + cb] = f;
                        const float y = Xc[s * NT + tid];
                        acc1 = fmaf(ex2(y), f, acc1);
                        acc2 = fmaf(ex2(uc - y), f, acc2);
                    }
                    cpart[cq * N + cb] = acc1;
                    cpart[TC * N + cq * N + cb] = acc2;
                }
                __syncthreads();
                {   // forward, row views: the samples back from W
                    float acc3 = 0.0f, acc4 = 0.0f;
                    if (x.rcnt > 0) {
                        const float ur = Ur[x.rk];
                        for (int s = 0; s < x.rcnt; ++s) {
                            const int b = x.rlo + x.rb0 + s;
                            const float f = W[(x.rk - colLo[b]) * WP + b];
                            const float y = XrT[s * NT + tid];
                            acc3 = fmaf(ex2(y), f, acc3);
                            acc4 = fmaf(ex2(ur - y), f, acc4);
                        }
                    }
                    rpart[tid] = acc3;
                    rpart[NT + tid] = acc4;
                }
                __syncthreads();
                if (tid < N) {
                    float p1 = 0.0f, p2 = 0.0f;
#pragma unroll
                    for (int q2 = 0; q2 < TC; ++q2) {
                        p1 += cpart[q2 * N + tid];
                        p2 += cpart[TC * N + q2 * N + tid];
                    }
                    pb_[tid] = p1;
                    pb_[N + tid] = p2;
                } else if (tid < 2 * N) {
                    const int* h = recs + rb * S::REC;
                    const int k = tid - N, kmin = h[kRecKmin], T = h[kRecT];
                    float p3 = 0.0f, p4 = 0.0f;
                    if (k >= kmin && k < kmin + h[kRecRows]) {
                        for (int q2 = 0; q2 < T; ++q2) {
                            p3 += rpart[(k - kmin) * T + q2];
                            p4 += rpart[NT + (k - kmin) * T + q2];
                        }
                    }
                    pb_[2 * N + k] = p3;
                    pb_[3 * N + k] = p4;
                }
                cl.sync();
                rec_copy(gi + 1 < ngrid ? gi + 1 : 0, rb ^ 1);
                {   // q = dx * (sum of the bands' partials, rank order), then
                    // dx r = dx S / q, or the Eq. 5 terms (rank 0) when scoring
                    const int vs = tid / N, j = tid % N;
                    float q = 0.0f;
                    for (int q2 = 0; q2 < NB; ++q2) q += remote(pb_, q2)[tid];
                    q *= dx;
                    const int v = vs == 0 ? v1 : (vs == 1 ? v2 : (vs == 2 ? v3 : v4));
                    const int bin = (vs & 1) ? N - 1 - j : j;
                    const float Sv = __ldg(Sg + (size_t)v * N + bin);
                    if (scoring) {
                        if (r == 0) lacc += loglik_term(Sv, q, a.include_lgamma && !a.lgS);
                    } else {
                        rr[tid] = q > 0.0f ? dx * (Sv / q) : 0.0f;
                    }
                }
                buf ^= 1;
                rec_wait();
                rb ^= 1;
                __syncthreads();
                if (scoring) continue;
                {   // back-projection weights G = dx sum_v a_v r_v of the grid's
                    // four views in one pass over the column runs (the row
                    // views' exponents in column-run order: XrC)
                    const float uc = Uc[cb];
                    const float r1 = rr[cb], r2 = rr[N + cb];
                    for (int s = 0; s < x.ccnt; ++s) {
                        const int k = x.clo + x.ck0 + s;
                        const float y = Xc[s * NT + tid];
                        const float z = XrC[s * NT + tid];
                        const float gc = fmaf(ex2(y), r1, ex2(uc - y) * r2);
                        W[(x.ck0 + s) * WP + cb] = gc + fmaf(ex2(z), rr[2 * N + k], ex2(Ur[k] - z) * rr[3 * N + k]);
                    }
                }
                __syncthreads();
                if (const int beta = colLo[kRecLat - kRecHdr])  // this grid's record
                    band_scatter5<N, NB>(W, Ab, colLo, colLen, R0, cs, sn, c, beta);
                else
                    band_scatter<N, NB>(W, Ab, colLo, colLen, R0, cs, sn, c);
            }
            if (scoring) break;
            // multiplicative update of the band's rows; the first row also
            // takes what the band above scattered into it
            cl.sync();
            for (int i = tid; i < rows * N; i += NT) {
                const int l = i / N + 1, j = i % N, pi = l * P + j + 1;
                float acc = Ab[pi];
                if (l == 1 && r > 0) acc += remote(Ab, r - 1)[(R0 - band_start<N, NB>(r - 1) + 1) * P + j + 1];
                const float sv = sens[i];
                Fb[pi] = sv > 0.0f ? Fb[pi] * acc / sv : 0.0f;
            }
            cl.sync();
            if (r < NB - 1)
                for (int j = tid; j < N; j += NT) Fb[(rows + 1) * P + j + 1] = remote(Fb, r + 1)[P + j + 1];
            for (int i = tid; i < BIMG; i += NT) Ab[i] = 0.0f;
            __syncthreads();
        }

        // ---- Eq. 5: deterministic block reduction of rank 0's float64 terms
        if (last && a.L) {
            for (int off = 16; off > 0; off >>= 1) lacc += __shfl_down_sync(0xffffffffu, lacc, off);
            if ((tid & 31) == 0) dred[tid >> 5] = lacc;
            __syncthreads();
            if (r == 0 && tid == 0) {
                double t = 0.0;
                for (int wi = 0; wi < NT / 32; ++wi) t += dred[wi];
                a.L[lidx] = a.include_lgamma && a.lgS ? t - *a.lgS : t;
                if (t == -INFINITY) atomicCAS(a.status, BOAC_OK, BOAC_ENONFINITE);
            }
        }

        // ---- F out (own rows), then hand over to a second part if cut
        for (int i = tid; i < rows * N; i += NT) Fc[(size_t)R0 * N + i] = Fb[(i / N + 1) * P + (i % N) + 1];
        __threadfence();
        cl.sync();  // F written by every band; no CTA still reads another's shared memory
        if (!last && r == 0 && tid == 0 && cand != a.withhold)
            asm volatile("st.release.gpu.global.s32 [%0], %1;" ::"l"(a.ready + cand), "r"(1) : "memory");
    }
}

// ---------------------------------------------------------------- host side
// Instantiated (image side, cluster size) pairs.
#define BOAC_BAND_CASES(X) \
    X(256, 5) X(256, 6) X(256, 8) X(128, 2) X(128, 4) X(128, 8) X(64, 2) X(64, 4) X(64, 8)

bool band_supported(int n, int V, int nb) {
    if (V % 4 != 0 || V < 4 || V > kMaxViews) return false;
#define X(NV, BV) if (n == NV && nb == BV) return true;
    BOAC_BAND_CASES(X)
#undef X
    return false;
}

size_t band_smem_bytes(int n, int nb) {
#define X(NV, BV) if (n == NV && nb == BV) return BandSmem<NV, BV>::BYTES;
    BOAC_BAND_CASES(X)
#undef X
    return 0;
}

size_t band_tab_floats(int n, int nb, int V) {
#define X(NV, BV) if (n == NV && nb == BV) return (size_t)(V / 4) * BandShape<NV, BV>::GSTRIDE;
    BOAC_BAND_CASES(X)
#undef X
    return 0;
}

size_t band_sens_floats(int n, int nb) {
#define X(NV, BV) if (n == NV && nb == BV) return (size_t)BandShape<NV, BV>::H * NV;
    BOAC_BAND_CASES(X)
#undef X
    return 0;
}

size_t band_geo_bytes(int n, int nb, int V) {
    return sizeof(int) * (size_t)nb * (V / 4) * (8 + 4 * (size_t)n);
}

template <int N, int NB>
static int set_smem_attr() {
    constexpr int kDev = 64;
    static bool done[kDev];
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kDev) return launch_status();
    if (!done[dev]) {
        if (cudaFuncSetAttribute(mlem_band_kernel<N, NB>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)BandSmem<N, NB>::BYTES) != cudaSuccess)
            return launch_status();
        done[dev] = true;
    }
    return BOAC_OK;
}

template <int N, int NB>
static int max_clusters_t() {
    constexpr int kDev = 64;
    static int cached[kDev];
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kDev) {
        cudaGetLastError();
        return 0;
    }
    if (cached[dev]) return cached[dev];
    if (set_smem_attr<N, NB>() != BOAC_OK) return 0;
    cudaLaunchConfig_t cfg = {};
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = NB;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.gridDim = dim3(NB * 64, 1, 1);
    cfg.blockDim = dim3(BandShape<N, NB>::NT, 1, 1);
    cfg.dynamicSmemBytes = BandSmem<N, NB>::BYTES;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    int n = 0;
    if (cudaOccupancyMaxActiveClusters(&n, mlem_band_kernel<N, NB>, &cfg) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    cached[dev] = n;
    return n;
}

int band_max_clusters(int n, int nb) {
#define X(NV, BV) if (n == NV && nb == BV) return max_clusters_t<NV, BV>();
    BOAC_BAND_CASES(X)
#undef X
    return 0;
}

template <int N, int NB>
static int band_launch_t(const FusedArgs& a, int clusters, cudaStream_t st) {
    int s = set_smem_attr<N, NB>();
    if (s != BOAC_OK) return s;
    if (cudaMemsetAsync(a.geo_bad, 0, sizeof(int), st) != cudaSuccess) return launch_status();
    band_records_kernel<N, NB><<<dim3(a.V / 4, NB), N, 0, st>>>(a.V, const_cast<int*>(a.geo), a.geo_bad);
    s = launch_status();
    if (s != BOAC_OK) return s;
    cudaLaunchConfig_t cfg = {};
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = NB;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.gridDim = dim3((unsigned)(clusters * NB), 1, 1);
    cfg.blockDim = dim3(BandShape<N, NB>::NT, 1, 1);
    cfg.dynamicSmemBytes = BandSmem<N, NB>::BYTES;
    cfg.stream = st;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    if (cudaLaunchKernelEx(&cfg, mlem_band_kernel<N, NB>, a) != cudaSuccess) return launch_status();
    return launch_status();
}

int band_launch(int n, int nb, const FusedArgs& a, int clusters, cudaStream_t st) {
    if (clusters < 1) return BOAC_EINVAL;
#define X(NV, BV) if (n == NV && nb == BV) return band_launch_t<NV, BV>(a, clusters, st);
    BOAC_BAND_CASES(X)
#undef X
    return BOAC_EUNSUPPORTED;
}

#undef BOAC_BAND_CASES

}  // namespace boac

#ifdef BOAC_CHECKED
namespace boac {
BOAC_FAULT_READER(bounds_faults_band)
}  // namespace boac
#endif
