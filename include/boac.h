/*
 * boac.h -- C ABI of the BOAC hot path on GB300 (sm_103a).
 *
 * Method: Koutsantonis et al., "A Bayesian Optimization Approach for
 * Attenuation Correction in SPECT Brain Imaging" (arXiv 2109.11920).  For
 * every candidate head geometry c_0..c_5 proposed by the Bayesian optimiser
 * the library rasterises the attenuation map (Eq. 3-4), applies the
 * attenuated Radon transform S = A^mu F (Eq. 1-2) and its exact adjoint,
 * runs a fixed number of MLEM iterations (Sec. III, step 3) and scores the
 * candidate with the Poisson log-likelihood (Eq. 5).
 *
 * Discretisation (the paper gives none; both this library and its test
 * oracle use this one):
 *   - image: n x n pixels of pixel_cm; pixel (i, j) (row i, column j) has its
 *     centre at x = (j - c) pixel_cm, y = (i - c) pixel_cm, c = (n - 1) / 2;
 *   - views: phi_v = 2 pi v / n_views, v = 0 .. n_views - 1;
 *   - detector: n_bins = n bins of bin_cm = pixel_cm, bin b at s = (b - c) bin_cm;
 *   - ray: n samples one pixel apart, sample k at t = (k - c) pixel_cm along
 *     (-sin phi, cos phi); the detector lies at t -> +infinity;
 *   - F and mu are sampled bilinearly at the ray samples (0 outside the grid);
 *   - attenuation of sample k: a = exp(-pixel_cm (mu_k / 2 + sum_{k' > k} mu_k'));
 *   - q(v, b) = pixel_cm * sum_k a_k F_k.
 *
 * Conventions for every entry point:
 *   - All array arguments are DEVICE pointers to caller-owned, contiguous,
 *     row-major float32 (or float64 where stated) memory on the current CUDA
 *     device.  The library allocates no device memory: operations that need
 *     scratch take a caller-allocated workspace (see boac_workspace_bytes).
 *     It holds two arrays of static device memory on every GPU that loads
 *     it: the 64 MiB scratch of boac_mlem_noalloc and 32 MiB of scatter
 *     schedules kept across calls for up to 8 geometries (the fused kernels
 *     build a geometry's schedule once; later geometries build it in the
 *     workspace on every call).
 *   - Work is enqueued asynchronously on `stream` (a cudaStream_t; NULL =
 *     the legacy default stream).  Return values report argument and launch
 *     errors only; kernel faults surface at the next synchronisation.
 *   - Return BOAC_OK (0) on success or a negative BOAC_E* status.  Nothing is
 *     enqueued when an argument check fails.
 *   - Geometry restrictions: 8 <= n <= 256 with n_bins == n and
 *     bin_cm == pixel_cm; 2 <= n_views <= 720 and n_views even for the
 *     fused path (boac_mlem, boac_score_grad).
 */
#ifndef BOAC_H
#define BOAC_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ---------------------------------------------------- */
#define BOAC_OK 0
#define BOAC_EINVAL (-1)       /* bad shape, null pointer, stride or mode   */
#define BOAC_ECUDA (-2)        /* a CUDA call or launch failed              */
#define BOAC_EWORKSPACE (-3)   /* workspace missing or too small            */
#define BOAC_EUNSUPPORTED (-4) /* valid geometry the library has no kernel for */
#define BOAC_ETIMEOUT (-5)     /* a bounded wait on the device ran out (see
                                  boac_workspace_status)                   */
#define BOAC_ENONFINITE (-6)   /* not an error of the call: some candidate's
                                  Eq. 5 score is -inf because q = 0 on a bin
                                  with S > 0 (boac_workspace_status; the
                                  candidate is the one whose L is -inf)     */

/* ---- types ------------------------------------------------------------- */
/* Scanner geometry (see the discretisation above). */
typedef struct {
    int n;          /* image side in pixels (also the ray sample count)    */
    int n_bins;     /* detector bins per view; must equal n                */
    int n_views;    /* views uniformly spaced over 360 degrees             */
    float pixel_cm; /* pixel size in cm                                    */
    float bin_cm;   /* bin pitch in cm; must equal pixel_cm                */
} boac_geom;

/* Tissue values of the model attenuation map (Eq. 4): brain mu_b and
 * cranium mu_c in cm^-1, cranium thickness dR in cm.  Fixed, not optimised
 * (Sec. II). */
typedef struct {
    float mu_b, mu_c, dR;
} boac_tissue;

enum { BOAC_RASTER_CENTER = 0, BOAC_RASTER_AREA = 1 };

/* Workspace queries: which operation the size is for. */
enum {
    BOAC_OP_PROJECT = 0,
    BOAC_OP_BACKPROJECT = 1,
    BOAC_OP_MLEM = 2,
    BOAC_OP_MLEM_PLAIN = 3,
    BOAC_OP_SCORE = 4,
    BOAC_OP_SCORE_GRAD = 5,
    BOAC_OP_MLEM_UNFUSED = 6
};

/* Human-readable name of a status code (static string, never NULL). */
const char *boac_status_string(int status);

/* ABI version of this library (incremented on incompatible changes). */
int boac_abi_version(void);

/* Bounds faults counted by a checked build of this library
 * (libboac_checked.so, compiled with -DBOAC_CHECKED; the paper has no
 * counterpart).  There the shared-memory index of every bilinear gather and
 * scatter of the fused, cluster and grouped kernels, and every entry of the
 * scatter schedule, is checked before use; an index out of range is counted
 * and the access skipped -- never a trap or a memory fault -- so a checked
 * run reports *faults > 0 instead of corrupting memory.  Synchronous: reads
 * the counters after the device work queued before it; reset != 0 clears
 * them.  Normal builds return BOAC_EUNSUPPORTED. */
int boac_bounds_faults(int *faults, int reset);

/* Device status left in a boac_mlem / boac_mlem_ragged workspace by the last
 * call that used it: BOAC_OK; BOAC_ETIMEOUT if a kernel gave up one of its
 * bounded waits (the affected candidates' scores are NaN and their images
 * unspecified; this takes precedence); else BOAC_ENONFINITE if some
 * candidate's score is -inf (Eq. 5 with q_i = 0 < S_i: the image explains
 * none of a bin's counts -- a valid result, reported per candidate by its
 * -inf in L, not a failure).  boac_mlem_plain, boac_score and boac_loglik
 * keep no status word: there the -inf in L is the only report.  The fused kernel splits the batch's iterations evenly over
 * its CTAs, so a candidate may be continued by a second CTA, which waits for
 * a flag from the first; the schedule leaves that wait a whole candidate's
 * worth of slack, and it gives up after a limit set by boac_set_wait_cycles
 * (default about 2 s).  Synchronous: copies the
 * word to *status after the device work queued before it has finished. */
int boac_workspace_status(const void *ws, size_t ws_bytes, int *status);

/* Limit, in GPU clock cycles, of the bounded hand-over wait described above
 * (the second part of a cut candidate waiting for the first part's flag),
 * for every launch that follows, process-wide.  cycles <= 0 restores the
 * default, 2^32 (about 2 s at 2 GHz).  Returns the previous limit.  A
 * shorter limit gives up sooner on a GPU shared with other work, where a
 * CTA of the launch may wait for an SM; a longer one tolerates more such
 * delay.  The paper has no counterpart (its GPU code is not published). */
long long boac_set_wait_cycles(long long cycles);

/* ---- test hook of the bounded hand-over wait ----------------------------
 * The paper has no counterpart.  Runs the fused MLEM kernel of launch
 * configuration `config` (the ids of boac_mlem_ragged) on exactly `holders`
 * CTAs (or clusters), all resident at once (BOAC_EUNSUPPORTED otherwise),
 * for B candidates of K iterations sharing one sinogram S [n_views][n_bins],
 * and makes the first part of candidate `withhold` (-1: none) keep its
 * hand-over flag to itself, so that the CTA running that candidate's second
 * part waits in vain until the limit of boac_set_wait_cycles runs out.  That
 * CTA then records BOAC_ETIMEOUT in the workspace status word
 * (boac_workspace_status), sets the candidate's score to NaN and returns;
 * every other candidate is computed as by boac_mlem, without the ln S! term.
 * Pick B, K and holders so that the work split cuts `withhold` (with
 * cap = max(ceil(B K / holders), K), the candidates whose iterations
 * [j K, (j+1) K) straddle a multiple of cap).  Nothing faults or hangs: the
 * wait is bounded and the context stays usable.
 *   ws  boac_test_mlem_handover_bytes(g, B, K, config, holders) bytes.
 * Errors: BOAC_EINVAL for bad arguments or a configuration the geometry
 * does not support; BOAC_EWORKSPACE. */
size_t boac_test_mlem_handover_bytes(const boac_geom *g, int B, int K,
                                     int config, int holders);
int boac_test_mlem_handover(const boac_geom *g, const float *mu,
                            const float *S, float *F, int K, int B, double *L,
                            int config, int holders, int withhold, void *ws,
                            size_t ws_bytes, void *stream);

/* Bytes of device workspace that `op` needs for B candidates of geometry g
 * on the current device (0 if none).  For BOAC_OP_SCORE_GRAD the size also
 * depends on K and ckpt_every: use boac_score_grad_workspace_bytes.
 * Returns 0 and sets nothing on invalid arguments. */
size_t boac_workspace_bytes(const boac_geom *g, int B, int op);

/* ---- Eq. 3-4: model attenuation map ------------------------------------
 * R(theta) = max(0, sum_{k=0..5} c_k P_k(cos theta)), theta = atan2(y, x)
 * (Eq. 3; P_k Legendre polynomials), then Eq. 4 at every pixel centre:
 *   CENTER: mu_b where r < R, mu_c where R <= r < R + dR, 0 beyond;
 *   AREA:   mu_b f(R) + mu_c (f(R + dR) - f(R)),
 *           f(R') = clamp(1/2 + (R' - r) / pixel_cm, 0, 1)
 *           (one-pixel radial ramp; differentiable in c).
 * Computed in float64, stored as float32.
 *   c   [B][6]     Legendre coefficients in cm (device, float32)
 *   mu  [B][n][n]  output, cm^-1 (device, float32)
 * Errors: BOAC_EINVAL for null pointers, B < 1, bad mode or geometry. */
int boac_rasterize_mu(const boac_geom *g, const boac_tissue *t, const float *c,
                      int B, int mode, float *mu, void *stream);

/* ---- Eq. 3-4 with per-candidate tissue values ----------------------------
 * The 9-parameter model p = (c_0..c_5, mu_b, mu_c, dR): the paper fixes
 * mu_b, mu_c and dR (Sec. II); here they may differ between candidates so
 * that an optimiser can move them too.  Same maps as boac_rasterize_mu.
 *   p   [B][9]     float32 (device): coefficients in cm, mu_b and mu_c in
 *                  cm^-1, dR in cm; a negative or NaN dR is taken as 0
 *   mu  [B][n][n]  output, cm^-1 (device, float32)
 * Errors: BOAC_EINVAL for null pointers, B < 1, bad mode or geometry. */
int boac_rasterize_mu_params(const boac_geom *g, const float *p, int B,
                             int mode, float *mu, void *stream);

/* ---- Eq. 1-2: forward projection q = A^mu F ----------------------------
 *   mu  [B][n][n], F [B][n][n]   (device, float32)
 *   q   [B][n_views][n_bins]     output (device, float32)
 * The attenuation is integrated along each ray on the fly; no workspace. */
int boac_project(const boac_geom *g, const float *mu, const float *F, int B,
                 float *q, void *stream);

/* ---- Eq. 2 adjoint: out = (A^mu)^T y -----------------------------------
 * Exact transpose of boac_project (same bilinear weights), deterministic:
 * for n = 64, 96, 128 with an even view count a race-free scatter of the
 * views that share a sample grid into per-grid images summed in grid order,
 * for other sizes a per-pixel gather.
 *   y   [B][n_views][n_bins] (device, float32); NULL means y = 1 everywhere
 *       (the MLEM sensitivity image)
 *   out [B][n][n]            output (device, float32)
 *   ws  workspace of boac_workspace_bytes(g, B, BOAC_OP_BACKPROJECT) bytes
 *       (holds the attenuation factors of every ray sample and the per-grid
 *       images). */
int boac_backproject(const boac_geom *g, const float *mu, const float *y,
                     int B, float *out, void *ws, size_t ws_bytes,
                     void *stream);

/* ---- MLEM (Sec. III step 3; Shepp & Vardi) ------------------------------
 * For each candidate b: sens = A^T 1, then K times
 *   q = A F;  r = S / q (0 where q <= 0);  F <- F * (A^T r) / sens
 * (0 where sens == 0).  Optionally scores the result with Eq. 5:
 *   L[b] = sum_i S_i ln q_i - q_i [- ln S_i!]   at q = A F^K,
 * reduced in float64 (0 ln q := 0 where S_i = 0; -inf where q_i = 0 < S_i).
 *   mu       [B][n][n]                         (device, float32)
 *   S        measured sinogram(s), [n_views][n_bins] per candidate,
 *            candidate b's at S + b * s_stride floats; s_stride = 0 shares
 *            one sinogram between all candidates
 *   F        [B][n][n] in: initial image (e.g. ones), out: F^K
 *   K        iterations (>= 0)
 *   L        [B] float64 output, or NULL to skip the score
 * boac_mlem is the batched path: one persistent fused kernel runs every
 * iteration of every candidate on chip.  n <= 128: one CTA per candidate,
 * or, with n_views % 4 == 0 where a cost model over the resident cluster
 * counts finds it faster (batches that cannot give every SM a candidate),
 * a thread-block cluster of 2 to 16 CTAs per candidate, each CTA on a share
 * of the sample grids; n = 256 with n_views % 4 == 0: a cluster per
 * candidate with the image split into bands of rows over its CTAs.
 * Batches too small to fill the GPU that take neither cluster form (at
 * most 32 candidates at n = 64 and 96, 16 at 128, 2 at 256, scaled by the
 * SM count / 152) run the unfused batched kernels of boac_mlem_unfused.  The choice depends on B,
 * so query the workspace with the same B.  boac_mlem_plain is the
 * launch-per-step path: one candidate at a time, separate project / ratio /
 * backproject / update kernels per iteration (the comparison baseline).
 * Workspace: boac_workspace_bytes(g, B, BOAC_OP_MLEM / BOAC_OP_MLEM_PLAIN). */
int boac_mlem(const boac_geom *g, const float *mu, const float *S,
              long long s_stride, float *F, int K, int B, double *L,
              int include_lgamma, void *ws, size_t ws_bytes, void *stream);
/* boac_mlem_unfused: the same MLEM over the whole batch with one launch per
 * step (attenuation table once; per iteration the grouped projector, the
 * ratio, the grouped back-projection and the update, each covering every
 * candidate, so one candidate spreads over many CTAs).  Same arguments,
 * conventions and errors as boac_mlem, except that any view count is
 * accepted (boac_mlem needs an even one); workspace boac_workspace_bytes(g,
 * B, BOAC_OP_MLEM_UNFUSED) (the attenuation tables, 4 n_views n^2 bytes per
 * candidate, dominate); deterministic; no device waits (the workspace status
 * word is set to 0). */
int boac_mlem_unfused(const boac_geom *g, const float *mu, const float *S,
                      long long s_stride, float *F, int K, int B, double *L,
                      int include_lgamma, void *ws, size_t ws_bytes,
                      void *stream);
int boac_mlem_plain(const boac_geom *g, const float *mu, const float *S,
                    long long s_stride, float *F, int K, int B, double *L,
                    int include_lgamma, void *ws, size_t ws_bytes,
                    void *stream);

/* ---- ragged batches -------------------------------------------------------
 * Candidates of different image sizes and iteration counts in one call
 * (Sec. III step 3 for every candidate; batching is this library's).  Each
 * candidate names a size class (a geometry in classes[]), its iteration count
 * K and the float offsets of its mu [n][n], sinogram [n_views][n] and image
 * F [n][n] (in: initial image, out: F^K) in three caller-owned device pools.
 * Its score (Eq. 5, as boac_mlem) goes to L[index in cands].  Per class, one
 * persistent fused kernel takes candidates from a work queue, largest K
 * first.  config[c] (host array, or NULL for defaults) picks class c's launch
 * shape: 2 * shape + pair, shape 0/1/2 = CTAs of 2n/4n/8n (<= 1024) threads,
 * pair = 1 for two views per sample grid instead of four (four needs
 * n_views % 4 == 0); with n_views % 4 == 0, configurations 6, 7 and 8 run
 * each candidate on a thread-block cluster of CTAs that split the image into
 * bands of rows: 5, 6 or 8 CTAs for n = 256 (the default there: the cluster
 * size that keeps the most SMs busy), 2, 4 or 8 for n = 128 (the default
 * for classes with few candidates).  An id that does not apply to a class
 * is BOAC_EINVAL.  The autotuner of the Python package chooses them.
 *   classes  [n_classes] geometries (host), 1 <= n_classes <= 8, sides
 *            64/96/128/256
 *   cands    [B] descriptors (host)
 *   ws       boac_mlem_ragged_workspace_bytes(...) bytes (device)
 * boac_mlem_ragged = boac_mlem_ragged_prepare (sorts the candidates and
 * copies their records into ws; not capturable in a CUDA graph: it copies
 * from pageable host memory) + boac_mlem_ragged_run (kernel launches only:
 * capturable, and replayable as long as ws keeps the prepared records). */
typedef struct {
    int cls;              /* size class: index into classes[]             */
    int K;                /* MLEM iterations (>= 0)                       */
    long long mu_off;     /* float offset of mu in mu_pool                */
    long long S_off;      /* float offset of the sinogram in S_pool       */
    long long F_off;      /* float offset of F in F_pool                  */
} boac_ragged_cand;

size_t boac_mlem_ragged_workspace_bytes(const boac_geom *classes, int n_classes,
                                        const boac_ragged_cand *cands, int B,
                                        const int *config);
int boac_mlem_ragged_prepare(const boac_geom *classes, int n_classes,
                             const boac_ragged_cand *cands, int B,
                             const int *config, void *ws, size_t ws_bytes,
                             void *stream);
int boac_mlem_ragged_run(const boac_geom *classes, int n_classes,
                         const boac_ragged_cand *cands, int B,
                         const float *mu_pool, const float *S_pool,
                         float *F_pool, double *L, int include_lgamma,
                         const int *config, void *ws, size_t ws_bytes,
                         void *stream);
int boac_mlem_ragged(const boac_geom *classes, int n_classes,
                     const boac_ragged_cand *cands, int B,
                     const float *mu_pool, const float *S_pool, float *F_pool,
                     double *L, int include_lgamma, const int *config,
                     void *ws, size_t ws_bytes, void *stream);

/* ---- boac_mlem without a workspace -------------------------------------
 * The paper has no counterpart: this is a convenience for callers that
 * cannot allocate device memory when they call the library (code running
 * under another framework's allocator or inside a callback where cudaMalloc
 * is not allowed, or a host process without an allocator of its own).
 * Same arguments and results as boac_mlem, minus the workspace (always the
 * one-CTA fused kernel, so results match boac_mlem's to float rounding where
 * boac_mlem picks another kernel for the batch size): the fused kernel's
 * scratch comes from a 64 MiB array built into the library, which every GPU
 * that loads the library keeps until the process exits.
 *   - Every call looks up that array's device address on the current device
 *     (cudaGetSymbolAddress); the first call on a device also loads the
 *     library's GPU code there, so make that first call before any stream
 *     capture.
 *   - L is required (BOAC_EINVAL if NULL): the status word of the bounded
 *     hand-over wait (see boac_workspace_status) lives in the built-in array,
 *     so here a candidate whose wait gave up shows only as a NaN in L.
 *   - Fewer candidates run at once when one slot's scratch (about
 *     n_views * n^2 / 2 + n^2 floats, plus three 256 x 257 images at n = 256)
 *     does not fit 64 MiB many times; BOAC_EWORKSPACE if not even one fits
 *     (never for n <= 128; at n = 256 above about 500 views).
 *   - Every call shares the one array: calls that can overlap on the GPU
 *     (different streams, or other threads) race and corrupt each other's
 *     results.  Serialise them.  Each call clears, on its stream, what must
 *     start at zero (the status word and the hand-over flags) and writes
 *     every other scratch entry before reading it.
 *   - Allocates nothing: no cudaMalloc, cudaFree or allocating library call. */
int boac_mlem_noalloc(const boac_geom *g, const float *mu, const float *S,
                      long long s_stride, float *F, int K, int B, double *L,
                      int include_lgamma, void *stream);

/* ---- Eq. 5: score of given images ---------------------------------------
 * L[b] = sum_i S_i ln q_i - q_i [- ln S_i!], q = A^mu F (float32 projection,
 * float64 reduction; same conventions as boac_mlem).
 *   ws  boac_workspace_bytes(g, B, BOAC_OP_SCORE) bytes (holds q). */
int boac_score(const boac_geom *g, const float *mu, const float *S,
               long long s_stride, const float *F, int B, int include_lgamma,
               double *L, void *ws, size_t ws_bytes, void *stream);

/* ---- d ln P / d c: gradient of the score through K MLEM iterations ------
 * The paper's optimiser is gradient-free (Sec. III); this gives it exact
 * gradients of the Eq. 5 score with respect to the Legendre coefficients of
 * Eq. 3, through the AREA rasterisation of Eq. 4 and K unrolled MLEM
 * iterations from F^0 = 1 (reverse mode; F^n is recomputed from checkpoints
 * stored every ckpt_every iterations, which changes memory, not results).
 *   t, c    tissue values and [B][6] float32 coefficients (device)
 *   S       sinogram(s) as for boac_mlem
 *   L       [B] float64 score, dL_dc [B][6] float64 gradient (device outputs)
 *   F_out   [B][n][n] F^K, or NULL
 *   ws      boac_score_grad_workspace_bytes(g, B, K, ckpt_every) bytes
 * Float32 arithmetic except the score and the final sum over pixels
 * (float64).  Where q = 0 < S (L = -inf) the gradient is taken as 0 there. */
size_t boac_score_grad_workspace_bytes(const boac_geom *g, int B, int K,
                                       int ckpt_every);
int boac_score_grad(const boac_geom *g, const boac_tissue *t, const float *c,
                    const float *S, long long s_stride, int K, int ckpt_every,
                    int B, int include_lgamma, double *L, double *dL_dc,
                    float *F_out, void *ws, size_t ws_bytes, void *stream);

/* boac_score_grad on the batched kernels of every step (one launch per
 * projection, back-projection and adjoint step), for comparison with the
 * fused kernel boac_score_grad takes for 64 / 96 / 128 images with a view
 * count divisible by 4.  Same arguments, results to float rounding, and
 * workspace (boac_score_grad_workspace_bytes covers both). */
int boac_score_grad_unfused(const boac_geom *g, const boac_tissue *t,
                            const float *c, const float *S, long long s_stride,
                            int K, int ckpt_every, int B, int include_lgamma,
                            double *L, double *dL_dc, float *F_out, void *ws,
                            size_t ws_bytes, void *stream);

/* The same score and its gradient in the 9-parameter model (see
 * boac_rasterize_mu_params): p [B][9] float32 (device) in, dL_dp [B][9]
 * float64 (device) out, in the order c_0..c_5, mu_b, mu_c, dR.  Through the
 * AREA map:
 *   dmu/dmu_b = f(R),  dmu/dmu_c = f(R + dR) - f(R),
 *   dmu/ddR   = mu_c f'(R + dR), taken as 0 where dR <= 0,
 * f' = 1/pixel_cm strictly inside a ramp and 0 elsewhere.  The first six
 * entries equal boac_score_grad's at the same tissue values.  Same
 * workspace (boac_score_grad_workspace_bytes), outputs and errors as
 * boac_score_grad. */
int boac_score_grad_params(const boac_geom *g, const float *p, const float *S,
                           long long s_stride, int K, int ckpt_every, int B,
                           int include_lgamma, double *L, double *dL_dp,
                           float *F_out, void *ws, size_t ws_bytes,
                           void *stream);

/* ---- The system matrix A^mu written out (Sec. III) ----------------------
 * The explicit-matrix counterpart of the matrix-free path, for comparison:
 * A[(v, b)][p] = pixel_cm * sum_k a_k w_k(p) over the ray samples k of bin b
 * of view v that read pixel p = i * n + j with bilinear weight w_k(p) (the
 * same samples, weights and attenuation factors as boac_project).  Rows
 * R = n_views * n_bins, columns n * n.
 *
 * Which pixels a row reads depends on the geometry only, so a boac_sysmat
 * holds one sparsity pattern, shared by every candidate: CSR row pointers
 * [R + 1] and column indices [nnz] (ascending within a row), and the CSR of
 * A^T (pixel pointers [n * n + 1], row indices [nnz], ascending).  Entries
 * whose weight happens to be exactly 0 are kept.  Values are per candidate,
 * interleaved by groups of 8 candidates so that one entry of a group is one
 * 32-byte sector: vals [G][2][nnz][8] float32, G = ceil(B / 8), with
 * vals[b / 8][0][e][b % 8] entry e of candidate b in the order of A and
 * vals[b / 8][1][e][b % 8] the same values in the order of A^T (zeros for
 * the candidates of the last group beyond B).
 *
 * boac_sysmat_create builds the pattern on the device (device memory of
 * about 16 bytes per nonzero, about 2 n nonzeros per row) and synchronises
 * `stream` twice; the caller owns the handle and frees it with
 * boac_sysmat_destroy.  Errors: BOAC_EINVAL (geometry, null out),
 * BOAC_ECUDA (allocation or launch), BOAC_EUNSUPPORTED (a consistency
 * check of the build failed, or a pixel is read by more than 4096 rows).
 * boac_sysmat_nnz returns the number of nonzeros (-1 for a null handle).
 * boac_sysmat_pattern copies the pattern into caller device buffers (any
 * may be NULL).
 * boac_sysmat_values fills vals for B candidates from mu [B][n][n]
 * (16-byte aligned).
 * boac_sysmat_project: q [B][R] = A F for F [B][n][n].
 * boac_sysmat_mlem: K MLEM iterations on F [B][n][n] in place (sens = A^T 1,
 * F <- F A^T(S / A F) / sens with the conventions of boac_mlem) and, when
 * L is not NULL, the Eq. 5 score of the result (float64 [B]); S and
 * s_stride as for boac_mlem; ws boac_sysmat_mlem_workspace_bytes(m, B)
 * bytes.  Deterministic: every sum runs in a fixed order. */
typedef struct boac_sysmat boac_sysmat;
int boac_sysmat_create(const boac_geom *g, boac_sysmat **out, void *stream);
int boac_sysmat_destroy(boac_sysmat *m);
long long boac_sysmat_nnz(const boac_sysmat *m);
int boac_sysmat_pattern(const boac_sysmat *m, int *row_ptr, int *col,
                        int *colT_ptr, int *rowT, void *stream);
int boac_sysmat_values(const boac_sysmat *m, const float *mu, int B,
                       float *vals, void *stream);
int boac_sysmat_project(const boac_sysmat *m, const float *vals,
                        const float *F, int B, float *q, void *stream);
size_t boac_sysmat_mlem_workspace_bytes(const boac_sysmat *m, int B);
int boac_sysmat_mlem(const boac_sysmat *m, const float *vals, const float *S,
                     long long s_stride, float *F, int K, int B, double *L,
                     int include_lgamma, void *ws, size_t ws_bytes,
                     void *stream);

/* Eq. 5 reduction alone, for expected counts q already on the device:
 *   q [B][n_views][n_bins] float32, S as above, L [B] float64 output. */
int boac_loglik(const boac_geom *g, const float *q, const float *S,
                long long s_stride, int B, int include_lgamma, double *L,
                void *stream);

#ifdef __cplusplus
}
#endif
#endif /* BOAC_H */
