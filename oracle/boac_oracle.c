/*
 * boac_oracle.c -- plain FP64 CPU oracle for the BOAC hot path
 * (Koutsantonis et al., "A Bayesian Optimization Approach for Attenuation
 * Correction in SPECT Brain Imaging", arXiv 2109.11920).
 *
 * TEST INFRASTRUCTURE.  Only the tests, the smoke check and the benchmark's
 * CPU-baseline leg use this file.  The CUDA library never links it, calls it
 * or shares a header with it.
 *
 * What it computes, step by step, in double precision, with no blocking,
 * fusion or reordering beyond the definitions:
 *
 *   Eq. 3   R(theta) = sum_{k=0..5} c_k P_k(cos theta), clamped at 0.
 *   Eq. 4   mu(r,theta): mu_b inside R, mu_c in the shell [R, R+dR), 0
 *           outside (CENTER mode: the pixel centre decides), or the same
 *           map with a radial linear ramp of width one pixel on each
 *           boundary (AREA mode, the differentiable reading).
 *   Eq. 1   the attenuated Radon transform, discretised as rotate-and-sum:
 *           N ray samples per bin spaced one pixel apart, bilinear sampling
 *           of F and mu at the rotated points, and the attenuation from the
 *           emission point to the detector taken as exp(-dx*(mu_k/2 +
 *           sum_{k'>k} mu_k')) (half of the own cell plus every cell between
 *           it and the detector).
 *   Eq. 2   S = A^mu F; the adjoint (A^mu)^T is an explicit scatter of
 *           dx*a*y to the four bilinear neighbours.
 *   MLEM    (Shepp-Vardi, cited in Sec. III): sens = A^T 1,
 *           F <- F * A^T(S / A F) / sens, with 0 where q <= 0 or sens == 0.
 *   Eq. 5   ln P = sum_i S_i ln q_i - q_i - ln S_i!  (0 ln q := 0 for S_i=0;
 *           -inf when q_i = 0 < S_i).
 *   grad    exact reverse-mode derivative of Eq. 5 after K MLEM iterations
 *           with respect to c_0..c_5 (AREA mode, F^0 = 1), and in the
 *           9-parameter form with respect to mu_b, mu_c and dR too (the
 *           paper keeps those fixed; this form lets them be optimised).
 *
 * Geometry (the paper gives none; this is the reading used on both sides):
 *   pixel (i,j), row i, column j, centre x=(j-c)dx, y=(i-c)dx, c=(n-1)/2;
 *   view v at phi_v = 2 pi v / V; bin b at s_b=(b-cb)ds, cb=(nb-1)/2;
 *   ray sample k at t_k=(k-c)dx; point p = s (cos,sin) + t (-sin,cos);
 *   the detector lies at t -> +infinity.
 *
 * Build: gcc -O2 -ffp-contract=off -fPIC -shared -lm -lpthread.
 */
#include <math.h>
#include <pthread.h>
#include <stdlib.h>
#include <string.h>

/* ------------------------------------------------------------------ */
/* Angles.  cos/sin of 2 pi v / V with the quadrant taken exactly, so that
 * views a multiple of 90 degrees apart are exact rotations of each other.  */
static void view_cos_sin(int v, int V, double *cs, double *sn)
{
    const double half_pi = 1.57079632679489661923;
    long long four_v = 4LL * (long long)v;
    int quadrant = (int)((four_v / V) % 4);
    long long rem = four_v % V;
    double th = half_pi * (double)rem / (double)V;
    double c = cos(th), s = sin(th);
    switch (quadrant) {
    case 0: *cs = c;  *sn = s;  break;
    case 1: *cs = -s; *sn = c;  break;
    case 2: *cs = -c; *sn = -s; break;
    default: *cs = s; *sn = -c; break;
    }
}

void orc_view_cos_sin(int v, int V, double *cs_sn)
{
    view_cos_sin(v, V, &cs_sn[0], &cs_sn[1]);
}

/* ------------------------------------------------------------------ */
/* Eq. 3: the first six Legendre polynomials (textbook closed forms).     */
void orc_legendre(double z, double *P)
{
    double z2 = z * z, z3 = z2 * z, z4 = z2 * z2, z5 = z4 * z;
    P[0] = 1.0;
    P[1] = z;
    P[2] = (3.0 * z2 - 1.0) / 2.0;
    P[3] = (5.0 * z3 - 3.0 * z) / 2.0;
    P[4] = (35.0 * z4 - 30.0 * z2 + 3.0) / 8.0;
    P[5] = (63.0 * z5 - 70.0 * z3 + 15.0 * z) / 8.0;
}

/* Pixel centre -> (r, cos theta).  theta = atan2(y, x), so cos theta = x/r;
 * at the origin theta is taken as 0.                                      */
static void pixel_polar(int n, double dx, int i, int j, double *r, double *z)
{
    double c = (n - 1) / 2.0;
    double x = (j - c) * dx, y = (i - c) * dx;
    *r = sqrt(x * x + y * y);
    *z = (*r > 0.0) ? x / *r : 1.0;
}

/* Eq. 3 unclamped, then clamped at zero.                                  */
static double boundary_raw(const double *coef, double z)
{
    double P[6];
    orc_legendre(z, P);
    double R = 0.0;
    for (int k = 0; k < 6; ++k) R += coef[k] * P[k];
    return R;
}

/* Radial ramp of width dx: fraction of the pixel inside radius Rp.       */
static double ramp(double Rp, double r, double dx)
{
    double f = 0.5 + (Rp - r) / dx;
    if (f < 0.0) f = 0.0;
    if (f > 1.0) f = 1.0;
    return f;
}

/* Eq. 4.  mode 0 = CENTER (hard classes at the pixel centre, half-open
 * intervals r<R, R<=r<R+dR), mode 1 = AREA (ramp).                        */
void orc_rasterize(int n, double dx, double mu_b, double mu_c, double dR,
                   const double *coef, int mode, double *mu)
{
    for (int i = 0; i < n; ++i)
        for (int j = 0; j < n; ++j) {
            double r, z;
            pixel_polar(n, dx, i, j, &r, &z);
            double R = boundary_raw(coef, z);
            if (R < 0.0) R = 0.0;
            double m;
            if (mode == 0) {
                if (r < R) m = mu_b;
                else if (r < R + dR) m = mu_c;
                else m = 0.0;
            } else {
                double fin = ramp(R, r, dx), fout = ramp(R + dR, r, dx);
                m = mu_b * fin + mu_c * (fout - fin);
            }
            mu[i * n + j] = m;
        }
}

/* ------------------------------------------------------------------ */
/* Projection geometry.                                                    */
typedef struct {
    int n, nb, V;
    double dx, ds;
} geom_t;

/* Continuous pixel index (u = column, w = row) of ray sample k of bin b.  */
static void ray_uw(const geom_t *g, double cs, double sn, int k, int b,
                   double *u, double *w)
{
    double c = (g->n - 1) / 2.0, cb = (g->nb - 1) / 2.0;
    double s = (b - cb) * g->ds, t = (k - c) * g->dx;
    double px = s * cs - t * sn, py = s * sn + t * cs;
    *u = c + px / g->dx;
    *w = c + py / g->dx;
}

/* Bilinear sample of image X at (u, w); neighbours outside the grid add 0. */
static double bilinear(int n, const double *X, double u, double w)
{
    double j0f = floor(u), i0f = floor(w);
    double au = u - j0f, aw = w - i0f;
    int j0 = (int)j0f, i0 = (int)i0f;
    double acc = 0.0;
    for (int di = 0; di < 2; ++di)
        for (int dj = 0; dj < 2; ++dj) {
            int i = i0 + di, j = j0 + dj;
            if (i < 0 || i >= n || j < 0 || j >= n) continue;
            double wt = (di ? aw : 1.0 - aw) * (dj ? au : 1.0 - au);
            acc += wt * X[i * n + j];
        }
    return acc;
}

/* Transpose of bilinear(): add val times each weight to the neighbours.  */
static void scatter(int n, double *X, double u, double w, double val)
{
    double j0f = floor(u), i0f = floor(w);
    double au = u - j0f, aw = w - i0f;
    int j0 = (int)j0f, i0 = (int)i0f;
    for (int di = 0; di < 2; ++di)
        for (int dj = 0; dj < 2; ++dj) {
            int i = i0 + di, j = j0 + dj;
            if (i < 0 || i >= n || j < 0 || j >= n) continue;
            double wt = (di ? aw : 1.0 - aw) * (dj ? au : 1.0 - au);
            X[i * n + j] += wt * val;
        }
}

/* Attenuation factors of every ray sample: a[(v*n + k)*nb + b].          */
static void attenuation_table(const geom_t *g, const double *mu, double *a)
{
    for (int v = 0; v < g->V; ++v) {
        double cs, sn;
        view_cos_sin(v, g->V, &cs, &sn);
        for (int b = 0; b < g->nb; ++b) {
            double suffix = 0.0; /* sum of mu samples between k and detector */
            for (int k = g->n - 1; k >= 0; --k) {
                double u, w;
                ray_uw(g, cs, sn, k, b, &u, &w);
                double m = bilinear(g->n, mu, u, w);
                a[((size_t)v * g->n + k) * g->nb + b] =
                    exp(-g->dx * (0.5 * m + suffix));
                suffix += m;
            }
        }
    }
}

void orc_attenuation(int n, int nb, int V, double dx, double ds,
                     const double *mu, double *a)
{
    geom_t g = {n, nb, V, dx, ds};
    attenuation_table(&g, mu, a);
}

/* q = A X using a precomputed table (Eq. 1 / Eq. 2).                     */
static void project_table(const geom_t *g, const double *a, const double *X,
                          double *q)
{
    for (int v = 0; v < g->V; ++v) {
        double cs, sn;
        view_cos_sin(v, g->V, &cs, &sn);
        for (int b = 0; b < g->nb; ++b) {
            double acc = 0.0;
            for (int k = 0; k < g->n; ++k) {
                double u, w;
                ray_uw(g, cs, sn, k, b, &u, &w);
                acc += a[((size_t)v * g->n + k) * g->nb + b] *
                       bilinear(g->n, X, u, w);
            }
            q[v * g->nb + b] = g->dx * acc;
        }
    }
}

/* out = A^T y using a precomputed table (explicit scatter).              */
static void backproject_table(const geom_t *g, const double *a,
                              const double *y, double *out)
{
    memset(out, 0, sizeof(double) * g->n * g->n);
    for (int v = 0; v < g->V; ++v) {
        double cs, sn;
        view_cos_sin(v, g->V, &cs, &sn);
        for (int b = 0; b < g->nb; ++b)
            for (int k = 0; k < g->n; ++k) {
                double u, w;
                ray_uw(g, cs, sn, k, b, &u, &w);
                double val = g->dx * a[((size_t)v * g->n + k) * g->nb + b] *
                             y[v * g->nb + b];
                scatter(g->n, out, u, w, val);
            }
    }
}

/* Public projector: attenuation computed on the fly along each ray.     */
void orc_project(int n, int nb, int V, double dx, double ds, const double *mu,
                 const double *F, double *q)
{
    geom_t g = {n, nb, V, dx, ds};
    for (int v = 0; v < V; ++v) {
        double cs, sn;
        view_cos_sin(v, V, &cs, &sn);
        for (int b = 0; b < nb; ++b) {
            double suffix = 0.0, acc = 0.0;
            for (int k = n - 1; k >= 0; --k) {
                double u, w;
                ray_uw(&g, cs, sn, k, b, &u, &w);
                double m = bilinear(n, mu, u, w);
                double a = exp(-dx * (0.5 * m + suffix));
                suffix += m;
                acc += a * bilinear(n, F, u, w);
            }
            q[v * nb + b] = dx * acc;
        }
    }
}

/* The system matrix A^mu written out (Sec. III: the "system matrix" linking
 * F to the sinogram, Eq. 2): A[(v*nb + b)*n*n + i*n + j] = dx * sum_k a_k w_k,
 * w_k the bilinear weight with which sample k of ray (v, b) reads pixel
 * (i, j), a_k its attenuation factor.  Dense, row-major [V*nb][n*n].       */
void orc_system_matrix(int n, int nb, int V, double dx, double ds,
                       const double *mu, double *A)
{
    geom_t g = {n, nb, V, dx, ds};
    size_t npix = (size_t)n * n;
    double *a = malloc(sizeof(double) * (size_t)V * n * nb);
    attenuation_table(&g, mu, a);
    memset(A, 0, sizeof(double) * (size_t)V * nb * npix);
    for (int v = 0; v < V; ++v) {
        double cs, sn;
        view_cos_sin(v, V, &cs, &sn);
        for (int b = 0; b < nb; ++b) {
            double *row = A + ((size_t)v * nb + b) * npix;
            for (int k = 0; k < n; ++k) {
                double u, w;
                ray_uw(&g, cs, sn, k, b, &u, &w);
                double j0f = floor(u), i0f = floor(w);
                double au = u - j0f, aw = w - i0f;
                double ak = a[((size_t)v * n + k) * nb + b];
                for (int di = 0; di < 2; ++di)
                    for (int dj = 0; dj < 2; ++dj) {
                        int i = (int)i0f + di, j = (int)j0f + dj;
                        if (i < 0 || i >= n || j < 0 || j >= n) continue;
                        double wt = (di ? aw : 1.0 - aw) * (dj ? au : 1.0 - au);
                        row[(size_t)i * n + j] += dx * ak * wt;
                    }
            }
        }
    }
    free(a);
}

/* Public back-projector: the explicit transpose of orc_project.          */
void orc_backproject(int n, int nb, int V, double dx, double ds,
                     const double *mu, const double *y, double *out)
{
    geom_t g = {n, nb, V, dx, ds};
    memset(out, 0, sizeof(double) * n * n);
    for (int v = 0; v < V; ++v) {
        double cs, sn;
        view_cos_sin(v, V, &cs, &sn);
        for (int b = 0; b < nb; ++b) {
            double suffix = 0.0;
            for (int k = n - 1; k >= 0; --k) {
                double u, w;
                ray_uw(&g, cs, sn, k, b, &u, &w);
                double m = bilinear(n, mu, u, w);
                double a = exp(-dx * (0.5 * m + suffix));
                suffix += m;
                scatter(n, out, u, w, dx * a * y[v * nb + b]);
            }
        }
    }
}

/* ------------------------------------------------------------------ */
/* MLEM (Shepp-Vardi) with a fixed iteration count (Sec. III, step 3).    */
static void mlem_table(const geom_t *g, const double *a, const double *sens,
                       const double *S, int K, double *F)
{
    int nbin = g->V * g->nb, npix = g->n * g->n;
    double *q = malloc(sizeof(double) * nbin);
    double *r = malloc(sizeof(double) * nbin);
    double *z = malloc(sizeof(double) * npix);
    for (int it = 0; it < K; ++it) {
        project_table(g, a, F, q);
        for (int i = 0; i < nbin; ++i) r[i] = (q[i] > 0.0) ? S[i] / q[i] : 0.0;
        backproject_table(g, a, r, z);
        for (int j = 0; j < npix; ++j)
            F[j] = (sens[j] > 0.0) ? F[j] * z[j] / sens[j] : 0.0;
    }
    free(q);
    free(r);
    free(z);
}

static void sensitivity(const geom_t *g, const double *a, double *sens)
{
    int nbin = g->V * g->nb;
    double *ones = malloc(sizeof(double) * nbin);
    for (int i = 0; i < nbin; ++i) ones[i] = 1.0;
    backproject_table(g, a, ones, sens);
    free(ones);
}

void orc_mlem(int n, int nb, int V, double dx, double ds, const double *mu,
              const double *S, int K, double *F)
{
    geom_t g = {n, nb, V, dx, ds};
    double *a = malloc(sizeof(double) * (size_t)V * n * nb);
    double *sens = malloc(sizeof(double) * n * n);
    attenuation_table(&g, mu, a);
    sensitivity(&g, a, sens);
    mlem_table(&g, a, sens, S, K, F);
    free(a);
    free(sens);
}

void orc_sensitivity(int n, int nb, int V, double dx, double ds,
                     const double *mu, double *sens)
{
    geom_t g = {n, nb, V, dx, ds};
    double *a = malloc(sizeof(double) * (size_t)V * n * nb);
    attenuation_table(&g, mu, a);
    sensitivity(&g, a, sens);
    free(a);
}

/* ------------------------------------------------------------------ */
/* Eq. 5: Poisson log-likelihood of S given the expected counts q.        */
double orc_loglik(int nbin, const double *S, const double *q, int include_lgamma)
{
    double L = 0.0;
    for (int i = 0; i < nbin; ++i) {
        double term;
        if (S[i] > 0.0) {
            if (!(q[i] > 0.0)) return -INFINITY;
            term = S[i] * log(q[i]) - q[i];
        } else {
            term = -q[i];
        }
        if (include_lgamma) term -= lgamma(S[i] + 1.0);
        L += term;
    }
    return L;
}

double orc_score(int n, int nb, int V, double dx, double ds, const double *mu,
                 const double *S, const double *F, int include_lgamma)
{
    double *q = malloc(sizeof(double) * V * nb);
    orc_project(n, nb, V, dx, ds, mu, F, q);
    double L = orc_loglik(V * nb, S, q, include_lgamma);
    free(q);
    return L;
}

/* ------------------------------------------------------------------ */
/* Reverse-mode gradient of Eq. 5 after K MLEM iterations from F^0 = 1,   */
/* with respect to the attenuation map (AREA rasterisation), then to the  */
/* Legendre coefficients and, for the 9-parameter form, to mu_b, mu_c and */
/* dR as well.                                                             */

/* abar[v,k,b] += dx * ybin[v,b] * (B_v X)(k,b): the derivative of either
 * <qbar, A X> (forward) or <zbar, A^T y> (backward) with respect to the
 * attenuation factor of sample (v,k,b).                                   */
static void accumulate_abar(const geom_t *g, const double *ybin,
                            const double *X, double *abar)
{
    for (int v = 0; v < g->V; ++v) {
        double cs, sn;
        view_cos_sin(v, g->V, &cs, &sn);
        for (int b = 0; b < g->nb; ++b) {
            double yb = ybin[v * g->nb + b];
            if (yb == 0.0) continue;
            for (int k = 0; k < g->n; ++k) {
                double u, w;
                ray_uw(g, cs, sn, k, b, &u, &w);
                abar[((size_t)v * g->n + k) * g->nb + b] +=
                    g->dx * yb * bilinear(g->n, X, u, w);
            }
        }
    }
}

/* Forward pass and reverse sweep: returns L and fills mubar[n*n] with
 * dL/dmu at every pixel (the caller owns mubar).                          */
static double score_mubar(int n, int nb, int V, double dx, double ds,
                          double mu_b, double mu_c, double dR,
                          const double *coef, const double *S, int K,
                          int include_lgamma, double *mubar, double *F_out)
{
    geom_t g = {n, nb, V, dx, ds};
    int npix = n * n, nbin = V * nb;
    size_t ntab = (size_t)V * n * nb;

    /* forward: mu, a, sens, and every iterate */
    double *mu = malloc(sizeof(double) * npix);
    orc_rasterize(n, dx, mu_b, mu_c, dR, coef, 1, mu);
    double *a = malloc(sizeof(double) * ntab);
    attenuation_table(&g, mu, a);
    double *sens = malloc(sizeof(double) * npix);
    sensitivity(&g, a, sens);

    double *F = malloc(sizeof(double) * (size_t)(K + 1) * npix);
    double *q = malloc(sizeof(double) * (size_t)(K + 1) * nbin);
    double *r = malloc(sizeof(double) * (size_t)K * nbin);
    double *z = malloc(sizeof(double) * (size_t)K * npix);
    for (int j = 0; j < npix; ++j) F[j] = 1.0;
    for (int it = 0; it < K; ++it) {
        double *Fi = F + (size_t)it * npix, *Fn = F + (size_t)(it + 1) * npix;
        double *qi = q + (size_t)it * nbin, *ri = r + (size_t)it * nbin;
        double *zi = z + (size_t)it * npix;
        project_table(&g, a, Fi, qi);
        for (int i = 0; i < nbin; ++i) ri[i] = (qi[i] > 0.0) ? S[i] / qi[i] : 0.0;
        backproject_table(&g, a, ri, zi);
        for (int j = 0; j < npix; ++j)
            Fn[j] = (sens[j] > 0.0) ? Fi[j] * zi[j] / sens[j] : 0.0;
    }
    double *qK = q + (size_t)K * nbin, *FK = F + (size_t)K * npix;
    project_table(&g, a, FK, qK);
    double L = orc_loglik(nbin, S, qK, include_lgamma);
    if (F_out) memcpy(F_out, FK, sizeof(double) * npix);

    /* reverse */
    double *abar = calloc(ntab, sizeof(double));
    double *Fbar = malloc(sizeof(double) * npix);
    double *Fbar_new = malloc(sizeof(double) * npix);
    double *sensbar = calloc(npix, sizeof(double));
    double *zbar = malloc(sizeof(double) * npix);
    double *qbar = malloc(sizeof(double) * nbin);
    double *rbar = malloc(sizeof(double) * nbin);
    double *tmp = malloc(sizeof(double) * npix);

    /* d L / d q^K */
    for (int i = 0; i < nbin; ++i) {
        if (S[i] > 0.0) qbar[i] = (qK[i] > 0.0) ? S[i] / qK[i] - 1.0 : 0.0;
        else qbar[i] = -1.0;
    }
    backproject_table(&g, a, qbar, Fbar);       /* Fbar = A^T qbar        */
    accumulate_abar(&g, qbar, FK, abar);

    for (int it = K - 1; it >= 0; --it) {
        double *Fi = F + (size_t)it * npix, *Fn = F + (size_t)(it + 1) * npix;
        double *qi = q + (size_t)it * nbin, *ri = r + (size_t)it * nbin;
        double *zi = z + (size_t)it * npix;
        /* F^{n+1} = F^n z / sens */
        for (int j = 0; j < npix; ++j) {
            if (sens[j] > 0.0) {
                zbar[j] = Fbar[j] * Fi[j] / sens[j];
                sensbar[j] -= Fbar[j] * Fn[j] / sens[j];
                Fbar_new[j] = Fbar[j] * zi[j] / sens[j];
            } else {
                zbar[j] = 0.0;
                Fbar_new[j] = 0.0;
            }
        }
        /* z = A^T r */
        project_table(&g, a, zbar, rbar);         /* rbar = A zbar         */
        accumulate_abar(&g, ri, zbar, abar);
        /* r = S / q */
        for (int i = 0; i < nbin; ++i)
            qbar[i] = (qi[i] > 0.0) ? -rbar[i] * S[i] / (qi[i] * qi[i]) : 0.0;
        /* q = A F^n */
        backproject_table(&g, a, qbar, tmp);
        for (int j = 0; j < npix; ++j) Fbar_new[j] += tmp[j];
        accumulate_abar(&g, qbar, Fi, abar);
        memcpy(Fbar, Fbar_new, sizeof(double) * npix);
    }
    /* sens = A^T 1 */
    {
        double *ones = malloc(sizeof(double) * nbin);
        for (int i = 0; i < nbin; ++i) ones[i] = 1.0;
        accumulate_abar(&g, ones, sensbar, abar);
        free(ones);
    }

    /* a = exp(-dx (m_k / 2 + sum_{k'>k} m_k')):
     * mbar_j = -dx (abar_j a_j / 2 + sum_{k<j} abar_k a_k).
     * mu samples are bilinear in mu, so mubar = sum_v B_v^T mbar_v.      */
    for (int j = 0; j < npix; ++j) mubar[j] = 0.0;
    for (int v = 0; v < V; ++v) {
        double cs, sn;
        view_cos_sin(v, V, &cs, &sn);
        for (int b = 0; b < nb; ++b) {
            double prefix = 0.0;
            for (int k = 0; k < n; ++k) {
                size_t idx = ((size_t)v * n + k) * nb + b;
                double aa = abar[idx] * a[idx];
                double mbar = -dx * (0.5 * aa + prefix);
                prefix += aa;
                double u, w;
                ray_uw(&g, cs, sn, k, b, &u, &w);
                scatter(n, mubar, u, w, mbar);
            }
        }
    }

    free(mu); free(a); free(sens); free(F); free(q); free(r); free(z);
    free(abar); free(Fbar); free(Fbar_new); free(sensbar); free(zbar);
    free(qbar); free(rbar); free(tmp);
    return L;
}

/* Chain rule through Eq. 4 (AREA) and Eq. 3:
 *   mu = mu_b f(R) + mu_c (f(R + dR) - f(R)),  R = max(0, sum c_k P_k(z)),
 *   f(R') = clamp(1/2 + (R' - r)/dx, 0, 1), f' = 1/dx strictly inside the ramp,
 *   dmu/dc_k  = ((mu_b - mu_c) f'(R) + mu_c f'(R + dR)) P_k(z)   [R > 0]
 *   dmu/dmu_b = f(R),  dmu/dmu_c = f(R + dR) - f(R),
 *   dmu/ddR   = mu_c f'(R + dR)                                  [dR > 0].
 * gc[6] always; gt[3] = (d/dmu_b, d/dmu_c, d/ddR) when not NULL.         */
static void grad_from_mubar(int n, double dx, double mu_b, double mu_c,
                            double dR, const double *coef,
                            const double *mubar, double *gc, double *gt)
{
    for (int k = 0; k < 6; ++k) gc[k] = 0.0;
    if (gt) gt[0] = gt[1] = gt[2] = 0.0;
    for (int i = 0; i < n; ++i)
        for (int j = 0; j < n; ++j) {
            double rr, zz;
            pixel_polar(n, dx, i, j, &rr, &zz);
            double Rraw = boundary_raw(coef, zz);
            double mb = mubar[i * n + j];
            if (gt) {
                double R = Rraw > 0.0 ? Rraw : 0.0;
                double fin = ramp(R, rr, dx), fout = ramp(R + dR, rr, dx);
                double e_out = 0.5 + (R + dR - rr) / dx;
                gt[0] += mb * fin;
                gt[1] += mb * (fout - fin);
                if (dR > 0.0 && e_out > 0.0 && e_out < 1.0) gt[2] += mb * mu_c / dx;
            }
            if (!(Rraw > 0.0)) continue;
            double R = Rraw;
            double e_in = 0.5 + (R - rr) / dx, e_out = 0.5 + (R + dR - rr) / dx;
            double d_in = (e_in > 0.0 && e_in < 1.0) ? 1.0 / dx : 0.0;
            double d_out = (e_out > 0.0 && e_out < 1.0) ? 1.0 / dx : 0.0;
            double dmu_dR = (mu_b - mu_c) * d_in + mu_c * d_out;
            if (dmu_dR == 0.0) continue;
            double P[6];
            orc_legendre(zz, P);
            double s = mb * dmu_dR;
            for (int k = 0; k < 6; ++k) gc[k] += s * P[k];
        }
}

/* Score and dL/dc_0..c_5 for fixed tissue values.                         */
double orc_score_grad(int n, int nb, int V, double dx, double ds, double mu_b,
                      double mu_c, double dR, const double *coef,
                      const double *S, int K, int include_lgamma,
                      double *grad, double *F_out)
{
    double *mubar = malloc(sizeof(double) * n * n);
    double L = score_mubar(n, nb, V, dx, ds, mu_b, mu_c, dR, coef, S, K,
                           include_lgamma, mubar, F_out);
    grad_from_mubar(n, dx, mu_b, mu_c, dR, coef, mubar, grad, NULL);
    free(mubar);
    return L;
}

/* The 9-parameter form p = (c_0..c_5, mu_b, mu_c, dR): score and dL/dp.
 * A negative dR is taken as 0 (the map of dR = 0, derivative 0).          */
double orc_score_grad_params(int n, int nb, int V, double dx, double ds,
                             const double *p, const double *S, int K,
                             int include_lgamma, double *grad, double *F_out)
{
    double dR = p[8] > 0.0 ? p[8] : 0.0;
    double *mubar = malloc(sizeof(double) * n * n);
    double L = score_mubar(n, nb, V, dx, ds, p[6], p[7], dR, p, S, K,
                           include_lgamma, mubar, F_out);
    grad_from_mubar(n, dx, p[6], p[7], dR, p, mubar, grad, grad + 6);
    free(mubar);
    return L;
}

/* ------------------------------------------------------------------ */
/* Batch drivers: candidates split over POSIX threads (one candidate per  */
/* task); each candidate runs the single-candidate code above unchanged.  */
typedef struct {
    int n, nb, V;
    double dx, ds;
    int B;
    const double *mu;      /* [B][n*n]                                     */
    const double *S;       /* [B][V*nb] rows s_stride apart (0 = shared)   */
    long long s_stride;
    const int *iters;      /* [B]                                          */
    double *F;             /* [B][n*n] in/out                              */
    double *L;             /* [B] or NULL                                  */
    int include_lgamma;
    int next;
    pthread_mutex_t lock;
} batch_job;

static void *batch_worker(void *arg)
{
    batch_job *j = (batch_job *)arg;
    int npix = j->n * j->n;
    for (;;) {
        pthread_mutex_lock(&j->lock);
        int c = j->next++;
        pthread_mutex_unlock(&j->lock);
        if (c >= j->B) break;
        const double *mu = j->mu + (size_t)c * npix;
        const double *S = j->S + (size_t)c * j->s_stride;
        double *F = j->F + (size_t)c * npix;
        orc_mlem(j->n, j->nb, j->V, j->dx, j->ds, mu, S, j->iters[c], F);
        if (j->L)
            j->L[c] = orc_score(j->n, j->nb, j->V, j->dx, j->ds, mu, S, F,
                                j->include_lgamma);
    }
    return NULL;
}

/* MLEM (+ optional score) for B candidates on nthreads host threads.     */
int orc_mlem_batch(int n, int nb, int V, double dx, double ds, int B,
                   const double *mu, const double *S, long long s_stride,
                   const int *iters, double *F, double *L, int include_lgamma,
                   int nthreads)
{
    batch_job job = {n, nb, V, dx, ds, B, mu, S, s_stride, iters, F, L,
                     include_lgamma, 0, PTHREAD_MUTEX_INITIALIZER};
    if (nthreads < 1) nthreads = 1;
    if (nthreads > B) nthreads = B;
    pthread_t *th = malloc(sizeof(pthread_t) * nthreads);
    for (int t = 0; t < nthreads; ++t)
        pthread_create(&th[t], NULL, batch_worker, &job);
    for (int t = 0; t < nthreads; ++t) pthread_join(th[t], NULL);
    free(th);
    return nthreads;
}
