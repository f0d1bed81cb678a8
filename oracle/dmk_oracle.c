/*
 * dmk_oracle.c -- plain FP64 CPU oracle for the discrete DMK evaluation pass
 * of Jiang & Greengard (arXiv 2308.00292).  TEST INFRASTRUCTURE ONLY: see
 * dmk_oracle.h.  Nothing here is shared with the CUDA path.
 *
 * Layout of the file, in the order of the paper:
 *   1. special functions: Legendre polynomials, Gauss-Legendre rules,
 *      Chebyshev polynomials of the first kind (Sec. 2.1)
 *   2. the prolate spheroidal wave function psi_0^c (App. A.5) by the
 *      Legendre-Galerkin form of the prolate differential operator,
 *      extended off [-1,1] by the eigen-relation of the operator F_c
 *   3. kernel splittings (Sec. 3.2 Gaussian; Sec. 3.6 PSWF) and their
 *      Fourier transforms (eqs. differencekernelft, differencekernelft3,
 *      windowedkernelft and the windowing of Sec. 4.x "Handling singularities")
 *   4. O1: the direct sum (eq. discretesum with zero self-interaction)
 *   5. the level-restricted adaptive tree (Sec. 3.2, Step 0)
 *   6. the DMK algorithm, Steps 0-5 of Sec. 3.4
 *   7. the 2D Laplace kernel log r: the Fourier-space splitting of Sec. 3.7
 *      at lambda = 0 in the plane, a quad-tree, and Steps 0-5 in 2D
 *
 * Readings of the paper taken here:
 *   - Fourier spacing h_l = 2 pi / (3 R_l): the difference kernel D_l has
 *     support radius R_l and colleague separations reach 2 R_l per
 *     coordinate, so its periodic images must sit 3 R_l apart (Poisson
 *     summation, eq. poissonsummation); the trapezoidal weight h_l^3 / (2 pi)^3
 *     is included in w_{l,m} (eqs. differencekernelft2 / wlmdef omit it).
 *   - D_l is applied at box level l for l = 0 .. L_max - 1; the root's only
 *     colleague is itself.
 *   - F_out(B) = B is not a leaf and holds sources; F_in(B) = B holds targets
 *     and some colleague has F_out.  The residual level of a pair is the
 *     level of the source's leaf.
 *   - Leaves at every level (including L_max) evaluate their local expansion.
 *   - The windowed root kernel of the PSWF splitting is
 *     What_0(k) = 8 pi sin^2(R_t k / 2) / k^2 * psi(k R_0 / c) / psi(0),
 *     R_t = (1 + sqrt 3) R_0 (truncated-kernel windowing of Sec. 4).
 *   - The PSWF self term is S_L(0) = psi(0) / (c_0 R_L).
 *   - A box holding more than n_s points is split unless all of them lie in
 *     one finest Morton cell (coincident points); otherwise duplicates would
 *     drive the tree to the depth cap, where their self terms rho S_L(0)
 *     grow like 2^L and the far field's eps-relative error no longer cancels.
 *   - Yukawa kernel exp(-lambda r) / r (lambda > 0), split in Fourier space
 *     (Sec. 3.7, eqs. yukawaPSWFkernels / yukawagaussiankernels, times the 4 pi
 *     of the kernel without its 1/(4 pi)): the unit-box map turns lambda into
 *     lambda S.  The PSWF mollified kernel has no closed form in physical
 *     space; it is the radial inverse transform
 *       S_l(r) = 2 / (pi psi(0) r) int_0^inf psi(sqrt(k^2 + lambda^2) R_l / c)
 *                k sin(k r) / (k^2 + lambda^2) dk.
 *     psi decays only like 1/x beyond x = 1, so the integral is taken as the
 *     Laplace mollifier Phi(r/R_l)/r (its lambda = 0 value, in closed form) plus
 *     the integral of the difference of the two integrands, which decays
 *     faster by (lambda R_l / c)^2 / x^2; that one by Gauss-Legendre panels up
 *     to x = sqrt(k^2 + lambda^2) R_l / c = 4.  The Gaussian one has the closed form
 *     (e^{-lambda r} erfc(a - r/sigma) - e^{lambda r} erfc(a + r/sigma)) / (2 r),
 *     a = lambda sigma / 2.  The windowed root kernel multiplies the mollifier by
 *     the transform of the kernel truncated at R_t:
 *       4 pi (k - e^{-lambda R_t} (lambda sin k R_t + k cos k R_t)) / (k (k^2 + lambda^2)).
 */
#include "dmk_oracle.h"

#include <complex.h>
#include <math.h>
#include <stdint.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef double complex cplx;

#ifndef M_PI
#define M_PI 3.14159265358979323846
#endif

/* ====================================================================== */
/* 1. Special functions                                                    */
/* ====================================================================== */

/* Legendre polynomial P_k(x) by the three-term recurrence. */
static double legendre_p(int k, double x)
{
    if (k == 0) return 1.0;
    double p0 = 1.0, p1 = x;
    for (int j = 1; j < k; ++j) {
        double p2 = ((2.0 * j + 1.0) * x * p1 - j * p0) / (j + 1.0);
        p0 = p1;
        p1 = p2;
    }
    return p1;
}

/* n-point Gauss-Legendre rule on [-1, 1] (Newton iteration on P_n). */
static void gauss_legendre(int n, double *x, double *w)
{
    for (int i = 0; i < n; ++i) {
        double z = cos(M_PI * (i + 0.75) / (n + 0.5));
        double dp = 1.0;
        for (int it = 0; it < 100; ++it) {
            double p0 = 1.0, p1 = z;
            for (int j = 1; j < n; ++j) {
                double p2 = ((2.0 * j + 1.0) * z * p1 - j * p0) / (j + 1.0);
                p0 = p1;
                p1 = p2;
            }
            /* p1 = P_n(z), p0 = P_{n-1}(z) */
            dp = n * (z * p1 - p0) / (z * z - 1.0);
            double dz = p1 / dp;
            z -= dz;
            if (fabs(dz) < 1e-16) break;
        }
        x[i] = z;
        w[i] = 2.0 / ((1.0 - z * z) * dp * dp);
    }
}

/* Chebyshev polynomial of the first kind from its definition
 * T_n(x) = cos(n arccos x), x in [-1, 1] (Sec. 2.1). */
static double cheb_t(int n, double x)
{
    if (x > 1.0) x = 1.0;
    if (x < -1.0) x = -1.0;
    return cos(n * acos(x));
}

/* derivative T_n'(x) = n U_{n-1}(x), with U_k the Chebyshev polynomials of the
 * second kind by their three-term recurrence (U_0 = 1, U_1 = 2x) */
static double cheb_dt(int n, double x)
{
    if (n == 0) return 0.0;
    if (x > 1.0) x = 1.0;
    if (x < -1.0) x = -1.0;
    double u0 = 1.0, u1 = 2.0 * x;
    if (n == 1) return 1.0;
    for (int k = 2; k < n; ++k) {
        double u2 = 2.0 * x * u1 - u0;
        u0 = u1;
        u1 = u2;
    }
    return n * u1;
}

/* Chebyshev nodes of the first kind r_i = cos(pi (i - 1/2) / p), i = 1..p. */
static void cheb_nodes(int p, double *t)
{
    for (int i = 1; i <= p; ++i) t[i - 1] = cos(M_PI * (i - 0.5) / p);
}

/* Inverse of a dense n x n matrix by Gauss-Jordan elimination with partial
 * pivoting.  a is overwritten.  Returns 0 on success. */
static int mat_inverse(int n, double *a, double *inv)
{
    for (int i = 0; i < n * n; ++i) inv[i] = 0.0;
    for (int i = 0; i < n; ++i) inv[i * n + i] = 1.0;
    for (int col = 0; col < n; ++col) {
        int piv = col;
        for (int r = col + 1; r < n; ++r)
            if (fabs(a[r * n + col]) > fabs(a[piv * n + col])) piv = r;
        if (a[piv * n + col] == 0.0) return -1;
        if (piv != col)
            for (int k = 0; k < n; ++k) {
                double t = a[col * n + k]; a[col * n + k] = a[piv * n + k]; a[piv * n + k] = t;
                t = inv[col * n + k]; inv[col * n + k] = inv[piv * n + k]; inv[piv * n + k] = t;
            }
        double d = a[col * n + col];
        for (int k = 0; k < n; ++k) { a[col * n + k] /= d; inv[col * n + k] /= d; }
        for (int r = 0; r < n; ++r) {
            if (r == col) continue;
            double f = a[r * n + col];
            if (f == 0.0) continue;
            for (int k = 0; k < n; ++k) {
                a[r * n + k] -= f * a[col * n + k];
                inv[r * n + k] -= f * inv[col * n + k];
            }
        }
    }
    return 0;
}

/* ====================================================================== */
/* 2. PSWF psi_0^c (App. A.5)                                              */
/* ====================================================================== */
/* psi_0^c is the eigenfunction of F_c[phi](x) = int_{-1}^1 phi(t) e^{icxt} dt
 * with the largest eigenvalue.  It is also the lowest eigenfunction of the
 * prolate operator L[psi] = -((1 - x^2) psi')' + c^2 x^2 psi, which is
 * tridiagonal in the orthonormal Legendre basis; psi_0 is even, so only even
 * degrees k = 0, 2, 4, ... enter.  Off [-1, 1] the eigen-relation
 * psi(x) = lambda_0^{-1} int_{-1}^1 psi(t) cos(c x t) dt is used. */

#define PSWF_NK 120 /* even Legendre degrees 0 .. 238 */
#define PSWF_NQ 600 /* quadrature nodes for the eigen-relation */

typedef struct {
    double c;
    int nk;                 /* number of significant even terms */
    double beta[PSWF_NK];   /* coefficient of sqrt((2k+1)/2) P_k, k = 2i */
    double lambda0, c0, c2, chi0;
    double xq[PSWF_NQ], wq[PSWF_NQ], psiq[PSWF_NQ];
} pswf_t;

static double pswf_series(const pswf_t *s, double x)
{
    /* sum_i beta_i sqrt((2k+1)/2) P_k(x), k = 2i, recurrence in k */
    double p0 = 1.0, p1 = x, acc = s->beta[0] * sqrt(0.5);
    int kmax = 2 * (s->nk - 1);
    for (int k = 1; k < kmax; ++k) {
        double p2 = ((2.0 * k + 1.0) * x * p1 - k * p0) / (k + 1.0);
        p0 = p1;
        p1 = p2;
        int kk = k + 1; /* p1 = P_kk */
        if ((kk & 1) == 0) acc += s->beta[kk / 2] * sqrt((2.0 * kk + 1.0) / 2.0) * p1;
    }
    return acc;
}

static void pswf_init(pswf_t *s, double c)
{
    memset(s, 0, sizeof(*s));
    s->c = c;
    int n = PSWF_NK;
    double d[PSWF_NK], e[PSWF_NK];
    for (int i = 0; i < n; ++i) {
        double k = 2.0 * i;
        double bk = (2.0 * k * k + 2.0 * k - 1.0) / ((2.0 * k - 1.0) * (2.0 * k + 3.0));
        d[i] = k * (k + 1.0) + c * c * bk;
        double ak = (k + 1.0) * (k + 2.0) / ((2.0 * k + 3.0) * sqrt((2.0 * k + 1.0) * (2.0 * k + 5.0)));
        e[i] = c * c * ak; /* couples i and i+1 */
    }
    /* smallest eigenvalue by Sturm-sequence bisection */
    double lo = 1e300, hi = d[0];
    for (int i = 0; i < n; ++i) {
        double r = fabs(i > 0 ? e[i - 1] : 0.0) + fabs(i < n - 1 ? e[i] : 0.0);
        if (d[i] - r < lo) lo = d[i] - r;
    }
    for (int it = 0; it < 400; ++it) {
        double mid = 0.5 * (lo + hi);
        int cnt = 0;
        double q = d[0] - mid;
        if (q < 0) ++cnt;
        for (int i = 1; i < n; ++i) {
            if (q == 0.0) q = 1e-300;
            q = d[i] - mid - e[i - 1] * e[i - 1] / q;
            if (q < 0) ++cnt;
        }
        if (cnt >= 1) hi = mid; else lo = mid;
        if (hi - lo <= 1e-15 * fabs(hi)) break;
    }
    double chi = 0.5 * (lo + hi);
    s->chi0 = chi;
    /* eigenvector by inverse iteration with a shift just below chi (the
     * shifted matrix is then positive definite, so the Thomas solve is safe) */
    double shift = chi - 1e-9 * (1.0 + fabs(chi));
    double v[PSWF_NK], cp[PSWF_NK], dp[PSWF_NK];
    for (int i = 0; i < n; ++i) v[i] = 1.0 / (1.0 + i);
    for (int it = 0; it < 6; ++it) {
        /* solve (T - shift I) y = v */
        double bb = d[0] - shift;
        cp[0] = e[0] / bb;
        dp[0] = v[0] / bb;
        for (int i = 1; i < n; ++i) {
            double den = (d[i] - shift) - e[i - 1] * cp[i - 1];
            cp[i] = (i < n - 1) ? e[i] / den : 0.0;
            dp[i] = (v[i] - e[i - 1] * dp[i - 1]) / den;
        }
        v[n - 1] = dp[n - 1];
        for (int i = n - 2; i >= 0; --i) v[i] = dp[i] - cp[i] * v[i + 1];
        double nrm = 0.0;
        for (int i = 0; i < n; ++i) nrm += v[i] * v[i];
        nrm = sqrt(nrm);
        for (int i = 0; i < n; ++i) v[i] /= nrm;
    }
    double vmax = 0.0;
    for (int i = 0; i < n; ++i) if (fabs(v[i]) > vmax) vmax = fabs(v[i]);
    s->nk = n;
    while (s->nk > 2 && fabs(v[s->nk - 1]) < 1e-19 * vmax) s->nk--;
    for (int i = 0; i < n; ++i) s->beta[i] = (i < s->nk) ? v[i] : 0.0;
    /* normalise psi(0) = 1 */
    double p0 = pswf_series(s, 0.0);
    for (int i = 0; i < n; ++i) s->beta[i] /= p0;
    /* int_{-1}^1 psi = sqrt(2) beta_0 (orthogonality); lambda_0 psi(0) = that */
    s->lambda0 = sqrt(2.0) * s->beta[0];
    s->c0 = s->beta[0] / sqrt(2.0);
    /* c_2 = int_0^1 x^2 psi(x) dx by Gauss-Legendre on [0, 1] */
    {
        double xg[200], wg[200];
        gauss_legendre(200, xg, wg);
        double acc = 0.0;
        for (int i = 0; i < 200; ++i) {
            double x = 0.5 * (xg[i] + 1.0);
            acc += 0.5 * wg[i] * x * x * pswf_series(s, x);
        }
        s->c2 = acc;
    }
    gauss_legendre(PSWF_NQ, s->xq, s->wq);
    for (int i = 0; i < PSWF_NQ; ++i) s->psiq[i] = pswf_series(s, s->xq[i]);
}

/* psi(x) for any real x: series on [-1, 1], eigen-relation outside. */
static double pswf_eval(const pswf_t *s, double x)
{
    double ax = fabs(x);
    if (ax <= 1.0) return pswf_series(s, ax);
    double acc = 0.0;
    for (int i = 0; i < PSWF_NQ; ++i) acc += s->wq[i] * s->psiq[i] * cos(s->c * x * s->xq[i]);
    return acc / s->lambda0;
}

/* psi(x1) - psi(x2) without cancellation, from the eigen-relation:
 * (1/lambda_0) int psi(t) (cos(c x1 t) - cos(c x2 t)) dt with the difference of
 * cosines written as -2 sin(c (x1 + x2) t / 2) sin(c (x1 - x2) t / 2).  Needed
 * where both arguments are small (the Yukawa Dhat_l near k = 0). */
static double pswf_diff(const pswf_t *s, double x1, double x2)
{
    double acc = 0.0;
    for (int i = 0; i < PSWF_NQ; ++i)
        acc += s->wq[i] * s->psiq[i] * sin(0.5 * s->c * (x1 + x2) * s->xq[i]) *
               sin(0.5 * s->c * (x1 - x2) * s->xq[i]);
    return -2.0 * acc / s->lambda0;
}

/* Phi(s) = c_0^{-1} int_0^s psi(t) dt for s in [0, 1]; 1 beyond (Sec. 3.6).
 * Uses int_0^s P_k = (P_{k+1}(s) - P_{k-1}(s)) / (2k + 1) for even k >= 2. */
static double pswf_Phi(const pswf_t *s, double x)
{
    if (x >= 1.0) return 1.0;
    if (x <= 0.0) return 0.0;
    double acc = s->beta[0] * sqrt(0.5) * x;
    for (int i = 1; i < s->nk; ++i) {
        int k = 2 * i;
        acc += s->beta[i] * sqrt((2.0 * k + 1.0) / 2.0) *
               (legendre_p(k + 1, x) - legendre_p(k - 1, x)) / (2.0 * k + 1.0);
    }
    return acc / s->c0;
}

/* ====================================================================== */
/* 3. Kernel splittings                                                    */
/* ====================================================================== */

#define YUK_LEVELS 22   /* levels 0 .. 21 */
#define YUK_PANELS 8    /* regular panels up to the cutoff */
#define YUK_NODES 24    /* Gauss-Legendre nodes per panel */
#define YUK_MAXP 40     /* regular plus graded panels */
#define YUK_NQ (YUK_MAXP * YUK_NODES)

typedef struct {
    oracle_params prm;
    pswf_t *pswf;   /* PSWF splitting only */
    double Rt;      /* truncation radius of the windowed root kernel */
    double hW;      /* root Fourier spacing */
    double lam;     /* Yukawa parameter in unit-box units (0: Laplace) */
    /* PSWF Yukawa: per level, nodes k_j and weights g_j of
     * S_l(r) = Phi(r / R_l) / r + sum_j g_j sin(k_j r) / r,
     * S_l(0) = psi(0) / (c_0 R_l) + sum_j g_j k_j */
    double (*yk)[YUK_NQ], (*yg)[YUK_NQ];
    int yn[YUK_LEVELS];
} split_t;

static double level_R(int l) { return ldexp(1.0, -l); }

static double gauss_sigma(const split_t *sp, int l) { return level_R(l) / sp->prm.delta; }

/* Yukawa: the level-l mollified kernel, the Laplace one plus the radial
 * quadrature of the difference */
static double yuk_pswf_S(const split_t *sp, int l, double r)
{
    double acc = 0.0, R = level_R(l);
    if (r == 0.0) {
        for (int j = 0; j < sp->yn[l]; ++j) acc += sp->yg[l][j] * sp->yk[l][j];
        return 1.0 / (sp->pswf->c0 * R) + acc;
    }
    for (int j = 0; j < sp->yn[l]; ++j) acc += sp->yg[l][j] * sin(sp->yk[l][j] * r);
    return (pswf_Phi(sp->pswf, r / R) + acc) / r;
}

static double yuk_gauss_S(double lam, double sg, double r)
{
    double a = 0.5 * lam * sg;
    if (r == 0.0) return 2.0 / (sqrt(M_PI) * sg) * exp(-a * a) - lam * erfc(a);
    return (exp(-lam * r) * erfc(a - r / sg) - exp(lam * r) * erfc(a + r / sg)) / (2.0 * r);
}

/* mollified kernel S_l(r); r = 0 gives its finite limit */
static double split_S(const split_t *sp, int l, double r)
{
    double R = level_R(l);
    if (sp->lam > 0.0) {
        if (sp->prm.splitting == ORACLE_PSWF) return yuk_pswf_S(sp, l, r);
        return yuk_gauss_S(sp->lam, gauss_sigma(sp, l), r);
    }
    if (sp->prm.splitting == ORACLE_PSWF) {
        if (r == 0.0) return 1.0 / (sp->pswf->c0 * R); /* psi(0) = 1 */
        return pswf_Phi(sp->pswf, r / R) / r;
    } else {
        double sg = gauss_sigma(sp, l);
        if (r == 0.0) return 2.0 / (sqrt(M_PI) * sg);
        return erf(r / sg) / r;
    }
}

/* residual kernel R_l(r) = K(r) - S_l(r), r > 0 */
static double split_R(const split_t *sp, int l, double r)
{
    double R = level_R(l);
    if (sp->lam > 0.0) {
        if (sp->prm.splitting == ORACLE_PSWF) return exp(-sp->lam * r) / r - yuk_pswf_S(sp, l, r);
        /* the closed form, without the cancellation of K - S_l */
        double sg = gauss_sigma(sp, l), a = 0.5 * sp->lam * sg;
        return (exp(-sp->lam * r) * erfc(r / sg - a) + exp(sp->lam * r) * erfc(r / sg + a)) / (2.0 * r);
    }
    if (sp->prm.splitting == ORACLE_PSWF) {
        return (1.0 - pswf_Phi(sp->pswf, r / R)) / r;
    } else {
        return erfc(r / gauss_sigma(sp, l)) / r;
    }
}

/* d/dr of the residual kernel R_l(r) = 1/r - S_l(r), r > 0:
 *   PSWF:     -Phi'(r/R)/(R r) - (1 - Phi(r/R))/r^2, Phi'(t) = psi(t)/c_0
 *   Gaussian: -2 exp(-r^2/sigma^2)/(sqrt(pi) sigma r) - erfc(r/sigma)/r^2 */
static double split_dR(const split_t *sp, int l, double r)
{
    double R = level_R(l);
    if (sp->prm.splitting == ORACLE_PSWF) {
        double t = r / R;
        double dphi = t < 1.0 ? pswf_eval(sp->pswf, t) / sp->pswf->c0 : 0.0;
        return -dphi / (R * r) - (1.0 - pswf_Phi(sp->pswf, t)) / (r * r);
    } else {
        double sg = gauss_sigma(sp, l);
        return -2.0 * exp(-(r * r) / (sg * sg)) / (sqrt(M_PI) * sg * r) - erfc(r / sg) / (r * r);
    }
}

/* Fourier transform of the difference kernel D_l at |k| */
static double split_Dhat(const split_t *sp, int l, double k)
{
    double R = level_R(l), R1 = level_R(l + 1);
    if (sp->lam > 0.0) {
        /* 4 pi [G_{l+1}(k) - G_l(k)] / (k^2 + lambda^2), G the mollifier in
         * the variable sqrt(k^2 + lambda^2) */
        double k2 = k * k + sp->lam * sp->lam, kk = sqrt(k2);
        if (sp->prm.splitting == ORACLE_PSWF) {
            const pswf_t *s = sp->pswf;
            return 4.0 * M_PI * pswf_diff(s, kk * R1 / s->c, kk * R / s->c) / k2;
        }
        double s0 = gauss_sigma(sp, l), s1 = gauss_sigma(sp, l + 1);
        /* e^{-a} - e^{-b} = e^{-a} (1 - e^{a - b}), without cancellation */
        double a = k2 * s1 * s1 / 4.0, b = k2 * s0 * s0 / 4.0;
        return 4.0 * M_PI * exp(-a) * (-expm1(a - b)) / k2;
    }
    if (sp->prm.splitting == ORACLE_PSWF) {
        const pswf_t *s = sp->pswf;
        if (k == 0.0) return 2.0 * M_PI * s->c2 / s->c0 * (R * R - R1 * R1);
        return 4.0 * M_PI * (pswf_eval(s, k * R1 / s->c) - pswf_eval(s, k * R / s->c)) / (k * k);
    } else {
        double s0 = gauss_sigma(sp, l), s1 = gauss_sigma(sp, l + 1);
        if (k == 0.0) return M_PI * (s0 * s0 - s1 * s1);
        return 4.0 * M_PI * (exp(-k * k * s1 * s1 / 4.0) - exp(-k * k * s0 * s0 / 4.0)) / (k * k);
    }
}

/* Fourier transform of the windowed root kernel W_0 at |k| */
static double split_What(const split_t *sp, double k)
{
    double Rt = sp->Rt;
    double win;
    if (sp->lam > 0.0) {
        double lam = sp->lam, k2 = k * k + lam * lam, kk = sqrt(k2);
        if (sp->prm.splitting == ORACLE_PSWF) win = pswf_eval(sp->pswf, kk / sp->pswf->c);
        else { double sg = gauss_sigma(sp, 0); win = exp(-k2 * sg * sg / 4.0); }
        /* transform of exp(-lambda r)/r truncated at Rt */
        double tr;
        if (k == 0.0) {
            /* 1 - e^{-x} (1 + x) = sum_{n >= 2} (-1)^n (n - 1) x^n / n!  (its
             * series for small x; -expm1(-x) - x e^{-x} otherwise), x = lambda R_t */
            double x = lam * Rt, v;
            if (x < 0.1) {
                double term = 0.5 * x * x;  /* x^n / n! at n = 2 */
                v = 0.0;
                for (int n = 2; n < 20; ++n) {
                    v += ((n & 1) ? -1.0 : 1.0) * (n - 1) * term;
                    term *= x / (n + 1);
                }
            } else {
                v = -expm1(-x) - x * exp(-x);
            }
            tr = 4.0 * M_PI * v / (lam * lam);
        }
        else {
            /* k - e^{-x} (lambda sin kR_t + k cos kR_t) as a sum without
             * cancellation: -k expm1(-x) + 2 k e^{-x} sin^2(k R_t / 2) - e^{-x} lambda sin kR_t */
            double x = lam * Rt, sn = sin(0.5 * k * Rt);
            double num = -k * expm1(-x) + 2.0 * k * exp(-x) * sn * sn - exp(-x) * lam * sin(k * Rt);
            tr = 4.0 * M_PI * num / (k * k2);
        }
        return tr * win;
    }
    if (sp->prm.splitting == ORACLE_PSWF) win = pswf_eval(sp->pswf, k / sp->pswf->c);
    else { double sg = gauss_sigma(sp, 0); win = exp(-k * k * sg * sg / 4.0); }
    if (k == 0.0) return 2.0 * M_PI * Rt * Rt * win;
    double sn = sin(Rt * k / 2.0);
    return 8.0 * M_PI * sn * sn / (k * k) * win;
}

/* difference-kernel spacing h_l: periodic images 3 R_l apart */
static double split_h(int l) { return 2.0 * M_PI / (3.0 * level_R(l)); }

/* Table 1 (PSWF parameters for the 3D Laplace kernel) */
static const double T1_eps[4] = {1e-3, 1e-6, 1e-9, 1e-12};
static const double T1_c[4] = {7.2462000846862793, 13.739999771118164,
                               20.736000061035156, 27.870000839233398};
static const int T1_N1[4] = {13, 25, 39, 53};
static const int T1_p[4] = {9, 18, 28, 38};
/* Gaussian columns of Table 1, used for the cross-check splitting.  N1^G is
 * read as 2 nf; nf is taken about 10% above N1^G / 2, where the Fourier
 * approximation of D_l reaches eps (pinned in the tests). */
static const int T1_nfG[4] = {12, 24, 36, 48};
static const int T1_pG[4] = {16, 30, 46, 62};

static int table_row(double eps)
{
    /* the row with the largest table precision that is <= eps */
    for (int i = 0; i < 4; ++i)
        if (T1_eps[i] <= eps * (1.0 + 1e-12)) return i;
    return 3;
}

void oracle_default_params(oracle_params *prm)
{
    if (prm->eps <= 0.0) prm->eps = 1e-6;
    int row = table_row(prm->eps);
    if (prm->max_level <= 0) prm->max_level = 20;
    if (prm->leaf_cap <= 0) prm->leaf_cap = 280;
    if (prm->splitting == ORACLE_PSWF) {
        if (prm->c <= 0.0) prm->c = T1_c[row];
        if (prm->p <= 0) prm->p = T1_p[row];
        if (prm->nf <= 0) prm->nf = (T1_N1[row] - 1) / 2;
        if (prm->n0 <= 0) {
            double Rt = 1.0 + sqrt(3.0);
            double hW = 2.0 * M_PI / (2.0 + Rt);
            prm->n0 = (int)ceil(prm->c / hW) + 1;
        }
    } else {
        if (prm->delta <= 0.0) {
            /* erfc(delta) = eps / 10 by bisection */
            double lo = 0.5, hi = 10.0, target = prm->eps / 10.0;
            for (int it = 0; it < 200; ++it) {
                double mid = 0.5 * (lo + hi);
                if (erfc(mid) > target) lo = mid; else hi = mid;
            }
            prm->delta = 0.5 * (lo + hi);
        }
        if (prm->gauss_b <= 0.0) prm->gauss_b = prm->delta;
        if (prm->p <= 0) prm->p = T1_pG[row];
        if (prm->nf <= 0) prm->nf = T1_nfG[row];
        if (prm->n0 <= 0) {
            double sg = 1.0 / prm->delta;
            double Rt = sqrt(3.0) + prm->gauss_b * sg;
            double hW = 2.0 * M_PI / (2.0 + Rt);
            double K = 2.0 * sqrt(log(100.0 / prm->eps)) / sg;
            prm->n0 = (int)ceil(K / hW);
        }
    }
}

static int split_init(split_t *sp, const oracle_params *in)
{
    memset(sp, 0, sizeof(*sp));
    sp->prm = *in;
    oracle_default_params(&sp->prm);
    if (sp->prm.splitting == ORACLE_PSWF) {
        sp->pswf = (pswf_t *)malloc(sizeof(pswf_t));
        if (!sp->pswf) return -1;
        pswf_init(sp->pswf, sp->prm.c);
        sp->Rt = 1.0 + sqrt(3.0);
    } else {
        sp->Rt = sqrt(3.0) + sp->prm.gauss_b / sp->prm.delta;
    }
    /* W_0 is supported within Rt + R_0; separations within the unit box are
     * at most 1 per coordinate, so the images must be 2 + Rt apart. */
    sp->hW = 2.0 * M_PI / (2.0 + sp->Rt);
    return 0;
}

/* set the Yukawa parameter (unit-box units) and, for the PSWF splitting, the
 * radial quadrature of every level's mollified kernel */
static int split_set_lambda(split_t *sp, double lam)
{
    sp->lam = lam;
    if (!(lam > 0.0) || sp->prm.splitting != ORACLE_PSWF) return 0;
    sp->yk = malloc(sizeof(*sp->yk) * YUK_LEVELS);
    sp->yg = malloc(sizeof(*sp->yg) * YUK_LEVELS);
    if (!sp->yk || !sp->yg) return -1;
    double xg[YUK_NODES], wg[YUK_NODES];
    gauss_legendre(YUK_NODES, xg, wg);
    const pswf_t *s = sp->pswf;
    for (int l = 0; l < YUK_LEVELS; ++l) {
        double R = level_R(l);
        /* k from 0 to where sqrt(k^2 + lambda^2) R / c = 4, in panels: the
         * factor k / (k^2 + lambda^2) varies on the scale lambda near k = 0
         * (poles at +-i lambda), so the first panels grow geometrically from
         * width lambda, then regular panels of width kmax / 8 follow */
        double x4 = 4.0 * s->c / R;
        double kmax = x4 > lam ? sqrt(x4 * x4 - lam * lam) : 0.0;
        double pw = kmax / YUK_PANELS;
        double br[YUK_MAXP + 1];
        int nb = 0;
        br[nb++] = 0.0;
        for (double b = lam; b < pw && nb < YUK_MAXP - YUK_PANELS; b *= 3.0) br[nb++] = b;
        double b0 = br[nb - 1];
        for (int q = 1; q <= YUK_PANELS; ++q) br[nb++] = b0 + (kmax - b0) * q / YUK_PANELS;
        int j = 0;
        for (int q = 0; q + 1 < nb; ++q) {
            double a = br[q], h = br[q + 1] - br[q];
            for (int i = 0; i < YUK_NODES; ++i, ++j) {
                double k = a + 0.5 * h * (xg[i] + 1.0), w = 0.5 * h * wg[i];
                double k2 = k * k + lam * lam;
                sp->yk[l][j] = k;
                sp->yg[l][j] = 2.0 / M_PI * w *
                               (pswf_eval(s, sqrt(k2) * R / s->c) * k / k2 - pswf_eval(s, k * R / s->c) / k);
            }
        }
        sp->yn[l] = j;
    }
    return 0;
}

static void split_free(split_t *sp)
{
    free(sp->pswf);
    free(sp->yk);
    free(sp->yg);
    sp->pswf = NULL;
    sp->yk = sp->yg = NULL;
}

/* ====================================================================== */
/* 4. O1: direct summation                                                 */
/* ====================================================================== */

void oracle_direct(const double *src, const double *rho, int64_t ns,
                   const double *tgt, int64_t nt, double *pot, int nthreads)
{
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#else
    (void)nthreads;
#endif
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t i = 0; i < nt; ++i) {
        double sum = 0.0, comp = 0.0; /* Neumaier compensated sum */
        double x = tgt[3 * i], y = tgt[3 * i + 1], z = tgt[3 * i + 2];
        for (int64_t j = 0; j < ns; ++j) {
            double dx = x - src[3 * j], dy = y - src[3 * j + 1], dz = z - src[3 * j + 2];
            double r2 = dx * dx + dy * dy + dz * dz;
            if (r2 == 0.0) continue;
            double term = rho[j] / sqrt(r2);
            double t = sum + term;
            if (fabs(sum) >= fabs(term)) comp += (sum - t) + term;
            else comp += (term - t) + sum;
            sum = t;
        }
        pot[i] = sum + comp;
    }
}

/* O1 for the Yukawa kernel: u_i = sum_{j : y_j != x_i} rho_j exp(-lambda r) / r */
void oracle_direct_yukawa(const double *src, const double *rho, int64_t ns,
                          const double *tgt, int64_t nt, double lambda, double *pot, int nthreads)
{
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#else
    (void)nthreads;
#endif
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t i = 0; i < nt; ++i) {
        double sum = 0.0, comp = 0.0;
        double x = tgt[3 * i], y = tgt[3 * i + 1], z = tgt[3 * i + 2];
        for (int64_t j = 0; j < ns; ++j) {
            double dx = x - src[3 * j], dy = y - src[3 * j + 1], dz = z - src[3 * j + 2];
            double r2 = dx * dx + dy * dy + dz * dz;
            if (r2 == 0.0) continue;
            double r = sqrt(r2);
            double term = rho[j] * exp(-lambda * r) / r;
            double t = sum + term;
            if (fabs(sum) >= fabs(term)) comp += (sum - t) + term;
            else comp += (term - t) + sum;
            sum = t;
        }
        pot[i] = sum + comp;
    }
}

/* O1 gradient: grad u(x_i) = sum_{j : y_j != x_i} rho_j (y_j - x_i) / |x_i - y_j|^3,
 * the derivative of eq. discretesum in the target position, with compensated
 * sums per component. */
void oracle_direct_grad(const double *src, const double *rho, int64_t ns,
                        const double *tgt, int64_t nt, double *grad, int nthreads)
{
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#else
    (void)nthreads;
#endif
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t i = 0; i < nt; ++i) {
        double sum[3] = {0.0, 0.0, 0.0}, comp[3] = {0.0, 0.0, 0.0};
        const double *x = &tgt[3 * i];
        for (int64_t j = 0; j < ns; ++j) {
            double d[3] = {src[3 * j] - x[0], src[3 * j + 1] - x[1], src[3 * j + 2] - x[2]};
            double r2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
            if (r2 == 0.0) continue;
            double f = rho[j] / (r2 * sqrt(r2));
            for (int a = 0; a < 3; ++a) {
                double term = f * d[a];
                double t = sum[a] + term;
                if (fabs(sum[a]) >= fabs(term)) comp[a] += (sum[a] - t) + term;
                else comp[a] += (term - t) + sum[a];
                sum[a] = t;
            }
        }
        for (int a = 0; a < 3; ++a) grad[3 * i + a] = sum[a] + comp[a];
    }
}

/* ====================================================================== */
/* 5. Level-restricted adaptive tree (Sec. 3.2; Step 0 of Sec. 3.4)        */
/* ====================================================================== */

typedef struct {
    int level;
    int64_t ix, iy, iz;
    int parent;
    int child[8];
    int64_t start, count; /* range in the point order array */
    int leaf;
    int64_t nsrc, ntgt;
    int col[27];
    int ncol;
    int fout, fin, has_local;
    double *proxy;
    cplx *Phi;
    double *local;
} obox;

typedef struct {
    int64_t n;            /* points in the union set */
    double *u;            /* unit-box coordinates [n][3] */
    int64_t *cell;        /* finest (level 21) cell [n][3] */
    double *q;            /* charge (0 for pure targets) */
    char *is_src, *is_tgt;
    int64_t *out_index;   /* target output slot or -1 */
    double S;             /* scale of the unit-box map */
} opoints;

typedef struct {
    obox *b;
    int nb, cap;
    int64_t *ord;          /* point order: boxes own contiguous ranges */
    int lev_start[23], lev_count[23];
    int nlev;              /* number of levels present (L_max + 1) */
} otree;

static uint64_t morton3(int64_t ix, int64_t iy, int64_t iz, int level)
{
    uint64_t m = 0;
    for (int b = 0; b < level; ++b) {
        m |= (uint64_t)((ix >> b) & 1) << (3 * b);
        m |= (uint64_t)((iy >> b) & 1) << (3 * b + 1);
        m |= (uint64_t)((iz >> b) & 1) << (3 * b + 2);
    }
    return m;
}

/* unique key of (level, cell): Morton code with a leading one bit */
static uint64_t cell_key(int level, int64_t ix, int64_t iy, int64_t iz)
{
    return morton3(ix, iy, iz, level) | ((uint64_t)1 << (3 * level));
}

static int cmp_u64(const void *a, const void *b)
{
    uint64_t x = *(const uint64_t *)a, y = *(const uint64_t *)b;
    return (x > y) - (x < y);
}

static int key_in(const uint64_t *keys, int n, uint64_t k)
{
    return n > 0 && bsearch(&k, keys, (size_t)n, sizeof(uint64_t), cmp_u64) != NULL;
}

static int tree_push(otree *t, const obox *b)
{
    if (t->nb == t->cap) {
        int nc = t->cap ? 2 * t->cap : 1024;
        obox *nbp = (obox *)realloc(t->b, (size_t)nc * sizeof(obox));
        if (!nbp) return -1;
        t->b = nbp;
        t->cap = nc;
    }
    t->b[t->nb++] = *b;
    return t->nb - 1;
}

/* Box at (level, ix, iy, iz) or -1; boxes of a level are in Morton order. */
static int tree_find(const otree *t, int level, int64_t ix, int64_t iy, int64_t iz)
{
    if (level >= t->nlev) return -1;
    int64_t lim = (int64_t)1 << level;
    if (ix < 0 || iy < 0 || iz < 0 || ix >= lim || iy >= lim || iz >= lim) return -1;
    uint64_t key = morton3(ix, iy, iz, level);
    int lo = t->lev_start[level], hi = lo + t->lev_count[level] - 1;
    while (lo <= hi) {
        int mid = (lo + hi) / 2;
        const obox *b = &t->b[mid];
        uint64_t mk = morton3(b->ix, b->iy, b->iz, level);
        if (mk == key) return mid;
        if (mk < key) lo = mid + 1; else hi = mid - 1;
    }
    return -1;
}

/* Top-down build: a box is split when it has more than leaf_cap points or
 * is in the forced set, and its level is below max_level. */
static int tree_build(otree *t, const opoints *P, const oracle_params *prm,
                      const uint64_t *forced, int nforced)
{
    t->nb = 0;
    for (int64_t i = 0; i < P->n; ++i) t->ord[i] = i;
    int64_t *tmp = (int64_t *)malloc((size_t)(P->n > 0 ? P->n : 1) * sizeof(int64_t));
    if (!tmp) return -1;
    obox root;
    memset(&root, 0, sizeof(root));
    root.parent = -1;
    for (int c = 0; c < 8; ++c) root.child[c] = -1;
    root.start = 0;
    root.count = P->n;
    if (tree_push(t, &root) < 0) { free(tmp); return -1; }
    t->nlev = 1;
    t->lev_start[0] = 0;
    t->lev_count[0] = 1;
    for (int l = 0; l < prm->max_level; ++l) {
        int s = t->lev_start[l], e = s + t->lev_count[l];
        int next_start = t->nb;
        for (int bi = s; bi < e; ++bi) {
            obox *b = &t->b[bi];
            /* capacity rule; a box whose points all share one finest cell
             * (exact or near duplicates) is never split by it */
            int same_cell = 1;
            if (b->count > prm->leaf_cap) {
                int64_t p0 = t->ord[b->start];
                for (int64_t k = b->start + 1; k < b->start + b->count && same_cell; ++k) {
                    int64_t pk = t->ord[k];
                    for (int d = 0; d < 3; ++d)
                        if (P->cell[3 * pk + d] != P->cell[3 * p0 + d]) same_cell = 0;
                }
            }
            int split = (b->count > prm->leaf_cap && !same_cell) ||
                        key_in(forced, nforced, cell_key(l, b->ix, b->iy, b->iz));
            if (!split) continue;
            /* stable partition of the box's points into the 8 octants */
            int64_t cnt[8] = {0}, off[8];
            int shift = 20 - l;
            for (int64_t k = b->start; k < b->start + b->count; ++k) {
                int64_t pi = t->ord[k];
                int oct = (int)(((P->cell[3 * pi] >> shift) & 1) | (((P->cell[3 * pi + 1] >> shift) & 1) << 1) |
                                (((P->cell[3 * pi + 2] >> shift) & 1) << 2));
                cnt[oct]++;
            }
            off[0] = b->start;
            for (int c = 1; c < 8; ++c) off[c] = off[c - 1] + cnt[c - 1];
            int64_t o2[8];
            memcpy(o2, off, sizeof(off));
            for (int64_t k = b->start; k < b->start + b->count; ++k) {
                int64_t pi = t->ord[k];
                int oct = (int)(((P->cell[3 * pi] >> shift) & 1) | (((P->cell[3 * pi + 1] >> shift) & 1) << 1) |
                                (((P->cell[3 * pi + 2] >> shift) & 1) << 2));
                tmp[o2[oct]++] = pi;
            }
            memcpy(t->ord + b->start, tmp + b->start, (size_t)b->count * sizeof(int64_t));
            int64_t bix = b->ix, biy = b->iy, biz = b->iz;
            for (int c = 0; c < 8; ++c) {
                if (cnt[c] == 0) continue;
                obox ch;
                memset(&ch, 0, sizeof(ch));
                ch.level = l + 1;
                ch.ix = 2 * bix + (c & 1);
                ch.iy = 2 * biy + ((c >> 1) & 1);
                ch.iz = 2 * biz + ((c >> 2) & 1);
                ch.parent = bi;
                for (int q = 0; q < 8; ++q) ch.child[q] = -1;
                ch.start = off[c];
                ch.count = cnt[c];
                int id = tree_push(t, &ch);
                if (id < 0) { free(tmp); return -1; }
                t->b[bi].child[c] = id;
                b = &t->b[bi];
            }
        }
        if (t->nb == next_start) break;
        t->lev_start[l + 1] = next_start;
        t->lev_count[l + 1] = t->nb - next_start;
        t->nlev = l + 2;
    }
    free(tmp);
    for (int i = 0; i < t->nb; ++i) {
        obox *b = &t->b[i];
        b->leaf = 1;
        for (int c = 0; c < 8; ++c) if (b->child[c] >= 0) b->leaf = 0;
    }
    return 0;
}

/* Level restriction: a non-empty leaf T at level a must not share a boundary
 * point with a non-leaf box at level a+1.  Leaves in violation are added to
 * the forced set and the tree is rebuilt until none remains; the result is
 * the smallest balanced refinement of the leaf-capacity tree. */
static int tree_build_balanced(otree *t, const opoints *P, const oracle_params *prm)
{
    uint64_t *forced = NULL;
    int nforced = 0, capf = 0;
    for (int iter = 0; iter < 64; ++iter) {
        if (tree_build(t, P, prm, forced, nforced) < 0) { free(forced); return -1; }
        int added = 0;
        for (int i = 0; i < t->nb; ++i) {
            obox *T = &t->b[i];
            if (!T->leaf) continue;
            int a = T->level;
            if (a + 1 >= t->nlev) continue;
            int viol = 0;
            for (int64_t jx = 2 * T->ix - 1; jx <= 2 * T->ix + 2 && !viol; ++jx)
                for (int64_t jy = 2 * T->iy - 1; jy <= 2 * T->iy + 2 && !viol; ++jy)
                    for (int64_t jz = 2 * T->iz - 1; jz <= 2 * T->iz + 2 && !viol; ++jz) {
                        int A = tree_find(t, a + 1, jx, jy, jz);
                        if (A >= 0 && !t->b[A].leaf) viol = 1;
                    }
            if (viol) {
                if (nforced == capf) {
                    capf = capf ? 2 * capf : 256;
                    uint64_t *nf = (uint64_t *)realloc(forced, (size_t)capf * sizeof(uint64_t));
                    if (!nf) { free(forced); return -1; }
                    forced = nf;
                }
                forced[nforced++] = cell_key(a, T->ix, T->iy, T->iz);
                added = 1;
            }
        }
        if (!added) { free(forced); return 0; }
        qsort(forced, (size_t)nforced, sizeof(uint64_t), cmp_u64);
    }
    free(forced);
    return -2;
}

static void tree_free(otree *t)
{
    for (int i = 0; i < t->nb; ++i) {
        free(t->b[i].proxy);
        free(t->b[i].Phi);
        free(t->b[i].local);
    }
    free(t->b);
    free(t->ord);
    memset(t, 0, sizeof(*t));
}

/* unit-box map of the union set (see dmk_oracle.h) */
static int points_init(opoints *P, const double *src, const double *rho, int64_t ns,
                       const double *tgt, int64_t nt)
{
    memset(P, 0, sizeof(*P));
    int same = (tgt == src && nt == ns);
    int64_t n = same ? ns : ns + nt;
    P->n = n;
    size_t nn = (size_t)(n > 0 ? n : 1);
    P->u = (double *)malloc(nn * 3 * sizeof(double));
    P->cell = (int64_t *)malloc(nn * 3 * sizeof(int64_t));
    P->q = (double *)malloc(nn * sizeof(double));
    P->is_src = (char *)malloc(nn);
    P->is_tgt = (char *)malloc(nn);
    P->out_index = (int64_t *)malloc(nn * sizeof(int64_t));
    if (!P->u || !P->cell || !P->q || !P->is_src || !P->is_tgt || !P->out_index) return -1;
    const double *xyz[2] = {src, tgt};
    double lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
    for (int64_t i = 0; i < n; ++i) {
        const double *x = (i < ns) ? &src[3 * i] : &tgt[3 * (i - ns)];
        for (int d = 0; d < 3; ++d) {
            if (x[d] < lo[d]) lo[d] = x[d];
            if (x[d] > hi[d]) hi[d] = x[d];
        }
    }
    (void)xyz;
    double S = 0.0;
    for (int d = 0; d < 3; ++d) if (n > 0 && hi[d] - lo[d] > S) S = hi[d] - lo[d];
    if (S == 0.0) S = 1.0;
    P->S = S;
    for (int64_t i = 0; i < n; ++i) {
        const double *x = (i < ns) ? &src[3 * i] : &tgt[3 * (i - ns)];
        for (int d = 0; d < 3; ++d) {
            volatile double diff = x[d] - lo[d];
            double u = diff / S;
            P->u[3 * i + d] = u;
            double f = floor(u * 2097152.0);
            int64_t c = (int64_t)f;
            if (c > 2097151) c = 2097151;
            if (c < 0) c = 0;
            P->cell[3 * i + d] = c;
        }
        if (same) {
            P->q[i] = rho[i];
            P->is_src[i] = 1;
            P->is_tgt[i] = 1;
            P->out_index[i] = i;
        } else if (i < ns) {
            P->q[i] = rho[i];
            P->is_src[i] = 1;
            P->is_tgt[i] = 0;
            P->out_index[i] = -1;
        } else {
            P->q[i] = 0.0;
            P->is_src[i] = 0;
            P->is_tgt[i] = 1;
            P->out_index[i] = i - ns;
        }
    }
    return 0;
}

static void points_free(opoints *P)
{
    free(P->u); free(P->cell); free(P->q); free(P->is_src); free(P->is_tgt); free(P->out_index);
    memset(P, 0, sizeof(*P));
}

static int tree_make(otree *t, const opoints *P, const oracle_params *prm)
{
    memset(t, 0, sizeof(*t));
    t->ord = (int64_t *)malloc((size_t)(P->n > 0 ? P->n : 1) * sizeof(int64_t));
    if (!t->ord) return -1;
    int rc = tree_build_balanced(t, P, prm);
    if (rc < 0) return rc;
    /* source / target counts, colleagues, flags */
    for (int i = 0; i < t->nb; ++i) {
        obox *b = &t->b[i];
        b->nsrc = b->ntgt = 0;
        for (int64_t k = b->start; k < b->start + b->count; ++k) {
            b->nsrc += P->is_src[t->ord[k]];
            b->ntgt += P->is_tgt[t->ord[k]];
        }
        b->ncol = 0;
        for (int dx = -1; dx <= 1; ++dx)
            for (int dy = -1; dy <= 1; ++dy)
                for (int dz = -1; dz <= 1; ++dz) {
                    int c = tree_find(t, b->level, b->ix + dx, b->iy + dy, b->iz + dz);
                    if (c >= 0) b->col[b->ncol++] = c;
                }
    }
    for (int i = 0; i < t->nb; ++i) t->b[i].fout = !t->b[i].leaf && t->b[i].nsrc > 0;
    for (int i = 0; i < t->nb; ++i) {
        obox *b = &t->b[i];
        b->fin = 0;
        if (b->ntgt == 0) continue;
        for (int k = 0; k < b->ncol; ++k) if (t->b[b->col[k]].fout) b->fin = 1;
    }
    return 0;
}

/* ====================================================================== */
/* 6. The DMK algorithm (Sec. 3.4)                                         */
/* ====================================================================== */

typedef struct {
    int p, nf, N1, n0, NW;
    double t[64];          /* Chebyshev nodes */
    double *Vinv;          /* [p][p], Vinv[n*p + i] */
    /* Step 1 operators, one dimension at a time */
    double *c2p[2];        /* [node i of parent][node k of child], child offset s = -1 / +1 */
    double *p2c[2];        /* [child coeff m][parent coeff n] = (V^{-1} E)[m][n] */
} ops_t;

/* 1-D anterpolation weights: a[i] = sum_n T_n(xi) Vinv[n][i] = U(xi, i) */
static void anterp_weights(const ops_t *o, double xi, double *a)
{
    int p = o->p;
    for (int i = 0; i < p; ++i) a[i] = 0.0;
    for (int n = 0; n < p; ++n) {
        double tn = cheb_t(n, xi);
        for (int i = 0; i < p; ++i) a[i] += tn * o->Vinv[n * p + i];
    }
}

static int ops_init(ops_t *o, int p, int nf, int n0)
{
    memset(o, 0, sizeof(*o));
    o->p = p; o->nf = nf; o->N1 = 2 * nf + 1; o->n0 = n0; o->NW = 2 * n0 + 1;
    cheb_nodes(p, o->t);
    double *V = (double *)malloc((size_t)p * p * sizeof(double));
    o->Vinv = (double *)malloc((size_t)p * p * sizeof(double));
    if (!V || !o->Vinv) return -1;
    /* V(i, j) = T_{j}(r_i) (0-based j) */
    for (int i = 0; i < p; ++i)
        for (int j = 0; j < p; ++j) V[i * p + j] = cheb_t(j, o->t[i]);
    if (mat_inverse(p, V, o->Vinv) != 0) { free(V); return -1; }
    free(V);
    for (int s = 0; s < 2; ++s) {
        double off = s ? 1.0 : -1.0;
        o->c2p[s] = (double *)malloc((size_t)p * p * sizeof(double));
        o->p2c[s] = (double *)malloc((size_t)p * p * sizeof(double));
        if (!o->c2p[s] || !o->p2c[s]) return -1;
        double a[64];
        /* T_c2p = U^T for the child's nodes seen in parent coordinates
         * (Lemma ctoplemma): child node k sits at (t_k + s) / 2 */
        for (int k = 0; k < p; ++k) {
            anterp_weights(o, 0.5 * (o->t[k] + off), a);
            for (int i = 0; i < p; ++i) o->c2p[s][i * p + k] = a[i];
        }
        /* T_p2c = V^{-1} E, E(k, n) = T_n((t_k + s) / 2) (Lemma ptoclemma) */
        for (int m = 0; m < p; ++m)
            for (int n = 0; n < p; ++n) {
                double acc = 0.0;
                for (int k = 0; k < p; ++k) acc += o->Vinv[m * p + k] * cheb_t(n, 0.5 * (o->t[k] + off));
                o->p2c[s][m * p + n] = acc;
            }
    }
    return 0;
}

static void ops_free(ops_t *o)
{
    free(o->Vinv);
    for (int s = 0; s < 2; ++s) { free(o->c2p[s]); free(o->p2c[s]); }
}

/* Apply a (nout x nin) complex matrix along one axis of a 3-D array. */
static void mode_apply_c(const cplx *M, int nout, int nin, const cplx *X, const int dims[3],
                         int axis, cplx *Y)
{
    int d0 = dims[0], d1 = dims[1], d2 = dims[2];
    int o0 = axis == 0 ? nout : d0, o1 = axis == 1 ? nout : d1, o2 = axis == 2 ? nout : d2;
    for (int a = 0; a < o0; ++a)
        for (int b = 0; b < o1; ++b)
            for (int c = 0; c < o2; ++c) {
                cplx acc = 0.0;
                for (int i = 0; i < nin; ++i) {
                    int xa = a, xb = b, xc = c, mo;
                    if (axis == 0) { xa = i; mo = a; } else if (axis == 1) { xb = i; mo = b; } else { xc = i; mo = c; }
                    acc += M[mo * nin + i] * X[((size_t)xa * d1 + xb) * d2 + xc];
                }
                Y[((size_t)a * o1 + b) * o2 + c] = acc;
            }
}

/* Y = (M (x) M (x) M) X for a real p^3 array and real (nout x nin) matrices
 * given per axis. */
static void tensor3_real(const double *Mx, const double *My, const double *Mz, int nout, int nin,
                         const double *X, double *Y, double *w1, double *w2)
{
    /* contract z, then y, then x */
    int n = nin, m = nout;
    for (int a = 0; a < n; ++a)
        for (int b = 0; b < n; ++b)
            for (int c = 0; c < m; ++c) {
                double acc = 0.0;
                for (int k = 0; k < n; ++k) acc += Mz[c * n + k] * X[(a * n + b) * n + k];
                w1[(a * n + b) * m + c] = acc;
            }
    for (int a = 0; a < n; ++a)
        for (int b = 0; b < m; ++b)
            for (int c = 0; c < m; ++c) {
                double acc = 0.0;
                for (int k = 0; k < n; ++k) acc += My[b * n + k] * w1[(a * n + k) * m + c];
                w2[(a * m + b) * m + c] = acc;
            }
    for (int a = 0; a < m; ++a)
        for (int b = 0; b < m; ++b)
            for (int c = 0; c < m; ++c) {
                double acc = 0.0;
                for (int k = 0; k < n; ++k) acc += Mx[a * n + k] * w2[(k * m + b) * m + c];
                Y[(a * m + b) * m + c] = acc;
            }
}

/* Proxy charges rho~ = U^T rho on a box's grid (Def. anterpdef, eq. proxynd). */
static void form_proxy(const ops_t *o, const opoints *P, const otree *t, const obox *b, double *proxy)
{
    int p = o->p;
    double R = level_R(b->level);
    double cx = (b->ix + 0.5) * R, cy = (b->iy + 0.5) * R, cz = (b->iz + 0.5) * R;
    double ax[64], ay[64], az[64];
    memset(proxy, 0, (size_t)p * p * p * sizeof(double));
    for (int64_t k = b->start; k < b->start + b->count; ++k) {
        int64_t pi = t->ord[k];
        if (!P->is_src[pi]) continue;
        double q = P->q[pi];
        anterp_weights(o, 2.0 * (P->u[3 * pi] - cx) / R, ax);
        anterp_weights(o, 2.0 * (P->u[3 * pi + 1] - cy) / R, ay);
        anterp_weights(o, 2.0 * (P->u[3 * pi + 2] - cz) / R, az);
        for (int i = 0; i < p; ++i)
            for (int j = 0; j < p; ++j) {
                double qij = q * ax[i] * ay[j];
                for (int l = 0; l < p; ++l) proxy[(i * p + j) * p + l] += qij * az[l];
            }
    }
}

/* Outgoing plane-wave expansion from proxy charges, eq. outgoingexpansion2:
 * Phi_m = sum_j exp(-i h k_m . (r_j - c_B)) rho~_j, h the spacing, nodes at
 * c_B + (R/2) t. */
static void prox2pw(const ops_t *o, double h, double R, int nmodes_half, const double *proxy, cplx *Phi)
{
    int p = o->p, N = 2 * nmodes_half + 1;
    cplx *E = (cplx *)malloc((size_t)N * p * sizeof(cplx));
    cplx *X = (cplx *)malloc((size_t)p * p * p * sizeof(cplx));
    cplx *Y1 = (cplx *)malloc((size_t)N * p * p * sizeof(cplx));
    cplx *Y2 = (cplx *)malloc((size_t)N * N * p * sizeof(cplx));
    for (int m = -nmodes_half; m <= nmodes_half; ++m)
        for (int j = 0; j < p; ++j) E[(m + nmodes_half) * p + j] = cexp(-I * h * m * 0.5 * R * o->t[j]);
    for (int i = 0; i < p * p * p; ++i) X[i] = proxy[i];
    int d0[3] = {p, p, p}, d1[3] = {N, p, p}, d2[3] = {N, N, p};
    mode_apply_c(E, N, p, X, d0, 0, Y1);
    mode_apply_c(E, N, p, Y1, d1, 1, Y2);
    mode_apply_c(E, N, p, Y2, d2, 2, Phi);
    free(E); free(X); free(Y1); free(Y2);
}

/* Local Chebyshev coefficients from an incoming expansion: values
 * sum_m exp(i h k_m . (r_n - c_B)) Psi_m on the grid (eq. incomingexpansion2),
 * real part, then V^{-1} per dimension (eq. localexpansion). */
static void pw2poly(const ops_t *o, double h, double R, int nmodes_half, const cplx *Psi, double *coef)
{
    int p = o->p, N = 2 * nmodes_half + 1;
    cplx *F = (cplx *)malloc((size_t)p * N * sizeof(cplx));
    cplx *Y1 = (cplx *)malloc((size_t)p * N * N * sizeof(cplx));
    cplx *Y2 = (cplx *)malloc((size_t)p * p * N * sizeof(cplx));
    cplx *Y3 = (cplx *)malloc((size_t)p * p * p * sizeof(cplx));
    double *vals = (double *)malloc((size_t)p * p * p * sizeof(double));
    double *w1 = (double *)malloc((size_t)p * p * p * sizeof(double));
    double *w2 = (double *)malloc((size_t)p * p * p * sizeof(double));
    for (int n = 0; n < p; ++n)
        for (int m = -nmodes_half; m <= nmodes_half; ++m)
            F[n * N + (m + nmodes_half)] = cexp(I * h * m * 0.5 * R * o->t[n]);
    int d0[3] = {N, N, N}, d1[3] = {p, N, N}, d2[3] = {p, p, N};
    mode_apply_c(F, p, N, Psi, d0, 0, Y1);
    mode_apply_c(F, p, N, Y1, d1, 1, Y2);
    mode_apply_c(F, p, N, Y2, d2, 2, Y3);
    for (int i = 0; i < p * p * p; ++i) vals[i] = creal(Y3[i]);
    tensor3_real(o->Vinv, o->Vinv, o->Vinv, p, p, vals, coef, w1, w2);
    free(F); free(Y1); free(Y2); free(Y3); free(vals); free(w1); free(w2);
}

/* Evaluate a local Chebyshev expansion at unit-box point u in box b. */
static double eval_local(const ops_t *o, const obox *b, const double *coef, const double *u)
{
    int p = o->p;
    double R = level_R(b->level);
    double tx[64], ty[64], tz[64];
    double xi[3];
    xi[0] = 2.0 * (u[0] - (b->ix + 0.5) * R) / R;
    xi[1] = 2.0 * (u[1] - (b->iy + 0.5) * R) / R;
    xi[2] = 2.0 * (u[2] - (b->iz + 0.5) * R) / R;
    for (int n = 0; n < p; ++n) {
        tx[n] = cheb_t(n, xi[0]);
        ty[n] = cheb_t(n, xi[1]);
        tz[n] = cheb_t(n, xi[2]);
    }
    double acc = 0.0;
    for (int a = 0; a < p; ++a)
        for (int bb = 0; bb < p; ++bb) {
            double s = 0.0;
            for (int c = 0; c < p; ++c) s += coef[(a * p + bb) * p + c] * tz[c];
            acc += tx[a] * ty[bb] * s;
        }
    return acc;
}

/* gradient (in unit-box coordinates) of the local expansion at u:
 * d/du_x sum coef[a][b][c] T_a(xi_x) T_b(xi_y) T_c(xi_z) = (2/R) sum coef T_a' T_b T_c, ... */
static void eval_local_grad(const ops_t *o, const obox *b, const double *coef, const double *u, double *g)
{
    int p = o->p;
    double R = level_R(b->level);
    double t[3][64], dt[3][64];
    double xi[3];
    xi[0] = 2.0 * (u[0] - (b->ix + 0.5) * R) / R;
    xi[1] = 2.0 * (u[1] - (b->iy + 0.5) * R) / R;
    xi[2] = 2.0 * (u[2] - (b->iz + 0.5) * R) / R;
    for (int d = 0; d < 3; ++d)
        for (int n = 0; n < p; ++n) {
            t[d][n] = cheb_t(n, xi[d]);
            dt[d][n] = cheb_dt(n, xi[d]);
        }
    double gx = 0.0, gy = 0.0, gz = 0.0;
    for (int a = 0; a < p; ++a)
        for (int bb = 0; bb < p; ++bb)
            for (int c = 0; c < p; ++c) {
                double v = coef[(a * p + bb) * p + c];
                gx += v * dt[0][a] * t[1][bb] * t[2][c];
                gy += v * t[0][a] * dt[1][bb] * t[2][c];
                gz += v * t[0][a] * t[1][bb] * dt[2][c];
            }
    g[0] = 2.0 * gx / R;
    g[1] = 2.0 * gy / R;
    g[2] = 2.0 * gz / R;
}

/* near-field list of a target leaf: source leaves whose Step-4 target set
 * (colleagues' subtrees and coarse neighbours) contains it */
typedef struct { int *s; int n, cap; } ilist;

static int ilist_push(ilist *L, int v)
{
    if (L->n == L->cap) {
        int nc = L->cap ? 2 * L->cap : 32;
        int *ns = (int *)realloc(L->s, (size_t)nc * sizeof(int));
        if (!ns) return -1;
        L->s = ns;
        L->cap = nc;
    }
    L->s[L->n++] = v;
    return 0;
}

static int add_subtree_leaves(const otree *t, int X, int S, ilist *lists)
{
    const obox *b = &t->b[X];
    if (b->leaf) return ilist_push(&lists[X], S);
    for (int c = 0; c < 8; ++c)
        if (b->child[c] >= 0 && add_subtree_leaves(t, b->child[c], S, lists) < 0) return -1;
    return 0;
}

static int run_dmk(const split_t *sp, const opoints *P, otree *t, double *ufar, double *unear,
                   double *gfar, double *gnear)
{
    const oracle_params *prm = &sp->prm;
    ops_t o;
    if (ops_init(&o, prm->p, prm->nf, prm->n0) != 0) { ops_free(&o); return -1; }
    int p = o.p, p3 = p * p * p;
    int N1 = o.N1, NF = N1 * N1 * N1;
    int nf = o.nf;
    int Lmax = t->nlev - 1;
    int rc = 0;

    for (int64_t i = 0; i < P->n; ++i) { ufar[i] = 0.0; unear[i] = 0.0; }

    /* ---- Step 2: upward pass ---------------------------------------- */
    /* proxy charges on every leaf with sources, from the sources */
#pragma omp parallel for schedule(dynamic, 1)
    for (int i = 0; i < t->nb; ++i) {
        obox *b = &t->b[i];
        if (!b->leaf || b->nsrc == 0) continue;
        b->proxy = (double *)malloc((size_t)p3 * sizeof(double));
        form_proxy(&o, P, t, b, b->proxy);
    }
    /* merge children into parents, finest level first (T_c2p) */
    for (int l = Lmax - 1; l >= 0; --l) {
        int s = t->lev_start[l], e = s + t->lev_count[l];
#pragma omp parallel for schedule(dynamic, 1)
        for (int i = s; i < e; ++i) {
            obox *b = &t->b[i];
            if (b->leaf || b->nsrc == 0) continue;
            b->proxy = (double *)calloc((size_t)p3, sizeof(double));
            double *tmp = (double *)malloc((size_t)p3 * sizeof(double));
            double *w1 = (double *)malloc((size_t)p3 * sizeof(double));
            double *w2 = (double *)malloc((size_t)p3 * sizeof(double));
            for (int c = 0; c < 8; ++c) {
                int ci = b->child[c];
                if (ci < 0 || !t->b[ci].proxy) continue;
                tensor3_real(o.c2p[c & 1], o.c2p[(c >> 1) & 1], o.c2p[(c >> 2) & 1], p, p,
                             t->b[ci].proxy, tmp, w1, w2);
                for (int k = 0; k < p3; ++k) b->proxy[k] += tmp[k];
            }
            free(tmp); free(w1); free(w2);
        }
    }

    /* weights w_{l,m} = (h_l / 2 pi)^3 Dhat_l(h_l |m|) */
    cplx *wl = (cplx *)malloc((size_t)NF * sizeof(cplx));

    /* ---- Step 3: downward pass --------------------------------------- */
    for (int l = 0; l <= Lmax; ++l) {
        int s = t->lev_start[l], e = s + t->lev_count[l];
        double R = level_R(l), h = split_h(l);
        double wscale = pow(h / (2.0 * M_PI), 3);
        for (int mx = -nf; mx <= nf; ++mx)
            for (int my = -nf; my <= nf; ++my)
                for (int mz = -nf; mz <= nf; ++mz) {
                    double km = h * sqrt((double)(mx * mx + my * my + mz * mz));
                    wl[((mx + nf) * N1 + (my + nf)) * N1 + (mz + nf)] = wscale * split_Dhat(sp, l, km);
                }
        /* outgoing expansions */
#pragma omp parallel for schedule(dynamic, 1)
        for (int i = s; i < e; ++i) {
            obox *b = &t->b[i];
            if (!b->fout) continue;
            b->Phi = (cplx *)malloc((size_t)NF * sizeof(cplx));
            prox2pw(&o, h, R, nf, b->proxy, b->Phi);
        }
        /* incoming expansions and local expansions */
#pragma omp parallel for schedule(dynamic, 1)
        for (int i = s; i < e; ++i) {
            obox *b = &t->b[i];
            if (!b->fin) continue;
            cplx *Psi = (cplx *)calloc((size_t)NF, sizeof(cplx));
            double *coef = (double *)malloc((size_t)p3 * sizeof(double));
            double cB[3] = {(b->ix + 0.5) * R, (b->iy + 0.5) * R, (b->iz + 0.5) * R};
            for (int k = 0; k < b->ncol; ++k) {
                const obox *S = &t->b[b->col[k]];
                if (!S->fout) continue;
                double d[3] = {cB[0] - (S->ix + 0.5) * R, cB[1] - (S->iy + 0.5) * R, cB[2] - (S->iz + 0.5) * R};
                for (int mx = -nf; mx <= nf; ++mx)
                    for (int my = -nf; my <= nf; ++my)
                        for (int mz = -nf; mz <= nf; ++mz) {
                            int idx = ((mx + nf) * N1 + (my + nf)) * N1 + (mz + nf);
                            double ph = h * (mx * d[0] + my * d[1] + mz * d[2]);
                            Psi[idx] += wl[idx] * cexp(I * ph) * S->Phi[idx];
                        }
            }
            pw2poly(&o, h, R, nf, Psi, coef);
            if (!b->local) b->local = (double *)calloc((size_t)p3, sizeof(double));
            for (int k = 0; k < p3; ++k) b->local[k] += coef[k];
            b->has_local = 1;
            free(Psi); free(coef);
        }
        /* the windowed kernel W_0 over the whole unit box, at the root */
        if (l == 0) {
            obox *b = &t->b[0];
            int n0 = o.n0, NW = o.NW;
            size_t NWF = (size_t)NW * NW * NW;
            double hW = sp->hW;
            if (!b->local) b->local = (double *)calloc((size_t)p3, sizeof(double));
            if (b->proxy) {
                cplx *PhiW = (cplx *)malloc(NWF * sizeof(cplx));
                double *coef = (double *)malloc((size_t)p3 * sizeof(double));
                prox2pw(&o, hW, 1.0, n0, b->proxy, PhiW);
                double ws = pow(hW / (2.0 * M_PI), 3);
                for (int mx = -n0; mx <= n0; ++mx)
                    for (int my = -n0; my <= n0; ++my)
                        for (int mz = -n0; mz <= n0; ++mz) {
                            size_t idx = ((size_t)(mx + n0) * NW + (my + n0)) * NW + (mz + n0);
                            double km = hW * sqrt((double)(mx * mx + my * my + mz * mz));
                            PhiW[idx] *= ws * split_What(sp, km);
                        }
                pw2poly(&o, hW, 1.0, n0, PhiW, coef);
                for (int k = 0; k < p3; ++k) b->local[k] += coef[k];
                free(PhiW); free(coef);
            }
            b->has_local = 1;
        }
        /* split local expansions to children (T_p2c) */
#pragma omp parallel for schedule(dynamic, 1)
        for (int i = s; i < e; ++i) {
            obox *b = &t->b[i];
            if (b->leaf || !b->has_local) continue;
            double *w1 = (double *)malloc((size_t)p3 * sizeof(double));
            double *w2 = (double *)malloc((size_t)p3 * sizeof(double));
            double *tmp = (double *)malloc((size_t)p3 * sizeof(double));
            for (int c = 0; c < 8; ++c) {
                int ci = b->child[c];
                if (ci < 0) continue;
                obox *ch = &t->b[ci];
                tensor3_real(o.p2c[c & 1], o.p2c[(c >> 1) & 1], o.p2c[(c >> 2) & 1], p, p, b->local, tmp, w1, w2);
                if (!ch->local) ch->local = (double *)calloc((size_t)p3, sizeof(double));
                for (int k = 0; k < p3; ++k) ch->local[k] += tmp[k];
                ch->has_local = 1;
            }
            free(w1); free(w2); free(tmp);
        }
        /* evaluate local expansions at the targets of the leaves */
#pragma omp parallel for schedule(dynamic, 1)
        for (int i = s; i < e; ++i) {
            obox *b = &t->b[i];
            if (!b->leaf || !b->has_local) continue;
            for (int64_t k = b->start; k < b->start + b->count; ++k) {
                int64_t pi = t->ord[k];
                if (!P->is_tgt[pi]) continue;
                ufar[pi] += eval_local(&o, b, b->local, &P->u[3 * pi]);
                if (gfar) {
                    double g[3];
                    eval_local_grad(&o, b, b->local, &P->u[3 * pi], g);
                    for (int d = 0; d < 3; ++d) gfar[3 * pi + d] += g[d];
                }
            }
        }
        /* expansions of this level are no longer needed */
        for (int i = s; i < e; ++i) {
            free(t->b[i].Phi);
            t->b[i].Phi = NULL;
        }
    }
    free(wl);

    /* ---- Step 4: direct interactions with the residual kernels -------- */
    ilist *lists = (ilist *)calloc((size_t)t->nb, sizeof(ilist));
    for (int S = 0; S < t->nb && rc == 0; ++S) {
        const obox *b = &t->b[S];
        if (!b->leaf || b->nsrc == 0) continue;
        /* colleagues (whole subtrees) */
        for (int k = 0; k < b->ncol; ++k)
            if (add_subtree_leaves(t, b->col[k], S, lists) < 0) rc = -1;
        /* coarse neighbours: leaves one level up sharing a boundary point */
        if (b->level > 0) {
            int lp = b->level - 1;
            int64_t px = b->ix >> 1, py = b->iy >> 1, pz = b->iz >> 1;
            for (int64_t qx = px - 1; qx <= px + 1; ++qx)
                for (int64_t qy = py - 1; qy <= py + 1; ++qy)
                    for (int64_t qz = pz - 1; qz <= pz + 1; ++qz) {
                        int X = tree_find(t, lp, qx, qy, qz);
                        if (X < 0 || !t->b[X].leaf) continue;
                        int adj = 2 * qx <= b->ix + 1 && 2 * qx + 2 >= b->ix &&
                                  2 * qy <= b->iy + 1 && 2 * qy + 2 >= b->iy &&
                                  2 * qz <= b->iz + 1 && 2 * qz + 2 >= b->iz;
                        if (adj && ilist_push(&lists[X], S) < 0) rc = -1;
                    }
        }
    }
    if (rc == 0) {
#pragma omp parallel for schedule(dynamic, 1)
        for (int T = 0; T < t->nb; ++T) {
            const obox *bt = &t->b[T];
            if (!bt->leaf || bt->ntgt == 0) continue;
            for (int64_t k = bt->start; k < bt->start + bt->count; ++k) {
                int64_t ti = t->ord[k];
                if (!P->is_tgt[ti]) continue;
                const double *x = &P->u[3 * ti];
                double acc = 0.0, gacc[3] = {0.0, 0.0, 0.0};
                for (int li = 0; li < lists[T].n; ++li) {
                    const obox *bs = &t->b[lists[T].s[li]];
                    double Rb = level_R(bs->level);
                    for (int64_t kk = bs->start; kk < bs->start + bs->count; ++kk) {
                        int64_t sj = t->ord[kk];
                        if (!P->is_src[sj]) continue;
                        const double *y = &P->u[3 * sj];
                        double dx = x[0] - y[0], dy = x[1] - y[1], dz = x[2] - y[2];
                        double r = sqrt(dx * dx + dy * dy + dz * dz);
                        if (r == 0.0 || r >= Rb) continue;
                        acc += P->q[sj] * split_R(sp, bs->level, r);
                        if (gnear) {
                            /* grad_x R(|x - y|) = R'(r) (x - y) / r */
                            double f = P->q[sj] * split_dR(sp, bs->level, r) / r;
                            gacc[0] += f * dx;
                            gacc[1] += f * dy;
                            gacc[2] += f * dz;
                        }
                    }
                }
                unear[ti] += acc;
                if (gnear)
                    for (int d = 0; d < 3; ++d) gnear[3 * ti + d] += gacc[d];
            }
        }
    }
    for (int i = 0; i < t->nb; ++i) free(lists[i].s);
    free(lists);

    /* ---- Step 5: self-interaction corrections ------------------------- */
    /* a target coincident with a source received rho S_L(0) through the far
     * field; remove it (the sum excludes coincident pairs) */
#pragma omp parallel for schedule(dynamic, 1)
    for (int T = 0; T < t->nb; ++T) {
        const obox *b = &t->b[T];
        if (!b->leaf || b->ntgt == 0 || b->nsrc == 0) continue;
        double S0 = split_S(sp, b->level, 0.0);
        for (int64_t k = b->start; k < b->start + b->count; ++k) {
            int64_t ti = t->ord[k];
            if (!P->is_tgt[ti]) continue;
            for (int64_t kk = b->start; kk < b->start + b->count; ++kk) {
                int64_t sj = t->ord[kk];
                if (!P->is_src[sj]) continue;
                if (P->u[3 * ti] == P->u[3 * sj] && P->u[3 * ti + 1] == P->u[3 * sj + 1] &&
                    P->u[3 * ti + 2] == P->u[3 * sj + 2])
                    unear[ti] -= P->q[sj] * S0;
            }
        }
    }
    ops_free(&o);
    return rc;
}

int oracle_dmk(const oracle_params *prm_in,
               const double *src, const double *rho, int64_t ns,
               const double *tgt, int64_t nt,
               double *pot, double *pot_far, double *pot_near)
{
    if (ns < 0 || nt < 0) return -1;
    if (nt == 0) return 0;
    split_t sp;
    if (split_init(&sp, prm_in) != 0) return -1;
#ifdef _OPENMP
    if (sp.prm.nthreads > 0) omp_set_num_threads(sp.prm.nthreads);
#endif
    opoints P;
    otree t;
    memset(&t, 0, sizeof(t));
    int rc = points_init(&P, src, rho, ns, tgt, nt);
    /* exp(-lambda |x - y|) = exp(-(lambda S) |u - v|) in the unit box */
    if (rc == 0) rc = split_set_lambda(&sp, sp.prm.lambda * P.S);
    if (rc == 0) rc = tree_make(&t, &P, &sp.prm);
    double *ufar = NULL, *unear = NULL;
    if (rc == 0) {
        ufar = (double *)malloc((size_t)P.n * sizeof(double));
        unear = (double *)malloc((size_t)P.n * sizeof(double));
        if (!ufar || !unear) rc = -1;
    }
    if (rc == 0) rc = run_dmk(&sp, &P, &t, ufar, unear, NULL, NULL);
    if (rc == 0) {
        for (int64_t i = 0; i < P.n; ++i) {
            int64_t o = P.out_index[i];
            if (o < 0) continue;
            pot[o] = (ufar[i] + unear[i]) / P.S;
            if (pot_far) pot_far[o] = ufar[i] / P.S;
            if (pot_near) pot_near[o] = unear[i] / P.S;
        }
    }
    free(ufar);
    free(unear);
    tree_free(&t);
    points_free(&P);
    split_free(&sp);
    return rc;
}

int oracle_dmk_grad(const oracle_params *prm_in,
                    const double *src, const double *rho, int64_t ns,
                    const double *tgt, int64_t nt,
                    double *pot, double *grad, double *grad_far, double *grad_near)
{
    if (ns < 0 || nt < 0) return -1;
    if (nt == 0) return 0;
    if (prm_in->lambda != 0.0) return -1; /* gradients: Laplace kernel only */
    split_t sp;
    if (split_init(&sp, prm_in) != 0) return -1;
#ifdef _OPENMP
    if (sp.prm.nthreads > 0) omp_set_num_threads(sp.prm.nthreads);
#endif
    opoints P;
    otree t;
    memset(&t, 0, sizeof(t));
    int rc = points_init(&P, src, rho, ns, tgt, nt);
    if (rc == 0) rc = tree_make(&t, &P, &sp.prm);
    double *ufar = NULL, *unear = NULL, *gf = NULL, *gn = NULL;
    if (rc == 0) {
        ufar = (double *)calloc((size_t)P.n, sizeof(double));
        unear = (double *)calloc((size_t)P.n, sizeof(double));
        gf = (double *)calloc((size_t)P.n * 3, sizeof(double));
        gn = (double *)calloc((size_t)P.n * 3, sizeof(double));
        if (!ufar || !unear || !gf || !gn) rc = -1;
    }
    if (rc == 0) rc = run_dmk(&sp, &P, &t, ufar, unear, gf, gn);
    if (rc == 0) {
        /* unit-box potentials scale by 1/S, their gradients by 1/S^2 */
        const double s2 = P.S * P.S;
        for (int64_t i = 0; i < P.n; ++i) {
            int64_t o = P.out_index[i];
            if (o < 0) continue;
            if (pot) pot[o] = (ufar[i] + unear[i]) / P.S;
            for (int d = 0; d < 3; ++d) {
                grad[3 * o + d] = (gf[3 * i + d] + gn[3 * i + d]) / s2;
                if (grad_far) grad_far[3 * o + d] = gf[3 * i + d] / s2;
                if (grad_near) grad_near[3 * o + d] = gn[3 * i + d] / s2;
            }
        }
    }
    free(ufar);
    free(unear);
    free(gf);
    free(gn);
    tree_free(&t);
    points_free(&P);
    split_free(&sp);
    return rc;
}

int64_t oracle_tree(const oracle_params *prm_in,
                    const double *src, int64_t ns, const double *tgt, int64_t nt,
                    int32_t *leaf_level, int64_t *leaf_cell,
                    int32_t *box_level, int64_t *box_cell, int32_t *box_leaf,
                    int64_t max_boxes)
{
    oracle_params prm = *prm_in;
    oracle_default_params(&prm);
    opoints P;
    otree t;
    memset(&t, 0, sizeof(t));
    double *dummy = (double *)calloc((size_t)(ns > 0 ? ns : 1), sizeof(double));
    int rc = points_init(&P, src, dummy, ns, tgt, nt);
    if (rc == 0) rc = tree_make(&t, &P, &prm);
    int64_t nb = rc == 0 ? t.nb : rc;
    if (rc == 0) {
        for (int i = 0; i < t.nb; ++i) {
            const obox *b = &t.b[i];
            if (b->leaf)
                for (int64_t k = b->start; k < b->start + b->count; ++k) {
                    int64_t pi = t.ord[k];
                    leaf_level[pi] = b->level;
                    leaf_cell[pi] = (int64_t)morton3(b->ix, b->iy, b->iz, b->level);
                }
            if (box_level && i < max_boxes) {
                box_level[i] = b->level;
                box_cell[i] = (int64_t)morton3(b->ix, b->iy, b->iz, b->level);
                box_leaf[i] = b->leaf;
            }
        }
    }
    tree_free(&t);
    points_free(&P);
    free(dummy);
    return nb;
}

/* ---- pin-test entry points -------------------------------------------- */

void oracle_pswf(double c, const double *x, int64_t n, double *out)
{
    pswf_t *s = (pswf_t *)malloc(sizeof(pswf_t));
    pswf_init(s, c);
    for (int64_t i = 0; i < n; ++i) out[i] = pswf_eval(s, x[i]);
    free(s);
}

void oracle_pswf_constants(double c, double *lambda0, double *c0, double *c2, double *chi0)
{
    pswf_t *s = (pswf_t *)malloc(sizeof(pswf_t));
    pswf_init(s, c);
    *lambda0 = s->lambda0;
    *c0 = s->c0;
    *c2 = s->c2;
    *chi0 = s->chi0;
    free(s);
}

void oracle_kernel(const oracle_params *prm, int what, int level,
                   const double *r, int64_t n, double *out)
{
    split_t sp;
    if (split_init(&sp, prm) != 0) return;
    if (split_set_lambda(&sp, prm->lambda) != 0) { split_free(&sp); return; }
    for (int64_t i = 0; i < n; ++i) {
        double x = r[i];
        switch (what) {
        case 0: out[i] = split_S(&sp, level, x); break;
        case 1: out[i] = split_R(&sp, level, x); break;
        case 2: out[i] = split_S(&sp, level + 1, x) - split_S(&sp, level, x); break;
        case 3: out[i] = split_Dhat(&sp, level, x); break;
        case 4: out[i] = split_What(&sp, x); break;
        default: out[i] = NAN;
        }
    }
    split_free(&sp);
}

double oracle_h(const oracle_params *prm, int level) { (void)prm; return split_h(level); }

double oracle_hW(const oracle_params *prm)
{
    split_t sp;
    if (split_init(&sp, prm) != 0) return NAN;
    double h = sp.hW;
    split_free(&sp);
    return h;
}

/* ====================================================================== */
/* 7. The 2D Laplace kernel log r (Sec. 3.7 at lambda = 0, in the plane)   */
/* ====================================================================== */
/*
 * u_i = sum_{j : y_j != x_i} rho_j log |x_i - y_j| for points in the plane.
 *
 * In two dimensions the transform of log r is -2 pi / k^2 (a finite part;
 * the delta term it leaves undetermined drops out of every piece below,
 * since each piece carries a factor that vanishes at k = 0).  The splitting
 * of Sec. 3.7 (eq. yukawaPSWFkernels at lambda = 0, psi(0) = 1) gives
 *   Dhat_l(k) = -2 pi (psi(k R_{l+1} / c) - psi(k R_l / c)) / k^2,
 *     Dhat_l(0) = -pi (c_2 / c_0) (R_l^2 - R_{l+1}^2),
 *   Rhat_L(k) = -2 pi (1 - psi(k R_L / c)) / k^2,
 * and the radial inverse transform of Rhat_L is the residual kernel
 *   R_L(r) = F(r / R_L),  F(rho) = -int_0^inf (1 - psi(k / c)) J_0(k rho) / k dk.
 * With int_0^inf (J_0(t) - [t < 1]) / t dt = log 2 - gamma (Euler's constant)
 * the tail of the slowly decaying part is summed in closed form:
 *   F(rho) = log(rho K / 2) + gamma - int_0^K (1 - psi(k / c) J_0(k rho)) / k dk,
 * exact up to the part of psi beyond k = K, taken as K = 4 c (psi(x) is below
 * psi(1) / (c x) there).  The integrand is smooth (O(k) at 0) and is summed
 * with Gauss-Legendre panels.  F(rho) - log rho is smooth, so the mollified
 * kernel log r - R_L(r) has the finite value at r = 0
 *   S_L(0) = log R_L - log(K / 2) - gamma + int_0^K (1 - psi(k / c)) / k dk,
 * which a coincident source adds through the far field (Step 5 removes it).
 * The windowed root kernel is the kernel truncated at R_t = 1 + sqrt 2 (the
 * diameter of the unit square plus the mollifier's radius R_0 = 1), times
 * the mollifier:
 *   What_0(k) = psi(k / c) 2 pi (R_t log R_t J_1(k R_t) / k - (1 - J_0(k R_t)) / k^2),
 *   What_0(0) = pi R_t^2 (log R_t - 1/2),
 * sampled with spacing h_W = 2 pi / (2 + R_t) (separations are at most 1 per
 * coordinate).  The difference kernels use the spacing h_l = 2 pi / (3 R_l)
 * of the 3D pass and weights (h / 2 pi)^2.  The Table 1 parameters (c, p,
 * nf) carry over: the transforms decay through psi in the same way, and the
 * 1/k^2 factor is the same as for 1/r in 3D.
 * The unit-box map (the 3D one restricted to two coordinates) turns
 * log |x - y| into log S + log |u - v|: the potential in input units adds
 * log S times the charge of the sources not coincident with the target.
 * The Gaussian splitting (Sec. 3.2 in the plane) serves as a cross-check:
 * with sigma_l = R_l / delta the same transforms with exp(-k^2 sigma^2 / 4) in
 * place of psi give the residual -E_1(r^2 / sigma_l^2) / 2 and the self value
 * log sigma_l - gamma / 2 in closed form.
 */

#define L2_PANELS 10
#define L2_NODES 20
#define L2_NQ (L2_PANELS * L2_NODES)
#define L2_EULER_GAMMA 0.57721566490153286061

typedef struct {
    oracle_params prm;
    pswf_t *pswf;
    double Rt, hW, K;
    double qk[L2_NQ], qw[L2_NQ], qpsi[L2_NQ]; /* nodes, weights / k, psi(k / c) */
    double G0;                                /* F(rho) - log rho at rho = 0 */
} split2_t;

/* Exponential integral E_1(x), x > 0: the power series
 * -gamma - log x - sum_k (-x)^k / (k k!) for x <= 1, and beyond it the
 * continued fraction E_1(x) = e^{-x} / (x + 1 - 1 / (x + 3 - 4 / (x + 5 - ...)))
 * by the modified Lentz method (Abramowitz & Stegun 5.1.11 and 5.1.22). */
static double expint_e1(double x)
{
    if (x <= 1.0) {
        double sum = 0.0, term = 1.0;
        for (int k = 1; k < 60; ++k) {
            term *= -x / k; /* (-x)^k / k! */
            double add = -term / k;
            sum += add;
            if (fabs(add) < 1e-18 * fabs(sum)) break;
        }
        return -L2_EULER_GAMMA - log(x) + sum;
    }
    double b = x + 1.0, c = 1e300, d = 1.0 / b, h = d;
    for (int i = 1; i < 500; ++i) {
        double an = -(double)i * i;
        b += 2.0;
        d = 1.0 / (an * d + b);
        c = b + an / c;
        double del = c * d;
        h *= del;
        if (fabs(del - 1.0) < 1e-16) break;
    }
    return h * exp(-x);
}

static int split2_init(split2_t *sp, const oracle_params *in)
{
    memset(sp, 0, sizeof(*sp));
    sp->prm = *in;
    if (sp->prm.splitting == ORACLE_GAUSSIAN) {
        /* the cross-check splitting, sigma_l = R_l / delta: Dhat_l, the window
         * and the residual -E_1(r^2 / sigma_L^2) / 2 in closed form */
        oracle_params tmp = sp->prm;
        tmp.n0 = 1;
        oracle_default_params(&tmp);
        double sg = 1.0 / tmp.delta;
        sp->Rt = sqrt(2.0) + tmp.gauss_b * sg;
        sp->hW = 2.0 * M_PI / (2.0 + sp->Rt);
        if (sp->prm.n0 <= 0) sp->prm.n0 = (int)ceil(2.0 * sqrt(log(100.0 / tmp.eps)) / sg / sp->hW);
        tmp.n0 = sp->prm.n0;
        sp->prm = tmp;
        return 0;
    }
    if (sp->prm.splitting != ORACLE_PSWF) return -1;
    sp->Rt = 1.0 + sqrt(2.0);
    sp->hW = 2.0 * M_PI / (2.0 + sp->Rt);
    /* the 3D defaults, with the root modes for the 2D window */
    oracle_params tmp = sp->prm;
    tmp.n0 = 1;
    oracle_default_params(&tmp);
    if (sp->prm.n0 <= 0) sp->prm.n0 = (int)ceil(tmp.c / sp->hW) + 1;
    tmp.n0 = sp->prm.n0;
    sp->prm = tmp;
    sp->pswf = (pswf_t *)malloc(sizeof(pswf_t));
    if (!sp->pswf) return -1;
    pswf_init(sp->pswf, sp->prm.c);
    sp->K = 4.0 * sp->prm.c;
    double xg[L2_NODES], wg[L2_NODES];
    gauss_legendre(L2_NODES, xg, wg);
    double acc = 0.0, pw = sp->K / L2_PANELS;
    for (int q = 0, j = 0; q < L2_PANELS; ++q)
        for (int i = 0; i < L2_NODES; ++i, ++j) {
            double k = pw * (q + 0.5 * (xg[i] + 1.0));
            sp->qk[j] = k;
            sp->qw[j] = 0.5 * pw * wg[i] / k;
            sp->qpsi[j] = pswf_eval(sp->pswf, k / sp->prm.c);
            acc += sp->qw[j] * (1.0 - sp->qpsi[j]);
        }
    sp->G0 = log(0.5 * sp->K) + L2_EULER_GAMMA - acc;
    return 0;
}

static void split2_free(split2_t *sp)
{
    free(sp->pswf);
    sp->pswf = NULL;
}

/* residual kernel R_l(r) = F(r / R_l), r > 0; Gaussian: -E_1(r^2 / sigma_l^2) / 2 */
static double split2_R(const split2_t *sp, int l, double r)
{
    if (sp->prm.splitting == ORACLE_GAUSSIAN) {
        double sg = level_R(l) / sp->prm.delta;
        return -0.5 * expint_e1(r * r / (sg * sg));
    }
    double rho = r / level_R(l), acc = 0.0;
    for (int j = 0; j < L2_NQ; ++j) acc += sp->qw[j] * (1.0 - sp->qpsi[j] * j0(sp->qk[j] * rho));
    return log(rho * 0.5 * sp->K) + L2_EULER_GAMMA - acc;
}

/* mollified kernel at r = 0: lim (log r - R_l(r)); Gaussian: log sigma_l - gamma / 2 */
static double split2_S0(const split2_t *sp, int l)
{
    if (sp->prm.splitting == ORACLE_GAUSSIAN) return log(level_R(l) / sp->prm.delta) - 0.5 * L2_EULER_GAMMA;
    return log(level_R(l)) - sp->G0;
}

static double split2_Dhat(const split2_t *sp, int l, double k)
{
    double R = level_R(l), R1 = level_R(l + 1);
    if (sp->prm.splitting == ORACLE_GAUSSIAN) {
        double s0 = R / sp->prm.delta, s1 = R1 / sp->prm.delta;
        if (k == 0.0) return -0.5 * M_PI * (s0 * s0 - s1 * s1);
        return -2.0 * M_PI * (exp(-k * k * s1 * s1 / 4.0) - exp(-k * k * s0 * s0 / 4.0)) / (k * k);
    }
    const pswf_t *s = sp->pswf;
    if (k == 0.0) return -M_PI * s->c2 / s->c0 * (R * R - R1 * R1);
    return -2.0 * M_PI * pswf_diff(s, k * R1 / s->c, k * R / s->c) / (k * k);
}

static double split2_What(const split2_t *sp, double k)
{
    double Rt = sp->Rt, win;
    if (sp->prm.splitting == ORACLE_GAUSSIAN) {
        double sg = 1.0 / sp->prm.delta;
        win = exp(-k * k * sg * sg / 4.0);
    } else {
        win = pswf_eval(sp->pswf, k / sp->pswf->c);
    }
    if (k == 0.0) return M_PI * Rt * Rt * (log(Rt) - 0.5) * win;
    return 2.0 * M_PI * (Rt * log(Rt) * j1(k * Rt) / k - (1.0 - j0(k * Rt)) / (k * k)) * win;
}

void oracle_direct_log2d(const double *src, const double *rho, int64_t ns,
                         const double *tgt, int64_t nt, double *pot, int nthreads)
{
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#else
    (void)nthreads;
#endif
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < nt; ++i) {
        double sum = 0.0, comp = 0.0;
        for (int64_t j = 0; j < ns; ++j) {
            double dx = tgt[2 * i] - src[2 * j], dy = tgt[2 * i + 1] - src[2 * j + 1];
            if (dx == 0.0 && dy == 0.0) continue;
            double v = rho[j] * 0.5 * log(dx * dx + dy * dy);
            double t = sum + v; /* Neumaier */
            if (fabs(sum) >= fabs(v)) comp += (sum - t) + v; else comp += (v - t) + sum;
            sum = t;
        }
        pot[i] = sum + comp;
    }
}

/* ---- quad-tree (the 3D rules of Sec. 3.2 Step 0 in two dimensions) ---- */

typedef struct {
    int level;
    int64_t ix, iy;
    int parent;
    int child[4];
    int64_t start, count;
    int leaf;
    int64_t nsrc, ntgt;
    int col[9];
    int ncol;
    int fout, fin, has_local;
    double *proxy;
    cplx *Phi;
    double *local;
} obox2;

typedef struct {
    int64_t n;
    double *u;          /* unit-box coordinates [n][2] */
    int64_t *cell;      /* finest (level 21) cell [n][2] */
    double *q;
    char *is_src, *is_tgt;
    int64_t *out_index;
    double S;
} opoints2;

typedef struct {
    obox2 *b;
    int nb, cap;
    int64_t *ord;
    int lev_start[23], lev_count[23];
    int nlev;
} otree2;

static uint64_t morton2(int64_t ix, int64_t iy, int level)
{
    uint64_t m = 0;
    for (int b = 0; b < level; ++b) {
        m |= (uint64_t)((ix >> b) & 1) << (2 * b);
        m |= (uint64_t)((iy >> b) & 1) << (2 * b + 1);
    }
    return m;
}

static uint64_t cell_key2(int level, int64_t ix, int64_t iy)
{
    return morton2(ix, iy, level) | ((uint64_t)1 << (2 * level));
}

static int tree2_push(otree2 *t, const obox2 *b)
{
    if (t->nb == t->cap) {
        int nc = t->cap ? 2 * t->cap : 1024;
        obox2 *nbp = (obox2 *)realloc(t->b, (size_t)nc * sizeof(obox2));
        if (!nbp) return -1;
        t->b = nbp;
        t->cap = nc;
    }
    t->b[t->nb++] = *b;
    return t->nb - 1;
}

static int tree2_find(const otree2 *t, int level, int64_t ix, int64_t iy)
{
    if (level >= t->nlev) return -1;
    int64_t lim = (int64_t)1 << level;
    if (ix < 0 || iy < 0 || ix >= lim || iy >= lim) return -1;
    uint64_t key = morton2(ix, iy, level);
    int lo = t->lev_start[level], hi = lo + t->lev_count[level] - 1;
    while (lo <= hi) {
        int mid = (lo + hi) / 2;
        uint64_t mk = morton2(t->b[mid].ix, t->b[mid].iy, level);
        if (mk == key) return mid;
        if (mk < key) lo = mid + 1; else hi = mid - 1;
    }
    return -1;
}

static int tree2_build(otree2 *t, const opoints2 *P, const oracle_params *prm,
                       const uint64_t *forced, int nforced)
{
    t->nb = 0;
    for (int64_t i = 0; i < P->n; ++i) t->ord[i] = i;
    int64_t *tmp = (int64_t *)malloc((size_t)(P->n > 0 ? P->n : 1) * sizeof(int64_t));
    if (!tmp) return -1;
    obox2 root;
    memset(&root, 0, sizeof(root));
    root.parent = -1;
    for (int c = 0; c < 4; ++c) root.child[c] = -1;
    root.count = P->n;
    if (tree2_push(t, &root) < 0) { free(tmp); return -1; }
    t->nlev = 1;
    t->lev_start[0] = 0;
    t->lev_count[0] = 1;
    for (int l = 0; l < prm->max_level; ++l) {
        int s = t->lev_start[l], e = s + t->lev_count[l];
        int next_start = t->nb;
        for (int bi = s; bi < e; ++bi) {
            obox2 *b = &t->b[bi];
            int same_cell = 1;
            if (b->count > prm->leaf_cap) {
                int64_t p0 = t->ord[b->start];
                for (int64_t k = b->start + 1; k < b->start + b->count && same_cell; ++k) {
                    int64_t pk = t->ord[k];
                    if (P->cell[2 * pk] != P->cell[2 * p0] || P->cell[2 * pk + 1] != P->cell[2 * p0 + 1])
                        same_cell = 0;
                }
            }
            int split = (b->count > prm->leaf_cap && !same_cell) ||
                        key_in(forced, nforced, cell_key2(l, b->ix, b->iy));
            if (!split) continue;
            int64_t cnt[4] = {0}, off[4], o2[4];
            int shift = 20 - l;
            for (int64_t k = b->start; k < b->start + b->count; ++k) {
                int64_t pi = t->ord[k];
                cnt[((P->cell[2 * pi] >> shift) & 1) | (((P->cell[2 * pi + 1] >> shift) & 1) << 1)]++;
            }
            off[0] = b->start;
            for (int c = 1; c < 4; ++c) off[c] = off[c - 1] + cnt[c - 1];
            memcpy(o2, off, sizeof(off));
            for (int64_t k = b->start; k < b->start + b->count; ++k) {
                int64_t pi = t->ord[k];
                tmp[o2[((P->cell[2 * pi] >> shift) & 1) | (((P->cell[2 * pi + 1] >> shift) & 1) << 1)]++] = pi;
            }
            memcpy(t->ord + b->start, tmp + b->start, (size_t)b->count * sizeof(int64_t));
            int64_t bix = b->ix, biy = b->iy;
            for (int c = 0; c < 4; ++c) {
                if (cnt[c] == 0) continue;
                obox2 ch;
                memset(&ch, 0, sizeof(ch));
                ch.level = l + 1;
                ch.ix = 2 * bix + (c & 1);
                ch.iy = 2 * biy + ((c >> 1) & 1);
                ch.parent = bi;
                for (int q = 0; q < 4; ++q) ch.child[q] = -1;
                ch.start = off[c];
                ch.count = cnt[c];
                int id = tree2_push(t, &ch);
                if (id < 0) { free(tmp); return -1; }
                t->b[bi].child[c] = id;
            }
        }
        if (t->nb == next_start) break;
        t->lev_start[l + 1] = next_start;
        t->lev_count[l + 1] = t->nb - next_start;
        t->nlev = l + 2;
    }
    free(tmp);
    for (int i = 0; i < t->nb; ++i) {
        obox2 *b = &t->b[i];
        b->leaf = 1;
        for (int c = 0; c < 4; ++c) if (b->child[c] >= 0) b->leaf = 0;
    }
    return 0;
}

/* level restriction, as in 3D: rebuild with violating leaves forced to split */
static int tree2_build_balanced(otree2 *t, const opoints2 *P, const oracle_params *prm)
{
    uint64_t *forced = NULL;
    int nforced = 0, capf = 0;
    for (int iter = 0; iter < 64; ++iter) {
        if (tree2_build(t, P, prm, forced, nforced) < 0) { free(forced); return -1; }
        int added = 0;
        for (int i = 0; i < t->nb; ++i) {
            obox2 *T = &t->b[i];
            if (!T->leaf || T->level + 1 >= t->nlev) continue;
            int viol = 0;
            for (int64_t jx = 2 * T->ix - 1; jx <= 2 * T->ix + 2 && !viol; ++jx)
                for (int64_t jy = 2 * T->iy - 1; jy <= 2 * T->iy + 2 && !viol; ++jy) {
                    int A = tree2_find(t, T->level + 1, jx, jy);
                    if (A >= 0 && !t->b[A].leaf) viol = 1;
                }
            if (viol) {
                if (nforced == capf) {
                    capf = capf ? 2 * capf : 256;
                    uint64_t *nfp = (uint64_t *)realloc(forced, (size_t)capf * sizeof(uint64_t));
                    if (!nfp) { free(forced); return -1; }
                    forced = nfp;
                }
                forced[nforced++] = cell_key2(T->level, T->ix, T->iy);
                added = 1;
            }
        }
        if (!added) { free(forced); return 0; }
        qsort(forced, (size_t)nforced, sizeof(uint64_t), cmp_u64);
    }
    free(forced);
    return -2;
}

static void tree2_free(otree2 *t)
{
    for (int i = 0; i < t->nb; ++i) {
        free(t->b[i].proxy);
        free(t->b[i].Phi);
        free(t->b[i].local);
    }
    free(t->b);
    free(t->ord);
    memset(t, 0, sizeof(*t));
}

static int points2_init(opoints2 *P, const double *src, const double *rho, int64_t ns,
                        const double *tgt, int64_t nt)
{
    memset(P, 0, sizeof(*P));
    int same = (tgt == src && nt == ns);
    int64_t n = same ? ns : ns + nt;
    P->n = n;
    size_t nn = (size_t)(n > 0 ? n : 1);
    P->u = (double *)malloc(nn * 2 * sizeof(double));
    P->cell = (int64_t *)malloc(nn * 2 * sizeof(int64_t));
    P->q = (double *)malloc(nn * sizeof(double));
    P->is_src = (char *)malloc(nn);
    P->is_tgt = (char *)malloc(nn);
    P->out_index = (int64_t *)malloc(nn * sizeof(int64_t));
    if (!P->u || !P->cell || !P->q || !P->is_src || !P->is_tgt || !P->out_index) return -1;
    double lo[2] = {INFINITY, INFINITY}, hi[2] = {-INFINITY, -INFINITY};
    for (int64_t i = 0; i < n; ++i) {
        const double *x = (i < ns) ? &src[2 * i] : &tgt[2 * (i - ns)];
        for (int d = 0; d < 2; ++d) {
            if (x[d] < lo[d]) lo[d] = x[d];
            if (x[d] > hi[d]) hi[d] = x[d];
        }
    }
    double S = 0.0;
    for (int d = 0; d < 2; ++d) if (n > 0 && hi[d] - lo[d] > S) S = hi[d] - lo[d];
    if (S == 0.0) S = 1.0;
    P->S = S;
    for (int64_t i = 0; i < n; ++i) {
        const double *x = (i < ns) ? &src[2 * i] : &tgt[2 * (i - ns)];
        for (int d = 0; d < 2; ++d) {
            volatile double diff = x[d] - lo[d];
            double u = diff / S;
            P->u[2 * i + d] = u;
            int64_t c = (int64_t)floor(u * 2097152.0);
            if (c > 2097151) c = 2097151;
            if (c < 0) c = 0;
            P->cell[2 * i + d] = c;
        }
        P->is_src[i] = same || i < ns;
        P->is_tgt[i] = same || i >= ns;
        P->q[i] = P->is_src[i] ? rho[i] : 0.0;
        P->out_index[i] = same ? i : (i < ns ? -1 : i - ns);
    }
    return 0;
}

static void points2_free(opoints2 *P)
{
    free(P->u); free(P->cell); free(P->q); free(P->is_src); free(P->is_tgt); free(P->out_index);
    memset(P, 0, sizeof(*P));
}

static int tree2_make(otree2 *t, const opoints2 *P, const oracle_params *prm)
{
    memset(t, 0, sizeof(*t));
    t->ord = (int64_t *)malloc((size_t)(P->n > 0 ? P->n : 1) * sizeof(int64_t));
    if (!t->ord) return -1;
    int rc = tree2_build_balanced(t, P, prm);
    if (rc < 0) return rc;
    for (int i = 0; i < t->nb; ++i) {
        obox2 *b = &t->b[i];
        b->nsrc = b->ntgt = 0;
        for (int64_t k = b->start; k < b->start + b->count; ++k) {
            b->nsrc += P->is_src[t->ord[k]];
            b->ntgt += P->is_tgt[t->ord[k]];
        }
        b->ncol = 0;
        for (int dx = -1; dx <= 1; ++dx)
            for (int dy = -1; dy <= 1; ++dy) {
                int c = tree2_find(t, b->level, b->ix + dx, b->iy + dy);
                if (c >= 0) b->col[b->ncol++] = c;
            }
    }
    for (int i = 0; i < t->nb; ++i) t->b[i].fout = !t->b[i].leaf && t->b[i].nsrc > 0;
    for (int i = 0; i < t->nb; ++i) {
        obox2 *b = &t->b[i];
        b->fin = 0;
        if (b->ntgt == 0) continue;
        for (int k = 0; k < b->ncol; ++k) if (t->b[b->col[k]].fout) b->fin = 1;
    }
    return 0;
}

/* ---- the 2D transforms: the 3D ones with one axis fewer ---------------- */

/* Y = (Mx (x) My) X for a real p^2 array */
static void tensor2_real(const double *Mx, const double *My, int p, const double *X, double *Y)
{
    double *w = (double *)malloc((size_t)p * p * sizeof(double));
    for (int a = 0; a < p; ++a)
        for (int b = 0; b < p; ++b) {
            double acc = 0.0;
            for (int k = 0; k < p; ++k) acc += My[b * p + k] * X[a * p + k];
            w[a * p + b] = acc;
        }
    for (int a = 0; a < p; ++a)
        for (int b = 0; b < p; ++b) {
            double acc = 0.0;
            for (int k = 0; k < p; ++k) acc += Mx[a * p + k] * w[k * p + b];
            Y[a * p + b] = acc;
        }
    free(w);
}

static void form_proxy2(const ops_t *o, const opoints2 *P, const otree2 *t, const obox2 *b, double *proxy)
{
    int p = o->p;
    double R = level_R(b->level);
    double cx = (b->ix + 0.5) * R, cy = (b->iy + 0.5) * R;
    double ax[64], ay[64];
    memset(proxy, 0, (size_t)p * p * sizeof(double));
    for (int64_t k = b->start; k < b->start + b->count; ++k) {
        int64_t pi = t->ord[k];
        if (!P->is_src[pi]) continue;
        anterp_weights(o, 2.0 * (P->u[2 * pi] - cx) / R, ax);
        anterp_weights(o, 2.0 * (P->u[2 * pi + 1] - cy) / R, ay);
        for (int i = 0; i < p; ++i)
            for (int j = 0; j < p; ++j) proxy[i * p + j] += P->q[pi] * ax[i] * ay[j];
    }
}

static void prox2pw2(const ops_t *o, double h, double R, int nh, const double *proxy, cplx *Phi)
{
    int p = o->p, N = 2 * nh + 1;
    cplx *E = (cplx *)malloc((size_t)N * p * sizeof(cplx));
    cplx *X = (cplx *)malloc((size_t)p * p * sizeof(cplx));
    cplx *Y1 = (cplx *)malloc((size_t)N * p * sizeof(cplx));
    for (int m = -nh; m <= nh; ++m)
        for (int j = 0; j < p; ++j) E[(m + nh) * p + j] = cexp(-I * h * m * 0.5 * R * o->t[j]);
    for (int i = 0; i < p * p; ++i) X[i] = proxy[i];
    int d0[3] = {p, p, 1}, d1[3] = {N, p, 1};
    mode_apply_c(E, N, p, X, d0, 0, Y1);
    mode_apply_c(E, N, p, Y1, d1, 1, Phi);
    free(E); free(X); free(Y1);
}

static void pw2poly2(const ops_t *o, double h, double R, int nh, const cplx *Psi, double *coef)
{
    int p = o->p, N = 2 * nh + 1;
    cplx *F = (cplx *)malloc((size_t)p * N * sizeof(cplx));
    cplx *Y1 = (cplx *)malloc((size_t)p * N * sizeof(cplx));
    cplx *Y2 = (cplx *)malloc((size_t)p * p * sizeof(cplx));
    double *vals = (double *)malloc((size_t)p * p * sizeof(double));
    for (int n = 0; n < p; ++n)
        for (int m = -nh; m <= nh; ++m) F[n * N + (m + nh)] = cexp(I * h * m * 0.5 * R * o->t[n]);
    int d0[3] = {N, N, 1}, d1[3] = {p, N, 1};
    mode_apply_c(F, p, N, Psi, d0, 0, Y1);
    mode_apply_c(F, p, N, Y1, d1, 1, Y2);
    for (int i = 0; i < p * p; ++i) vals[i] = creal(Y2[i]);
    tensor2_real(o->Vinv, o->Vinv, p, vals, coef);
    free(F); free(Y1); free(Y2); free(vals);
}

static double eval_local2(const ops_t *o, const obox2 *b, const double *coef, const double *u)
{
    int p = o->p;
    double R = level_R(b->level);
    double tx[64], ty[64];
    double xi = 2.0 * (u[0] - (b->ix + 0.5) * R) / R, yi = 2.0 * (u[1] - (b->iy + 0.5) * R) / R;
    for (int n = 0; n < p; ++n) {
        tx[n] = cheb_t(n, xi);
        ty[n] = cheb_t(n, yi);
    }
    double acc = 0.0;
    for (int a = 0; a < p; ++a) {
        double s = 0.0;
        for (int b2 = 0; b2 < p; ++b2) s += coef[a * p + b2] * ty[b2];
        acc += tx[a] * s;
    }
    return acc;
}

static int add_subtree_leaves2(const otree2 *t, int X, int S, ilist *lists)
{
    const obox2 *b = &t->b[X];
    if (b->leaf) return ilist_push(&lists[X], S);
    for (int c = 0; c < 4; ++c)
        if (b->child[c] >= 0 && add_subtree_leaves2(t, b->child[c], S, lists) < 0) return -1;
    return 0;
}

/* Steps 2-5 of Sec. 3.4 in the plane (unit-box potentials) */
static int run_dmk2(const split2_t *sp, const opoints2 *P, otree2 *t, double *ufar, double *unear)
{
    const oracle_params *prm = &sp->prm;
    ops_t o;
    if (ops_init(&o, prm->p, prm->nf, prm->n0) != 0) { ops_free(&o); return -1; }
    int p = o.p, p2 = p * p, N1 = o.N1, NF = N1 * N1, nf = o.nf;
    int Lmax = t->nlev - 1, rc = 0;
    for (int64_t i = 0; i < P->n; ++i) { ufar[i] = 0.0; unear[i] = 0.0; }

    /* Step 2: proxy charges on source leaves, merged upward (T_c2p) */
#pragma omp parallel for schedule(dynamic, 1)
    for (int i = 0; i < t->nb; ++i) {
        obox2 *b = &t->b[i];
        if (!b->leaf || b->nsrc == 0) continue;
        b->proxy = (double *)malloc((size_t)p2 * sizeof(double));
        form_proxy2(&o, P, t, b, b->proxy);
    }
    for (int l = Lmax - 1; l >= 0; --l) {
        int s = t->lev_start[l], e = s + t->lev_count[l];
#pragma omp parallel for schedule(dynamic, 1)
        for (int i = s; i < e; ++i) {
            obox2 *b = &t->b[i];
            if (b->leaf || b->nsrc == 0) continue;
            b->proxy = (double *)calloc((size_t)p2, sizeof(double));
            double *tmp = (double *)malloc((size_t)p2 * sizeof(double));
            for (int c = 0; c < 4; ++c) {
                int ci = b->child[c];
                if (ci < 0 || !t->b[ci].proxy) continue;
                tensor2_real(o.c2p[c & 1], o.c2p[(c >> 1) & 1], p, t->b[ci].proxy, tmp);
                for (int k = 0; k < p2; ++k) b->proxy[k] += tmp[k];
            }
            free(tmp);
        }
    }

    /* Step 3: downward pass */
    cplx *wl = (cplx *)malloc((size_t)NF * sizeof(cplx));
    for (int l = 0; l <= Lmax; ++l) {
        int s = t->lev_start[l], e = s + t->lev_count[l];
        double R = level_R(l), h = split_h(l), ws = (h / (2.0 * M_PI)) * (h / (2.0 * M_PI));
        for (int mx = -nf; mx <= nf; ++mx)
            for (int my = -nf; my <= nf; ++my)
                wl[(mx + nf) * N1 + (my + nf)] = ws * split2_Dhat(sp, l, h * sqrt((double)(mx * mx + my * my)));
#pragma omp parallel for schedule(dynamic, 1)
        for (int i = s; i < e; ++i) {
            obox2 *b = &t->b[i];
            if (!b->fout) continue;
            b->Phi = (cplx *)malloc((size_t)NF * sizeof(cplx));
            prox2pw2(&o, h, R, nf, b->proxy, b->Phi);
        }
#pragma omp parallel for schedule(dynamic, 1)
        for (int i = s; i < e; ++i) {
            obox2 *b = &t->b[i];
            if (!b->fin) continue;
            cplx *Psi = (cplx *)calloc((size_t)NF, sizeof(cplx));
            double *coef = (double *)malloc((size_t)p2 * sizeof(double));
            double cB[2] = {(b->ix + 0.5) * R, (b->iy + 0.5) * R};
            for (int k = 0; k < b->ncol; ++k) {
                const obox2 *S = &t->b[b->col[k]];
                if (!S->fout) continue;
                double d[2] = {cB[0] - (S->ix + 0.5) * R, cB[1] - (S->iy + 0.5) * R};
                for (int mx = -nf; mx <= nf; ++mx)
                    for (int my = -nf; my <= nf; ++my) {
                        int idx = (mx + nf) * N1 + (my + nf);
                        Psi[idx] += wl[idx] * cexp(I * h * (mx * d[0] + my * d[1])) * S->Phi[idx];
                    }
            }
            pw2poly2(&o, h, R, nf, Psi, coef);
            if (!b->local) b->local = (double *)calloc((size_t)p2, sizeof(double));
            for (int k = 0; k < p2; ++k) b->local[k] += coef[k];
            b->has_local = 1;
            free(Psi); free(coef);
        }
        if (l == 0) {
            /* the windowed root kernel over the unit square */
            obox2 *b = &t->b[0];
            int n0 = o.n0, NW = o.NW;
            if (!b->local) b->local = (double *)calloc((size_t)p2, sizeof(double));
            if (b->proxy) {
                cplx *PhiW = (cplx *)malloc((size_t)NW * NW * sizeof(cplx));
                double *coef = (double *)malloc((size_t)p2 * sizeof(double));
                prox2pw2(&o, sp->hW, 1.0, n0, b->proxy, PhiW);
                double wsw = (sp->hW / (2.0 * M_PI)) * (sp->hW / (2.0 * M_PI));
                for (int mx = -n0; mx <= n0; ++mx)
                    for (int my = -n0; my <= n0; ++my)
                        PhiW[(mx + n0) * NW + (my + n0)] *=
                            wsw * split2_What(sp, sp->hW * sqrt((double)(mx * mx + my * my)));
                pw2poly2(&o, sp->hW, 1.0, n0, PhiW, coef);
                for (int k = 0; k < p2; ++k) b->local[k] += coef[k];
                free(PhiW); free(coef);
            }
            b->has_local = 1;
        }
        /* local expansions to the children (T_p2c) */
#pragma omp parallel for schedule(dynamic, 1)
        for (int i = s; i < e; ++i) {
            obox2 *b = &t->b[i];
            if (b->leaf || !b->has_local) continue;
            double *tmp = (double *)malloc((size_t)p2 * sizeof(double));
            for (int c = 0; c < 4; ++c) {
                int ci = b->child[c];
                if (ci < 0) continue;
                obox2 *ch = &t->b[ci];
                tensor2_real(o.p2c[c & 1], o.p2c[(c >> 1) & 1], p, b->local, tmp);
                if (!ch->local) ch->local = (double *)calloc((size_t)p2, sizeof(double));
                for (int k = 0; k < p2; ++k) ch->local[k] += tmp[k];
                ch->has_local = 1;
            }
            free(tmp);
        }
#pragma omp parallel for schedule(dynamic, 1)
        for (int i = s; i < e; ++i) {
            obox2 *b = &t->b[i];
            if (!b->leaf || !b->has_local) continue;
            for (int64_t k = b->start; k < b->start + b->count; ++k) {
                int64_t pi = t->ord[k];
                if (P->is_tgt[pi]) ufar[pi] += eval_local2(&o, b, b->local, &P->u[2 * pi]);
            }
        }
        for (int i = s; i < e; ++i) {
            free(t->b[i].Phi);
            t->b[i].Phi = NULL;
        }
    }
    free(wl);

    /* Step 4: residual kernels over the same lists as in 3D */
    ilist *lists = (ilist *)calloc((size_t)t->nb, sizeof(ilist));
    for (int S = 0; S < t->nb && rc == 0; ++S) {
        const obox2 *b = &t->b[S];
        if (!b->leaf || b->nsrc == 0) continue;
        for (int k = 0; k < b->ncol; ++k)
            if (add_subtree_leaves2(t, b->col[k], S, lists) < 0) rc = -1;
        if (b->level > 0) {
            int lp = b->level - 1;
            int64_t px = b->ix >> 1, py = b->iy >> 1;
            for (int64_t qx = px - 1; qx <= px + 1; ++qx)
                for (int64_t qy = py - 1; qy <= py + 1; ++qy) {
                    int X = tree2_find(t, lp, qx, qy);
                    if (X < 0 || !t->b[X].leaf) continue;
                    int adj = 2 * qx <= b->ix + 1 && 2 * qx + 2 >= b->ix && 2 * qy <= b->iy + 1 && 2 * qy + 2 >= b->iy;
                    if (adj && ilist_push(&lists[X], S) < 0) rc = -1;
                }
        }
    }
    if (rc == 0) {
#pragma omp parallel for schedule(dynamic, 1)
        for (int T = 0; T < t->nb; ++T) {
            const obox2 *bt = &t->b[T];
            if (!bt->leaf || bt->ntgt == 0) continue;
            for (int64_t k = bt->start; k < bt->start + bt->count; ++k) {
                int64_t ti = t->ord[k];
                if (!P->is_tgt[ti]) continue;
                const double *x = &P->u[2 * ti];
                double acc = 0.0;
                for (int li = 0; li < lists[T].n; ++li) {
                    const obox2 *bs = &t->b[lists[T].s[li]];
                    double Rb = level_R(bs->level);
                    for (int64_t kk = bs->start; kk < bs->start + bs->count; ++kk) {
                        int64_t sj = t->ord[kk];
                        if (!P->is_src[sj]) continue;
                        double dx = x[0] - P->u[2 * sj], dy = x[1] - P->u[2 * sj + 1];
                        double r = sqrt(dx * dx + dy * dy);
                        if (r == 0.0 || r >= Rb) continue;
                        acc += P->q[sj] * split2_R(sp, bs->level, r);
                    }
                }
                unear[ti] += acc;
            }
        }
    }
    for (int i = 0; i < t->nb; ++i) free(lists[i].s);
    free(lists);

    /* Step 5: a coincident source added rho S_L(0) through the far field */
#pragma omp parallel for schedule(dynamic, 1)
    for (int T = 0; T < t->nb; ++T) {
        const obox2 *b = &t->b[T];
        if (!b->leaf || b->ntgt == 0 || b->nsrc == 0) continue;
        double S0 = split2_S0(sp, b->level);
        for (int64_t k = b->start; k < b->start + b->count; ++k) {
            int64_t ti = t->ord[k];
            if (!P->is_tgt[ti]) continue;
            for (int64_t kk = b->start; kk < b->start + b->count; ++kk) {
                int64_t sj = t->ord[kk];
                if (P->is_src[sj] && P->u[2 * ti] == P->u[2 * sj] && P->u[2 * ti + 1] == P->u[2 * sj + 1])
                    unear[ti] -= P->q[sj] * S0;
            }
        }
    }
    ops_free(&o);
    return rc;
}

int oracle_dmk_log2d(const oracle_params *prm_in,
                     const double *src, const double *rho, int64_t ns,
                     const double *tgt, int64_t nt,
                     double *pot, double *pot_far, double *pot_near)
{
    if (ns < 0 || nt < 0) return -1;
    if (nt == 0) return 0;
    split2_t sp;
    if (split2_init(&sp, prm_in) != 0) { split2_free(&sp); return -1; }
#ifdef _OPENMP
    if (sp.prm.nthreads > 0) omp_set_num_threads(sp.prm.nthreads);
#endif
    opoints2 P;
    otree2 t;
    memset(&t, 0, sizeof(t));
    int rc = points2_init(&P, src, rho, ns, tgt, nt);
    if (rc == 0) rc = tree2_make(&t, &P, &sp.prm);
    double *ufar = NULL, *unear = NULL;
    if (rc == 0) {
        ufar = (double *)malloc((size_t)P.n * sizeof(double));
        unear = (double *)malloc((size_t)P.n * sizeof(double));
        if (!ufar || !unear) rc = -1;
    }
    if (rc == 0) rc = run_dmk2(&sp, &P, &t, ufar, unear);
    if (rc == 0) {
        /* log S times the charge of the sources not coincident with the target */
        double qtot = 0.0, logS = log(P.S);
        for (int64_t j = 0; j < P.n; ++j) if (P.is_src[j]) qtot += P.q[j];
        for (int T = 0; T < t.nb; ++T) {
            const obox2 *b = &t.b[T];
            if (!b->leaf) continue;
            for (int64_t k = b->start; k < b->start + b->count; ++k) {
                int64_t ti = t.ord[k], o = P.out_index[ti];
                if (o < 0) continue;
                double qc = 0.0;
                for (int64_t kk = b->start; kk < b->start + b->count; ++kk) {
                    int64_t sj = t.ord[kk];
                    if (P.is_src[sj] && P.u[2 * ti] == P.u[2 * sj] && P.u[2 * ti + 1] == P.u[2 * sj + 1])
                        qc += P.q[sj];
                }
                pot[o] = ufar[ti] + unear[ti] + logS * (qtot - qc);
                if (pot_far) pot_far[o] = ufar[ti];
                if (pot_near) pot_near[o] = unear[ti];
            }
        }
    }
    free(ufar);
    free(unear);
    tree2_free(&t);
    points2_free(&P);
    split2_free(&sp);
    return rc;
}

void oracle_kernel_log2d(const oracle_params *prm, int what, int level,
                         const double *r, int64_t n, double *out)
{
    split2_t sp;
    if (split2_init(&sp, prm) != 0) { split2_free(&sp); return; }
    for (int64_t i = 0; i < n; ++i) {
        double x = r[i];
        switch (what) {
        case 0: out[i] = split2_S0(&sp, level); break;
        case 1: out[i] = split2_R(&sp, level, x); break;
        case 3: out[i] = split2_Dhat(&sp, level, x); break;
        case 4: out[i] = split2_What(&sp, x); break;
        default: out[i] = NAN;
        }
    }
    split2_free(&sp);
}

double oracle_hW_log2d(const oracle_params *prm)
{
    split2_t sp;
    if (split2_init(&sp, prm) != 0) { split2_free(&sp); return NAN; }
    double h = sp.hW;
    split2_free(&sp);
    return h;
}

int oracle_n0_log2d(const oracle_params *prm)
{
    split2_t sp;
    if (split2_init(&sp, prm) != 0) { split2_free(&sp); return -1; }
    int n0 = sp.prm.n0;
    split2_free(&sp);
    return n0;
}

int64_t oracle_tree_log2d(const oracle_params *prm_in, const double *src, int64_t ns,
                          int32_t *leaf_level, int64_t *leaf_ix, int64_t *leaf_iy)
{
    split2_t sp;
    if (split2_init(&sp, prm_in) != 0) { split2_free(&sp); return -1; }
    double *dummy = (double *)calloc((size_t)(ns > 0 ? ns : 1), sizeof(double));
    opoints2 P;
    otree2 t;
    memset(&t, 0, sizeof(t));
    int rc = points2_init(&P, src, dummy, ns, src, ns);
    if (rc == 0) rc = tree2_make(&t, &P, &sp.prm);
    int64_t nb = rc == 0 ? t.nb : rc;
    if (rc == 0)
        for (int i = 0; i < t.nb; ++i) {
            const obox2 *b = &t.b[i];
            if (!b->leaf) continue;
            for (int64_t k = b->start; k < b->start + b->count; ++k) {
                int64_t pi = t.ord[k];
                leaf_level[pi] = b->level;
                leaf_ix[pi] = b->ix;
                leaf_iy[pi] = b->iy;
            }
        }
    tree2_free(&t);
    points2_free(&P);
    free(dummy);
    split2_free(&sp);
    return nb;
}
