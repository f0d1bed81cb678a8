// plan_math.cpp -- host-side tables of a DMK plan ("Step 1: Precomputation",
// Sec. 3.4 of arXiv 2308.00292) for the 3D Laplace kernel with the PSWF
// kernel splitting of Sec. 3.6.
//
// Box geometry used throughout the library: the unit box is [0,1]^3 (level 0),
// a box at level l has side R_l = 2^-l, and Chebyshev coordinates in a box are
// xi = 2 (x - c_B) / R_l in [-1, 1].
//
// Tables produced here (all one-dimensional, level independent):
//   * Chebyshev nodes t_j = cos(pi (j + 1/2) / p), j = 0..p-1 (Sec. 2.1)
//   * shift matrices A_s[n][m], s = -1/+1: T_n((xi + s)/2) = sum_m A_s[n][m] T_m(xi).
//     They map child Chebyshev moments to parent moments (Lemma ctoplemma,
//     T_c2p) and, transposed, parent coefficients to child coefficients
//     (Lemma ptoclemma, T_p2c); both are exact for degree < p.
//   * plane-wave matrices F[m][n] = sum_j exp(-i theta m t_j) Vinv[n][j] with
//     theta = h_l R_l / 2 = pi / 3: they turn Chebyshev moments into the
//     outgoing expansion of eq. outgoingexpansion2 (T_prox2pw), and conj(F)^T
//     turns an incoming expansion into Chebyshev coefficients (eqs.
//     incomingexpansion2 and localexpansion, T_pw2poly).
//   * translation weights w(|m|^2) = (1/27) Dhat((2 pi / 3)|m|) at R = 1, so that
//     w_{l,m} = w(|m|^2) / R_l (eqs. wlmdef, differencekernelft3 with the
//     trapezoidal weight (h_l/2pi)^3 and h_l = 2 pi / (3 R_l)).
//   * root weights wW(|m|^2) = (hW / 2pi)^3 What_0(hW |m|) for the windowed
//     kernel of eq. windowedkernelft2, What_0(k) = 8 pi sin^2(R_t k / 2)/k^2
//     psi(k/c)/psi(0), R_t = 1 + sqrt 3, hW = 2 pi / (3 + sqrt 3).
//   * the residual polynomial q(t) = Phi(sqrt t)/sqrt t on t in [0, 1], so that
//     R_l(r) = 1/r - q(r^2 / R_l^2) / R_l for r < R_l (eq. newkernels).
#include "dmk_internal.h"

#include <algorithm>
#include <cmath>
#include <complex>
#include <vector>

namespace dmk {

namespace {

// Table 1 of the paper: eps, c, N1 = 2 nf + 1, p.
struct Row { double eps, c; int N1, p; };
const Row kTable1[4] = {
    {1e-3, 7.2462000846862793, 13, 9},
    {1e-6, 13.739999771118164, 25, 18},
    {1e-9, 20.736000061035156, 39, 28},
    {1e-12, 27.870000839233398, 53, 38},
};

// Gauss-Legendre rule on [-1, 1] by Newton's method on P_n.
void gl_rule(int n, std::vector<double> &x, std::vector<double> &w) {
    x.resize(n);
    w.resize(n);
    for (int i = 0; i < (n + 1) / 2; ++i) {
        double z = std::cos(M_PI * (i + 0.75) / (n + 0.5));
        double dp = 0.0;
        for (int it = 0; it < 50; ++it) {
            double pm = 1.0, pc = z;
            for (int k = 2; k <= n; ++k) {
                double pn = ((2.0 * k - 1.0) * z * pc - (k - 1.0) * pm) / k;
                pm = pc;
                pc = pn;
            }
            dp = n * (pm - z * pc) / (1.0 - z * z);
            double dz = pc / dp;
            z -= dz;
            if (std::fabs(dz) < 1e-16) break;
        }
        x[i] = -z;
        x[n - 1 - i] = z;
        w[i] = w[n - 1 - i] = 2.0 / ((1.0 - z * z) * dp * dp);
    }
}

// Cyclic Jacobi eigen-decomposition of a dense symmetric matrix (row-major).
// On return a holds the eigenvalues on its diagonal and v the eigenvectors
// (columns).
void jacobi_eigen(int n, std::vector<double> &a, std::vector<double> &v) {
    v.assign((size_t)n * n, 0.0);
    for (int i = 0; i < n; ++i) v[(size_t)i * n + i] = 1.0;
    for (int sweep = 0; sweep < 100; ++sweep) {
        double off = 0.0, tot = 0.0;
        for (int i = 0; i < n; ++i)
            for (int j = 0; j < n; ++j) {
                double x = a[(size_t)i * n + j] * a[(size_t)i * n + j];
                tot += x;
                if (i != j) off += x;
            }
        if (off <= 1e-30 * tot) break;
        for (int p = 0; p < n - 1; ++p)
            for (int q = p + 1; q < n; ++q) {
                double apq = a[(size_t)p * n + q];
                if (std::fabs(apq) < 1e-300) continue;
                double app = a[(size_t)p * n + p], aqq = a[(size_t)q * n + q];
                double theta = (aqq - app) / (2.0 * apq);
                double t = (theta >= 0 ? 1.0 : -1.0) / (std::fabs(theta) + std::sqrt(theta * theta + 1.0));
                double c = 1.0 / std::sqrt(t * t + 1.0), s = t * c;
                for (int k = 0; k < n; ++k) {
                    double akp = a[(size_t)k * n + p], akq = a[(size_t)k * n + q];
                    a[(size_t)k * n + p] = c * akp - s * akq;
                    a[(size_t)k * n + q] = s * akp + c * akq;
                }
                for (int k = 0; k < n; ++k) {
                    double apk = a[(size_t)p * n + k], aqk = a[(size_t)q * n + k];
                    a[(size_t)p * n + k] = c * apk - s * aqk;
                    a[(size_t)q * n + k] = s * apk + c * aqk;
                }
                for (int k = 0; k < n; ++k) {
                    double vkp = v[(size_t)k * n + p], vkq = v[(size_t)k * n + q];
                    v[(size_t)k * n + p] = c * vkp - s * vkq;
                    v[(size_t)k * n + q] = s * vkp + c * vkq;
                }
            }
    }
}

}  // namespace

// ---- PSWF psi_0^c ---------------------------------------------------------
// psi_0^c is the ground state of the prolate operator -((1-x^2) psi')' + c^2 x^2
// psi, whose matrix in the orthonormal Legendre basis couples degrees k and
// k +- 2 only; psi_0 is even.  Outside [-1, 1] psi is continued by the
// eigen-relation lambda_0 psi(x) = int_{-1}^1 psi(t) exp(i c x t) dt (App. A.5).
Pswf::Pswf(double c_) : c(c_) {
    const int n = 64;  // even degrees 0..126
    std::vector<double> a((size_t)n * n, 0.0), v;
    for (int i = 0; i < n; ++i) {
        double k = 2.0 * i;
        a[(size_t)i * n + i] = k * (k + 1.0) + c * c * (2.0 * k * (k + 1.0) - 1.0) / ((2.0 * k + 3.0) * (2.0 * k - 1.0));
        if (i + 1 < n) {
            double off = c * c * (k + 1.0) * (k + 2.0) / ((2.0 * k + 3.0) * std::sqrt((2.0 * k + 1.0) * (2.0 * k + 5.0)));
            a[(size_t)i * n + i + 1] = off;
            a[(size_t)(i + 1) * n + i] = off;
        }
    }
    jacobi_eigen(n, a, v);
    int imin = 0;
    for (int i = 1; i < n; ++i)
        if (a[(size_t)i * n + i] < a[(size_t)imin * n + imin]) imin = i;
    chi0 = a[(size_t)imin * n + imin];
    coef.resize(n);
    for (int i = 0; i < n; ++i) coef[i] = v[(size_t)i * n + imin] * std::sqrt((4.0 * i + 1.0) / 2.0);
    double p0 = eval_inside(0.0);
    for (double &x : coef) x /= p0;  // psi(0) = 1
    gl_rule(400, qx, qw);
    qpsi.resize(qx.size());
    double integral = 0.0;
    for (size_t i = 0; i < qx.size(); ++i) {
        qpsi[i] = eval_inside(qx[i]);
        integral += qw[i] * qpsi[i];
    }
    lambda0 = integral;  // psi(0) = 1
    c0 = 0.5 * lambda0;  // c_0 = int_0^1 psi = lambda_0 psi(0) / 2 (Sec. 3.6)
    // x^2 = P_0/3 + 2 P_2/3, so int_0^1 x^2 psi only sees the P_0 and P_2 terms
    c2 = 0.5 * (coef[0] * 2.0 / 3.0 + coef[1] * 4.0 / 15.0);
}

// coef[i] multiplies P_{2i}(x) (coefficients already include the Legendre
// normalisation).
double Pswf::eval_inside(double x) const {
    double acc = coef[0];
    double pm = 1.0, pc = x;  // P_0, P_1
    int kmax = 2 * (int)(coef.size() - 1);
    for (int k = 2; k <= kmax; ++k) {
        double pn = ((2.0 * k - 1.0) * x * pc - (k - 1.0) * pm) / k;
        pm = pc;
        pc = pn;
        if ((k & 1) == 0) acc += coef[k / 2] * pc;
    }
    return acc;
}

double Pswf::operator()(double x) const {
    double ax = std::fabs(x);
    if (ax <= 1.0) return eval_inside(ax);
    double acc = 0.0;
    for (size_t i = 0; i < qx.size(); ++i) acc += qw[i] * qpsi[i] * std::cos(c * ax * qx[i]);
    return acc / lambda0;
}

// psi(x1) - psi(x2) = lambda_0^{-1} int psi(t) (cos c x1 t - cos c x2 t) dt with
// cos a - cos b = -2 sin((a + b)/2) sin((a - b)/2): no cancellation when both
// arguments are small
double Pswf::diff(double x1, double x2) const {
    double acc = 0.0;
    for (size_t i = 0; i < qx.size(); ++i)
        acc += qw[i] * qpsi[i] * std::sin(0.5 * c * (x1 + x2) * qx[i]) * std::sin(0.5 * c * (x1 - x2) * qx[i]);
    return -2.0 * acc / lambda0;
}

// Phi(s) = c_0^{-1} int_0^s psi, by Gauss-Legendre quadrature on [0, s].
double Pswf::Phi(double s) const {
    if (s >= 1.0) return 1.0;
    if (s <= 0.0) return 0.0;
    static thread_local std::vector<double> gx, gw;
    if (gx.empty()) gl_rule(80, gx, gw);
    double acc = 0.0;
    for (size_t i = 0; i < gx.size(); ++i) acc += gw[i] * eval_inside(0.5 * s * (gx[i] + 1.0));
    return 0.5 * s * acc / c0;
}

// ---- Chebyshev fits -----------------------------------------------------------
namespace {
// Chebyshev coefficients of f on t in [0, 1] from its values at the 64 points
// t_j = (1 + cos(pi (j + 1/2) / 64)) / 2, truncated where the tail falls below tol
std::vector<double> cheb_fit(const std::vector<double> &vals, double tol) {
    const int nc = (int)vals.size();
    std::vector<double> ch(nc, 0.0);
    for (int k = 0; k < nc; ++k) {
        double acc = 0.0;
        for (int j = 0; j < nc; ++j) acc += vals[j] * std::cos(M_PI * k * (j + 0.5) / nc);
        ch[k] = acc * (k == 0 ? 1.0 : 2.0) / nc;
    }
    int deg = nc - 1;
    double tail = 0.0;
    while (deg > 2 && tail + std::fabs(ch[deg]) < tol) { tail += std::fabs(ch[deg]); --deg; }
    ch.resize(deg + 1);
    return ch;
}

// monomial coefficients in x = 2t - 1 of a Chebyshev series (for Horner)
std::vector<double> cheb_to_mono(const std::vector<double> &ch) {
    const int deg = (int)ch.size() - 1;
    std::vector<double> mono(deg + 1, 0.0), Tm2(deg + 1, 0.0), Tm1(deg + 1, 0.0), Tc(deg + 1, 0.0);
    Tm2[0] = 1.0;
    mono[0] += ch[0];
    if (deg >= 1) { Tm1[1] = 1.0; mono[1] += ch[1]; }
    for (int k = 2; k <= deg; ++k) {
        std::fill(Tc.begin(), Tc.end(), 0.0);
        for (int i = 0; i < k; ++i) Tc[i + 1] += 2.0 * Tm1[i];
        for (int i = 0; i <= k - 2; ++i) Tc[i] -= Tm2[i];
        for (int i = 0; i <= k; ++i) mono[i] += ch[k] * Tc[i];
        Tm2 = Tm1;
        Tm1 = Tc;
    }
    return mono;
}

double cheb_node01(int j, int nc) { return 0.5 * (std::cos(M_PI * (j + 0.5) / nc) + 1.0); }
}  // namespace

// ---- plan tables ------------------------------------------------------------
int build_tables(double eps, int p_override, int nf_override, Tables &tb, std::string &err) {
    int row = 3;
    for (int i = 0; i < 4; ++i)
        if (kTable1[i].eps <= eps * (1.0 + 1e-12)) { row = i; break; }
    tb.eps = eps;
    tb.c = kTable1[row].c;
    tb.p = p_override > 0 ? p_override : kTable1[row].p;
    tb.nf = nf_override > 0 ? nf_override : (kTable1[row].N1 - 1) / 2;
    if (tb.p > kMaxP || tb.nf > kMaxNf) { err = "p or nf above the library limits"; return -1; }
    const int p = tb.p, nf = tb.nf;
    Pswf psi(tb.c);
    tb.psi0_over_c0 = 1.0 / psi.c0;

    // Chebyshev nodes and T_n(t_j) by the three-term recurrence
    tb.t.resize(p);
    for (int j = 0; j < p; ++j) tb.t[j] = std::cos(M_PI * (j + 0.5) / p);
    std::vector<double> T((size_t)p * p);  // T[n][j]
    for (int j = 0; j < p; ++j) {
        double t0 = 1.0, t1 = tb.t[j];
        T[j] = 1.0;
        if (p > 1) T[(size_t)1 * p + j] = t1;
        for (int n = 2; n < p; ++n) {
            double t2 = 2.0 * tb.t[j] * t1 - t0;
            T[(size_t)n * p + j] = t2;
            t0 = t1;
            t1 = t2;
        }
    }
    // V^{-1}[n][j] from the discrete orthogonality of T_n at the nodes
    std::vector<double> Vinv((size_t)p * p);
    for (int n = 0; n < p; ++n)
        for (int j = 0; j < p; ++j) Vinv[(size_t)n * p + j] = (n == 0 ? 1.0 : 2.0) / p * T[(size_t)n * p + j];

    // A_s: coefficient-space recurrence, y = (xi + s)/2, T_{n+1}(y) = 2 y T_n(y) - T_{n-1}(y),
    // using xi T_m = (T_{m+1} + T_{|m-1|}) / 2.
    for (int si = 0; si < 2; ++si) {
        double s = si ? 1.0 : -1.0;
        std::vector<std::vector<double>> P(p, std::vector<double>(p + 1, 0.0));
        P[0][0] = 1.0;
        if (p > 1) { P[1][0] = 0.5 * s; P[1][1] = 0.5; }
        for (int n = 1; n + 1 < p; ++n) {
            std::vector<double> xiT(p + 1, 0.0);  // xi * T_n(y) in the T_m(xi) basis
            for (int m = 0; m <= n; ++m) {
                double a = P[n][m];
                if (a == 0.0) continue;
                if (m + 1 <= p) xiT[m + 1] += 0.5 * a;
                xiT[m == 0 ? 1 : m - 1] += 0.5 * a;
            }
            for (int m = 0; m <= n + 1 && m < p; ++m)
                P[n + 1][m] = xiT[m] + s * P[n][m] - P[n - 1][m];
        }
        tb.A[si].assign((size_t)p * p, 0.0);
        for (int n = 0; n < p; ++n)
            for (int m = 0; m < p; ++m) tb.A[si][(size_t)n * p + m] = P[n][m];
    }

    // F[m][n], m in [-nf, nf]: moments -> outgoing expansion, theta = pi/3
    const int N1 = 2 * nf + 1;
    const double theta = M_PI / 3.0;
    tb.Fr.assign((size_t)N1 * p, 0.0);
    tb.Fi.assign((size_t)N1 * p, 0.0);
    for (int mi = 0; mi < N1; ++mi) {
        int m = mi - nf;
        for (int n = 0; n < p; ++n) {
            std::complex<double> acc = 0.0;
            for (int j = 0; j < p; ++j) acc += std::polar(1.0, -theta * m * tb.t[j]) * Vinv[(size_t)n * p + j];
            tb.Fr[(size_t)mi * p + n] = acc.real();
            tb.Fi[(size_t)mi * p + n] = acc.imag();
        }
    }

    // translation weights w(s), s = |m|^2, at R = 1: (1/3)^3 Dhat((2 pi/3) sqrt s),
    // Dhat(k) = 4 pi [psi(k/(2c)) - psi(k/c)] / k^2, Dhat(0) = 2 pi (c2/c0)(1 - 1/4)
    const int ns = 3 * nf * nf + 1;
    tb.w.resize(ns);
    for (int s = 0; s < ns; ++s) {
        double dhat;
        if (s == 0) {
            dhat = 2.0 * M_PI * psi.c2 / psi.c0 * 0.75;
        } else {
            double k = 2.0 * M_PI / 3.0 * std::sqrt((double)s);
            dhat = 4.0 * M_PI * (psi(k / (2.0 * tb.c)) - psi(k / tb.c)) / (k * k);
        }
        tb.w[s] = dhat / 27.0;
    }

    // root term: windowed kernel of the unit box
    const double Rt = 1.0 + std::sqrt(3.0);
    tb.hW = 2.0 * M_PI / (2.0 + Rt);
    tb.n0 = (int)std::ceil(tb.c / tb.hW) + 1;
    if (tb.n0 > kMaxNf) { err = "root mode count above the library limit"; return -1; }
    const int NW = 2 * tb.n0 + 1;
    const double thetaW = 0.5 * tb.hW;  // nodes at c_root + t/2
    tb.FWr.assign((size_t)NW * p, 0.0);
    tb.FWi.assign((size_t)NW * p, 0.0);
    for (int mi = 0; mi < NW; ++mi) {
        int m = mi - tb.n0;
        for (int n = 0; n < p; ++n) {
            std::complex<double> acc = 0.0;
            for (int j = 0; j < p; ++j) acc += std::polar(1.0, -thetaW * m * tb.t[j]) * Vinv[(size_t)n * p + j];
            tb.FWr[(size_t)mi * p + n] = acc.real();
            tb.FWi[(size_t)mi * p + n] = acc.imag();
        }
    }
    const int nsW = 3 * tb.n0 * tb.n0 + 1;
    tb.wW.resize(nsW);
    const double scale = std::pow(tb.hW / (2.0 * M_PI), 3);
    for (int s = 0; s < nsW; ++s) {
        double k = tb.hW * std::sqrt((double)s);
        double what;
        if (s == 0) {
            what = 2.0 * M_PI * Rt * Rt;
        } else {
            double sn = std::sin(0.5 * Rt * k);
            what = 8.0 * M_PI * sn * sn / (k * k) * psi(k / tb.c);
        }
        tb.wW[s] = scale * what;
    }

    // residual polynomial q(t) = Phi(sqrt t)/sqrt t: Chebyshev interpolation on
    // t in [0, 1] at 64 points, truncated where the coefficients fall below the
    // target accuracy
    {
        const int nc = 64;
        std::vector<double> vals(nc);
        for (int j = 0; j < nc; ++j) {
            double s = std::sqrt(cheb_node01(j, nc));
            vals[j] = (s == 0.0) ? tb.psi0_over_c0 : psi.Phi(s) / s;
        }
        double tol = 1e-3 * eps * tb.psi0_over_c0;
        tol = std::max(tol, 1e-15 * tb.psi0_over_c0);
        tb.qcheb = cheb_fit(vals, tol);
        tb.qmono = cheb_to_mono(tb.qcheb);
    }
    tb.psi_grid.resize(257);
    for (int k = 0; k <= 256; ++k) tb.psi_grid[k] = psi(k / 64.0);
    return 0;
}


// ---- Yukawa kernel (Sec. 3.7) ------------------------------------------------
// The Fourier-space splitting replaces k by sqrt(k^2 + lambda^2) in the
// mollifier psi(k R_l / c) / psi(0) and divides by k^2 + lambda^2:
//   Dhat_l(k) = 4 pi [psi(kk R_{l+1} / c) - psi(kk R_l / c)] / kk^2,  kk^2 = k^2 + lambda^2,
//   What_0(k) = psi(kk / c) That(k),  That the transform of exp(-lambda r)/r cut at R_t,
//   S_l(r)    = 2 / (pi r) int_0^inf psi(kk R_l / c) k sin(k r) / kk^2 dk.
// S_l is evaluated as the Laplace mollifier Phi(r / R_l) / r (its lambda = 0
// value) plus the radial transform of the difference of the integrands, which
// decays fast; the residual is R_l(r) = exp(-lambda r) / r - S_l(r).
namespace {
// psi on [0, X] as a Chebyshev interpolant (psi itself beyond X)
struct PsiProxy {
    const Pswf &psi;
    double X;
    std::vector<double> a;
    PsiProxy(const Pswf &p, double xmax) : psi(p), X(xmax) {
        const int n = std::min(1024, (int)(0.6 * p.c * X) + 100);
        std::vector<double> f(n);
        for (int j = 0; j < n; ++j) f[j] = psi(0.5 * X * (std::cos(M_PI * (j + 0.5) / n) + 1.0));
        a.assign(n, 0.0);
        for (int k = 0; k < n; ++k) {
            double acc = 0.0;
            for (int j = 0; j < n; ++j) acc += f[j] * std::cos(M_PI * k * (j + 0.5) / n);
            a[k] = acc * (k == 0 ? 1.0 : 2.0) / n;
        }
    }
    double operator()(double x) const {
        x = std::fabs(x);
        if (x > X) return psi(x);
        const double u = 2.0 * x / X - 1.0;
        double b1 = 0.0, b2 = 0.0;  // Clenshaw
        for (int k = (int)a.size() - 1; k >= 1; --k) {
            const double b0 = 2.0 * u * b1 - b2 + a[k];
            b2 = b1;
            b1 = b0;
        }
        return u * b1 - b2 + a[0];
    }
    // psi(x1) - psi(x2); the eigen-relation form where both are small
    double diff(double x1, double x2) const {
        if (std::max(std::fabs(x1), std::fabs(x2)) < 0.25) return psi.diff(x1, x2);
        return (*this)(x1) - (*this)(x2);
    }
};

// 1 - e^{-x} (1 + x) without cancellation
double one_minus_exp_1px(double x) {
    if (x < 0.1) {
        double term = 0.5 * x * x, v = 0.0;
        for (int n = 2; n < 20; ++n) {
            v += ((n & 1) ? -1.0 : 1.0) * (n - 1) * term;
            term *= x / (n + 1);
        }
        return v;
    }
    return -std::expm1(-x) - x * std::exp(-x);
}
}  // namespace

int build_yukawa_tables(const Tables &tb, double lam, int nlev, YukawaTables &yt, std::string &err) {
    if (!(lam > 0.0) || nlev < 1 || nlev > kMaxLevel + 1) { err = "Yukawa tables: bad lambda or level count"; return -1; }
    Pswf psi(tb.c);
    const double c = tb.c;
    const int nf = tb.nf, ns = 3 * nf * nf + 1, n0 = tb.n0, nsW = 3 * n0 * n0 + 1;
    // largest psi argument: translation weights, root weights, quadrature
    double X = 4.5;
    X = std::max(X, std::sqrt((4.0 * M_PI * M_PI / 9.0) * (ns - 1) + lam * lam) / c);
    X = std::max(X, std::sqrt(tb.hW * tb.hW * (nsW - 1) + lam * lam) / c);
    X = std::min(X, 40.0);
    PsiProxy ps(psi, X);

    yt.lam = lam;
    yt.nlev = nlev;
    // translation weights (h_l / 2 pi)^3 Dhat_l(h_l |m|), h_l = 2 pi / (3 R_l)
    yt.wl.assign((size_t)nlev * ns, 0.0);
    for (int l = 0; l < nlev; ++l) {
        const double R = std::ldexp(1.0, -l);
        const double h = 2.0 * M_PI / (3.0 * R), sc = std::pow(1.0 / (3.0 * R), 3);
        for (int s = 0; s < ns; ++s) {
            const double k2 = h * h * s + lam * lam, kk = std::sqrt(k2);
            yt.wl[(size_t)l * ns + s] = sc * 4.0 * M_PI * ps.diff(0.5 * kk * R / c, kk * R / c) / k2;
        }
    }
    // root weights
    const double Rt = 1.0 + std::sqrt(3.0), scW = std::pow(tb.hW / (2.0 * M_PI), 3);
    yt.wW.assign(nsW, 0.0);
    for (int s = 0; s < nsW; ++s) {
        const double k = tb.hW * std::sqrt((double)s), k2 = k * k + lam * lam;
        const double xt = lam * Rt;
        double tr;
        if (s == 0) {
            tr = 4.0 * M_PI * one_minus_exp_1px(xt) / (lam * lam);
        } else {
            const double sn = std::sin(0.5 * k * Rt);
            const double num = -k * std::expm1(-xt) + 2.0 * k * std::exp(-xt) * sn * sn - std::exp(-xt) * lam * std::sin(k * Rt);
            tr = 4.0 * M_PI * num / (k * k2);
        }
        yt.wW[s] = scW * ps(std::sqrt(k2) / c) * tr;
    }
    // residual polynomials: q_l(t) = R_l S_l(R_l sqrt t)
    std::vector<double> gx, gw;
    gl_rule(24, gx, gw);
    const int nc = 64;
    std::vector<std::vector<double>> monos(nlev);
    int qdeg = 2;
    for (int l = 0; l < nlev; ++l) {
        const double R = std::ldexp(1.0, -l);
        // panels in k: graded from width lambda near 0 (poles at +-i lambda),
        // then 8 regular panels up to sqrt(k^2 + lambda^2) R / c = 4
        const double x4 = 4.0 * c / R, kmax = x4 > lam ? std::sqrt(x4 * x4 - lam * lam) : 0.0, pw = kmax / 8.0;
        std::vector<double> br{0.0};
        for (double b = lam; b < pw && br.size() < 32; b *= 3.0) br.push_back(b);
        const double b0 = br.back();
        for (int q = 1; q <= 8; ++q) br.push_back(b0 + (kmax - b0) * q / 8.0);
        std::vector<double> kn, gn;  // nodes, weights x integrand without sin(k r)
        for (size_t q = 0; q + 1 < br.size(); ++q) {
            const double a = br[q], hq = br[q + 1] - br[q];
            for (int i = 0; i < 24; ++i) {
                const double k = a + 0.5 * hq * (gx[i] + 1.0), k2 = k * k + lam * lam;
                kn.push_back(k);
                gn.push_back(2.0 / M_PI * 0.5 * hq * gw[i] * (ps(std::sqrt(k2) * R / c) * k / k2 - ps(k * R / c) / k));
            }
        }
        std::vector<double> vals(nc);
        for (int j = 0; j < nc; ++j) {
            const double t = cheb_node01(j, nc), st = std::sqrt(t), r = R * st;
            double acc = 0.0;
            if (st == 0.0) {
                for (size_t i = 0; i < kn.size(); ++i) acc += gn[i] * kn[i];
                vals[j] = tb.psi0_over_c0 + R * acc;
            } else {
                for (size_t i = 0; i < kn.size(); ++i) acc += gn[i] * std::sin(kn[i] * r);
                vals[j] = psi.Phi(st) / st + acc / st;
            }
        }
        // the mollifier carries the transform of psi beyond x = 1 (where psi is
        // below eps but not zero): high Chebyshev modes of size ~1e-3 eps,
        // dropped up to 2e-2 eps S_l(0) in all
        double vmax = 0.0;  // q_l(0), the largest value
        for (double v : vals) vmax = std::max(vmax, std::fabs(v));
        const double tol = std::max(2e-2 * tb.eps * vmax, 1e-15 * tb.psi0_over_c0);
        monos[l] = cheb_to_mono(cheb_fit(vals, tol));
        qdeg = std::max(qdeg, (int)monos[l].size() - 1);
    }
    if (qdeg > kMaxYukawaDegree) { err = "Yukawa residual polynomial degree above 62"; return -1; }
    // rows [degree, c_0 .. c_qdeg]: each level is evaluated at its own degree
    // (large lambda R_l needs high degrees at the coarse levels only)
    yt.qdeg = qdeg;
    yt.qmono.assign((size_t)nlev * (qdeg + 2), 0.0);
    for (int l = 0; l < nlev; ++l) {
        yt.qmono[(size_t)l * (qdeg + 2)] = (double)(monos[l].size() - 1);
        for (size_t d = 0; d < monos[l].size(); ++d) yt.qmono[(size_t)l * (qdeg + 2) + 1 + d] = monos[l][d];
    }
    return 0;
}

// ---- 2D Laplace kernel log r (Sec. 3.7 at lambda = 0, in the plane) -----------
// log r transforms to -2 pi / k^2 in two dimensions, so (psi(0) = 1)
//   Dhat_l(k) = -2 pi [psi(k R_{l+1} / c) - psi(k R_l / c)] / k^2, Dhat_l(0) = -pi (c2 / c0) (R_l^2 - R_{l+1}^2),
// and with h_l = 2 pi / (3 R_l) the weight (h_l / 2 pi)^2 Dhat_l(h_l |m|) is the
// same at every level.  The residual's transform -2 pi (1 - psi(k R / c)) / k^2
// inverts to R_l(r) = F(r / R_l), F(rho) = -int_0^inf (1 - psi(k / c)) J_0(k rho) / k dk;
// the integral of (J_0(t) - [t < 1]) / t over (0, inf) is log 2 - gamma, which
// leaves F(rho) = log rho + G(rho^2) with
//   G(t) = log(K / 2) + gamma - int_0^K (1 - psi(k / c) J_0(k sqrt t)) / k dk,
// psi negligible beyond K = 4 c.  The root window is the kernel cut at
// R_t = 1 + sqrt 2 times psi(k / c):
//   What(k) = psi(k / c) 2 pi (R_t log R_t J_1(k R_t) / k - (1 - J_0(k R_t)) / k^2).
int build_log2d_tables(const Tables &tb, Log2dTables &t2, std::string &err) {
    const int p = tb.p, nf = tb.nf;
    const double c = tb.c;
    Pswf psi(c);
    // translation weights at R = 1: (1/3)^2 Dhat((2 pi / 3) sqrt s)
    t2.w.resize(2 * nf * nf + 1);
    for (int s = 0; s <= 2 * nf * nf; ++s) {
        double dhat;
        if (s == 0) {
            dhat = -M_PI * psi.c2 / psi.c0 * 0.75;
        } else {
            const double k = 2.0 * M_PI / 3.0 * std::sqrt((double)s);
            dhat = -2.0 * M_PI * psi.diff(k / (2.0 * c), k / c) / (k * k);
        }
        t2.w[s] = dhat / 9.0;
    }
    // root window
    const double Rt = 1.0 + std::sqrt(2.0);
    t2.hW = 2.0 * M_PI / (2.0 + Rt);
    t2.n0 = (int)std::ceil(c / t2.hW) + 1;
    if (t2.n0 > kMaxNf) { err = "root mode count above the library limit"; return -1; }
    const int NW = 2 * t2.n0 + 1;
    t2.FWr.assign((size_t)NW * p, 0.0);
    t2.FWi.assign((size_t)NW * p, 0.0);
    for (int mi = 0; mi < NW; ++mi) {
        const int m = mi - t2.n0;
        for (int n = 0; n < p; ++n) {
            std::complex<double> acc = 0.0;
            for (int j = 0; j < p; ++j) {
                // V^{-1}[n][j] = (n ? 2 : 1) / p T_n(t_j), T_n(cos a) = cos(n a)
                const double vinv = (n == 0 ? 1.0 : 2.0) / p * std::cos(n * M_PI * (j + 0.5) / p);
                acc += std::polar(1.0, -0.5 * t2.hW * m * tb.t[j]) * vinv;
            }
            t2.FWr[(size_t)mi * p + n] = acc.real();
            t2.FWi[(size_t)mi * p + n] = acc.imag();
        }
    }
    t2.wW.resize(2 * t2.n0 * t2.n0 + 1);
    const double scW = (t2.hW / (2.0 * M_PI)) * (t2.hW / (2.0 * M_PI));
    for (int s = 0; s <= 2 * t2.n0 * t2.n0; ++s) {
        const double k = t2.hW * std::sqrt((double)s);
        double what;
        if (s == 0)
            what = M_PI * Rt * Rt * (std::log(Rt) - 0.5);
        else
            what = 2.0 * M_PI * (Rt * std::log(Rt) * std::cyl_bessel_j(1.0, k * Rt) / k -
                                 (1.0 - std::cyl_bessel_j(0.0, k * Rt)) / (k * k)) * psi(k / c);
        t2.wW[s] = scW * what;
    }
    // G(t) on [0, 1]: 16 Gauss-Legendre panels of 24 nodes on [0, K], then a
    // Chebyshev interpolant at 64 points in t, cut where its tail is below
    // 1e-3 eps of max(1, |G|)
    const double K = 4.0 * c, gamma = 0.57721566490153286061;
    std::vector<double> gx, gw, kk, wk, ps;
    gl_rule(24, gx, gw);
    const int panels = 16;
    for (int q = 0; q < panels; ++q)
        for (int i = 0; i < 24; ++i) {
            const double k = K / panels * (q + 0.5 * (gx[i] + 1.0));
            kk.push_back(k);
            wk.push_back(0.5 * K / panels * gw[i] / k);
            ps.push_back(psi(k / c));
        }
    auto G = [&](double t) {
        const double r = std::sqrt(t);
        double acc = 0.0;
        for (size_t j = 0; j < kk.size(); ++j) acc += wk[j] * (1.0 - ps[j] * std::cyl_bessel_j(0.0, kk[j] * r));
        return std::log(0.5 * K) + gamma - acc;
    };
    const int nc = 64;
    std::vector<double> vals(nc);
    double gmax = 1.0;
    for (int j = 0; j < nc; ++j) {
        vals[j] = G(cheb_node01(j, nc));
        gmax = std::max(gmax, std::fabs(vals[j]));
    }
    t2.g = cheb_fit(vals, 1e-3 * tb.eps * gmax);
    t2.G0 = G(0.0);
    // the monomial form costs one FMA per degree instead of two; keep it if it
    // reproduces the Chebyshev sum within 1e-4 eps (its coefficients grow with
    // the degree, about 6e7 at the 1e-12 row, where it does not)
    std::vector<double> mono = cheb_to_mono(t2.g);
    double dev = 0.0;
    for (int j = 0; j <= 256; ++j) {
        const double x = -1.0 + j / 128.0;
        double b1 = 0.0, b2 = 0.0, h = 0.0;
        for (int k = (int)t2.g.size() - 1; k >= 1; --k) {
            const double b0 = 2.0 * x * b1 - b2 + t2.g[k];
            b2 = b1;
            b1 = b0;
        }
        for (int k = (int)mono.size() - 1; k >= 0; --k) h = h * x + mono[k];
        dev = std::max(dev, std::fabs(x * b1 - b2 + t2.g[0] - h));
    }
    t2.gmono.clear();
    if (dev <= 1e-4 * tb.eps * gmax) t2.gmono = mono;
    return 0;
}

}  // namespace dmk
