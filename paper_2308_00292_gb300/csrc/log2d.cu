// log2d.cu -- the DMK evaluation pass for the 2D Laplace kernel log r
// (Sec. 3.7 at lambda = 0 in the plane; Steps 0-5 of Sec. 3.4 in two
// dimensions), FP64 throughout.
//
// The tree is the library's 3D builder run on the points lifted to z = 0: the
// builder only creates cells that hold points and only forces splits of
// non-empty cells, so every box lies in the z = 0 layer and the octree is the
// quad-tree of the points (octants 0-3 are the quadrants, colleagues with
// dz = 0 are the 2D colleagues, and the near lists are the 2D ones).
//
// Per box the expansions are p^2 Chebyshev moments / local coefficients and
// (2 nf + 1)^2 plane waves.  At these sizes a box's transforms are a few
// hundred thousand flops, far below a tensor-core tile, so every kernel is a
// block per box on the CUDA cores with the box's arrays in shared memory.
//   k2_moments   Step 2: M[a][b] = sum_j q_j T_a(xi_j) T_b(eta_j) of a leaf
//   k2_c2p       Step 2: parent moments from the children (coefficient shifts)
//   k2_outgoing  Step 3: Phi[m] = sum F[mx][a] F[my][b] M[a][b] (F_out boxes)
//   k2_local     Step 3: p2c of the parent's coefficients, the incoming
//                expansion of the colleagues (translation phases are cube
//                roots of unity), the root window at level 0
//   k2_eval      Step 3: local expansions at the targets
//   k2_near      Step 4-5: residual kernel log(r / R) + G(r^2 / R^2) over the
//                near lists; coincident pairs remove rho S_L(0)
//   k2_finalize  input order; log|x - y| = log S + log|u - v| adds log S times
//                the charge of the non-coincident sources
#include "dmk_internal.h"
#include "dev_util.h"
#include "log2d.h"

#include <algorithm>
#include <cmath>
#include <vector>

namespace dmk {
namespace {

constexpr int kT = 256;                       // threads per block
constexpr int kPer = (kMaxP * kMaxP + kT - 1) / kT;  // p^2 entries per thread

#define L2CK(x)                                                              \
    do {                                                                     \
        cudaError_t e_ = (x);                                                \
        if (e_ != cudaSuccess) {                                             \
            err = std::string("CUDA: ") + cudaGetErrorString(e_);            \
            return DMK_ERR_CUDA;                                             \
        }                                                                    \
    } while (0)

inline unsigned nblk(int64_t n, int t) { return (unsigned)((n + t - 1) / t); }

__device__ __forceinline__ void cell2(const TreeView &tv, int b, int &ix, int &iy) {
    int iz;
    box_decode_d(tv.bkey[b], tv.blevel[b], ix, iy, iz);
}

// Chebyshev polynomials T_0 .. T_{p-1} at x
__device__ __forceinline__ void cheb_row(double x, int p, double *T) {
    T[0] = 1.0;
    if (p > 1) T[1] = x;
    for (int n = 2; n < p; ++n) T[n] = 2.0 * x * T[n - 1] - T[n - 2];
}

// ---- Step 2: moments of the source leaves -----------------------------------
__global__ void __launch_bounds__(kT) k2_moments(TreeView tv, Log2dDev d, double *mom) {
    const int b = blockIdx.x;
    if (!(tv.bflags[b] & BF_LEAF) || tv.bnsrc[b] == 0) return;
    __shared__ double Tx[32][kMaxP], Ty[32][kMaxP];
    const int p = d.p, pp = p * p, tid = threadIdx.x;
    int ix, iy;
    cell2(tv, b, ix, iy);
    const double R = level_R(tv.blevel[b]), cx = (ix + 0.5) * R, cy = (iy + 0.5) * R;
    const double s2R = (double)(2u << tv.blevel[b]);  // 2 / R, a power of two
    double acc[kPer];
#pragma unroll
    for (int j = 0; j < kPer; ++j) acc[j] = 0.0;
    const int s0 = tv.bstart[b], n = tv.bcount[b];
    for (int c0 = 0; c0 < n; c0 += 32) {
        if (tid < 64) {  // warp 0 the x rows (times the charge), warp 1 the y rows
            const int i = tid & 31, k = s0 + c0 + i;
            double *row = tid < 32 ? Tx[i] : Ty[i];
            if (c0 + i < n) {
                // 2 (x - c) / R, an exact scaling
                cheb_row(tid < 32 ? (tv.ux[k] - cx) * s2R : (tv.uy[k] - cy) * s2R, p, row);
                if (tid < 32) {
                    const double qk = tv.q[k];
                    for (int a = 0; a < p; ++a) row[a] *= qk;  // q_j T_a(xi_j)
                }
            } else {
                for (int a = 0; a < p; ++a) row[a] = 0.0;
            }
        }
        __syncthreads();
#pragma unroll
        for (int j = 0; j < kPer; ++j) {
            const int e = tid + j * kT;
            if (e < pp) {
                const int a = e / p, bb = e - a * p;
                double s = 0.0;
                for (int i = 0; i < 32; ++i) s += Tx[i][a] * Ty[i][bb];
                acc[j] += s;
            }
        }
        __syncthreads();
    }
#pragma unroll
    for (int j = 0; j < kPer; ++j) {
        const int e = tid + j * kT;
        if (e < pp) mom[(size_t)b * pp + e] = acc[j];
    }
}

// ---- Step 2: parent moments from the children ------------------------------
// T_n((xi + s) / 2) = sum_m A_s[n][m] T_m(xi): M_P[n][n'] = sum A_sx[n][k] A_sy[n'][k'] M_C[k][k']
__global__ void __launch_bounds__(kT) k2_c2p(TreeView tv, Log2dDev d, int lstart, double *mom) {
    const int b = lstart + blockIdx.x;
    if ((tv.bflags[b] & BF_LEAF) || tv.bnsrc[b] == 0) return;
    __shared__ double MC[kMaxP * kMaxP], Y[kMaxP * kMaxP];
    const int p = d.p, pp = p * p, tid = threadIdx.x;
    // M_P = sum_C A_sx(C) (M_C A_sy(C)^T): the children with the same x half share
    // A_sx, so Y_C = M_C A_sy(C)^T is summed per x half (in the threads' registers,
    // which own the same entries of Y and of M_P) and A_sx is applied once per half
    double ys[2][kPer];
#pragma unroll
    for (int j = 0; j < kPer; ++j) ys[0][j] = ys[1][j] = 0.0;
    const uint8_t mask = tv.bcmask[b];
    int ci = tv.bchild0[b], halves = 0;
    for (int oc = 0; oc < 8; ++oc) {
        if (!(mask & (1u << oc))) continue;
        const int c = ci++;
        if (tv.bnsrc[c] == 0) continue;
        const int hx = oc & 1;
        halves |= 1 << hx;
        const double *Ay = d.A + (size_t)((oc >> 1) & 1) * pp;
        __syncthreads();
        for (int e = tid; e < pp; e += kT) MC[e] = mom[(size_t)c * pp + e];
        __syncthreads();
        // Y[k][n'] = sum_k' A_sy[n'][k'] M_C[k][k'] (A_s[n][m] = 0 for m > n)
#pragma unroll
        for (int j = 0; j < kPer; ++j) {
            const int e = tid + j * kT;
            if (e < pp) {
                const int k = e / p, n2 = e - k * p;
                double s = 0.0;
                for (int k2 = 0; k2 <= n2; ++k2) s += Ay[n2 * p + k2] * MC[k * p + k2];
                if (hx) ys[1][j] += s;
                else ys[0][j] += s;
            }
        }
    }
    double acc[kPer];
#pragma unroll
    for (int j = 0; j < kPer; ++j) acc[j] = 0.0;
    for (int hx = 0; hx < 2; ++hx) {
        if (!(halves & (1 << hx))) continue;
        const double *Ax = d.A + (size_t)hx * pp;
        __syncthreads();
#pragma unroll
        for (int j = 0; j < kPer; ++j) {
            const int e = tid + j * kT;
            if (e < pp) Y[e] = hx ? ys[1][j] : ys[0][j];
        }
        __syncthreads();
#pragma unroll
        for (int j = 0; j < kPer; ++j) {
            const int e = tid + j * kT;
            if (e < pp) {
                const int n1 = e / p, n2 = e - n1 * p;
                double s = 0.0;
                for (int k = 0; k <= n1; ++k) s += Ax[n1 * p + k] * Y[k * p + n2];
                acc[j] += s;
            }
        }
    }
#pragma unroll
    for (int j = 0; j < kPer; ++j) {
        const int e = tid + j * kT;
        if (e < pp) mom[(size_t)b * pp + e] = acc[j];
    }
}

// The moments are real, so the plane waves are Hermitian, Phi[-m] = conj(Phi[m]),
// and only the half spectrum m_x = 0 ... nh (nh = (N - 1) / 2, rows nh + 1 of N
// complex values) is formed, stored and translated.  F[m][a] approximates
// exp(-i theta m xi) by T_0 ... T_{p-1}: its cosine part is even and its sine
// part odd, so F is real for even a and imaginary for odd a (the other part
// is rounding, taken as zero), and each complex product is a real one.

// Phi[mx][my] = sum_a sum_b F[mx][a] F[my][b] M[a][b], mx = 0 ... nh, into phi
// ((nh + 1) x N complex, interleaved); M and the workspace Y ((nh + 1) x p
// complex) in shared memory
__device__ void pw_from_moments(const double *M, const double *Fr, const double *Fi, int p, int N, double *Yr,
                                double *Yi, double *phi) {
    const int tid = threadIdx.x, nh = (N - 1) / 2, NH = nh + 1;
    // Y[mx][b] = sum_a F[mx][a] M[a][b]: real part over even a, imaginary over odd a
    for (int e = tid; e < NH * p; e += kT) {
        const int mx = e / p, bb = e - mx * p;
        const double *fr = Fr + (size_t)(mx + nh) * p, *fi = Fi + (size_t)(mx + nh) * p;
        double sr = 0.0, si = 0.0;
        for (int a = 0; a < p; a += 2) sr += fr[a] * M[a * p + bb];
        for (int a = 1; a < p; a += 2) si += fi[a] * M[a * p + bb];
        Yr[e] = sr;
        Yi[e] = si;
    }
    __syncthreads();
    // Phi[mx][my] = sum_b F[my][b] Y[mx][b]: F[my][b] = Fr (b even) or i Fi (b odd),
    // and F[-my] = conj(F[my]).  With E = sum_{b even} Fr[m][b] Y[mx][b] and
    // O = sum_{b odd} Fi[m][b] Y[mx][b] (complex, m >= 0):
    // Phi[mx][m] = E + i O and Phi[mx][-m] = E - i O
    for (int e = tid; e < NH * NH; e += kT) {
        const int mx = e / NH, m = e - mx * NH;
        const double *fr = Fr + (size_t)(m + nh) * p, *fi = Fi + (size_t)(m + nh) * p, *yr = Yr + mx * p,
                     *yi = Yi + mx * p;
        double er = 0.0, ei = 0.0, orr = 0.0, oi = 0.0;
        for (int bb = 0; bb < p; bb += 2) {
            er += fr[bb] * yr[bb];
            ei += fr[bb] * yi[bb];
        }
        for (int bb = 1; bb < p; bb += 2) {
            orr += fi[bb] * yr[bb];
            oi += fi[bb] * yi[bb];
        }
        double *pp = phi + 2 * (mx * N + nh + m), *pm = phi + 2 * (mx * N + nh - m);
        pp[0] = er - oi;
        pp[1] = ei + orr;
        if (m > 0) {
            pm[0] = er + oi;
            pm[1] = ei - orr;
        }
    }
    __syncthreads();
}

// c[n][n'] = Re sum_{all m} conj(F[mx][n]) conj(F[my][n']) Psi[mx][my] from the
// half spectrum Psi ((nh + 1) x N complex interleaved, the rows mx >= 1 already
// doubled: the terms at m and -m are conjugate; overwritten); the workspace Z
// (p x (nh + 1), two real arrays) in shared memory
__device__ void coef_from_pw(double *Psi, const double *Fr, const double *Fi, int p, int N, double *Zr,
                             double *Zi, double *acc /* kPer per thread */) {
    const int tid = threadIdx.x, nh = (N - 1) / 2, NH = nh + 1;
    // Z[n][my] = sum_mx conj(F[mx][n]) Psi[mx][my]: conj(F) = Fr (n even) or -i Fi (n odd).
    // The second contraction needs only Zs[n][m] = Re Z[n][m] + Re Z[n][-m] (n' even:
    // Fr[-m] = Fr[m]) and Za[n][m] = Im Z[n][m] - Im Z[n][-m] (n' odd: Fi[-m] = -Fi[m]),
    // m = 0 ... nh (Zs[n][0] = Re Z[n][0], Za[n][0] = 0).  So Psi's columns are first
    // replaced in place by their sums (column +m) and differences (column -m), m >= 1,
    // and each of Zs, Za is one real contraction over mx.  Stored in Zr and Zi as
    // p x (nh + 1).
    for (int e = tid; e < NH * nh; e += kT) {
        const int mx = e / nh, m = e - mx * nh + 1;
        double *pp = Psi + 2 * (mx * N + nh + m), *pm = Psi + 2 * (mx * N + nh - m);
        const double ar = pp[0], ai = pp[1], br = pm[0], bi = pm[1];
        pp[0] = ar + br;
        pp[1] = ai + bi;
        pm[0] = ar - br;
        pm[1] = ai - bi;
    }
    __syncthreads();
    for (int e = tid; e < p * NH; e += kT) {
        const int n = e / NH, m = e - n * NH;
        const double *ps = Psi + 2 * (nh + m), *pa = Psi + 2 * (nh - m);
        double zs = 0.0, za = 0.0;
        if (!(n & 1)) {
            for (int mx = 0; mx < NH; ++mx) {
                const double f = Fr[(mx + nh) * p + n];
                zs += f * ps[2 * mx * N];
                za += f * pa[2 * mx * N + 1];
            }
        } else {
            for (int mx = 0; mx < NH; ++mx) {
                const double f = Fi[(mx + nh) * p + n];
                zs += f * ps[2 * mx * N + 1];
                za -= f * pa[2 * mx * N];
            }
        }
        Zr[e] = zs;
        Zi[e] = m ? za : 0.0;
    }
    __syncthreads();
    // c[n][n'] = Re sum_my conj(F[my][n']) Z[n][my] = sum_m Fr[m][n'] Zs[n][m] (n' even)
    // or sum_m Fi[m][n'] Za[n][m] (n' odd), m = 0 ... nh
#pragma unroll
    for (int j = 0; j < kPer; ++j) {
        const int e = tid + j * kT;
        if (e < p * p) {
            const int n = e / p, n2 = e - n * p;
            const double *F = ((n2 & 1) ? Fi : Fr) + (size_t)nh * p + n2, *Z = ((n2 & 1) ? Zi : Zr) + n * NH;
            double s = 0.0;
            for (int m = 0; m < NH; ++m) s += F[m * p] * Z[m];
            acc[j] += s;
        }
    }
    __syncthreads();
}

// ---- Step 3: outgoing expansions of the F_out boxes -------------------------
__global__ void __launch_bounds__(kT) k2_outgoing(TreeView tv, Log2dDev d, const double *mom, double *phi) {
    const int b = blockIdx.x;
    if (!(tv.bflags[b] & BF_FOUT)) return;
    extern __shared__ double sm[];
    const int p = d.p, pp = p * p, N = d.N1, NH = d.nf + 1;
    double *M = sm, *Yr = M + pp, *Yi = Yr + NH * p, *P = Yi + NH * p;
    for (int e = threadIdx.x; e < pp; e += kT) M[e] = mom[(size_t)b * pp + e];
    __syncthreads();
    pw_from_moments(M, d.Fr, d.Fi, p, N, Yr, Yi, P);
    double *out = phi + (size_t)tv.bslot[b] * 2 * NH * N;
    for (int e = threadIdx.x; e < 2 * NH * N; e += kT) out[e] = P[e];
}

// ---- Step 3: local expansions of the boxes of one level ---------------------
__global__ void __launch_bounds__(kT) k2_local(TreeView tv, Log2dDev d, int level, int lstart, const double *mom,
                                               const double *phi, double *loc) {
    const int b = lstart + blockIdx.x;
    if (tv.bntgt[b] == 0) return;
    extern __shared__ double sm[];
    const int p = d.p, pp = p * p, N = d.N1, NW = d.NW, NM = N > NW ? N : NW;
    // Psi holds a half spectrum, (NM + 1) / 2 rows of NM
    double *CP = sm, *Y = CP + pp, *Psi = Y + pp, *Zr = Psi + NM * (NM + 1), *Zi = Zr + p * NM;
    const int tid = threadIdx.x;
    double acc[kPer];
#pragma unroll
    for (int j = 0; j < kPer; ++j) acc[j] = 0.0;
    int ix, iy;
    cell2(tv, b, ix, iy);
    // the parent's expansion in this box's coordinates: c[k][k'] = sum A_sx[n][k] A_sy[n'][k'] c_P[n][n']
    if (level > 0) {
        const int P = tv.bparent[b];
        const double *Ax = d.A + (size_t)(ix & 1) * pp, *Ay = d.A + (size_t)(iy & 1) * pp;
        for (int e = tid; e < pp; e += kT) CP[e] = loc[(size_t)P * pp + e];
        __syncthreads();
        for (int e = tid; e < pp; e += kT) {  // Y[n][k'] = sum_n' A_sy[n'][k'] c_P[n][n'] (A_s[n'][k'] = 0 for k' > n')
            const int n = e / p, k2 = e - n * p;
            double s = 0.0;
            for (int n2 = k2; n2 < p; ++n2) s += Ay[n2 * p + k2] * CP[n * p + n2];
            Y[e] = s;
        }
        __syncthreads();
#pragma unroll
        for (int j = 0; j < kPer; ++j) {
            const int e = tid + j * kT;
            if (e < pp) {
                const int k = e / p, k2 = e - k * p;
                double s = 0.0;
                for (int n = k; n < p; ++n) s += Ax[n * p + k] * Y[n * p + k2];
                acc[j] += s;
            }
        }
        __syncthreads();
    }
    // incoming plane waves from the F_out colleagues: w(|m|^2) omega^{m . delta}
    if (tv.bflags[b] & BF_FIN) {
        const int nf = d.nf, NH = nf + 1;
        __shared__ const double *s_ph[9];  // the colleague at (dx, dy) = (c / 3 - 1, c % 3 - 1), or null
        if (tid < 9) {
            const int S = tv.bcol[(size_t)b * 27 + 9 * (tid / 3) + 3 * (tid % 3) + 1];
            s_ph[tid] = (S >= 0 && (tv.bflags[S] & BF_FOUT)) ? phi + (size_t)tv.bslot[S] * 2 * NH * N : nullptr;
        }
        __syncthreads();
        // delta = c_B - c_S = -(dx, dy) R: the phase exp(i (2 pi / 3) m . delta / R) is a
        // cube root of unity, c + i s with c in {1, -1/2} and s in {0, +-sqrt(3)/2}, so
        // Psi = w (U + i V) with U = sum c Phi_S and V = sum s Phi_S; half spectrum
        // mx = 0 ... nf, the rows mx >= 1 doubled
        for (int e = tid; e < NH * N; e += kT) {
            const int mx = e / N, my = e % N - nf;
            double ur = 0.0, ui = 0.0, vr = 0.0, vi = 0.0;
#pragma unroll
            for (int c = 0; c < 9; ++c) {
                const double *ph = s_ph[c];
                if (!ph) continue;
                const int dx = c / 3 - 1, dy = c % 3 - 1;
                int r = (-(mx * dx + my * dy)) % 3;
                if (r < 0) r += 3;
                const double cr = r == 0 ? 1.0 : -0.5,
                             ci = r == 0 ? 0.0 : (r == 1 ? 0.86602540378443864676 : -0.86602540378443864676);
                const double pr = ph[2 * e], pi = ph[2 * e + 1];
                ur = fma(cr, pr, ur);
                ui = fma(cr, pi, ui);
                vr = fma(ci, pr, vr);
                vi = fma(ci, pi, vi);
            }
            const double w = (mx ? 2.0 : 1.0) * d.w[mx * mx + my * my];
            Psi[2 * e] = w * (ur - vi);
            Psi[2 * e + 1] = w * (ui + vr);
        }
        __syncthreads();
        coef_from_pw(Psi, d.Fr, d.Fi, p, N, Zr, Zi, acc);
    }
    // the windowed root kernel over the unit square
    if (level == 0 && tv.bnsrc[b] > 0) {
        for (int e = tid; e < pp; e += kT) CP[e] = mom[(size_t)b * pp + e];
        __syncthreads();
        pw_from_moments(CP, d.FWr, d.FWi, p, NW, Zr, Zi, Psi);
        const int n0 = d.n0;
        for (int e = tid; e < (n0 + 1) * NW; e += kT) {
            const int mx = e / NW, my = e % NW - n0;
            const double w = (mx ? 2.0 : 1.0) * d.wW[mx * mx + my * my];
            Psi[2 * e] *= w;
            Psi[2 * e + 1] *= w;
        }
        __syncthreads();
        coef_from_pw(Psi, d.FWr, d.FWi, p, NW, Zr, Zi, acc);
    }
#pragma unroll
    for (int j = 0; j < kPer; ++j) {
        const int e = tid + j * kT;
        if (e < pp) loc[(size_t)b * pp + e] = acc[j];
    }
}

// ---- Step 3: local expansions at the targets ---------------------------------
__global__ void __launch_bounds__(kT) k2_eval(TreeView tv, Log2dDev d, const int32_t *pleaf, const double *loc,
                                              double *ufar) {
    const int64_t k = (int64_t)blockIdx.x * kT + threadIdx.x;
    if (k >= tv.n) return;
    if (!(tv.pflag[k] & 2)) { ufar[k] = 0.0; return; }
    const int b = pleaf[k], p = d.p;
    int ix, iy;
    cell2(tv, b, ix, iy);
    const double R = level_R(tv.blevel[b]);
    const double s2R = (double)(2u << tv.blevel[b]);  // 2 / R, a power of two: exact scaling
    const double xi = (tv.ux[k] - (ix + 0.5) * R) * s2R, eta = (tv.uy[k] - (iy + 0.5) * R) * s2R;
    double Ty[kMaxP];
    cheb_row(eta, p, Ty);
    const double *c = loc + (size_t)b * p * p;
    double acc = 0.0, t0 = 1.0, t1 = xi;
    for (int a = 0; a < p; ++a) {
        const double ta = a == 0 ? 1.0 : (a == 1 ? xi : 2.0 * xi * t1 - t0);
        if (a >= 2) { t0 = t1; t1 = ta; }
        double s = 0.0;
        for (int bb = 0; bb < p; ++bb) s += c[a * p + bb] * Ty[bb];
        acc += ta * s;
    }
    ufar[k] = acc;
}

// ---- Steps 4-5: residual kernels over the near lists ------------------------
// A block of kNW warps per target leaf.  The sources of the leaf's near list are
// staged in shared memory, kCH at a time, with FP32 offsets from the leaf's
// centre for screening.  A warp takes kS targets at a time: its lanes screen
// 32 candidates per step in FP32 against a threshold that cannot reject a
// pair inside the support, append the survivors (target slot, source) to one
// queue, and evaluate the queue 32 pairs at a time in FP64 into per-lane,
// per-slot sums in shared memory, so that the FP64 pipe (the bound: GB300
// issues FP64 at about 1/62 of its FP32 rate) sees only pairs that are evaluated,
// with one partly filled step per kS targets.  The lanes' sums of a target
// are then added in a fixed butterfly order (results do not depend on timing).
//
// Per pair inside the support (t = r^2 / R^2 < 1, exact since 1/R^2 = 4^l):
//   (1/2) log t + G(2t - 1),
// with log t = e ln 2 + log m, t = m 2^e, m in [1, 2), by Tang's table-driven
// method: log m = -log F_k + log1p(m F_k - 1), F_k ~ 1 / (1 + (k + 1/2)/256) for
// the leading 8 bits k of m's fraction, so |m F_k - 1| <= 2^-9, and log1p by
// its Taylor series to degree 5 (remainder below 5e-18).  The tables hold
// -(1/2) log F_k and g_0 - (e/2) ln 2 (e = -1 ... -255; smaller t, and
// subnormal r^2, take CUDA's log).  G by Horner in monomials (MONO) or by
// Clenshaw in Chebyshev polynomials.  Coincident pairs remove q S_L(0) and
// count their charge for the log S term.
//
// MIX (the mixed path, eps >= 1e-7): the same staging, screening and queue;
// each pair in FP32 from hi/lo offsets in leaf units (the separation keeps its
// relative accuracy however close the points), logf, and Clenshaw on G's
// Chebyshev series cut for FP32; per-lane sums (hi, lo) by TwoSum.  Pairs with
// r^2 below 2^-100 leaf units squared (coincident ones among them) take FP64.
constexpr int kNW = 4, kNT = 32 * kNW;  // warps, threads per block
constexpr int kCH = 512;                // sources staged per chunk
constexpr int kS = 4;                   // targets in flight per warp (one queue, one flush)
constexpr int kLvl = 32;                // level table (levels 0 .. kMaxLevel, then the no-source mark)
constexpr int kNoSrc = kLvl - 1;
static_assert(kMaxLevel < kNoSrc, "level table");

template <bool MONO, bool MIX>
__global__ void __launch_bounds__(kNT) k2_near(TreeView tv, Log2dDev d, const int32_t *tleaves, const int32_t *nl_off,
                                               const int32_t *nl_src, double *unear, double *qco,
                                               unsigned long long *n_inside) {
    __shared__ double sx[kCH], sy[kCH], sq[kCH];
    __shared__ float sox[kCH], soy[kCH];
    // MIX: leaf-unit offsets from the leaf's centre as FP32 (hi, lo) pairs, FP32 charges
    __shared__ float sxh[MIX ? kCH : 1], sxl[MIX ? kCH : 1], syh[MIX ? kCH : 1], syl[MIX ? kCH : 1],
        sqf[MIX ? kCH : 1], thl[MIX ? kNW : 1][kS][4];
    __shared__ float4 gf4[MIX ? 16 : 1];
    __shared__ float l_R2f[MIX ? kLvl : 1], l_s2f[MIX ? kLvl : 1], l_S0f[MIX ? kLvl : 1];
    __shared__ uint8_t slev[kCH];
    __shared__ uint16_t queue[kNW][64];           // (slot << 10) | source
    __shared__ double accS[kNW][kS][32], qcS[kNW][kS][32], txS[kNW][kS], tyS[kNW][kS];
    __shared__ double lgF[256], lgL[256], lgE[256], g[64];
    __shared__ double l_x2[kLvl], l_S0[kLvl];
    __shared__ long long l_R2[kLvl];
    __shared__ float l_thr[kLvl];
    __shared__ unsigned s_inside;
    const int i = blockIdx.x, T = tleaves[i], tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
    const int gdeg = d.gdeg, a = tv.blevel[T];
    int ix, iy;
    cell2(tv, T, ix, iy);
    const double Bt = level_R(a), cx = (ix + 0.5) * Bt, cy = (iy + 0.5) * Bt;
    for (int e = tid; e < 256; e += kNT) {
        lgF[e] = d.lgF[e];
        lgL[e] = d.lgL[e];
        lgE[e] = d.lgE[e];
    }
    for (int e = tid; e <= gdeg; e += kNT) g[e] = d.g[e];
    if (MIX)
        for (int e = tid; e < d.gcn4; e += kNT) gf4[e] = reinterpret_cast<const float4 *>(d.gcf)[e];
    if (MIX && tid < kLvl) {
        // leaf units: r^2 < R_l^2 as r_leaf^2 < 4^(a - l), t = r_leaf^2 4^(l - a)
        const bool ok = tid <= kMaxLevel;
        l_R2f[tid] = ok ? ldexpf(1.0f, 2 * (a - tid)) : -1.0f;
        l_s2f[tid] = ok ? ldexpf(1.0f, 2 * (tid - a)) : 0.0f;
        l_S0f[tid] = ok ? (float)(log(level_R(tid)) - d.G0) : 0.0f;
    }
    if (tid < kLvl) {
        if (tid <= kMaxLevel) {
            const double R = level_R(tid);
            l_x2[tid] = 2.0 / (R * R);                // x = 2 t - 1 = r^2 (2 / R^2) - 1
            l_S0[tid] = log(R) - d.G0;                // mollified kernel at r = 0
            l_R2[tid] = __double_as_longlong(R * R);  // r^2 < R^2 compared as bit patterns
            // The FP32 offsets from the leaf's centre are off by at most
            // 2^-24 (|x_t - c| + |x_s - c|) + 2^-24 |dx| per axis, below
            // 2^-24 (4 R + B_t) for a pair inside the support; 2^-21 (4 R + B_t)
            // per axis and the relative factor cover that and the rounding of
            // the three FP32 operations with room.
            const double rr = R + (4.0 * R + Bt) * 0x1p-21;
            l_thr[tid] = __double2float_ru(rr * rr * (1.0 + 0x1p-20));
        } else {
            l_x2[tid] = l_S0[tid] = 0.0;
            l_R2[tid] = 0;
            l_thr[tid] = -1.0f;  // rejects every candidate
        }
    }
    if (tid == 0) s_inside = 0;
    const int t0 = tv.bstart[T], nt = tv.bcount[T];
    uint16_t *qw = queue[w];
    unsigned inside = 0;  // pairs inside the support evaluated by this thread
    const unsigned below = (1u << lane) - 1u;

    const double rBt = 1.0 / Bt;  // 2^a, exact
    // MIX: one queued pair in FP32 (separations from the hi/lo offsets keep their
    // relative accuracy however close the points), the lane's sums of the slot
    // an unevaluated FP32 pair (hi, lo) updated by TwoSum
    auto pair_mix = [&](int e) {
        const int j = e & 1023, sl = e >> 10;
        float2 &acc = reinterpret_cast<float2 *>(&accS[w][sl][0])[lane];
        const float dx = (thl[w][sl][0] - sxh[j]) + (thl[w][sl][1] - sxl[j]);
        const float dy = (thl[w][sl][2] - syh[j]) + (thl[w][sl][3] - syl[j]);
        const float r2 = fmaf(dy, dy, dx * dx);
        const int l = slev[j];
        if (!(r2 < l_R2f[l])) return;  // outside the support (or NaN)
        ++inside;
        float term;
        if (r2 < 0x1p-100f) {
            // coincident, or so close that r^2 leaves the FP32 range: FP64
            const double ddx = txS[w][sl] - sx[j], ddy = tyS[w][sl] - sy[j], r2d = fma(ddy, ddy, ddx * ddx);
            if (r2d == 0.0) {
                qcS[w][sl][lane] += sq[j];
                term = -sqf[j] * l_S0f[l];
            } else {
                term = (float)(sq[j] * (0.5 * log(r2d * (0.5 * l_x2[l])) + d.G0));
            }
        } else {
            const float t = r2 * l_s2f[l], x2 = fmaf(4.0f, t, -2.0f);  // 2 x, x = 2 t - 1
            // Clenshaw, four coefficients per shared-memory load
            float b1 = 0.0f, b2 = 0.0f, b0;
            for (int gi = d.gcn4 - 1; gi >= 1; --gi) {
                const float4 c = gf4[gi];
                b0 = fmaf(x2, b1, c.w - b2), b2 = b1, b1 = b0;
                b0 = fmaf(x2, b1, c.z - b2), b2 = b1, b1 = b0;
                b0 = fmaf(x2, b1, c.y - b2), b2 = b1, b1 = b0;
                b0 = fmaf(x2, b1, c.x - b2), b2 = b1, b1 = b0;
            }
            const float4 c = gf4[0];
            b0 = fmaf(x2, b1, c.w - b2), b2 = b1, b1 = b0;
            b0 = fmaf(x2, b1, c.z - b2), b2 = b1, b1 = b0;
            b0 = fmaf(x2, b1, c.y - b2), b2 = b1, b1 = b0;
            const float G = fmaf(0.5f * x2, b1, c.x - b2);
            term = sqf[j] * fmaf(0.5f, logf(t), G);
        }
        const float sum = acc.x + term, bv = sum - acc.x;
        acc.y += (acc.x - (sum - bv)) + (term - bv);
        acc.x = sum;
    };

    // one queued pair (target slot, staged source) into the lane's sums of the slot
    auto pair = [&](int e) {
        if (MIX) {
            pair_mix(e);
            return;
        }
        const int j = e & 1023, sl = e >> 10;
        double &acc = accS[w][sl][lane], &qc = qcS[w][sl][lane];
        const double dx = txS[w][sl] - sx[j], dy = tyS[w][sl] - sy[j];
        const double r2 = fma(dy, dy, dx * dx);
        const int l = slev[j];
        const long long rb = __double_as_longlong(r2);
        if (!(rb < l_R2[l])) return;  // outside the support (or NaN)
        ++inside;
        const double q = sq[j];
        if (rb == 0) {
            acc = fma(-q, l_S0[l], acc);
            qc += q;
            return;
        }
        const double x = fma(r2, l_x2[l], -1.0);
        double G, b2 = 0.0;  // G(x) = G x + g_0 (monomials) or x b_1 - b_2 + g_0 (Clenshaw, b_1 in G)
        if (MONO) {
            G = g[gdeg];
            for (int n = gdeg - 1; n >= 1; --n) G = fma(G, x, g[n]);
        } else {
            const double x2 = 2.0 * x;
            G = 0.0;
            for (int n = gdeg; n >= 1; --n) {
                const double b0 = fma(x2, G, g[n] - b2);
                b2 = G;
                G = b0;
            }
        }
        const int hi = __double2hiint(r2), be = (hi >> 20) & 0x7ff;
        const int et = be - 1023 + 2 * l;  // exponent of t = r^2 4^l
        double s;                          // g_0 + (1/2) log t
        if (be != 0 && et >= -255) {
            const int k = (hi >> 12) & 0xff;
            const double m = __hiloint2double((hi & 0x000fffff) | 0x3ff00000, __double2loint(r2));
            const double r = fma(m, lgF[k], -1.0);
            double h = fma(r, 0.1, -0.125);  // (1/2) log1p(r) = r (1/2 - r/4 + r^2/6 - r^3/8 + r^4/10)
            h = fma(h, r, 1.0 / 6.0);
            h = fma(h, r, -0.25);
            h = fma(h, r, 0.5);
            s = lgE[-et] + (lgL[k] + h * r);
        } else {
            s = g[0] + 0.5 * log(r2 * (0.5 * l_x2[l]));
        }
        const double v = MONO ? fma(G, x, s) : fma(x, G, s - b2);
        acc = fma(q, v, acc);
    };

    const int li0 = nl_off[i], li1 = nl_off[i + 1];
    int nch = 0, chunk = 0;  // sources staged, chunks processed (block-uniform)
    auto process = [&]() {
        __syncthreads();
        // warp w takes the targets w + kNW (s + kS g), s = 0 ... kS - 1, as group g
        for (int k0 = w; k0 < nt; k0 += kNW * kS) {
#pragma unroll
            for (int sl = 0; sl < kS; ++sl) accS[w][sl][lane] = qcS[w][sl][lane] = 0.0;
            if (lane < kS && k0 + kNW * lane < nt) {
                const double xt = tv.ux[t0 + k0 + kNW * lane], yt = tv.uy[t0 + k0 + kNW * lane];
                txS[w][lane] = xt;
                tyS[w][lane] = yt;
                if (MIX) {
                    const double ox = (xt - cx) * rBt, oy = (yt - cy) * rBt;
                    const float hx = (float)ox, hy = (float)oy;
                    thl[w][lane][0] = hx;
                    thl[w][lane][1] = (float)(ox - hx);
                    thl[w][lane][2] = hy;
                    thl[w][lane][3] = (float)(oy - hy);
                }
            }
            __syncwarp();
            int qn = 0;
            for (int sl = 0; sl < kS; ++sl) {
                const int k = k0 + kNW * sl;
                if (k >= nt || !(tv.pflag[t0 + k] & 2)) continue;
                const float tx = (float)(txS[w][sl] - cx), ty = (float)(tyS[w][sl] - cy);
                for (int j0 = 0; j0 < nch; j0 += 32) {
                    const int j = j0 + lane;
                    bool in = false;
                    if (j < nch) {
                        const float ex = tx - sox[j], ey = ty - soy[j];
                        in = fmaf(ey, ey, ex * ex) <= l_thr[slev[j]];
                    }
                    const unsigned m = __ballot_sync(0xffffffffu, in);
                    if (in) qw[qn + __popc(m & below)] = (uint16_t)((sl << 10) | j);
                    qn += __popc(m);
                    if (qn >= 32) {
                        __syncwarp();
                        pair(qw[lane]);
                        qn -= 32;
                        __syncwarp();
                        if (lane < qn) qw[lane] = qw[32 + lane];
                        __syncwarp();
                    }
                }
            }
            __syncwarp();
            if (lane < qn) pair(qw[lane]);
            __syncwarp();
            for (int sl = 0; sl < kS; ++sl) {
                const int k = k0 + kNW * sl, pk = t0 + k;
                if (k >= nt || !(tv.pflag[pk] & 2)) continue;
                double acc, qc = qcS[w][sl][lane];
                if (MIX) {
                    float2 a2 = reinterpret_cast<const float2 *>(&accS[w][sl][0])[lane];
                    for (int o = 16; o > 0; o >>= 1) {
                        const float oh = __shfl_xor_sync(0xffffffffu, a2.x, o),
                                    ol = __shfl_xor_sync(0xffffffffu, a2.y, o);
                        const float sum = a2.x + oh, bv = sum - a2.x;
                        a2.y = (a2.y + ol) + ((a2.x - (sum - bv)) + (oh - bv));
                        a2.x = sum;
                    }
                    acc = (double)a2.x + (double)a2.y;
                } else {
                    acc = accS[w][sl][lane];
                    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
                }
                // coincident sources (the target itself among them) are rare: one
                // lane's charge is taken as it is, more are summed like acc
                const unsigned mq = __ballot_sync(0xffffffffu, __double_as_longlong(qc) != 0);
                if (__popc(mq) > 1) {
                    for (int o = 16; o > 0; o >>= 1) qc += __shfl_xor_sync(0xffffffffu, qc, o);
                } else {
                    qc = __shfl_sync(0xffffffffu, qc, mq ? __ffs(mq) - 1 : 0);
                }
                if (lane == 0) {
                    unear[pk] = chunk ? unear[pk] + acc : acc;
                    qco[pk] = chunk ? qco[pk] + qc : qc;
                }
            }
            __syncwarp();
        }
        __syncthreads();
        nch = 0;
        ++chunk;
    };
    for (int li = li0; li < li1; ++li) {
        const int S = nl_src[li], s0 = tv.bstart[S], ns = tv.bcount[S], l = tv.blevel[S];
        for (int o = 0; o < ns;) {
            const int take = min(ns - o, kCH - nch);
            for (int e = tid; e < take; e += kNT) {
                const int ks = s0 + o + e, js = nch + e;
                const double xs = tv.ux[ks], ys = tv.uy[ks];
                sx[js] = xs;
                sy[js] = ys;
                sq[js] = tv.q[ks];
                sox[js] = (float)(xs - cx);
                soy[js] = (float)(ys - cy);
                slev[js] = (uint8_t)((tv.pflag[ks] & 1) ? l : kNoSrc);
                if (MIX) {
                    const double ox = (xs - cx) * rBt, oy = (ys - cy) * rBt;
                    const float hx = (float)ox, hy = (float)oy;
                    sxh[js] = hx;
                    sxl[js] = (float)(ox - hx);
                    syh[js] = hy;
                    syl[js] = (float)(oy - hy);
                    sqf[js] = (float)tv.q[ks];
                }
            }
            nch += take;
            o += take;
            if (nch == kCH) process();
        }
    }
    if (nch > 0) process();
    inside = __reduce_add_sync(0xffffffffu, inside);
    __syncthreads();
    if (lane == 0) atomicAdd(&s_inside, inside);
    __syncthreads();
    if (tid == 0) atomicAdd(n_inside, (unsigned long long)s_inside);
}

__global__ void k2_lift(const double *x2, int64_t n, double *x3) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    x3[3 * i] = x2[2 * i];
    x3[3 * i + 1] = x2[2 * i + 1];
    x3[3 * i + 2] = 0.0;
}

// total source charge in a fixed order: kQB blocks sum fixed ranges (threads
// strided, then a tree), one block adds the partial sums
constexpr int kQB = 304, kQT = 256;
__global__ void __launch_bounds__(kQT) k2_qsum_part(const double *q, const uint8_t *pflag, int64_t n, double *part) {
    __shared__ double s[kQT];
    const int64_t per = (n + kQB - 1) / kQB, lo = per * blockIdx.x, hi = min(n, lo + per);
    double a = 0.0;
    for (int64_t k = lo + threadIdx.x; k < hi; k += kQT) a += (pflag[k] & 1) ? q[k] : 0.0;
    s[threadIdx.x] = a;
    __syncthreads();
    for (int h = kQT / 2; h > 0; h >>= 1) {
        if ((int)threadIdx.x < h) s[threadIdx.x] += s[threadIdx.x + h];
        __syncthreads();
    }
    if (threadIdx.x == 0) part[blockIdx.x] = s[0];
}

__global__ void __launch_bounds__(kQB) k2_qsum(const double *part, double *out) {
    __shared__ double s[512];
    s[threadIdx.x] = part[threadIdx.x];
    if (threadIdx.x + kQB < 512) s[threadIdx.x + kQB] = 0.0;
    __syncthreads();
    for (int h = 256; h > 0; h >>= 1) {
        if ((int)threadIdx.x < h) s[threadIdx.x] += s[threadIdx.x + h];
        __syncthreads();
    }
    if (threadIdx.x == 0) *out = s[0];
}

__global__ void k2_finalize(int64_t n, const uint8_t *pflag, const int32_t *pout, const double *ufar,
                            const double *unear, const double *qco, const double *qtot, const Frame *frame,
                            double *pot) {
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n || !(pflag[k] & 2)) return;
    pot[pout[k]] = ufar[k] + unear[k] + log(frame->S) * (*qtot - qco[k]);
}

}  // namespace

int run_log2d(const Log2dDev &d, TreeBuilder &tree, Workspace &ws, Log2dBufs &bf, const double *src, int64_t ns,
              const double *charges, const double *tgt, int64_t nt, int leaf_cap, int max_level, double *pot,
              cudaStream_t st, const cudaEvent_t near_ev[2], std::string &err) {
    if (nt == 0) return DMK_OK;
    const bool same = (tgt == src && nt == ns);
    if (ws.ensure(bf.x3, std::max<int64_t>(ns, 1) * 24) || (!same && ws.ensure(bf.t3, nt * 24))) {
        err = "device allocation failed (2D points)";
        return DMK_ERR_OOM;
    }
    if (ns > 0) {
        k2_lift<<<nblk(ns, 256), 256, 0, st>>>(src, ns, (double *)bf.x3.p);
        launch_tick();
    }
    if (!same) {
        k2_lift<<<nblk(nt, 256), 256, 0, st>>>(tgt, nt, (double *)bf.t3.p);
        launch_tick();
    }
    L2CK(cudaGetLastError());
    const double *x3 = (const double *)bf.x3.p, *t3 = same ? x3 : (const double *)bf.t3.p;
    int rc = tree.build(x3, ns, charges, same ? nullptr : t3, same ? 0 : nt, same, leaf_cap, max_level, 0, st, err);
    if (rc) return rc;
    const TreeView tv = tree.view();
    const int p = d.p, pp = p * p, N = d.N1, NW = d.NW, NM = std::max(N, NW);
    const int64_t n = tv.n;
    if (ws.ensure(bf.mom, (int64_t)tv.nb * pp * 8) || ws.ensure(bf.loc, (int64_t)tv.nb * pp * 8) ||
        ws.ensure(bf.phi, (int64_t)std::max(tree.nslots, 1) * 2 * (d.nf + 1) * N * 8) || ws.ensure(bf.ufar, n * 8) ||
        ws.ensure(bf.unear, n * 8) || ws.ensure(bf.qco, n * 8) || ws.ensure(bf.qtot, 8) || ws.ensure(bf.cnt, 8) ||
        ws.ensure(bf.qpart, kQB * 8)) {
        err = "device allocation failed (2D expansions)";
        return DMK_ERR_OOM;
    }
    double *mom = (double *)bf.mom.p, *loc = (double *)bf.loc.p, *phi = (double *)bf.phi.p;
    double *ufar = (double *)bf.ufar.p, *unear = (double *)bf.unear.p, *qco = (double *)bf.qco.p;
    L2CK(cudaMemsetAsync(unear, 0, n * 8, st));
    L2CK(cudaMemsetAsync(qco, 0, n * 8, st));
    L2CK(cudaMemsetAsync(bf.cnt.p, 0, 8, st));
    // Step 2
    k2_moments<<<tv.nb, kT, 0, st>>>(tv, d, mom);
    launch_tick();
    for (int l = tv.nlev - 2; l >= 0; --l) {
        if (tv.lev_count[l] == 0) continue;
        k2_c2p<<<tv.lev_count[l], kT, 0, st>>>(tv, d, tv.lev_start[l], mom);
        launch_tick();
    }
    L2CK(cudaGetLastError());
    // Step 3
    const size_t smo = (size_t)(pp + (N + 1) * p + (N + 1) * N) * 8;  // half spectra: (N + 1) / 2 rows
    const size_t sml = (size_t)(2 * pp + NM * (NM + 1) + 2 * p * NM) * 8;
    L2CK(cudaFuncSetAttribute(k2_outgoing, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smo));
    L2CK(cudaFuncSetAttribute(k2_local, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sml));
    if (tree.nslots > 0) {
        k2_outgoing<<<tv.nb, kT, smo, st>>>(tv, d, mom, phi);
        launch_tick();
    }
    for (int l = 0; l < tv.nlev; ++l) {
        if (tv.lev_count[l] == 0) continue;
        k2_local<<<tv.lev_count[l], kT, sml, st>>>(tv, d, l, tv.lev_start[l], mom, phi, loc);
        launch_tick();
    }
    k2_eval<<<nblk(n, kT), kT, 0, st>>>(tv, d, (const int32_t *)tree.pleaf.p, loc, ufar);
    launch_tick();
    L2CK(cudaGetLastError());
    // Steps 4-5
    if (near_ev[0]) L2CK(cudaEventRecord(near_ev[0], st));
    if (tree.ntleaves > 0) {
        auto *cnt = (unsigned long long *)bf.cnt.p;
        const int32_t *tl = (const int32_t *)tree.tleaves.p, *no = (const int32_t *)tree.nl_off.p,
                      *ns_ = (const int32_t *)tree.nl_src.p;
        if (d.mixed)
            k2_near<false, true><<<tree.ntleaves, kNT, 0, st>>>(tv, d, tl, no, ns_, unear, qco, cnt);
        else if (d.gmono)
            k2_near<true, false><<<tree.ntleaves, kNT, 0, st>>>(tv, d, tl, no, ns_, unear, qco, cnt);
        else
            k2_near<false, false><<<tree.ntleaves, kNT, 0, st>>>(tv, d, tl, no, ns_, unear, qco, cnt);
        launch_tick();
    }
    if (near_ev[1]) L2CK(cudaEventRecord(near_ev[1], st));
    k2_qsum_part<<<kQB, kQT, 0, st>>>(tv.q, tv.pflag, n, (double *)bf.qpart.p);
    k2_qsum<<<1, kQB, 0, st>>>((const double *)bf.qpart.p, (double *)bf.qtot.p);
    launch_tick();
    k2_finalize<<<nblk(n, 256), 256, 0, st>>>(n, tv.pflag, (const int32_t *)tree.pout.p, ufar, unear, qco,
                                              (const double *)bf.qtot.p, (const Frame *)tree.frame.p, pot);
    launch_tick();
    launch_tick();
    L2CK(cudaGetLastError());
    return DMK_OK;
}

}  // namespace dmk
