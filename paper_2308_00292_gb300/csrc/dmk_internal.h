// dmk_internal.h -- internal declarations of libdmk (not part of the ABI).
#pragma once

#include <atomic>
#include <cstdint>
#include <string>
#include <vector>

#include <cuda_runtime.h>

namespace dmk {

// Record the thread-local detail returned by dmk_last_error_detail().
void set_error_detail(const std::string &m);

// Number of kernels this library has launched (reported per evaluation).
extern std::atomic<long long> g_launches;
inline void launch_tick() { g_launches.fetch_add(1, std::memory_order_relaxed); }

constexpr int kMaxP = 40;       // Chebyshev order limit (Table 1 goes to 38)
constexpr int kMaxNf = 28;      // Fourier half-width limit (Table 1 goes to 26)
constexpr int kMaxLevel = 20;   // deepest tree level; Morton cells have 21 bits
constexpr int kMortonBits = 21;

// ---------------------------------------------------------------- plan math
struct Pswf {
    explicit Pswf(double c);
    double operator()(double x) const;   // psi_0^c(x), psi(0) = 1
    double Phi(double s) const;          // c_0^{-1} int_0^s psi (1 for s >= 1)
    double eval_inside(double x) const;  // Legendre series, |x| <= 1
    double diff(double x1, double x2) const;  // psi(x1) - psi(x2) without cancellation
    double c, chi0 = 0, lambda0 = 0, c0 = 0, c2 = 0;
    std::vector<double> coef, qx, qw, qpsi;
};

struct Tables {
    double eps = 0, c = 0, hW = 0, psi0_over_c0 = 0;
    int p = 0, nf = 0, n0 = 0;
    std::vector<double> t, A[2], Fr, Fi, FWr, FWi, w, wW, qcheb, qmono, psi_grid;
};

int build_tables(double eps, int p_override, int nf_override, Tables &tb, std::string &err);

// Yukawa kernel exp(-lambda r)/r (Sec. 3.7, Fourier-space splitting) at a
// unit-box lambda: level-dependent translation weights w_l(|m|^2) (not scaled
// by 1/R_l), root weights wW(|m|^2) and residual polynomials q_l, monomials in
// 2 t - 1, t = r^2 / R_l^2, with S_l(r) = q_l(t) / R_l; row l of qmono is
// [degree of level l, c_0 .. c_qdeg] (zero padded), qdeg the largest degree.
constexpr int kMaxYukawaDegree = 62;
struct YukawaTables {
    double lam = -1.0;
    int nlev = 0, qdeg = 0;
    std::vector<double> wl, wW, qmono;  // [nlev][3 nf^2 + 1], [3 n0^2 + 1], [nlev][qdeg + 2]
};
int build_yukawa_tables(const Tables &tb, double lam, int nlev, YukawaTables &yt, std::string &err);

// The 2D Laplace kernel log r (Sec. 3.7 at lambda = 0 in the plane), on top of
// the dimension-free parts of Tables (t, A, Fr, Fi): translation weights
// w(|m|^2), the same at every level, the root window's spacing, modes, F
// matrix and weights, and the Chebyshev coefficients g (in x = 2t - 1) of the
// smooth part G of the residual, R_l(r) = log(r / R_l) + G(r^2 / R_l^2).
struct Log2dTables {
    double hW = 0, G0 = 0;
    int n0 = 0;
    std::vector<double> w, FWr, FWi, wW, g;  // [2 nf^2 + 1], [NW][p] x 2, [2 n0^2 + 1], [gdeg + 1]
    // g as monomials in 2 t - 1 (Horner) where that form keeps its accuracy,
    // else empty (the device then sums the Chebyshev series)
    std::vector<double> gmono;
};
int build_log2d_tables(const Tables &tb, Log2dTables &t2, std::string &err);

// ---------------------------------------------------------------- device views
// Plan tables on the device, in the working precision T.
template <typename T>
struct DevTables {
    int p, nf, N1, nh;       // nh = nf + 1 (stored half spectrum m_z >= 0)
    int n0, NW, nhW;
    int qdeg;
    const T *A;              // [2][p][p]
    const T *Fr, *Fi;        // [N1][p]   F[m][n], m = index - nf
    const T *FWr, *FWi;      // [NW][p]
    const T *w;              // [3 nf^2 + 1], at R = 1
    const T *wW;             // [3 n0^2 + 1]
    const T *qmono;          // [qdeg + 1], q(t) = sum qmono[k] (2t-1)^k
    // Yukawa kernel (null / 0 for Laplace): per-level translation weights
    // [nlev][3 nf^2 + 1] (already including 1/R_l), per-level residual
    // polynomials [nlev][qdeg + 1], lambda in unit-box units
    const T *wl;
    const T *ql;
    T lam;
};

// Box flags
enum : uint8_t { BF_LEAF = 1, BF_FOUT = 2, BF_FIN = 4 };

struct TreeView {
    int64_t n;               // points (sorted Morton order)
    const double *ux, *uy, *uz;   // unit-box coordinates
    const double *q;              // charge (0 for a target-only point)
    const uint8_t *pflag;         // bit 0 source, bit 1 target
    int nb;                       // boxes (by level, Morton order within a level)
    const uint64_t *bkey;         // Morton cell at the box's level
    const int8_t *blevel;
    const int32_t *bstart, *bcount, *bparent, *bchild0;
    const uint8_t *bcmask;        // octants present among the children
    const uint8_t *bflags;        // BF_*
    const int32_t *bnsrc, *bntgt;
    const int32_t *bcol;          // [nb][27] colleagues (-1 absent), k = 9(dx+1)+3(dy+1)+(dz+1)
    const int32_t *bslot;         // expansion slot of a non-leaf box, -1 for leaves
    int lev_start[kMaxLevel + 2];
    int lev_count[kMaxLevel + 2];
    int nlev;
};

// ---------------------------------------------------------------- helpers
__host__ __device__ inline double level_R(int l) {
    return 1.0 / (double)(1u << l);
}

// device-wide exclusive scan of int32 (n elements); total written to *d_total
void scan_exclusive_i32(const int32_t *d_in, int32_t *d_out, int64_t n, int32_t *d_total,
                        void *tmp, size_t tmp_bytes, cudaStream_t st);
size_t scan_tmp_bytes(int64_t n);

// LSD radix sort of (63-bit key, u32 value) pairs, stable.
void radix_sort_pairs(uint64_t *keys, uint32_t *vals, uint64_t *keys_alt, uint32_t *vals_alt,
                      int64_t n, int bits, void *tmp, size_t tmp_bytes, cudaStream_t st,
                      uint64_t **keys_out, uint32_t **vals_out);
size_t radix_tmp_bytes(int64_t n);

}  // namespace dmk
