// passes.cu -- the upward pass, the plane-wave (dual-space) downward pass and
// the residual near field of the discrete DMK algorithm (Steps 2-5 of Sec. 3.4
// of arXiv 2308.00292), templated on the working precision T, the Chebyshev
// order P and the Fourier half-width NF (the (P, NF) pairs of Table 1).
//
// Representations (all per box, box side R, Chebyshev coordinate
// xi = 2 (x - c_B) / R):
//   moments     M[a][b][c] = sum_j T_a(xi_x) T_b(xi_y) T_c(xi_z) rho_j over the
//               sources of a non-leaf box.  Proxy charges of Def. anterpdef are
//               rho~ = V^-T M, so M carries the same information; the library
//               folds V^-T into the plane-wave matrix F.
//   outgoing    Phi[my][mx][mz], m in [-nf, nf]^2 x [0, nf]: the half spectrum of
//               eq. outgoingexpansion2 (Phi_{-m} = conj(Phi_m) for real charges);
//               the m_z index is padded to an even count (nz_pad).
//   local       Lambda[a][b][c], Chebyshev coefficients of the far field in the
//               box (eq. localexpansion).
//
// Parity of the 1-D plane-wave matrix.  F[m][n] = sum_j exp(-i theta m t_j)
// Vinv[n][j] is real and even in m for even n and imaginary and odd in m for
// odd n (the Chebyshev nodes are symmetric and T_n has the parity of n).  Every
// contraction with F or with G = conj(F)^T therefore splits into an even part
// over m >= 0 and an odd part over m > 0, which the kernels use: the mode
// products touch only non-negative modes and real coefficients.  hs[n][m'] is
// Re F[m'][n] for even n and Im F[m'][n] for odd n, m' = 0..NF.
//
// Kernels:
//   k_upward   level by level, finest first: moments of a non-leaf box from the
//              sources of its leaf children (anterpolation onto the parent grid,
//              eq. proxynd) and from the moments of its non-leaf children (T_c2p,
//              Lemma ctoplemma, exact triangular shift matrices)
//   k_prox2pw  every F_out box: Phi = (F x F x F) M  (T_prox2pw)
//   k_root     the windowed kernel W_0 at the root (eq. windowedkernelft2)
//   k_local    level by level, coarsest first, every box with targets:
//              Lambda = T_p2c(Lambda_parent) (Lemma ptoclemma) plus, for F_in
//              boxes, the incoming expansion of eq. diagonaltranslation (the
//              phases are cube roots of unity because h_l R_l = 2 pi / 3) and its
//              conversion to Chebyshev coefficients (T_pw2poly); leaves then
//              evaluate Lambda at their targets (Step 3 "Evaluate local
//              expansions")
//   k_near     residual kernels R_{L(j)} over the interaction lists (Step 4),
//              including the self correction of Step 5 (r = 0 terms)
#include "passes.h"
#include "incoming.h"
#include "tc.h"
#include "dev_util.h"

#include <algorithm>
#include <cstdio>

namespace dmk {

constexpr int kThreads = 256;
constexpr int kCH = 32;  // points per staging chunk in k_upward

template <typename T> struct Cplx;
template <> struct Cplx<float> { using type = float2; };
template <> struct Cplx<double> { using type = double2; };


// A buffer of a kernel's layout.  With SM (the single-precision kernels, whose
// buffers the host checks to lie in shared memory) the pointer is formed from
// the shared array alone, so that the compiler emits shared-memory accesses
// instead of generic ones.
template <typename U, bool SM = false>
__device__ __forceinline__ U *buf_ptr(const BufLayout &lay, int i, char *sm, char *slab) {
    if constexpr (SM) return reinterpret_cast<U *>(sm + lay.off[i]);
    return lay.in_smem[i] ? reinterpret_cast<U *>(sm + lay.off[i])
                          : reinterpret_cast<U *>(slab + (size_t)blockIdx.x * lay.slab_bytes + lay.off[i]);
}

// the kernels whose buffers must all lie in shared memory
template <typename T, int P> constexpr bool all_smem() { return sizeof(T) == 4 && P <= 20; }

static bool layout_in_smem(const BufLayout &lay) {
    for (int i = 0; i < lay.n; ++i)
        if (!lay.in_smem[i]) return false;
    return true;
}

// the stored half spectrum pads m_z to an even count so that two adjacent
// modes form one aligned 16-byte (single) or 32-byte (double) pair
template <int NF> __host__ __device__ constexpr int nz_pad() { return (NF + 2) & ~1; }

template <typename C2> struct C2x2 { C2 a, b; };
__device__ __forceinline__ C2x2<float2> ld_pair(const float2 *p) {
    const float4 v = *reinterpret_cast<const float4 *>(p);
    return {make_float2(v.x, v.y), make_float2(v.z, v.w)};
}
__device__ __forceinline__ C2x2<double2> ld_pair(const double2 *p) {
    return {p[0], p[1]};
}

template <typename C2, typename T>
__device__ __forceinline__ void cfma(C2 &acc, T h, const C2 &v) {
    acc.x += h * v.x;
    acc.y += h * v.y;
}

// hs[n][m'] = Re F[m'][n] (n even) or Im F[m'][n] (n odd), m' = 0..NF
template <typename T, int P, int NF>
__device__ __forceinline__ void load_hs(const DevTables<T> &tb, T *hs) {
    constexpr int NH = NF + 1;
    for (int i = threadIdx.x; i < P * NH; i += blockDim.x) {
        const int n = i / NH, m = i % NH;
        hs[i] = (n & 1) ? tb.Fi[(m + NF) * P + n] : tb.Fr[(m + NF) * P + n];
    }
}

// four consecutive values (16-byte aligned) from shared memory
template <typename T> __device__ __forceinline__ void ld4(const T *p, T (&v)[4]);
template <> __device__ __forceinline__ void ld4<float>(const float *p, float (&v)[4]) {
    const float4 t = *reinterpret_cast<const float4 *>(p);
    v[0] = t.x; v[1] = t.y; v[2] = t.z; v[3] = t.w;
}
template <> __device__ __forceinline__ void ld4<double>(const double *p, double (&v)[4]) {
    const double2 t0 = *reinterpret_cast<const double2 *>(p), t1 = *reinterpret_cast<const double2 *>(p + 2);
    v[0] = t0.x; v[1] = t0.y; v[2] = t1.x; v[3] = t1.y;
}

// padded row strides of the upward pass's staging buffers (multiples of 4)
template <int P> struct UpShape {
    static constexpr int PS = (P + 3) & ~3, YS = (P * P + 3) & ~3;
    // tensor-core anterpolation D[bc][a] = sum_j T_b(y_j) T_c(z_j) rho_j T_a(x_j):
    // bc on MT tiles of 128 TMEM lanes, a padded to NA columns (N), points in
    // chunks of KC (K); operands TF32 hi + lo
    static constexpr int MT = (P * P + 127) / 128, NA = (P + 15) / 16 * 16, KC = 16;
    static constexpr int TCOLS = MT * NA <= 32 ? 32 : (MT * NA <= 64 ? 64 : (MT * NA <= 128 ? 128 : 256));
    static constexpr bool TC_OK = MT * NA <= 256;
    static constexpr int A_FL = MT * 128 * KC, B_FL = NA * KC;  // floats per operand part
    static constexpr int TC_SCR = 2 * A_FL + 2 * B_FL + 3 * KC * PS;
};

// One axis of the child-to-parent moment shift on a P^3 array:
// out[.., n, ..] (+)= sum_{m <= n} A[n][m] in[.., m, ..] along axis AX (0 = z,
// the fastest index, 1 = y, 2 = x); two rows per thread, A from shared memory.
template <typename T, int P, int AX, int NT, bool ACC>
__device__ __forceinline__ void shift_up(const T *__restrict__ A, const T *in, T *out) {
    constexpr int s = AX == 0 ? 1 : (AX == 1 ? P : P * P);
    if constexpr (P > 20) {  // large orders: one output per thread (registers)
        for (int i = threadIdx.x; i < P * P * P; i += NT) {
            const int n = AX == 0 ? i % P : (AX == 1 ? (i / P) % P : i / (P * P));
            const int b = i - n * s;
            T acc = 0;
            for (int m = 0; m <= n; ++m) acc += A[n * P + m] * in[b + m * s];
            if (ACC) out[i] += acc; else out[i] = acc;
        }
        return;
    }
    constexpr bool TWO = true;
    constexpr int RR = P * P, H = TWO ? (RR + 1) / 2 : RR;
    auto base = [](int r) { return AX == 0 ? r * P : (AX == 1 ? (r / P) * P * P + r % P : r); };
    for (int t = threadIdx.x; t < H; t += NT) {
        const int r0 = t, r1 = t + H;
        const bool has1 = TWO && r1 < RR;
        const int b0 = base(r0), b1 = has1 ? base(r1) : b0;
        T o0[P], o1[P];
#pragma unroll
        for (int n = 0; n < P; ++n) o0[n] = o1[n] = (T)0;
#pragma unroll
        for (int m = 0; m < P; ++m) {
            const T v0 = in[b0 + m * s], v1 = in[b1 + m * s];
#pragma unroll
            for (int n = m; n < P; ++n) {
                const T a = A[n * P + m];
                o0[n] += a * v0;
                if (TWO) o1[n] += a * v1;
            }
        }
#pragma unroll
        for (int n = 0; n < P; ++n) {
            if (ACC) out[b0 + n * s] += o0[n]; else out[b0 + n * s] = o0[n];
        }
        if (has1) {
#pragma unroll
            for (int n = 0; n < P; ++n) {
                if (ACC) out[b1 + n * s] += o1[n]; else out[b1 + n * s] = o1[n];
            }
        }
    }
}

// ---------------------------------------------------------------------------
// Upward pass (Step 2)
// ---------------------------------------------------------------------------
// Tensor-core anterpolation of ntot points (ranges lstart / lpre) onto the
// grid of a box (centre cc, scale s2R): acc[a][b][c] += sum_j rho_j T_a(x_j)
// T_b(y_j) T_c(z_j) as D[bc][a] = sum_j Y[bc][j] X[a][j] with Y = T_b(y) T_c(z)
// and X = rho T_a(x), KC points per MMA batch; operands split into TF32 hi +
// lo (D = A_lo B_hi + A_hi B_lo + A_hi B_hi).  D accumulates kFlush batches in
// TMEM and is then added to acc by the CUDA cores in round-to-nearest FP32, so
// no sum runs through the tensor core's adder for more than kFlush batches:
// all batches at once missed the 1e-6 bar, and 4 batches per flush raised the
// rel-L2 error of 2e4 uniform points from 5.1e-7 to 6.3e-7, so each batch is
// flushed.  Called by the whole CTA.
template <int P>
__device__ void anterpolate_tc(const TreeView &tv, const double (&cc)[3], double s2R, const int *lstart,
                               const int *lpre, int ntot, float *scr, uint32_t tmem, uint64_t *bar, uint32_t &phase,
                               float *acc, int *tc_err) {
    using U = UpShape<P>;
    constexpr int KC = U::KC, PS = U::PS;
    float *Ah = scr, *Al = Ah + U::A_FL, *Bh = Al + U::A_FL, *Bl = Bh + U::B_FL;
    float *stg = Bl + U::B_FL;  // [3][KC][PS]: rho T_a(x), T_b(y), T_c(z)
    const int tid = threadIdx.x;
    constexpr uint32_t lbo = 128, sbo = KC * 32;
    bool ok = true;
    // threads 0 .. 3 KC - 1 hold one coordinate (and charge) of the next batch,
    // loaded one batch ahead
    auto fetch = [&](int p, double &u, double &w) {
        const int ax = tid / KC, j = tid % KC;
        u = 0.0;
        w = 1.0;
        if (p + j < ntot) {
            int seg = 0;
            while (seg < 7 && lpre[seg + 1] <= p + j) ++seg;
            const int kk = lstart[seg] + (p + j - lpre[seg]);
            u = ax == 0 ? tv.ux[kk] : (ax == 1 ? tv.uy[kk] : tv.uz[kk]);
            if (ax == 0) w = tv.q[kk];
        }
    };
    double un = 0.0, wn = 1.0;
    if (tid < 3 * KC) fetch(0, un, wn);
    constexpr int kFlush = 1;
    bool pending = false;     // a batch's MMAs were issued but not yet waited for
    uint32_t pend_par = 0;
    for (int p0 = 0; p0 < ntot; p0 += KC) {
        const int np = min(KC, ntot - p0), bi = p0 / KC;
        if (tid < 3 * KC) {
            const int ax = tid / KC, j = tid % KC;
            float *o = stg + (ax * KC + j) * PS;
            const double u = un, wq = wn;
            if (p0 + KC < ntot) fetch(p0 + KC, un, wn);
            if (j < np) {
                const float xi = (float)((u - cc[ax]) * s2R);
                const float w = (float)wq;
                float t0 = 1.f, t1 = xi;
                o[0] = w;
                if (P > 1) o[1] = w * xi;
#pragma unroll
                for (int n = 2; n < P; ++n) {
                    const float t2 = 2.f * xi * t1 - t0;
                    o[n] = w * t2;
                    t0 = t1;
                    t1 = t2;
                }
            } else {
#pragma unroll
                for (int n = 0; n < P; ++n) o[n] = 0.f;
            }
        }
        // the previous batch's MMAs read the operands: they must be done
        if (pending && tid == 0) ok = tc::mbar_wait(bar, pend_par, 2000000000ll) && ok;
        __syncthreads();
        // A operand: row bc, column j (K-major core matrices), 4 points per float4;
        // a fixed trip count, unrolled, so that the loads of all of a thread's
        // elements are in flight together
#pragma unroll
        for (int t = tid; t < U::A_FL / 4; t += kThreads) {
            const int r8 = t & 7, k4 = (t >> 3) % (KC / 4), bc = ((t >> 3) / (KC / 4)) * 8 + r8;
            float h[4], l[4];
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const int j = 4 * k4 + q;
                const float v = bc < P * P ? stg[(KC + j) * PS + bc / P] * stg[(2 * KC + j) * PS + bc % P] : 0.f;
                tc::split_tf32(v, h[q], l[q]);
            }
            reinterpret_cast<float4 *>(Ah)[t] = make_float4(h[0], h[1], h[2], h[3]);
            reinterpret_cast<float4 *>(Al)[t] = make_float4(l[0], l[1], l[2], l[3]);
        }
        // B operand: row a, column j
#pragma unroll
        for (int t = tid; t < U::B_FL / 4; t += kThreads) {
            const int r8 = t & 7, k4 = (t >> 3) % (KC / 4), a = ((t >> 3) / (KC / 4)) * 8 + r8;
            float h[4], l[4];
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const int j = 4 * k4 + q;
                const float v = a < P ? stg[j * PS + a] : 0.f;
                tc::split_tf32(v, h[q], l[q]);
            }
            reinterpret_cast<float4 *>(Bh)[t] = make_float4(h[0], h[1], h[2], h[3]);
            reinterpret_cast<float4 *>(Bl)[t] = make_float4(l[0], l[1], l[2], l[3]);
        }
        tc::fence_proxy_async();
        tc::fence_before_sync();
        __syncthreads();
        tc::fence_after_sync();
        if (tid == 0) {
            const uint32_t aH = tc::smem_addr(Ah), aL = tc::smem_addr(Al);
            const uint32_t bH = tc::smem_addr(Bh), bL = tc::smem_addr(Bl);
            const uint32_t id = tc::idesc_tf32(128, U::NA);
#pragma unroll
            for (int mt = 0; mt < U::MT; ++mt) {
                const uint32_t aoff = (uint32_t)(mt * 128 / 8) * sbo, dcol = tmem + (uint32_t)(mt * U::NA);
#pragma unroll
                for (int ks = 0; ks < KC / 8; ++ks) {
                    const uint32_t ko = (uint32_t)ks * 256;
                    tc::mma_tf32(dcol, tc::sdesc(aL + aoff + ko, lbo, sbo), tc::sdesc(bH + ko, lbo, sbo), id,
                                 ks > 0 || bi % kFlush != 0);
                    tc::mma_tf32(dcol, tc::sdesc(aH + aoff + ko, lbo, sbo), tc::sdesc(bL + ko, lbo, sbo), id, true);
                    tc::mma_tf32(dcol, tc::sdesc(aH + aoff + ko, lbo, sbo), tc::sdesc(bH + ko, lbo, sbo), id, true);
                }
            }
            tc::commit(bar);
        }
        const uint32_t par = phase;
        phase ^= 1u;
        if (bi % kFlush != kFlush - 1 && p0 + KC < ntot) {
            pending = true;
            pend_par = par;
            continue;
        }
        pending = false;
        // every thread waits for the batch, then adds its share of D to acc:
        // warp w reads TMEM lanes 32 (w mod 4) .. + 31 of the tiles w / 4, w / 4 + 2, ...
        ok = tc::mbar_wait(bar, par, 2000000000ll) && ok;  // about 1 s
        const bool wok = __all_sync(0xffffffffu, ok);
        tc::fence_after_sync();
        if (wok) {
            const int warp = tid >> 5, lane = tid & 31, nw = kThreads >> 5;
#pragma unroll
            for (int mt = warp >> 2; mt < U::MT; mt += nw >> 2) {
                const int bc = mt * 128 + (warp & 3) * 32 + lane;
                const uint32_t trow = tmem + ((uint32_t)((warp & 3) * 32) << 16) + (uint32_t)(mt * U::NA);
                float d[(P + 7) / 8][8];
#pragma unroll
                for (int c8 = 0; c8 < (P + 7) / 8; ++c8) tc::ld_x8(trow + (uint32_t)(c8 * 8), d[c8]);
                tc::ld_wait();
                if (bc < P * P) {
#pragma unroll
                    for (int c8 = 0; c8 < (P + 7) / 8; ++c8)
#pragma unroll
                        for (int q = 0; q < 8; ++q) {
                            const int a = c8 * 8 + q;
                            if (a < P) acc[a * P * P + bc] += d[c8][q];
                        }
                }
            }
        }
        tc::fence_before_sync();
        __syncthreads();
        tc::fence_after_sync();
    }
    if (!ok && (tid & 31) == 0) atomicExch(tc_err, 1);
}

// ---------------------------------------------------------------------------
// Single-precision upward pass of every level in one launch (k_anterp)
// ---------------------------------------------------------------------------
// Shapes: compute threads hold the register tiles of the anterpolation, one
// (a, b pair) item each; three staging warps form the Chebyshev rows of the
// next chunk of points meanwhile (double-buffered, one barrier per chunk).
template <int P> struct AntShape {
    static constexpr int PS = (P + 3) & ~3, NBP = (P + 1) / 2, NIT = P * NBP;
    static constexpr int NC = (NIT + 31) / 32 * 32;  // compute threads
    static constexpr int NS = 3 * kCH;               // staging threads: (axis, point)
    static constexpr int NT = NC + NS;
    static constexpr int P3 = P * P * P, P3P = (P3 + 31) / 32 * 32;
    static constexpr int STG = 3 * kCH * PS;         // floats of one staging buffer
    static constexpr int WRK = 2 * STG > P3P ? 2 * STG : P3P;  // staging buffers, or the shift scratch
    static constexpr int NPEN = (P * P + 1) / 2;     // pencil pairs of one shift axis
    static constexpr size_t SMEM = ((size_t)P3P + WRK + 2 * P * PS) * sizeof(float);
    static constexpr bool OK = NPEN <= NT;
};

// Chebyshev row of one coordinate of one point, times the charge for x:
// o[n] = w T_n(xi), n < P, zero-padded to PS
template <int P>
__device__ __forceinline__ void cheb_row(float *o, float xi, float w) {
    float t0 = 1.f, t1 = xi;
    o[0] = w;
    if (P > 1) o[1] = w * xi;
#pragma unroll
    for (int n = 2; n < P; ++n) {
        const float t2 = 2.f * xi * t1 - t0;
        o[n] = w * t2;
        t0 = t1;
        t1 = t2;
    }
#pragma unroll
    for (int n = P; n < AntShape<P>::PS; ++n) o[n] = 0.f;
}

// acc[a][b][c] += sum_j rho_j T_a(x_j) T_b(y_j) T_c(z_j) over the ntot points
// of the ranges (lstart, lpre) on the grid of centre cc and scale s2R.  A
// compute thread keeps M[a][b][c] and M[a][b+1][c] for every c in registers and
// adds point by point, two points per step (one FMA per moment and point, with
// rho T_a(x) T_b(y) formed once per (a, b)); a chunk's sums go to acc in
// shared memory, so every moment is a sum of chunk sums of kCH points.
// Staging threads load coordinates one chunk ahead of the rows they form.
// Called by the whole CTA after acc is zeroed; ends with a barrier.
template <int P>
__device__ __forceinline__ void anterpolate_pipe(const TreeView &tv, const double (&cc)[3], double s2R,
                                                 const int *lstart, const int *lpre, int ntot, float *stg,
                                                 float *acc) {
    using S = AntShape<P>;
    constexpr int PS = S::PS, NBP = S::NBP;
    const int tid = threadIdx.x;
    const bool stager = tid >= S::NC;
    const int sidx = tid - S::NC, ax = sidx / kCH, j = sidx % kCH;
    const double cax = ax == 0 ? cc[0] : (ax == 1 ? cc[1] : cc[2]);
    // the coordinate (and, for x, the charge) of point p of the ranges
    auto fetch = [&](int p, double &u, double &w) {
        u = cax;
        w = 0.0;
        if (p < ntot) {
            int seg = 0;
            while (seg < 7 && lpre[seg + 1] <= p) ++seg;
            const int kk = lstart[seg] + (p - lpre[seg]);
            u = ax == 0 ? tv.ux[kk] : (ax == 1 ? tv.uy[kk] : tv.uz[kk]);
            w = ax == 0 ? tv.q[kk] : 1.0;
        }
    };
    double un = 0.0, wn = 0.0;
    if (stager) {
        fetch(j, un, wn);
        cheb_row<P>(stg + (ax * kCH + j) * PS, (float)((un - cax) * s2R), (float)wn);
        fetch(kCH + j, un, wn);
    }
    __syncthreads();
    const int a = tid / NBP, b0 = 2 * (tid % NBP);
    const bool has1 = b0 + 1 < P;
    for (int c = 0, p0 = 0; p0 < ntot; ++c, p0 += kCH) {
        const float *cur = stg + (c & 1) * S::STG;
        if (stager) {
            if (p0 + kCH < ntot) {
                float *nxt = stg + ((c + 1) & 1) * S::STG;
                cheb_row<P>(nxt + (ax * kCH + j) * PS, (float)((un - cax) * s2R), (float)wn);
                fetch(p0 + 2 * kCH + j, un, wn);
            }
        } else if (tid < S::NIT) {
            const int np = min(kCH, ntot - p0);
            // the moments of rows b0 and b0 + 1 as pairs of consecutive c, so that
            // the packed FMA (two lanes of a 64-bit register pair, each rounded
            // like fmaf) takes the T_c(z) pairs as they come from shared memory
            float2 c0[PS / 2], c1[PS / 2];
#pragma unroll
            for (int k = 0; k < PS / 2; ++k) c0[k] = c1[k] = make_float2(0.f, 0.f);
            // two points per step (a row past np is staged as zeros)
            for (int jj = 0; jj < np; jj += 2) {
                const float *X0 = cur + jj * PS, *Y0 = cur + (kCH + jj) * PS;
                const float4 *Z0 = reinterpret_cast<const float4 *>(cur + (2 * kCH + jj) * PS);
                const float4 *Z1 = reinterpret_cast<const float4 *>(cur + (2 * kCH + jj + 1) * PS);
                const float xa0 = X0[a], xa1 = X0[PS + a];
                const float s00 = xa0 * Y0[b0], s01 = has1 ? xa0 * Y0[b0 + 1] : 0.f;
                const float s10 = xa1 * Y0[PS + b0], s11 = has1 ? xa1 * Y0[PS + b0 + 1] : 0.f;
                const float2 d00 = make_float2(s00, s00), d01 = make_float2(s01, s01);
                const float2 d10 = make_float2(s10, s10), d11 = make_float2(s11, s11);
#pragma unroll
                for (int c4 = 0; c4 < PS / 4; ++c4) {
                    const float4 z = Z0[c4], y = Z1[c4];
                    const float2 za0 = make_float2(z.x, z.y), za1 = make_float2(z.z, z.w);
                    const float2 zb0 = make_float2(y.x, y.y), zb1 = make_float2(y.z, y.w);
                    c0[2 * c4] = __ffma2_rn(d10, zb0, __ffma2_rn(d00, za0, c0[2 * c4]));
                    c0[2 * c4 + 1] = __ffma2_rn(d10, zb1, __ffma2_rn(d00, za1, c0[2 * c4 + 1]));
                    c1[2 * c4] = __ffma2_rn(d11, zb0, __ffma2_rn(d01, za0, c1[2 * c4]));
                    c1[2 * c4 + 1] = __ffma2_rn(d11, zb1, __ffma2_rn(d01, za1, c1[2 * c4 + 1]));
                }
            }
            // this thread's own rows of acc: no other thread touches them
            float *r0 = acc + (a * P + b0) * P;
#pragma unroll
            for (int k = 0; k < P; ++k) {
                r0[k] += (k & 1) ? c0[k >> 1].y : c0[k >> 1].x;
                if (has1) r0[P + k] += (k & 1) ? c1[k >> 1].y : c1[k >> 1].x;
            }
        }
        __syncthreads();
    }
}

// One axis of the exact child-to-parent shift (Lemma ctoplemma) on pencils:
// out[.., n, ..] = sum_{m <= n} A[n][m] in[.., m, ..] along axis AX (0 = the
// fastest index c, 1 = b, 2 = a), two pencils per thread, each read whole into
// registers first (so out may be in).  A is P x PS in shared memory, zero above
// the diagonal.  MODE 0: in from global memory (L2, bypassing L1); 1: in and
// out in shared memory; 2: out += (accumulate).
template <int P, int AX, int MODE>
__device__ __forceinline__ void shift_pencils(const float *A, const float *in, float *out) {
    using S = AntShape<P>;
    constexpr int PS = S::PS;
    constexpr int s = AX == 0 ? 1 : (AX == 1 ? P : P * P);
    auto base = [](int r) { return AX == 0 ? r * P : (AX == 1 ? (r / P) * P * P + r % P : r); };
    const int t = threadIdx.x;
    if (t < S::NPEN) {
        const int r0 = t, r1 = t + S::NPEN;
        const bool has1 = r1 < P * P;
        const int e0 = base(r0), e1 = has1 ? base(r1) : e0;
        float v0[PS], v1[PS];
#pragma unroll
        for (int m = 0; m < P; ++m) {
            v0[m] = MODE == 0 ? __ldcg(in + e0 + m * s) : in[e0 + m * s];
            v1[m] = MODE == 0 ? __ldcg(in + e1 + m * s) : in[e1 + m * s];
        }
#pragma unroll
        for (int m = P; m < PS; ++m) v0[m] = v1[m] = 0.f;
#pragma unroll
        for (int n = 0; n < P; ++n) {
            const float4 *Ar = reinterpret_cast<const float4 *>(A + n * PS);
            float o0 = 0.f, o1 = 0.f;
#pragma unroll
            for (int m4 = 0; m4 <= n / 4; ++m4) {
                const float4 w = Ar[m4];
                o0 = fmaf(w.x, v0[4 * m4], o0);
                o1 = fmaf(w.x, v1[4 * m4], o1);
                o0 = fmaf(w.y, v0[4 * m4 + 1], o0);
                o1 = fmaf(w.y, v1[4 * m4 + 1], o1);
                o0 = fmaf(w.z, v0[4 * m4 + 2], o0);
                o1 = fmaf(w.z, v1[4 * m4 + 2], o1);
                o0 = fmaf(w.w, v0[4 * m4 + 3], o0);
                o1 = fmaf(w.w, v1[4 * m4 + 3], o1);
            }
            if (MODE == 2) {
                out[e0 + n * s] += o0;
                if (has1) out[e1 + n * s] += o1;
            } else {
                out[e0 + n * s] = o0;
                if (has1) out[e1 + n * s] = o1;
            }
        }
    }
}

// Persistent CTAs take the expansion slots from a work counter.  For its box B
// a CTA anterpolates the sources of B's leaf children onto B's grid (a root
// that is a leaf anterpolates its own sources, for the windowed term W_0) and
// stores the result in M[slot(B)].  The child-to-parent shifts need no
// per-level launch: a box counts arrivals in cnt[slot] -- its own
// anterpolation and the completion of each non-leaf child holding sources --
// and the CTA whose arrival completes the count adds the shifted moments of
// those children to the box's own, then arrives at the parent.  No CTA waits
// for another, and every box's sum is formed by one CTA in octant order, so
// the result does not depend on scheduling.  cnt must be zero on entry.
template <int P>
__global__ void __launch_bounds__(AntShape<P>::NT, 2) k_anterp(TreeView tv, const float *Atab, int nslots,
                                                            const int32_t *slot2box, float *M, int *ctr, int *cnt) {
    using S = AntShape<P>;
    constexpr int P3 = S::P3, PS = S::PS;
    constexpr unsigned FULL = 0xffffffffu;
    extern __shared__ __align__(128) char sm[];
    float *acc = reinterpret_cast<float *>(sm);
    float *wrk = acc + S::P3P;          // staging buffers [2][3][kCH][PS], or the shift scratch [P3]
    float *As = wrk + S::WRK;           // shift matrices A_{-1}, A_{+1}: [2][P][PS]
    __shared__ int s_item, s_lstart[8], s_lpre[9], s_nnl, s_last;
    __shared__ int s_kids[8];           // non-leaf children with sources, in octant order (octant << 27 | box)
    const int tid = threadIdx.x, lane = tid & 31;
    for (int i = tid; i < 2 * P * PS; i += S::NT) {
        const int h = i / (P * PS), n = (i / PS) % P, m = i % PS;
        As[i] = m <= n && m < P ? Atab[h * P * P + n * P + m] : 0.f;
    }
    // warp 0: the children of box X -- the point ranges of its leaf children
    // with sources (when ranges is set) and its non-leaf children with sources.
    // The leading barrier: every warp has read the previous box's s_nnl and
    // s_kids (a box without non-leaf children reaches here with no barrier
    // after that read) before warp 0 overwrites them
    auto children = [&](int X, bool ranges) {
        __syncthreads();
        if (tid < 32) {
            const bool selfleaf = (tv.bflags[X] & BF_LEAF) != 0;
            const unsigned cm = selfleaf ? 0u : tv.bcmask[X];
            const int c0 = tv.bchild0[X];
            bool leafk = false, nonleaf = false;
            int st = 0, ct = 0;
            if (selfleaf) {
                if (lane == 0 && tv.bnsrc[X] > 0) {
                    leafk = true;
                    st = tv.bstart[X];
                    ct = tv.bcount[X];
                }
            } else if (lane < 8 && ((cm >> lane) & 1u)) {
                const int D = c0 + __popc(cm & ((1u << lane) - 1u));
                const bool src = tv.bnsrc[D] > 0, lf = (tv.bflags[D] & BF_LEAF) != 0;
                leafk = src && lf;
                nonleaf = src && !lf;
                if (leafk) {
                    st = tv.bstart[D];
                    ct = tv.bcount[D];
                }
                if (nonleaf) st = D;
            }
            const unsigned nm = __ballot_sync(FULL, nonleaf);
            if (nonleaf) s_kids[__popc(nm & ((1u << lane) - 1u))] = (lane << 27) | st;
            if (lane == 0) s_nnl = __popc(nm);
            if (ranges) {
                const unsigned lm = __ballot_sync(FULL, leafk);
                int pre = leafk ? ct : 0;
#pragma unroll
                for (int o = 1; o < 8; o <<= 1) {
                    const int v = __shfl_up_sync(FULL, pre, o);
                    if (lane >= o) pre += v;
                }
                const int tot = __shfl_sync(FULL, pre, 7);
                const int k = __popc(lm & ((1u << lane) - 1u));
                if (leafk) {
                    s_lstart[k] = st;
                    s_lpre[k] = pre - ct;
                }
                if (lane >= __popc(lm) && lane < 9) s_lpre[lane] = tot;
            }
        }
        __syncthreads();
    };
    for (;;) {
        // every thread has read the previous item (a skipped item comes straight
        // back here) before thread 0 takes the next
        __syncthreads();
        if (tid == 0) s_item = atomicAdd(ctr, 1);
        __syncthreads();
        const int slot = s_item;
        if (slot >= nslots) break;
        const int B = slot2box[slot];
        if (((tv.bflags[B] & BF_LEAF) && tv.blevel[B] != 0) || tv.bnsrc[B] == 0) continue;
        const int l = tv.blevel[B];
        int ix, iy, iz;
        box_decode_d(tv.bkey[B], l, ix, iy, iz);
        const double R = level_R(l), s2R = 2.0 / R;
        const double cc[3] = {(ix + 0.5) * R, (iy + 0.5) * R, (iz + 0.5) * R};
        for (int i = tid; i < P3; i += S::NT) acc[i] = 0.f;
        children(B, true);
        const int ntot = s_lpre[8];
        if (ntot > 0) anterpolate_pipe<P>(tv, cc, s2R, s_lstart, s_lpre, ntot, wrk, acc);
        float *Mo = M + (size_t)slot * P3;
        for (int i = tid; i < P3; i += S::NT) Mo[i] = acc[i];
        // arrivals, climbing while this CTA completes a box
        int X = B;
        bool own = true;  // acc holds X's own moments
        for (;;) {
            __threadfence();
            __syncthreads();
            if (tid == 0) s_last = atomicAdd(cnt + tv.bslot[X], 1) == s_nnl;
            __syncthreads();
            if (!s_last) break;
            __threadfence();
            const int nnl = s_nnl;
            if (nnl > 0) {
                float *MX = M + (size_t)tv.bslot[X] * P3;
                if (!own)
                    for (int i = tid; i < P3; i += S::NT) acc[i] = __ldcg(MX + i);
                for (int k = 0; k < nnl; ++k) {
                    const int e = s_kids[k], oc = e >> 27, D = e & ((1 << 27) - 1);
                    const float *MD = M + (size_t)tv.bslot[D] * P3;
                    __syncthreads();  // wrk and acc free (previous child done, acc loaded)
                    shift_pencils<P, 0, 0>(As + ((oc >> 2) & 1) * P * PS, MD, wrk);
                    __syncthreads();
                    shift_pencils<P, 1, 1>(As + ((oc >> 1) & 1) * P * PS, wrk, wrk);
                    __syncthreads();
                    shift_pencils<P, 2, 2>(As + (oc & 1) * P * PS, wrk, acc);
                }
                __syncthreads();
                for (int i = tid; i < P3; i += S::NT) MX[i] = acc[i];
            }
            const int par = tv.bparent[X];
            if (par < 0) break;
            X = par;
            own = false;
            children(X, false);
        }
    }
}

template <typename T, int P>
__global__ void __launch_bounds__(kThreads) k_upward(TreeView tv, DevTables<T> tb, int lstart, int lcount, T *M,
                                                     BufLayout lay, char *slab, int *tc_err) {
    extern __shared__ __align__(128) char sm[];
    using U = UpShape<P>;
    constexpr int P3 = P * P * P;
    constexpr int PS = U::PS, YS = U::YS;
    constexpr int NAG = (P + 3) / 4, NBCG = (P * P + 3) / 4;
    // the single-precision orders whose register tiles fit run in k_anterp; the
    // tensor-core form stays for the other single-precision orders
    constexpr bool kTC = sizeof(T) == 4 && U::TC_OK;
    __shared__ __align__(8) uint64_t s_bar;
    __shared__ uint32_t s_tmem;
    uint32_t phase = 0;
    if constexpr (kTC) {
        if ((threadIdx.x >> 5) == 0) tc::tmem_alloc(&s_tmem, U::TCOLS);
        if (threadIdx.x == 0) tc::mbar_init(&s_bar, 1);
        tc::fence_before_sync();
        __syncthreads();
        tc::fence_after_sync();
    }
    T *acc = buf_ptr<T, all_smem<T, P>()>(lay, 0, sm, slab);
    // scratch shared by the two phases: staging + Y for the sources of leaf
    // children, then two P^3 buffers for the moment shifts of non-leaf children
    T *scr = buf_ptr<T, all_smem<T, P>()>(lay, 1, sm, slab);
    T *As = buf_ptr<T, all_smem<T, P>()>(lay, 2, sm, slab);   // shift matrices A_{-1}, A_{+1}
    T *stg = scr;                           // [3][kCH][PS]
    T *Y = scr + 3 * kCH * PS;              // [kCH][YS]
    T *b0 = scr, *b1 = scr + P3;
    __shared__ int s_lstart[8], s_lpre[9];
    const int tid = threadIdx.x;
    for (int i = tid; i < 2 * P * P; i += kThreads) As[i] = tb.A[i];
    for (int it = blockIdx.x; it < lcount; it += gridDim.x) {
        const int B = lstart + it;
        const bool selfleaf = (tv.bflags[B] & BF_LEAF) != 0;
        // a leaf's sources go to its parent's grid; a root that is a leaf
        // anterpolates onto its own grid (for the windowed term W_0)
        if (selfleaf && tv.blevel[B] != 0) continue;
        if (tv.bnsrc[B] == 0) continue;
        for (int i = tid; i < P3; i += kThreads) acc[i] = (T)0;
        const int l = tv.blevel[B];
        int ix, iy, iz;
        box_decode_d(tv.bkey[B], l, ix, iy, iz);
        const double R = level_R(l), s2R = 2.0 / R;
        const double cc[3] = {(ix + 0.5) * R, (iy + 0.5) * R, (iz + 0.5) * R};
        __syncthreads();
        const int c0 = tv.bchild0[B];
        const unsigned cm = selfleaf ? 1u : tv.bcmask[B];
        // point ranges of the leaf children (with sources), streamed as one sequence
        if (tid == 0) {
            int k = 0, nl = 0, tot = 0;
            for (int oc = 0; oc < 8; ++oc) {
                if (!(cm & (1u << oc))) continue;
                const int D = selfleaf ? B : c0 + k;
                ++k;
                if (tv.bnsrc[D] == 0 || !(selfleaf || (tv.bflags[D] & BF_LEAF))) continue;
                s_lstart[nl] = tv.bstart[D];
                s_lpre[nl] = tot;
                tot += tv.bcount[D];
                ++nl;
            }
            for (int q = nl; q < 9; ++q) s_lpre[q] = tot;
        }
        __syncthreads();
        const int ntot = s_lpre[8];
        if constexpr (kTC) {
            if (ntot > 0) anterpolate_tc<P>(tv, cc, s2R, s_lstart, s_lpre, ntot, scr, s_tmem, &s_bar, phase, acc,
                                             tc_err);
        } else {
            {
                // anterpolation of the leaf children's sources onto this box's grid
                for (int p0 = 0; p0 < ntot; p0 += kCH) {
                    const int np = min(kCH, ntot - p0);
                    for (int t = tid; t < 3 * kCH; t += kThreads) {
                        const int ax = t / kCH, j = t % kCH;
                        T *o = stg + (ax * kCH + j) * PS;
                        if (j < np) {
                            int seg = 0;
                            while (seg < 7 && s_lpre[seg + 1] <= p0 + j) ++seg;
                            const int kk = s_lstart[seg] + (p0 + j - s_lpre[seg]);
                            const double u = ax == 0 ? tv.ux[kk] : (ax == 1 ? tv.uy[kk] : tv.uz[kk]);
                            const T xi = (T)((u - cc[ax]) * s2R);
                            const T w = ax == 0 ? (T)tv.q[kk] : (T)1;
                            T t0 = (T)1, t1 = xi;
                            o[0] = w;
                            if (P > 1) o[1] = w * xi;
#pragma unroll
                            for (int n = 2; n < P; ++n) {
                                T t2 = (T)2 * xi * t1 - t0;
                                o[n] = w * t2;
                                t0 = t1;
                                t1 = t2;
                            }
                        } else {
#pragma unroll
                            for (int n = 0; n < P; ++n) o[n] = (T)0;
                        }
                    }
                    __syncthreads();
                    // M[a][bc] += sum_j X[j][a] Y[j][bc], X = rho T_a(x), Y = T_b(y) T_c(z)
                    for (int i = tid; i < kCH * YS; i += kThreads) {
                        const int j = i / YS, bc = i % YS;
                        Y[i] = bc < P * P ? stg[(kCH + j) * PS + bc / P] * stg[(2 * kCH + j) * PS + bc % P] : (T)0;
                    }
                    __syncthreads();
                    for (int tile = tid; tile < NAG * NBCG; tile += kThreads) {
                        const int ag = tile / NBCG, bg = tile % NBCG;
                        T r[4][4];
#pragma unroll
                        for (int i = 0; i < 4; ++i)
#pragma unroll
                            for (int k = 0; k < 4; ++k) r[i][k] = (T)0;
                        for (int j = 0; j < np; ++j) {
                            T x[4], y[4];
                            ld4(stg + j * PS + ag * 4, x);
                            ld4(Y + j * YS + bg * 4, y);
#pragma unroll
                            for (int i = 0; i < 4; ++i)
#pragma unroll
                                for (int k = 0; k < 4; ++k) r[i][k] += x[i] * y[k];
                        }
#pragma unroll
                        for (int i = 0; i < 4; ++i) {
                            const int a = ag * 4 + i;
                            if (a >= P) continue;
#pragma unroll
                            for (int k = 0; k < 4; ++k) {
                                const int bc = bg * 4 + k;
                                if (bc < P * P) acc[a * P * P + bc] += r[i][k];
                            }
                        }
                    }
                    __syncthreads();
                }
            }
        }
        int k = 0;
        for (int oc = 0; oc < 8 && !selfleaf; ++oc) {
            if (!(cm & (1u << oc))) continue;
            const int D = c0 + k;
            ++k;
            if (tv.bnsrc[D] == 0 || (tv.bflags[D] & BF_LEAF)) continue;
            {
                // T_c2p: parent moments from child moments, exact
                const T *Mc = M + (size_t)tv.bslot[D] * P3;
                for (int i = tid; i < P3; i += kThreads) b0[i] = Mc[i];
                __syncthreads();
                shift_up<T, P, 0, kThreads, false>(As + ((oc >> 2) & 1) * P * P, b0, b1);
                __syncthreads();
                shift_up<T, P, 1, kThreads, false>(As + ((oc >> 1) & 1) * P * P, b1, b0);
                __syncthreads();
                shift_up<T, P, 2, kThreads, true>(As + (oc & 1) * P * P, b0, acc);
                __syncthreads();
            }
        }
        T *Mo = M + (size_t)tv.bslot[B] * P3;
        for (int i = tid; i < P3; i += kThreads) Mo[i] = acc[i];
        __syncthreads();
    }
    if constexpr (kTC) {
        tc::fence_before_sync();
        __syncthreads();
        tc::fence_after_sync();
        if ((threadIdx.x >> 5) == 0) tc::tmem_dealloc(s_tmem, U::TCOLS);
    }
}

// ---------------------------------------------------------------------------
// Outgoing expansions (Step 3, T_prox2pw), parity-split
// ---------------------------------------------------------------------------
// PLANE: the plane-major layout of the tensor-core incoming pass,
// Phi[slot][m_z][m_y][m_x] with m_x padded to an even count; otherwise
// Phi[slot][m_y][m_x][m_z] with m_z padded to an even count
template <typename T, int P, int NF, bool PLANE>
__global__ void __launch_bounds__(kThreads) k_prox2pw(TreeView tv, DevTables<T> tb, int nslots,
                                                      const int32_t *slot2box, const T *M,
                                                      typename Cplx<T>::type *Phi, BufLayout lay, char *slab) {
    using C2 = typename Cplx<T>::type;
    extern __shared__ __align__(128) char sm[];
    constexpr int P3 = P * P * P, NH = NF + 1, N1 = 2 * NF + 1;
    T *Mb = buf_ptr<T, all_smem<T, P>()>(lay, 0, sm, slab);
    C2 *T1 = buf_ptr<C2, all_smem<T, P>()>(lay, 1, sm, slab);  // [a][b][mz]
    C2 *T2 = buf_ptr<C2, all_smem<T, P>()>(lay, 2, sm, slab);  // [a][my + NF][mz]
    T *hs = buf_ptr<T, all_smem<T, P>()>(lay, 3, sm, slab);    // [n][m']
    const int tid = threadIdx.x;
    load_hs<T, P, NF>(tb, hs);
    constexpr int NHP = nz_pad<NF>(), MXP = (N1 + 1) & ~1;
    const size_t stride = PLANE ? (size_t)NH * N1 * MXP : (size_t)N1 * N1 * NHP;
    // element (m_y, m_x, m_z) of a box's array (indices from 0)
    auto at = [](int my, int mx, int mz) -> size_t {
        return PLANE ? ((size_t)mz * N1 + my) * MXP + mx : (size_t)(my * N1 + mx) * NHP + mz;
    };
    for (int slot = blockIdx.x; slot < nslots; slot += gridDim.x) {
        const int B = slot2box[slot];
        if (!(tv.bflags[B] & BF_FOUT)) continue;
        __syncthreads();
        const T *Ms = M + (size_t)slot * P3;
        for (int i = tid; i < P3; i += kThreads) Mb[i] = Ms[i];
        __syncthreads();
        // z: T1[a][b][mz] = sum_{c even} Fr M + i sum_{c odd} Fi M, mz >= 0
        for (int ab = tid; ab < P * P; ab += kThreads) {
            T E[NH], O[NH];
#pragma unroll
            for (int m = 0; m < NH; ++m) E[m] = O[m] = (T)0;
            const T *row = Mb + ab * P;
#pragma unroll 2
            for (int c = 0; c < P; ++c) {
                const T v = row[c];
                const T *h = hs + c * NH;
                if (c & 1) {
#pragma unroll
                    for (int m = 0; m < NH; ++m) O[m] += h[m] * v;
                } else {
#pragma unroll
                    for (int m = 0; m < NH; ++m) E[m] += h[m] * v;
                }
            }
#pragma unroll
            for (int m = 0; m < NH; ++m) T1[ab * NH + m] = C2{E[m], O[m]};
        }
        __syncthreads();
        // y: T2[a][+-my'][mz] = E +- i O
        for (int it = tid; it < P * NH * NH; it += kThreads) {
            const int a = it / (NH * NH), r = it % (NH * NH), myp = r / NH, mz = r % NH;
            C2 E{0, 0}, O{0, 0};
            for (int b = 0; b < P; ++b) {
                const C2 t = T1[(a * P + b) * NH + mz];
                const T h = hs[b * NH + myp];
                if (b & 1) cfma(O, h, t); else cfma(E, h, t);
            }
            T2[(a * N1 + NF + myp) * NH + mz] = C2{E.x - O.y, E.y + O.x};
            if (myp > 0) T2[(a * N1 + NF - myp) * NH + mz] = C2{E.x + O.y, E.y - O.x};
        }
        __syncthreads();
        // x: Phi[my][+-mx'][mz] = E +- i O
        C2 *out = Phi + (size_t)slot * stride;
        for (int it = tid; it < N1 * NH * NH; it += kThreads) {
            // consecutive threads write consecutive elements: m_z fastest, or m_x in
            // the plane-major layout
            int my, mxp, mz;
            if (PLANE) {
                mz = it / (N1 * NH);
                my = (it / NH) % N1;
                mxp = it % NH;
            } else {
                my = it / (NH * NH);
                mxp = (it / NH) % NH;
                mz = it % NH;
            }
            C2 E{0, 0}, O{0, 0};
            for (int a = 0; a < P; ++a) {
                const C2 t = T2[(a * N1 + my) * NH + mz];
                const T h = hs[a * NH + mxp];
                if (a & 1) cfma(O, h, t); else cfma(E, h, t);
            }
            out[at(my, NF + mxp, mz)] = C2{E.x - O.y, E.y + O.x};
            if (mxp > 0) out[at(my, NF - mxp, mz)] = C2{E.x + O.y, E.y - O.x};
        }
    }
}

// ---------------------------------------------------------------------------
// Roots: windowed kernel W_0 over each system's unit box (global scratch per CTA)
// ---------------------------------------------------------------------------
template <typename T, int P>
__global__ void __launch_bounds__(kThreads) k_root(TreeView tv, DevTables<T> tb, const T *M, int nroots, T *LamW_all,
                                                   typename Cplx<T>::type *scr_all, size_t scr_elems) {
    using C2 = typename Cplx<T>::type;
    constexpr int P3 = P * P * P;
    const int n0 = tb.n0, NW = tb.NW, nh = tb.nhW;
    const T *Fr = tb.FWr, *Fi = tb.FWi;
    const int tid = threadIdx.x;
    C2 *scr = scr_all + (size_t)blockIdx.x * scr_elems;
    // one root (system) per iteration: the roots are boxes 0 .. nroots - 1
    for (int r = blockIdx.x; r < nroots; r += gridDim.x) {
    T *LamW = LamW_all + (size_t)r * P3;
    __syncthreads();
    if (tv.bnsrc[r] == 0 || tv.bslot[r] < 0) {
        for (int i = tid; i < P3; i += kThreads) LamW[i] = (T)0;
        continue;
    }
    const T *Mroot = M + (size_t)tv.bslot[r] * P3;
    C2 *T1 = scr;                                  // [a][b][mz]
    C2 *T2 = T1 + P * P * nh;                      // [a][my][mz]
    C2 *Ph = T2 + P * NW * nh;                     // [my][mx][mz]
    C2 *U1 = Ph + NW * NW * nh;                    // [a][my][mz]
    C2 *U2 = U1 + P * NW * nh;                     // [a][b][mz]
    for (int i = tid; i < P * P * nh; i += kThreads) {
        const int mz = i % nh, ab = i / nh;
        T re = 0, im = 0;
        for (int c = 0; c < P; ++c) {
            re += Fr[(mz + n0) * P + c] * Mroot[ab * P + c];
            im += Fi[(mz + n0) * P + c] * Mroot[ab * P + c];
        }
        T1[i] = C2{re, im};
    }
    __syncthreads();
    for (int i = tid; i < P * NW * nh; i += kThreads) {
        const int mz = i % nh, my = (i / nh) % NW, a = i / (nh * NW);
        T re = 0, im = 0;
        for (int b = 0; b < P; ++b) {
            const C2 t = T1[(a * P + b) * nh + mz];
            const T fr = Fr[my * P + b], fi = Fi[my * P + b];
            re += fr * t.x - fi * t.y;
            im += fr * t.y + fi * t.x;
        }
        T2[i] = C2{re, im};
    }
    __syncthreads();
    for (int i = tid; i < NW * NW * nh; i += kThreads) {
        const int mz = i % nh, mx = (i / nh) % NW, my = i / (nh * NW);
        T re = 0, im = 0;
        for (int a = 0; a < P; ++a) {
            const C2 t = T2[(a * NW + my) * nh + mz];
            const T fr = Fr[mx * P + a], fi = Fi[mx * P + a];
            re += fr * t.x - fi * t.y;
            im += fr * t.y + fi * t.x;
        }
        const int mxv = mx - n0, myv = my - n0;
        const T w = tb.wW[mxv * mxv + myv * myv + mz * mz];
        Ph[i] = C2{re * w, im * w};
    }
    __syncthreads();
    // back to Chebyshev coefficients: G[n][m] = conj(F[m][n])
    for (int i = tid; i < P * NW * nh; i += kThreads) {
        const int mz = i % nh, my = (i / nh) % NW, a = i / (nh * NW);
        T re = 0, im = 0;
        for (int mx = 0; mx < NW; ++mx) {
            const C2 t = Ph[(my * NW + mx) * nh + mz];
            const T gr = Fr[mx * P + a], gi = -Fi[mx * P + a];
            re += gr * t.x - gi * t.y;
            im += gr * t.y + gi * t.x;
        }
        U1[i] = C2{re, im};
    }
    __syncthreads();
    for (int i = tid; i < P * P * nh; i += kThreads) {
        const int mz = i % nh, b = (i / nh) % P, a = i / (nh * P);
        T re = 0, im = 0;
        for (int my = 0; my < NW; ++my) {
            const C2 t = U1[(a * NW + my) * nh + mz];
            const T gr = Fr[my * P + b], gi = -Fi[my * P + b];
            re += gr * t.x - gi * t.y;
            im += gr * t.y + gi * t.x;
        }
        U2[i] = C2{re, im};
    }
    __syncthreads();
    for (int i = tid; i < P3; i += kThreads) {
        const int c = i % P, ab = i / P;
        T s = 0;
        for (int mz = 0; mz < nh; ++mz) {
            const C2 t = U2[ab * nh + mz];
            const T cz = mz == 0 ? (T)1 : (T)2;
            s += cz * (Fr[(mz + n0) * P + c] * t.x + Fi[(mz + n0) * P + c] * t.y);
        }
        LamW[i] = s;
    }
    }
}

// ---------------------------------------------------------------------------
// Local expansions and leaf evaluation (Step 3), parity-split
// ---------------------------------------------------------------------------
constexpr int kLThreads = 512;
constexpr int kECH = 32;  // targets per evaluation chunk

// One axis of a Chebyshev re-expansion on a P^3 array: out[.., m, ..] =
// sum_{n >= m} A[n][m] in[.., n, ..] along axis AX (0 = z, the fastest index,
// 1 = y, 2 = x).  A is P rows of PA = (P + 3) & ~3 entries, zero above the
// diagonal (m > n), so single precision reads a row's entries four at a time.
// Each thread owns one row (two when the rows outnumber the threads) of P
// outputs in registers.
template <typename T, int P> constexpr int shift_pad() { return (P + 3) & ~3; }
template <typename T, int P, int AX, int NT>
__device__ __forceinline__ void shift_pass(const T *__restrict__ A, const T *in, T *out) {
    constexpr int PA = shift_pad<T, P>();
    constexpr int s = AX == 0 ? 1 : (AX == 1 ? P : P * P);
    if constexpr (P > 20) {  // large orders: one output per thread (registers)
        for (int i = threadIdx.x; i < P * P * P; i += NT) {
            const int m = AX == 0 ? i % P : (AX == 1 ? (i / P) % P : i / (P * P));
            const int b = i - m * s;
            T acc = 0;
            for (int n = m; n < P; ++n) acc += A[n * PA + m] * in[b + n * s];
            out[i] = acc;
        }
        return;
    }
    constexpr bool TWO = P * P > NT;
    constexpr int RR = P * P, H = TWO ? (RR + 1) / 2 : RR;
    auto base = [](int r) { return AX == 0 ? r * P : (AX == 1 ? (r / P) * P * P + r % P : r); };
    for (int t = threadIdx.x; t < H; t += NT) {
        const int r0 = t, r1 = t + H;
        const bool has1 = TWO && r1 < RR;
        const int b0 = base(r0), b1 = has1 ? base(r1) : b0;
        T o0[PA], o1[PA];
#pragma unroll
        for (int m = 0; m < PA; ++m) o0[m] = o1[m] = (T)0;
#pragma unroll
        for (int n = 0; n < P; ++n) {
            const T v0 = in[b0 + n * s], v1 = in[b1 + n * s];
            if constexpr (sizeof(T) == 4) {
                const float4 *Ar = reinterpret_cast<const float4 *>(A + n * PA);
#pragma unroll
                for (int m4 = 0; m4 <= n / 4; ++m4) {
                    const float4 w = Ar[m4];
                    o0[4 * m4] += w.x * v0;
                    o0[4 * m4 + 1] += w.y * v0;
                    o0[4 * m4 + 2] += w.z * v0;
                    o0[4 * m4 + 3] += w.w * v0;
                    if (TWO) {
                        o1[4 * m4] += w.x * v1;
                        o1[4 * m4 + 1] += w.y * v1;
                        o1[4 * m4 + 2] += w.z * v1;
                        o1[4 * m4 + 3] += w.w * v1;
                    }
                }
            } else {
#pragma unroll
                for (int m = 0; m <= n; ++m) {
                    const T a = A[n * PA + m];
                    o0[m] += a * v0;
                    if (TWO) o1[m] += a * v1;
                }
            }
        }
#pragma unroll
        for (int m = 0; m < P; ++m) out[b0 + m * s] = o0[m];
        if (has1) {
#pragma unroll
            for (int m = 0; m < P; ++m) out[b1 + m * s] = o1[m];
        }
    }
}

// Work split of a contraction with `base` independent outputs per coefficient
// index (P of them) over `threads` threads: the index is cut into G groups of
// ceil(P / G) per thread item, and base * G items run in ceil(base G / threads)
// rounds between barriers.  Per inner step an item loads its inputs (~2
// instructions) and updates its accumulators (~3 each), so G minimises
// rounds x (2 + 3 ceil(P / G)), the time to the barrier, with at most max_per
// accumulators per item (registers); ties go to fewer groups.
constexpr int best_groups(int base, int P, int threads, int max_per) {
    int best = P, cost = 1 << 30;
    for (int G = 1; G <= P; ++G) {
        const int per = (P + G - 1) / G;
        if (per > max_per) continue;
        const int c = ((base * G + threads - 1) / threads) * (2 + 3 * per);
        if (c < cost) { cost = c; best = G; }
    }
    return best;
}

template <int P, int NF> struct LocalShape {
    static constexpr int NH = NF + 1, N1 = 2 * NF + 1;
    // phase B: a-groups, a per group (two complex accumulators per a)
    static constexpr int AG = best_groups(NH * NH, P, 512, 8), AC = (P + AG - 1) / AG;
    static constexpr int BG = best_groups(P * NH, P, 512, 10), BC = (P + BG - 1) / BG;  // phase C
    static constexpr int CG = best_groups(P * P, P, 512, 20), CC = (P + CG - 1) / CG;   // phase D
    // tensor-core leaf evaluation D[j][ab] = sum_c T_c(z_j) Lambda[ab][c]:
    // 128 targets per tile (M), ab padded to NP (N, multiple of 16, split into
    // at most two MMAs of <= 256 columns), c padded to KP (K, multiple of 8)
    static constexpr int TM = 128;
    static constexpr int NP = (P * P + 15) / 16 * 16, KP = (P + 7) / 8 * 8;
    static constexpr int NA = NP <= 256 ? NP : (NP / 2 + 15) / 16 * 16, NB = NP - NA;
    static constexpr int TCOLS = NP <= 128 ? 128 : (NP <= 256 ? 256 : 512);
    static constexpr bool TC_OK = NP <= 512 && NA <= 256 && NB <= 256;  // accumulator fits in TMEM
    // shared memory of the tensor-core evaluation: buffer 1 holds B_hi, A_hi,
    // A_lo, buffer 2 holds B_lo (floats)
    static constexpr int TC_BUF1 = NP * KP + 2 * TM * KP, TC_BUF2 = NP * KP;
};

// asynchronous 8-byte global -> shared copies (Ampere-style cp.async)
__device__ __forceinline__ void cp_async8(void *dst_smem, const void *src) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(tc::smem_addr(dst_smem)), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }

// T_0(x) .. T_{P-1}(x) by the three-term recurrence
template <int P> __device__ __forceinline__ void cheb_row(float x, float (&t)[P]) {
    t[0] = 1.f;
    if (P > 1) t[1] = x;
#pragma unroll
    for (int n = 2; n < P; ++n) t[n] = 2.f * x * t[n - 1] - t[n - 2];
}

// T_n(x) and T_n'(x) by their recurrences (T'_{n+1} = 2 T_n + 2 x T'_n - T'_{n-1})
template <int P> __device__ __forceinline__ void cheb_row_d(float x, float (&t)[P], float (&dt)[P]) {
    t[0] = 1.f;
    dt[0] = 0.f;
    if (P > 1) {
        t[1] = x;
        dt[1] = 1.f;
    }
#pragma unroll
    for (int n = 2; n < P; ++n) {
        t[n] = 2.f * x * t[n - 1] - t[n - 2];
        dt[n] = 2.f * t[n - 1] + 2.f * x * dt[n - 1] - dt[n - 2];
    }
}

// the same column range for the potential and its x and y derivatives:
// u = sum T_a T_b D, gx = sum T'_a T_b D, gy = sum T_a T'_b D
template <int P, int C0, int C1>
__device__ __forceinline__ void eval_part_g(uint32_t trow, const float (&tx)[P], const float (&ty)[P],
                                            const float (&dtx)[P], const float (&dty)[P], float &u, float &gx,
                                            float &gy) {
    constexpr int B = 4;
    float su = 0.f, sx = 0.f, sy = 0.f, acc = 0.f, accd = 0.f;
#pragma unroll
    for (int c = C0; c < C1; c += B) {
        float d[B][8];
#pragma unroll
        for (int g = 0; g < B; ++g)
            if (c + g < C1) tc::ld_x8(trow + (uint32_t)((c + g) * 8), d[g]);
        tc::ld_wait();
#pragma unroll
        for (int g = 0; g < B; ++g)
#pragma unroll
            for (int q = 0; q < 8; ++q) {
                const int n = (c + g) * 8 + q;
                if (c + g < C1 && n < P * P) {
                    acc += ty[n % P] * d[g][q];
                    accd += dty[n % P] * d[g][q];
                    if (n % P == P - 1) {
                        su += tx[n / P] * acc;
                        sx += dtx[n / P] * acc;
                        sy += tx[n / P] * accd;
                        acc = accd = 0.f;
                    }
                }
            }
    }
    constexpr int nlast = (8 * C1 < P * P ? 8 * C1 : P * P) - 1;
    if (nlast >= 8 * C0 && nlast % P != P - 1) {
        su += tx[nlast / P] * acc;
        sx += dtx[nlast / P] * acc;
        sy += tx[nlast / P] * accd;
    }
    u = su;
    gx = sx;
    gy = sy;
}

// sum over the accumulator columns n = 8 C0 .. 8 C1 - 1 (n = a P + b) of this
// thread's TMEM lane: T_a(x) T_b(y) D[n], up to six 8-column chunks per wait
template <int P, int C0, int C1>
__device__ __forceinline__ float eval_part(uint32_t trow, const float (&tx)[P], const float (&ty)[P]) {
    constexpr int B = 6;
    float sum = 0.f, acc = 0.f;
#pragma unroll
    for (int c = C0; c < C1; c += B) {
        float d[B][8];
#pragma unroll
        for (int g = 0; g < B; ++g)
            if (c + g < C1) tc::ld_x8(trow + (uint32_t)((c + g) * 8), d[g]);
        tc::ld_wait();
#pragma unroll
        for (int g = 0; g < B; ++g)
#pragma unroll
            for (int q = 0; q < 8; ++q) {
                const int n = (c + g) * 8 + q;
                if (c + g < C1 && n < P * P) {
                    acc += ty[n % P] * d[g][q];
                    if (n % P == P - 1) {
                        sum += tx[n / P] * acc;
                        acc = 0.f;
                    }
                }
            }
    }
    // a row a cut by the end of the range
    constexpr int nlast = (8 * C1 < P * P ? 8 * C1 : P * P) - 1;
    if (nlast >= 8 * C0 && nlast % P != P - 1) sum += tx[nlast / P] * acc;
    return sum;
}

// Shared state of the tensor-core leaf evaluation.
struct TcEval {
    float *Bh, *Bl, *Ah, *Al;  // operands (K-major, TF32 hi and lo)
    uint64_t *bar;             // MMA completion
    uint32_t tmem;             // accumulator base
    int *pending;              // an MMA batch outlived its wait
    float *red;                // partial sums of column groups 1..3: [4 values][3][128]
    int *err;                  // device error word
};

// point of position gp in a table of point ranges (starts rs, prefix offsets ro)
__device__ __forceinline__ int range_point(const int *rs, const int *ro, int gp) {
    int r = 0;
    while (gp >= ro[r + 1]) ++r;
    return rs[r] + gp - ro[r];
}

// Tensor cores: evaluate the Chebyshev expansion Lev (P^3, box centre cc,
// scale s2R = 2 / R) at the points of nr ranges: D[j][ab] = sum_c T_c(z_j)
// Lev[ab][c] for 128 points at a time (points on the TMEM lanes), then each
// point's threads form u_j = sum_a T_a(x_j) sum_b T_b(y_j) D[j][ab].  Operands
// are split into TF32 hi + lo and D = A_lo B_hi + A_hi B_lo + A_hi B_hi.  The
// first 128 points' coordinates are in xyz (fetched by cp.async).  With gfar,
// also the gradient in unit-box coordinates: d/dx and d/dy from the same D with
// T'_a or T'_b, d/dz from a second MMA with the A operand T'_c(z).  Called by
// the whole CTA.
template <int P, int NF>
__device__ void tc_eval(const TreeView &tv, const float *Lev, const double (&cc)[3], double s2R, const int *rs,
                        const int *ro, int nr, const double (*xyz)[128], const TcEval &st, uint32_t &phase,
                        double *ufar, double *gfar) {
    using S = LocalShape<P, NF>;
    const int tid = threadIdx.x, warp = tid >> 5;
    const int ntot = ro[nr];
    // B operand: row ab, column c of Lev; one float4 (4 columns) per step
    // (unrolled: a fixed trip count, all loads of a thread in flight together)
#pragma unroll
    for (int t = tid; t < S::NP * S::KP / 4; t += kLThreads) {
        const int r = t & 7, k4 = (t >> 3) % (S::KP / 4), n = ((t >> 3) / (S::KP / 4)) * 8 + r;
        float h[4], l[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int k = 4 * k4 + q;
            const float v = (n < P * P && k < P) ? Lev[n * P + k] : 0.f;
            tc::split_tf32(v, h[q], l[q]);
        }
        reinterpret_cast<float4 *>(st.Bh)[t] = make_float4(h[0], h[1], h[2], h[3]);
        reinterpret_cast<float4 *>(st.Bl)[t] = make_float4(l[0], l[1], l[2], l[3]);
    }
    cp_async_wait_all();
    __syncthreads();
    for (int p0 = 0; p0 < ntot; p0 += S::TM) {
        const int np = min(S::TM, ntot - p0);
        const bool first = p0 == 0;  // coordinates already in xyz
        // this thread's epilogue point
        const int jq = min(tid & (S::TM - 1), np - 1);
        const int pq = range_point(rs, ro, p0 + jq);
        const double xq = first ? xyz[0][jq] : tv.ux[pq];
        const double yq = first ? xyz[1][jq] : tv.uy[pq];
        // A operand row j = T_c(z_j) (deriv: T_c'(z_j)), c < P, zero rows past the points
        auto build_a = [&](bool deriv) {
            if (tid >= S::TM) return;
            const int j = tid;
            float tz[S::KP], dz[S::KP];
#pragma unroll
            for (int n = 0; n < S::KP; ++n) tz[n] = dz[n] = 0.f;
            if (j < np) {
                const float zi = (float)(((first ? xyz[2][j] : tv.uz[pq]) - cc[2]) * s2R);
                tz[0] = 1.f;
                if (P > 1) {
                    tz[1] = zi;
                    dz[1] = 1.f;
                }
#pragma unroll
                for (int n = 2; n < P; ++n) {
                    tz[n] = 2.f * zi * tz[n - 1] - tz[n - 2];
                    dz[n] = 2.f * tz[n - 1] + 2.f * zi * dz[n - 1] - dz[n - 2];
                }
            }
#pragma unroll
            for (int k4 = 0; k4 < S::KP / 4; ++k4) {
                float h[4], l[4];
#pragma unroll
                for (int q = 0; q < 4; ++q) tc::split_tf32(deriv ? dz[4 * k4 + q] : tz[4 * k4 + q], h[q], l[q]);
                const int o = ((j >> 3) * (S::KP / 4) + k4) * 8 + (j & 7);
                reinterpret_cast<float4 *>(st.Ah)[o] = make_float4(h[0], h[1], h[2], h[3]);
                reinterpret_cast<float4 *>(st.Al)[o] = make_float4(l[0], l[1], l[2], l[3]);
            }
        };
        auto issue = [&]() {
            if (tid != 0) return;
            constexpr uint32_t lbo = 128, sbo = S::KP * 32;
            const uint32_t aH = tc::smem_addr(st.Ah), aL = tc::smem_addr(st.Al);
            const uint32_t bH = tc::smem_addr(st.Bh), bL = tc::smem_addr(st.Bl);
#pragma unroll
            for (int h = 0; h < (S::NB > 0 ? 2 : 1); ++h) {
                const int n0 = h ? S::NA : 0;
                const uint32_t id = tc::idesc_tf32(S::TM, h ? S::NB : S::NA);
                const uint32_t boff = (uint32_t)(n0 / 8) * sbo, dcol = st.tmem + (uint32_t)n0;
#pragma unroll
                for (int ks = 0; ks < S::KP / 8; ++ks) {
                    const uint32_t ko = (uint32_t)ks * 256;
                    tc::mma_tf32(dcol, tc::sdesc(aL + ko, lbo, sbo), tc::sdesc(bH + boff + ko, lbo, sbo), id, ks > 0);
                    tc::mma_tf32(dcol, tc::sdesc(aH + ko, lbo, sbo), tc::sdesc(bL + boff + ko, lbo, sbo), id, true);
                    tc::mma_tf32(dcol, tc::sdesc(aH + ko, lbo, sbo), tc::sdesc(bH + boff + ko, lbo, sbo), id, true);
                }
            }
            tc::commit(st.bar);
        };
        // every warp waits; warps w, w + 4, w + 8, w + 12 share TMEM lanes
        // 32 (w mod 4) .. + 31 (points j) and split the ab columns
        auto wait = [&]() {
            bool ok = tc::mbar_wait(st.bar, phase, 2000000000ll);  // about 1 s
            ok = __all_sync(0xffffffffu, ok);
            tc::fence_after_sync();
            phase ^= 1u;
            if (!ok && (tid & 31) == 0) {
                atomicExch(st.err, 1);
                *st.pending = 1;
            }
            return ok;
        };
        const int j = tid & (S::TM - 1), cg = tid >> 7;
        const uint32_t trow = st.tmem + ((uint32_t)((warp & 3) * 32) << 16);
        constexpr int NC = S::NP / 8;  // 8-column chunks
        auto red = [&](int v, int g) -> float & { return st.red[(v * 3 + g) * 128 + j]; };
        build_a(false);
        tc::fence_proxy_async();
        tc::fence_before_sync();
        __syncthreads();
        tc::fence_after_sync();
        issue();
        const bool ok = wait();
        float tx[P], ty[P], dtx[P], dty[P];
        cheb_row_d<P>((float)((xq - cc[0]) * s2R), tx, dtx);
        cheb_row_d<P>((float)((yq - cc[1]) * s2R), ty, dty);
        float pu = 0.f, pgx = 0.f, pgy = 0.f, pgz = 0.f;
        if (ok && !gfar) {
            switch (cg) {
            case 0: pu = eval_part<P, 0, NC / 4>(trow, tx, ty); break;
            case 1: pu = eval_part<P, NC / 4, NC / 2>(trow, tx, ty); break;
            case 2: pu = eval_part<P, NC / 2, 3 * NC / 4>(trow, tx, ty); break;
            default: pu = eval_part<P, 3 * NC / 4, NC>(trow, tx, ty); break;
            }
        } else if (ok) {
            switch (cg) {
            case 0: eval_part_g<P, 0, NC / 4>(trow, tx, ty, dtx, dty, pu, pgx, pgy); break;
            case 1: eval_part_g<P, NC / 4, NC / 2>(trow, tx, ty, dtx, dty, pu, pgx, pgy); break;
            case 2: eval_part_g<P, NC / 2, 3 * NC / 4>(trow, tx, ty, dtx, dty, pu, pgx, pgy); break;
            default: eval_part_g<P, 3 * NC / 4, NC>(trow, tx, ty, dtx, dty, pu, pgx, pgy); break;
            }
        }
        if (gfar) {
            // d/dz: a second MMA with T_c'(z) once every warp has read the first D
            build_a(true);
            tc::fence_proxy_async();
            tc::fence_before_sync();
            __syncthreads();
            tc::fence_after_sync();
            issue();
            if (wait()) {
                switch (cg) {
                case 0: pgz = eval_part<P, 0, NC / 4>(trow, tx, ty); break;
                case 1: pgz = eval_part<P, NC / 4, NC / 2>(trow, tx, ty); break;
                case 2: pgz = eval_part<P, NC / 2, 3 * NC / 4>(trow, tx, ty); break;
                default: pgz = eval_part<P, 3 * NC / 4, NC>(trow, tx, ty); break;
                }
            }
        }
        if (cg > 0) {
            red(0, cg - 1) = pu;
            if (gfar) {
                red(1, cg - 1) = pgx;
                red(2, cg - 1) = pgy;
                red(3, cg - 1) = pgz;
            }
        }
        tc::fence_before_sync();
        __syncthreads();
        // added to the (zeroed) far field: a target may take two expansions, its
        // parent's and its own incoming one
        if (cg == 0 && j < np && (tv.pflag[pq] & 2)) {
            ufar[pq] += (double)(pu + red(0, 0) + red(0, 1) + red(0, 2));
            if (gfar) {
                gfar[3 * (size_t)pq + 0] += (double)(pgx + red(1, 0) + red(1, 1) + red(1, 2)) * s2R;
                gfar[3 * (size_t)pq + 1] += (double)(pgy + red(2, 0) + red(2, 1) + red(2, 2)) * s2R;
                gfar[3 * (size_t)pq + 2] += (double)(pgz + red(3, 0) + red(3, 1) + red(3, 2)) * s2R;
            }
        }
    }
}

// cp.async of the coordinates of the first 128 points of a range table
__device__ __forceinline__ void fetch_xyz(const TreeView &tv, const int *rs, const int *ro, int nr,
                                          double (*xyz)[128]) {
    const int n0 = min(128, ro[nr]);
    for (int t = threadIdx.x; t < 3 * 128; t += blockDim.x) {
        const int ax = t >> 7, j = t & 127;
        if (j < n0) {
            const int pt = range_point(rs, ro, j);
            cp_async8(&xyz[ax][j], (ax == 0 ? tv.ux : (ax == 1 ? tv.uy : tv.uz)) + pt);
        }
    }
    cp_async_commit();
}

template <typename T, int P, int NF>
__global__ void __launch_bounds__(kLThreads, 1) k_local(TreeView tv, DevTables<T> tb, int level, int lstart,
                                                        int lcount, const typename Cplx<T>::type *Phi, T *Lam,
                                                        const T *LamW, double *ufar, BufLayout lay, char *slab,
                                                        unsigned long long *flops, int *tc_err, int *run_ctr,
                                                        double *gfar, typename Cplx<T>::type *psig,
                                                        const T *lam_in, const int32_t *bfin, int lstr) {
    using C2 = typename Cplx<T>::type;
    using S = LocalShape<P, NF>;
    constexpr int NH = S::NH, N1 = S::N1, P3 = P * P * P, NHP = nz_pad<NF>();
    // single precision evaluates the leaves on the tensor cores (3xTF32)
    constexpr bool kTC = sizeof(T) == 4 && S::TC_OK;
    extern __shared__ __align__(128) char sm[];
    T *Ls = buf_ptr<T, all_smem<T, P>()>(lay, 0, sm, slab);
    C2 *PsE = buf_ptr<C2, all_smem<T, P>()>(lay, 1, sm, slab);  // [my + NF][mx'][mz]; PsO follows
    C2 *PsO = PsE + N1 * NH * NHP;
    C2 *T2 = PsE;                              // [a][b][mz], reuses the Psi buffers
    C2 *T1e = buf_ptr<C2, all_smem<T, P>()>(lay, 2, sm, slab);  // [a][my'][mz]; T1o follows
    C2 *T1o = T1e + P * NH * NH;
    T *hs = buf_ptr<T, all_smem<T, P>()>(lay, 3, sm, slab);
    T *ev = buf_ptr<T, all_smem<T, P>()>(lay, 4, sm, slab);     // [2][3][kECH][P]: T_n and T_n' of the evaluation chunk
    T *As = buf_ptr<T, all_smem<T, P>()>(lay, 5, sm, slab);     // shift matrices A_{-1}, A_{+1}
    __shared__ int s_ncol;
    __shared__ int s_cslot[27];
    __shared__ int s_cd[27][3];
    __shared__ int s_blk[64];  // slots of the F_out boxes of a sibling group's 4 x 4 x 4 block
    __shared__ int s_gtr;      // the group pass runs: bit 8, and the octants it keeps (F_in siblings)
    __shared__ __align__(8) uint64_t s_bar;  // MMA completion
    __shared__ uint32_t s_tmem;              // TMEM accumulator base
    __shared__ int s_pending;                // an MMA batch outlived its wait
    __shared__ float s_red[4 * 3 * 128];     // partial leaf sums (and gradients) of column groups 1..3
    __shared__ float2 s_ud[27 * 27];         // translation phases per colleague and residue class
    __shared__ double s_xyz[3][128];         // a leaf's first 128 points, fetched while its expansion forms
    const int tid = threadIdx.x, warp = tid >> 5;
    uint32_t phase = 0;
    if constexpr (kTC) {
        if (warp == 0) tc::tmem_alloc(&s_tmem, S::TCOLS);
        if (tid == 0) {
            tc::mbar_init(&s_bar, 1);
            s_pending = 0;
        }
        tc::fence_before_sync();
        __syncthreads();
        tc::fence_after_sync();
    }
    load_hs<T, P, NF>(tb, hs);
    {
        // the shift matrices with rows padded to shift_pad entries, zero above the diagonal
        constexpr int PA = shift_pad<T, P>();
        for (int i = tid; i < 2 * P * PA; i += kLThreads) {
            const int h = i / (P * PA), n = (i / PA) % P, m = i % PA;
            As[i] = (m < P && m <= n) ? tb.A[h * P * P + n * P + m] : (T)0;
        }
    }
    const size_t pstride = (size_t)N1 * N1 * NHP;
    const T invR = (T)(double)(1u << level);
    const T kH = (T)0.86602540378443864676;  // sqrt(3)/2
    T *Pl = buf_ptr<T, all_smem<T, P>()>(lay, 6, sm, slab);     // the parent's Lambda, kept for its next children
    int cur_parent = -1;
    __shared__ int s_run;
    __shared__ int s_grs[8], s_gro[9], s_gnr, s_gntgt;  // a sibling group's leaves evaluated in the parent
    __shared__ int s_brs[1], s_bro[2];                  // one leaf
    __shared__ double s_gxyz[3][128];                   // the group's first 128 points
    TcEval st{};
    if constexpr (kTC) {
        st.Bh = reinterpret_cast<float *>(PsE);
        st.Ah = st.Bh + S::NP * S::KP;
        st.Al = st.Ah + S::TM * S::KP;
        st.Bl = reinterpret_cast<float *>(T1e);
        st.bar = &s_bar;
        st.tmem = s_tmem;
        st.pending = &s_pending;
        st.red = s_red;
        st.err = tc_err;
    }
    auto parent_of = [&](int i) { return level > 0 ? tv.bparent[lstart + i] : -1; };
    // runs of 8 consecutive boxes from a work counter, moved to whole sibling
    // groups (children of one parent are adjacent in Morton order): a run
    // leaves a group that started in the previous run to that run's CTA and
    // finishes the group it ends in
    for (;;) {
        __syncthreads();
        if (tid == 0) s_run = atomicAdd(run_ctr, 1);
        __syncthreads();
        const int r0 = s_run * 8;
        if (r0 >= lcount) break;
        const int r1 = min(r0 + 8, lcount);
        int a0 = r0, a1 = r1;
        if (level > 0) {
            if (r0 > 0) {
                const int pp = parent_of(r0 - 1);
                while (a0 < r1 && parent_of(a0) == pp) ++a0;
            }
            while (a1 < lcount && parent_of(a1) == parent_of(a1 - 1)) ++a1;
        }
        for (int g0 = a0, g1 = a0; g0 < a1; g0 = g1) {
            const int Pg = parent_of(g0);
            g1 = g0 + 1;
            while (level > 0 && g1 < a1 && parent_of(g1) == Pg) ++g1;
            // leaves without incoming expansion keep their parent's Lambda: T_p2c is
            // an exact re-expansion, so they evaluate the parent's polynomial in the
            // parent's coordinates, all of the group's together (tensor-core path)
            int gnr = 0;
            if (kTC && level > 0) {
                __syncthreads();
                if (tid < 32) {
                    // warp 0, a lane per sibling (at most eight): the leaves with
                    // targets, their point ranges in sibling order
                    const int i = g0 + tid;
                    bool in = false;
                    int st0 = 0, ct = 0, ntg = 0;
                    if (tid < 8 && i < g1) {
                        const int b = lstart + i;
                        const uint8_t f = tv.bflags[b];
                        ntg = tv.bntgt[b];
                        in = (f & BF_LEAF) && !(!lam_in && (f & BF_FIN)) && ntg > 0;
                        if (in) {
                            st0 = tv.bstart[b];
                            ct = tv.bcount[b];
                        }
                    }
                    const unsigned inm = __ballot_sync(0xffffffffu, in);
                    int off = in ? ct : 0, nt = in ? ntg : 0;
#pragma unroll
                    for (int o = 1; o < 8; o <<= 1) {
                        const int v = __shfl_up_sync(0xffffffffu, off, o);
                        if (tid >= o) off += v;
                        nt += __shfl_xor_sync(0xffffffffu, nt, o);
                    }
                    const int k = __popc(inm & ((1u << tid) - 1u));
                    if (in) {
                        s_grs[k] = st0;
                        s_gro[k] = off - ct;
                    }
                    if (tid == 7) {
                        const int n = __popc(inm);
                        s_gro[n] = off;
                        s_gnr = n;
                        s_gntgt = nt;
                    }
                }
                __syncthreads();
                gnr = s_gnr;
                if (gnr > 0) fetch_xyz(tv, s_grs, s_gro, gnr, s_gxyz);
            }
            // ---- incoming expansions of the whole sibling group at once: the
            // colleagues of the 8 children of a parent lie in the 4 x 4 x 4 block of
            // the children of the parent's colleagues, and the phase omega^(m . delta)
            // factorises over the axes, so three 3-tap passes over the block (z, then
            // y, then x) form all siblings' Psi = w_l sum_S omega^(m . delta) Phi_S
            // while reading each colleague's Phi once instead of once per sibling.
            // The results go to this block's scratch, one plane-wave array per octant.
            bool gtr = false;
            if (level > 0 && !lam_in) {
                __syncthreads();
                if (tid < 32) {
                    // warp 0: the block's F_out slots (lane k: the parent's colleague k),
                    // and the Phi reads of both ways: the group pass reads every F_out
                    // box of the block once, writes and re-reads 8 + n_fin arrays; the
                    // per-box pass reads each F_in sibling's F_out colleagues
                    const int lane = tid;
                    for (int q = lane; q < 64; q += 32) s_blk[q] = -1;
                    __syncwarp();
                    int present = 0, sumcol = 0, nfin = 0;
                    unsigned keep = 0;  // octants of the incoming siblings
                    const int Pg = parent_of(g0);
                    if (lane < 27) {
                        const int C = tv.bcol[(size_t)Pg * 27 + lane];
                        if (C >= 0 && !(tv.bflags[C] & BF_LEAF)) {
                            const int dx = lane / 9 - 1, dy = (lane / 3) % 3 - 1, dz = lane % 3 - 1;
                            const unsigned cm = tv.bcmask[C];
                            int D = tv.bchild0[C];
                            for (int oc = 0; oc < 8; ++oc) {
                                if (!(cm & (1u << oc))) continue;
                                const int Dc = D++;
                                // block position of the child (octant bit 0 = x, 1 = y, 2 = z)
                                const int X = 2 * dx + (oc & 1) + 1, Y = 2 * dy + ((oc >> 1) & 1) + 1,
                                          Z = 2 * dz + ((oc >> 2) & 1) + 1;
                                if (X < 0 || X > 3 || Y < 0 || Y > 3 || Z < 0 || Z > 3) continue;
                                if (tv.bflags[Dc] & BF_FOUT) {
                                    s_blk[(X * 4 + Y) * 4 + Z] = tv.bslot[Dc];
                                    ++present;
                                }
                            }
                        }
                    }
                    for (int t = lane; t < (g1 - g0) * 27; t += 32) {
                        const int b = lstart + g0 + t / 27, k = t % 27;
                        if (!(tv.bflags[b] & BF_FIN) || tv.bntgt[b] == 0) continue;
                        const int Sb = tv.bcol[(size_t)b * 27 + k];
                        if (Sb >= 0 && (tv.bflags[Sb] & BF_FOUT)) ++sumcol;
                        if (k == 0) {
                            ++nfin;
                            keep |= 1u << (unsigned)(tv.bkey[b] & 7ull);
                        }
                    }
#pragma unroll
                    for (int o = 16; o > 0; o >>= 1) {
                        present += __shfl_xor_sync(0xffffffffu, present, o);
                        sumcol += __shfl_xor_sync(0xffffffffu, sumcol, o);
                        nfin += __shfl_xor_sync(0xffffffffu, nfin, o);
                        keep |= __shfl_xor_sync(0xffffffffu, keep, o);
                    }
                    // reads of the group pass: the block's F_out boxes once, and its
                    // result written and re-read once per incoming sibling
                    if (lane == 0) s_gtr = (nfin >= 2 && present + 2 * nfin < sumcol) ? (int)(256u | keep) : 0;
                }
                __syncthreads();
                gtr = s_gtr != 0;
            }
            if (gtr) {
                const unsigned gkeep = (unsigned)s_gtr & 255u;
                C2 *gout = psig + (size_t)blockIdx.x * 8 * pstride;
                const T kc = (T)-0.5;
                for (int i = tid; i < N1 * N1 * NH; i += kLThreads) {
                    const int mz = i % NH, mx = (i / NH) % N1, my = i / (NH * N1);
                    const int mxv = mx - NF, myv = my - NF;
                    // omega^(m r) for r = 1 per axis: (cos, sin) of 2 pi (m mod 3) / 3;
                    // r = -1 is its conjugate
                    const int rx = (mxv % 3 + 3) % 3, ry = (myv % 3 + 3) % 3, rz = mz % 3;
                    const T cx = rx ? kc : (T)1, sx = rx == 0 ? (T)0 : (rx == 1 ? kH : -kH);
                    const T cy = ry ? kc : (T)1, sy = ry == 0 ? (T)0 : (ry == 1 ? kH : -kH);
                    const T cz = rz ? kc : (T)1, sz = rz == 0 ? (T)0 : (rz == 1 ? kH : -kH);
                    // v + w * omega^(+m) and * omega^(-m)
                    auto rp = [](C2 v, T c, T sn) { return C2{c * v.x - sn * v.y, c * v.y + sn * v.x}; };
                    auto rm = [](C2 v, T c, T sn) { return C2{c * v.x + sn * v.y, c * v.y - sn * v.x}; };
                    auto add = [](C2 &a, C2 b) { a.x += b.x; a.y += b.y; };
                    const size_t off = (size_t)(my * N1 + mx) * NHP + mz;
                    C2 out[8];
#pragma unroll
                    for (int q = 0; q < 8; ++q) out[q] = C2{0, 0};
#pragma unroll
                    for (int X = 0; X < 4; ++X) {
                        C2 yy[4] = {C2{0, 0}, C2{0, 0}, C2{0, 0}, C2{0, 0}};  // [oy][oz]
                        bool anyx = false;
#pragma unroll
                        for (int Y = 0; Y < 4; ++Y) {
                            const int *bl = s_blk + (X * 4 + Y) * 4;
                            if (bl[0] < 0 && bl[1] < 0 && bl[2] < 0 && bl[3] < 0) continue;
                            anyx = true;
                            C2 v[4];
#pragma unroll
                            for (int Z = 0; Z < 4; ++Z) v[Z] = bl[Z] >= 0 ? Phi[(size_t)bl[Z] * pstride + off] : C2{0, 0};
                            // z: sibling oz at 1 + oz takes Z = oz, oz + 1, oz + 2 (delta 1, 0, -1)
                            C2 z0 = rp(v[0], cz, sz), z1 = rp(v[1], cz, sz);
                            add(z0, v[1]);
                            add(z1, v[2]);
                            add(z0, rm(v[2], cz, sz));
                            add(z1, rm(v[3], cz, sz));
                            // y: sibling oy takes Y = oy (delta 1), oy + 1 (0), oy + 2 (-1)
                            if (Y <= 1) {  // oy = Y: delta 1;  Y = 1 also oy = 0 with delta 0
                                const int oy = Y;
                                add(yy[oy * 2 + 0], rp(z0, cy, sy));
                                add(yy[oy * 2 + 1], rp(z1, cy, sy));
                            }
                            if (Y >= 1 && Y <= 2) {  // delta 0 for oy = Y - 1
                                add(yy[(Y - 1) * 2 + 0], z0);
                                add(yy[(Y - 1) * 2 + 1], z1);
                            }
                            if (Y >= 2) {  // delta -1 for oy = Y - 2
                                add(yy[(Y - 2) * 2 + 0], rm(z0, cy, sy));
                                add(yy[(Y - 2) * 2 + 1], rm(z1, cy, sy));
                            }
                        }
                        if (!anyx) continue;
                        // x: sibling ox takes X = ox (delta 1), ox + 1 (0), ox + 2 (-1)
#pragma unroll
                        for (int q = 0; q < 4; ++q) {
                            if (X <= 1) add(out[q * 2 + X], rp(yy[q], cx, sx));
                            if (X >= 1 && X <= 2) add(out[q * 2 + (X - 1)], yy[q]);
                            if (X >= 2) add(out[q * 2 + (X - 2)], rm(yy[q], cx, sx));
                        }
                    }
                    const int sq = mxv * mxv + myv * myv + mz * mz;
                    const T w = tb.wl ? tb.wl[(size_t)level * (3 * NF * NF + 1) + sq] : tb.w[sq] * invR;
                    // out[(oy * 2 + oz) * 2 + ox] belongs to octant ox | oy << 1 | oz << 2
#pragma unroll
                    for (int q = 0; q < 8; ++q) {
                        const int ox = q & 1, oz = (q >> 1) & 1, oy = q >> 2;
                        const int oc = ox | (oy << 1) | (oz << 2);
                        if (gkeep & (1u << oc)) gout[(size_t)oc * pstride + off] = C2{w * out[q].x, w * out[q].y};
                    }
                }
                __syncthreads();
            }
            for (int it = g0; it < g1; ++it) {
                const int B = lstart + it;
                if (tv.bntgt[B] == 0) continue;
                const uint8_t fl = tv.bflags[B];
                if (kTC && level > 0 && (fl & BF_LEAF) && !(fl & BF_FIN)) continue;  // in the group
                __syncthreads();
                if constexpr (kTC) {
                    if (fl & BF_LEAF) {
                        if (tid == 0) {
                            s_brs[0] = tv.bstart[B];
                            s_bro[0] = 0;
                            s_bro[1] = tv.bcount[B];
                        }
                        __syncthreads();
                        fetch_xyz(tv, s_brs, s_bro, 1, s_xyz);
                        if (lam_in && level > 0) {
                            // an incoming leaf: its parent's expansion is evaluated with its
                            // sibling group (in the parent's frame, exact since T_p2c is an
                            // exact re-expansion); here its own incoming expansion is added
                            int ix, iy, iz;
                            box_decode_d(tv.bkey[B], level, ix, iy, iz);
                            const double R = level_R(level), s2R = 2.0 / R;
                            const double cc[3] = {(ix + 0.5) * R, (iy + 0.5) * R, (iz + 0.5) * R};
                            if (tid == 0) atomicAdd(flops, 2ull * (P * P * P + P * P + P) * tv.bntgt[B]);
                            tc_eval<P, NF>(tv, (const float *)(lam_in + (size_t)bfin[B] * lstr), cc, s2R, s_brs, s_bro,
                                           1, s_xyz, st, phase, ufar, gfar);
                            continue;
                        }
                    }
                }
                // ---- parent's local expansion re-centred on this machine (T_p2c), or the root term
                if (level == 0) {
                    // a root: the windowed term of its system (roots are boxes 0 ..)
                    for (int i = tid; i < P3; i += kLThreads) Ls[i] = LamW[(size_t)B * P3 + i];
                } else {
                    T *b0 = reinterpret_cast<T *>(PsE);
                    T *b1 = reinterpret_cast<T *>(PsO);
                    const int Pb = tv.bparent[B];
                    if (Pb != cur_parent) {
                        const T *Lp = Lam + (size_t)tv.bslot[Pb] * P3;
                        for (int i = tid; i < P3; i += kLThreads) Pl[i] = Lp[i];
                        cur_parent = Pb;
                        __syncthreads();
                    }
                    const int oc = (int)(tv.bkey[B] & 7ull);
                    // child coefficient b_m = sum_{n >= m} A_s[n][m] a_n along z, then y, then x
                    constexpr int PA = shift_pad<T, P>();
                    shift_pass<T, P, 0, kLThreads>(As + ((oc >> 2) & 1) * P * PA, Pl, b1);
                    __syncthreads();
                    shift_pass<T, P, 1, kLThreads>(As + ((oc >> 1) & 1) * P * PA, b1, b0);
                    __syncthreads();
                    shift_pass<T, P, 2, kLThreads>(As + (oc & 1) * P * PA, b0, Ls);
                }
                __syncthreads();
                // ---- incoming expansion from F_out colleagues -> Chebyshev coefficients,
                // formed for all levels by the tensor-core incoming pass when lam_in is given
                if ((fl & BF_FIN) && lam_in) {
                    // lstr is a multiple of 4 and Ls is 128-byte aligned: whole float4 rows,
                    // every load of a thread in flight before the adds
                    const T *li = lam_in + (size_t)bfin[B] * lstr;
                    if constexpr (sizeof(T) == 4) {
                        constexpr int NV = (P3 + 3) / 4, PER = (NV + kLThreads - 1) / kLThreads;
                        float4 v[PER];
#pragma unroll
                        for (int k = 0; k < PER; ++k) {
                            const int i = tid + k * kLThreads;
                            v[k] = i < NV ? __ldg(reinterpret_cast<const float4 *>(li) + i) : make_float4(0, 0, 0, 0);
                        }
#pragma unroll
                        for (int k = 0; k < PER; ++k) {
                            const int i = 4 * (tid + k * kLThreads);
                            if (i < P3) Ls[i] += v[k].x;
                            if (i + 1 < P3) Ls[i + 1] += v[k].y;
                            if (i + 2 < P3) Ls[i + 2] += v[k].z;
                            if (i + 3 < P3) Ls[i + 3] += v[k].w;
                        }
                    } else {
                        for (int i = tid; i < P3; i += kLThreads) Ls[i] += li[i];
                    }
                    __syncthreads();
                } else if (fl & BF_FIN) {
                    if (tid == 0) {
                        int nc = 0;
                        for (int k = 0; k < 27; ++k) {
                            const int Sb = tv.bcol[(size_t)B * 27 + k];
                            if (Sb < 0 || !(tv.bflags[Sb] & BF_FOUT)) continue;
                            s_cslot[nc] = tv.bslot[Sb];
                            // delta = (c_B - c_S) / R = -(dx, dy, dz), stored mod 3 as 0..2
                            s_cd[nc][0] = (1 - k / 9 + 3) % 3;
                            s_cd[nc][1] = (1 - (k / 3) % 3 + 3) % 3;
                            s_cd[nc][2] = (1 - k % 3 + 3) % 3;
                            ++nc;
                        }
                        s_ncol = nc;
                    }
                    __syncthreads();
                    const int ncol = s_ncol;
                    // phase of colleague j for modes of residue class r = (m_x, m_y, m_z) mod 3
                    // (r = r_x + 3 r_y + 9 r_z): omega^k with k = r . delta_j mod 3, kept as
                    // (k != 0, +1 / -1 / 0 for k = 1 / 2 / 0) for the sum T - 1.5 U + i (sqrt3/2) D
                    for (int t = tid; t < (gtr ? 0 : 27 * ncol); t += kLThreads) {
                        const int j = t / 27, r = t % 27;
                        const int k = ((r % 3) * s_cd[j][0] + ((r / 3) % 3) * s_cd[j][1] + (r / 9) * s_cd[j][2]) % 3;
                        s_ud[t] = make_float2(k ? 1.f : 0.f, k == 1 ? 1.f : (k == 2 ? -1.f : 0.f));
                    }
                    __syncthreads();
                    // phase A: Psi = w_l * sum_S omega^(m.delta) Phi_S, folded into even/odd in m_x;
                    // a thread takes two adjacent m_z (one 16-byte load per colleague and sign
                    // of m_x), four colleagues per step for memory-level parallelism
                    if (gtr) {
                        // the group pass formed this box's Psi: fold it into even/odd in m_x
                        const C2 *g = psig + ((size_t)blockIdx.x * 8 + (size_t)(tv.bkey[B] & 7ull)) * pstride;
                        for (int i = tid; i < N1 * NH * NH; i += kLThreads) {
                            const int mz = i % NH, mxp = (i / NH) % NH, my = i / (NH * NH);
                            const C2 psp = g[(size_t)(my * N1 + NF + mxp) * NHP + mz];
                            const size_t o = (size_t)(my * NH + mxp) * NHP + mz;
                            if (mxp > 0) {
                                const C2 psm = g[(size_t)(my * N1 + NF - mxp) * NHP + mz];
                                PsE[o] = C2{psp.x + psm.x, psp.y + psm.y};
                                PsO[o] = C2{psp.x - psm.x, psp.y - psm.y};
                            } else {
                                PsE[o] = psp;
                                PsO[o] = C2{0, 0};
                            }
                        }
                    }
                    for (int i = tid; i < (gtr ? 0 : N1 * NH * (NHP / 2)); i += kLThreads) {
                        const int my = i / (NH * (NHP / 2)), r = i % (NH * (NHP / 2)), mxp = r / (NHP / 2);
                        const int mz0 = 2 * (r % (NHP / 2));
                        const int myv = my - NF;
                        const int rxp = mxp % 3, rxm = (3 - rxp) % 3, ry = (myv % 3 + 3) % 3;
                        const int rz0 = mz0 % 3, rz1 = (mz0 + 1) % 3;
                        const float2 *udp0 = s_ud + rxp + 3 * ry + 9 * rz0, *udp1 = s_ud + rxp + 3 * ry + 9 * rz1;
                        const float2 *udm0 = s_ud + rxm + 3 * ry + 9 * rz0, *udm1 = s_ud + rxm + 3 * ry + 9 * rz1;
                        C2 Tp[2] = {}, Up[2] = {}, Dp[2] = {}, Tm[2] = {}, Um[2] = {}, Dm[2] = {};
                        const size_t off_p = (size_t)(my * N1 + NF + mxp) * NHP + mz0;
                        const size_t off_m = (size_t)(my * N1 + NF - mxp) * NHP + mz0;
                        if (mxp > 0) {
#pragma unroll 4
                            for (int j = 0; j < ncol; ++j) {
                                const C2 *ph = Phi + (size_t)s_cslot[j] * pstride;
                                const C2x2<C2> vp = ld_pair(ph + off_p), vm = ld_pair(ph + off_m);
                                const float2 cp0 = udp0[27 * j], cp1 = udp1[27 * j];
                                const float2 cm0 = udm0[27 * j], cm1 = udm1[27 * j];
                                Tp[0].x += vp.a.x; Tp[0].y += vp.a.y;
                                Tp[1].x += vp.b.x; Tp[1].y += vp.b.y;
                                cfma(Up[0], (T)cp0.x, vp.a);
                                cfma(Dp[0], (T)cp0.y, vp.a);
                                cfma(Up[1], (T)cp1.x, vp.b);
                                cfma(Dp[1], (T)cp1.y, vp.b);
                                Tm[0].x += vm.a.x; Tm[0].y += vm.a.y;
                                Tm[1].x += vm.b.x; Tm[1].y += vm.b.y;
                                cfma(Um[0], (T)cm0.x, vm.a);
                                cfma(Dm[0], (T)cm0.y, vm.a);
                                cfma(Um[1], (T)cm1.x, vm.b);
                                cfma(Dm[1], (T)cm1.y, vm.b);
                            }
                        } else {
#pragma unroll 4
                            for (int j = 0; j < ncol; ++j) {
                                const C2x2<C2> vp = ld_pair(Phi + (size_t)s_cslot[j] * pstride + off_p);
                                const float2 cp0 = udp0[27 * j], cp1 = udp1[27 * j];
                                Tp[0].x += vp.a.x; Tp[0].y += vp.a.y;
                                Tp[1].x += vp.b.x; Tp[1].y += vp.b.y;
                                cfma(Up[0], (T)cp0.x, vp.a);
                                cfma(Dp[0], (T)cp0.y, vp.a);
                                cfma(Up[1], (T)cp1.x, vp.b);
                                cfma(Dp[1], (T)cp1.y, vp.b);
                            }
                        }
#pragma unroll
                        for (int h = 0; h < 2; ++h) {
                            const int mz = mz0 + h;
                            if (mz >= NH) continue;
                            const int sq = mxp * mxp + myv * myv + mz * mz;
                            const T w = tb.wl ? tb.wl[(size_t)level * (3 * NF * NF + 1) + sq] : tb.w[sq] * invR;
                            // S0 + omega S1 + omega^2 S2 = T - 1.5 U + i (sqrt3/2) D
                            const C2 psp{w * (Tp[h].x - (T)1.5 * Up[h].x - kH * Dp[h].y),
                                         w * (Tp[h].y - (T)1.5 * Up[h].y + kH * Dp[h].x)};
                            const size_t o = (size_t)(my * NH + mxp) * NHP + mz;
                            if (mxp > 0) {
                                const C2 psm{w * (Tm[h].x - (T)1.5 * Um[h].x - kH * Dm[h].y),
                                             w * (Tm[h].y - (T)1.5 * Um[h].y + kH * Dm[h].x)};
                                PsE[o] = C2{psp.x + psm.x, psp.y + psm.y};
                                PsO[o] = C2{psp.x - psm.x, psp.y - psm.y};
                            } else {
                                PsE[o] = psp;
                                PsO[o] = C2{0, 0};
                            }
                        }
                    }
                    __syncthreads();
                    // phase B: contract m_x -> a, for m_y = +-my'; fold into even/odd in m_y
                    for (int i = tid; i < NH * NH * S::AG; i += kLThreads) {
                        const int ag = i / (NH * NH), r = i % (NH * NH), myp = r / NH, mz = r % NH;
                        C2 ap[S::AC], am[S::AC];
#pragma unroll
                        for (int k = 0; k < S::AC; ++k) ap[k] = am[k] = C2{0, 0};
                        const int rp = (NF + myp) * NH, rm = (NF - myp) * NH;
                        for (int mxp = 0; mxp <= NF; ++mxp) {
                            const C2 ep = PsE[(rp + mxp) * NHP + mz], em = PsE[(rm + mxp) * NHP + mz];
                            const C2 op = PsO[(rp + mxp) * NHP + mz], om = PsO[(rm + mxp) * NHP + mz];
#pragma unroll
                            for (int k = 0; k < S::AC; ++k) {
                                const int a = ag + S::AG * k;
                                if (a < P) {
                                    const T h = hs[a * NH + mxp];
                                    if (a & 1) { cfma(ap[k], h, op); cfma(am[k], h, om); }
                                    else { cfma(ap[k], h, ep); cfma(am[k], h, em); }
                                }
                            }
                        }
#pragma unroll
                        for (int k = 0; k < S::AC; ++k) {
                            const int a = ag + S::AG * k;
                            if (a >= P) continue;
                            C2 vp = ap[k], vm = am[k];
                            if (a & 1) {  // times -i
                                vp = C2{vp.y, -vp.x};
                                vm = C2{vm.y, -vm.x};
                            }
                            const int o = (a * NH + myp) * NH + mz;
                            if (myp > 0) {
                                T1e[o] = C2{vp.x + vm.x, vp.y + vm.y};
                                T1o[o] = C2{vp.x - vm.x, vp.y - vm.y};
                            } else {
                                T1e[o] = vp;
                                T1o[o] = C2{0, 0};
                            }
                        }
                    }
                    __syncthreads();
                    // phase C: contract m_y -> b
                    for (int i = tid; i < P * NH * S::BG; i += kLThreads) {
                        const int bg = i / (P * NH), r = i % (P * NH), a = r / NH, mz = r % NH;
                        C2 acc[S::BC];
#pragma unroll
                        for (int k = 0; k < S::BC; ++k) acc[k] = C2{0, 0};
                        for (int myp = 0; myp <= NF; ++myp) {
                            const C2 te = T1e[(a * NH + myp) * NH + mz], to = T1o[(a * NH + myp) * NH + mz];
#pragma unroll
                            for (int k = 0; k < S::BC; ++k) {
                                const int b = bg + S::BG * k;
                                if (b < P) {
                                    const T h = hs[b * NH + myp];
                                    if (b & 1) cfma(acc[k], h, to); else cfma(acc[k], h, te);
                                }
                            }
                        }
#pragma unroll
                        for (int k = 0; k < S::BC; ++k) {
                            const int b = bg + S::BG * k;
                            if (b >= P) continue;
                            C2 v = acc[k];
                            if (b & 1) v = C2{v.y, -v.x};
                            T2[(a * P + b) * NH + mz] = v;
                        }
                    }
                    __syncthreads();
                    // phase D: contract m_z -> c (real part; m_z < 0 through Hermitian symmetry)
                    for (int i = tid; i < P * P * S::CG; i += kLThreads) {
                        const int cg = i / (P * P), ab = i % (P * P);
                        T acc[S::CC];
#pragma unroll
                        for (int k = 0; k < S::CC; ++k) acc[k] = (T)0;
                        for (int mz = 0; mz <= NF; ++mz) {
                            const C2 t = T2[ab * NH + mz];
                            const T cz = mz ? (T)2 : (T)1;
#pragma unroll
                            for (int k = 0; k < S::CC; ++k) {
                                const int c = cg + S::CG * k;
                                if (c < P) acc[k] += cz * hs[c * NH + mz] * ((c & 1) ? t.y : t.x);
                            }
                        }
#pragma unroll
                        for (int k = 0; k < S::CC; ++k) {
                            const int c = cg + S::CG * k;
                            if (c < P) Ls[ab * P + c] += acc[k];
                        }
                    }
                    __syncthreads();
                }
                if (tid == 0) {
                    // algorithmic flops of this box: p2c (3 triangular passes), the
                    // translation (one complex multiply-add per mode and colleague) and
                    // the three parity-split contractions, and the leaf evaluation
                    unsigned long long f = level > 0 ? 3ull * P * P * (P * (P + 1) / 2) * 2 : 0ull;
                    if ((fl & BF_FIN) && !lam_in)
                        f += 8ull * N1 * N1 * NH * s_ncol + 8ull * P * NH * NH * NH + 4ull * P * P * NH * NH +
                             2ull * P * P * P * NH;
                    if (fl & BF_LEAF) f += 2ull * (P * P * P + P * P + P) * tv.bntgt[B];
                    atomicAdd(flops, f);
                }
                if (!(fl & BF_LEAF)) {
                    T *Lo = Lam + (size_t)tv.bslot[B] * P3;
                    for (int i = tid; i < P3; i += kLThreads) Lo[i] = Ls[i];
                    continue;
                }
                // ---- leaf: evaluate the local expansion at its targets
                int ix, iy, iz;
                box_decode_d(tv.bkey[B], level, ix, iy, iz);
                const double R = level_R(level), s2R = 2.0 / R;
                const double cc[3] = {(ix + 0.5) * R, (iy + 0.5) * R, (iz + 0.5) * R};
                if constexpr (kTC) {
                    tc_eval<P, NF>(tv, Ls, cc, s2R, s_brs, s_bro, 1, s_xyz, st, phase, ufar, gfar);
                } else {
                    const int s = tv.bstart[B], e = s + tv.bcount[B];
                    T *dev = ev + 3 * kECH * P;  // derivatives T_n' (gradient pass)
                    for (int p0 = s; p0 < e; p0 += kECH) {
                        const int np = min(kECH, e - p0);
                        for (int t = tid; t < 3 * kECH; t += kLThreads) {
                            const int ax = t / kECH, j = t % kECH;
                            T *o = ev + (ax * kECH + j) * P, *od = dev + (ax * kECH + j) * P;
                            if (j < np) {
                                const int kk = p0 + j;
                                const double u = ax == 0 ? tv.ux[kk] : (ax == 1 ? tv.uy[kk] : tv.uz[kk]);
                                const T xi = (T)((u - cc[ax]) * s2R);
                                T t0 = (T)1, t1 = xi, d0 = (T)0, d1 = (T)1;
                                o[0] = (T)1;
                                od[0] = (T)0;
                                if (P > 1) {
                                    o[1] = xi;
                                    od[1] = (T)1;
                                }
#pragma unroll
                                for (int n = 2; n < P; ++n) {
                                    const T t2 = (T)2 * xi * t1 - t0;
                                    const T d2 = (T)2 * t1 + (T)2 * xi * d1 - d0;
                                    o[n] = t2;
                                    od[n] = d2;
                                    t0 = t1;
                                    t1 = t2;
                                    d0 = d1;
                                    d1 = d2;
                                }
                            } else {
#pragma unroll
                                for (int n = 0; n < P; ++n) o[n] = od[n] = (T)0;
                            }
                        }
                        __syncthreads();
                        // pass 0: W = sum_c Lambda T_c(z) -> u, d/dx, d/dy; pass 1 (gradient):
                        // W = sum_c Lambda T_c'(z) -> d/dz
                        for (int pass = 0; pass < (gfar ? 2 : 1); ++pass) {
                            // W[j][ab] = sum_c Lambda[ab][c] Z_c(z_j): 4 x 4 register tiles over (ab, j)
                            T *W = reinterpret_cast<T *>(PsE);
                            const T *tzs = (pass ? dev : ev) + 2 * kECH * P;
                            constexpr int NABG = (P * P + 3) / 4;
                            for (int tile = tid; tile < NABG * (kECH / 4); tile += kLThreads) {
                                const int jg = tile % (kECH / 4), abg = tile / (kECH / 4);
                                T acc[4][4];
#pragma unroll
                                for (int i = 0; i < 4; ++i)
#pragma unroll
                                    for (int k = 0; k < 4; ++k) acc[i][k] = (T)0;
#pragma unroll
                                for (int c = 0; c < P; ++c) {
                                    T l[4], z[4];
#pragma unroll
                                    for (int i = 0; i < 4; ++i) {
                                        const int ab = abg * 4 + i;
                                        l[i] = ab < P * P ? Ls[ab * P + c] : (T)0;
                                    }
#pragma unroll
                                    for (int k = 0; k < 4; ++k) z[k] = tzs[(jg * 4 + k) * P + c];
#pragma unroll
                                    for (int i = 0; i < 4; ++i)
#pragma unroll
                                        for (int k = 0; k < 4; ++k) acc[i][k] += l[i] * z[k];
                                }
#pragma unroll
                                for (int i = 0; i < 4; ++i) {
                                    const int ab = abg * 4 + i;
                                    if (ab < P * P)
#pragma unroll
                                        for (int k = 0; k < 4; ++k) W[(jg * 4 + k) * (P * P) + ab] = acc[i][k];
                                }
                            }
                            __syncthreads();
                            // sum_a X_a(x_j) sum_b Y_b(y_j) W[j][a][b]: 16 threads per target
                            const int j = tid >> 4, g = tid & 15;
                            const T *tx = ev + j * P, *ty = ev + (kECH + j) * P;
                            const T *dtx = dev + j * P, *dty = dev + (kECH + j) * P;
                            const T *Wj = W + j * (P * P);
                            T su = 0, sx = 0, sy = 0;
                            for (int a = g; a < P; a += 16) {
                                T sa = 0, sda = 0;
#pragma unroll
                                for (int b = 0; b < P; ++b) {
                                    sa += ty[b] * Wj[a * P + b];
                                    if (gfar && pass == 0) sda += dty[b] * Wj[a * P + b];
                                }
                                su += tx[a] * sa;
                                if (gfar && pass == 0) {
                                    sx += dtx[a] * sa;
                                    sy += tx[a] * sda;
                                }
                            }
#pragma unroll
                            for (int o = 8; o > 0; o >>= 1) {
                                su += __shfl_xor_sync(0xffffffffu, su, o);
                                sx += __shfl_xor_sync(0xffffffffu, sx, o);
                                sy += __shfl_xor_sync(0xffffffffu, sy, o);
                            }
                            if (g == 0 && j < np && (tv.pflag[p0 + j] & 2)) {
                                const size_t pk = (size_t)(p0 + j);
                                if (pass == 0) {
                                    ufar[pk] = (double)su;
                                    if (gfar) {
                                        gfar[3 * pk + 0] = (double)sx * s2R;
                                        gfar[3 * pk + 1] = (double)sy * s2R;
                                    }
                                } else {
                                    gfar[3 * pk + 2] = (double)su * s2R;
                                }
                            }
                            __syncthreads();
                        }
                    }
                }
            }
            if constexpr (kTC) {
                if (gnr > 0) {
                    // the group's leaves: the parent's expansion in the parent's frame
                    if (Pg != cur_parent) {
                        __syncthreads();
                        const T *Lp = Lam + (size_t)tv.bslot[Pg] * P3;
                        for (int i = tid; i < P3; i += kLThreads) Pl[i] = Lp[i];
                        cur_parent = Pg;
                    }
                    __syncthreads();
                    int ix, iy, iz;
                    box_decode_d(tv.bkey[Pg], level - 1, ix, iy, iz);
                    const double R = level_R(level - 1), s2R = 2.0 / R;
                    const double cc[3] = {(ix + 0.5) * R, (iy + 0.5) * R, (iz + 0.5) * R};
                    if (tid == 0) atomicAdd(flops, 2ull * (P * P * P + P * P + P) * (unsigned long long)s_gntgt);
                    tc_eval<P, NF>(tv, Pl, cc, s2R, s_grs, s_gro, gnr, s_gxyz, st, phase, ufar, gfar);
                }
            }
        }
    }
    if constexpr (kTC) {
        // an MMA batch that outlived its wait must finish before TMEM is freed
        if (s_pending && tid < 32) {
            const bool done = tc::mbar_wait(&s_bar, phase ^ 1u, 2000000000ll);
            (void)done;
        }
        tc::fence_before_sync();
        __syncthreads();
        tc::fence_after_sync();
        if (warp == 0) tc::tmem_dealloc(s_tmem, S::TCOLS);
    }
}

__global__ void k_finalize(int64_t n, const uint8_t *pflag, const int32_t *pout, const double *ufar,
                           const double *unear, const double *gfar, const double *gnear, const Frame *frame,
                           const int32_t *psys, int mode, double *pot, double *grad) {
    int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n || !(pflag[k] & 2)) return;
    // mode 0: both parts, 1: far part only, 2: near part only; unit-box
    // potentials scale by 1/S, their gradients by 1/S^2 (S of the point's system)
    const double S = frame[psys ? psys[k] : 0].S;
    const double v = (mode == 2 ? 0.0 : ufar[k]) + (mode == 1 ? 0.0 : unear[k]);
    const int64_t o = pout[k];
    pot[o] = v / S;
    if (grad)
        for (int d = 0; d < 3; ++d)
            grad[3 * o + d] = ((mode == 2 ? 0.0 : gfar[3 * k + d]) + (mode == 1 ? 0.0 : gnear[3 * k + d])) / (S * S);
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
static BufLayout make_layout(const std::vector<size_t> &sizes, size_t smem_limit) {
    BufLayout lay{};
    lay.n = (int)sizes.size();
    size_t so = 0, go = 0;
    for (int i = 0; i < lay.n; ++i) {
        size_t sz = (sizes[i] + 127) & ~(size_t)127;
        if (so + sz <= smem_limit) {
            lay.in_smem[i] = 1;
            lay.off[i] = so;
            so += sz;
        } else {
            lay.in_smem[i] = 0;
            lay.off[i] = go;
            go += sz;
        }
    }
    lay.smem_bytes = so;
    lay.slab_bytes = go;
    return lay;
}

#define PCK(x)                                                             \
    do {                                                                   \
        cudaError_t e_ = (x);                                              \
        if (e_ != cudaSuccess) {                                           \
            err = std::string(#x) + ": " + cudaGetErrorString(e_);         \
            return DMK_ERR_CUDA;                                           \
        }                                                                  \
    } while (0)

// the tensor-core incoming pass serves the single-precision path at the
// (P, NF) shapes it supports
template <typename T, int P, int NF> constexpr bool incoming_tc() {
    if constexpr (sizeof(T) == 4 && ((P == 9 && NF == 6) || (P == 18 && NF == 12) || (P == 19 && NF == 12)))
        return InShape<P, NF>::OK;
    return false;
}

template <typename T, int P, int NF> static int run_incoming(const IncomingArgs &a, cudaStream_t st, std::string &err) {
    if constexpr (incoming_tc<T, P, NF>()) {
        const int rc = launch_incoming<P, NF>(a, st, err);
        return rc ? rc : 0;
    }
    err = "tensor-core incoming pass requested for an unsupported shape";
    return DMK_ERR_INTERNAL;
}

template <typename T, int P, int NF>
static int run_passes_P(PassCtx &cx, std::string &err) {
    using C2 = typename Cplx<T>::type;
    constexpr int P3 = P * P * P, NH = NF + 1, N1 = 2 * NF + 1;
    TreeView tv = cx.tree->view();
    const DevTables<T> &tb = *reinterpret_cast<const DevTables<T> *>(cx.tables);
    if (tb.nf != NF || tb.p != P) { err = "table shape mismatch"; return DMK_ERR_INTERNAL; }
    cudaStream_t st = cx.st;
    Workspace &ws = *cx.ws;
    const int nslots = cx.tree->nslots;
    const size_t smem_limit = cx.smem_limit;
    const int64_t n = tv.n;
    const int maxgrid = cx.num_sms * 8;

    if (ws.ensure(cx.bufs->M, (int64_t)nslots * P3 * sizeof(T)) ||
        ws.ensure(cx.bufs->Lam, (int64_t)nslots * P3 * sizeof(T)) ||
        ws.ensure(cx.bufs->LamW, (int64_t)tv.lev_count[0] * P3 * sizeof(T)) || ws.ensure(cx.bufs->ufar, n * 8) ||
        ws.ensure(cx.bufs->unear, n * 8) || ws.ensure(cx.bufs->counter, 256)) {
        err = "device allocation failed (expansions)";
        return DMK_ERR_OOM;
    }
    T *M = (T *)cx.bufs->M.p;
    T *Lam = (T *)cx.bufs->Lam.p;
    T *LamW = (T *)cx.bufs->LamW.p;
    double *ufar = (double *)cx.bufs->ufar.p;
    double *unear = (double *)cx.bufs->unear.p;
    PCK(cudaMemsetAsync(ufar, 0, n * 8, st));
    PCK(cudaMemsetAsync(unear, 0, n * 8, st));
    // gradient pass: far and near gradients of every point (n x 3)
    double *gfar = nullptr, *gnear = nullptr;
    if (cx.grad) {
        if (ws.ensure(cx.bufs->gfar, n * 24) || ws.ensure(cx.bufs->gnear, n * 24)) {
            err = "device allocation failed (gradients)";
            return DMK_ERR_OOM;
        }
        gfar = (double *)cx.bufs->gfar.p;
        gnear = (double *)cx.bufs->gnear.p;
        PCK(cudaMemsetAsync(gfar, 0, n * 24, st));
        PCK(cudaMemsetAsync(gnear, 0, n * 24, st));
    }
    // device words: [0] near work queue, [2..3] pairs inside R_L, [4..5] local
    // flops, [6] tensor-core wait error, [8..9] incoming reads, [10..11] pairs
    // screened by the near field, [12] the upward pass's work queue, [32 + l]
    // level-l work queue of k_local
    PCK(cudaMemsetAsync(cx.bufs->counter.p, 0, 256, st));

    // ---- residual near field and self corrections, on the side stream: it
    // needs only the tree, and fills the SMs the per-level far-field launches
    // leave idle
    PCK(cudaEventRecord(cx.fork, st));
    PCK(cudaStreamWaitEvent(cx.side, cx.fork, 0));
    cudaEventRecord(cx.nev[0], cx.side);
    // the diagnostic modes skip the half they do not return: far part only (1),
    // near part only (2)
    const bool do_far = cx.mode != 2, do_near = cx.mode != 1;
    if (cx.tree->ntleaves > 0 && do_near) {
        NearArgs na{tv,
                    cx.tree->ntleaves,
                    (const int32_t *)cx.tree->tleaves.p,
                    (const int32_t *)cx.tree->nl_off.p,
                    (const int32_t *)cx.tree->nl_src.p,
                    cx.tree->plocal.p,
                    (const float4 *)cx.tree->plocal_lo.p,
                    tb.ql ? (const void *)tb.ql : (const void *)tb.qmono,
                    tb.qdeg,
                    unear,
                    gnear,
                    (int *)cx.bufs->counter.p,
                    tb.ql != nullptr,
                    (double)tb.lam,
                    tv.nlev};
        int rc_near = launch_near(sizeof(T) == 4, na, cx.num_sms, cx.side);
        if (rc_near == 1) { err = "residual polynomial degree outside 2..30"; return DMK_ERR_UNSUPPORTED; }
        if (rc_near == 3) { err = "the Yukawa near field has no gradient pass"; return DMK_ERR_UNSUPPORTED; }
        if (rc_near) { err = "near-field launch failed"; return DMK_ERR_CUDA; }
        PCK(cudaGetLastError());
    }
    cudaEventRecord(cx.nev[1], cx.side);
    PCK(cudaEventRecord(cx.join, cx.side));
    // ---- upward pass (finest level first)
    cudaEventRecord(cx.ev[1], st);
    {
        size_t scr = std::max((size_t)2 * P3, (size_t)kCH * (3 * UpShape<P>::PS + UpShape<P>::YS)) * sizeof(T);
        if (sizeof(T) == 4 && UpShape<P>::TC_OK) scr = std::max(scr, (size_t)UpShape<P>::TC_SCR * sizeof(float));
        BufLayout lay = make_layout({P3 * sizeof(T), scr, (size_t)2 * P * P * sizeof(T)}, smem_limit - 1024);
        if (all_smem<T, P>() && !layout_in_smem(lay)) {
            err = "upward pass: buffers do not fit in shared memory";
            return DMK_ERR_INTERNAL;
        }
        if (sizeof(T) == 4 && UpShape<P>::TC_OK && !lay.in_smem[1]) {
            err = "tensor-core operands of the upward pass do not fit in shared memory";
            return DMK_ERR_INTERNAL;
        }
        PCK(cudaFuncSetAttribute(k_upward<T, P>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)lay.smem_bytes));
        // single precision: the whole upward pass (anterpolation and the
        // child-to-parent shifts of every level) in one launch; otherwise level
        // by level, finest first
        constexpr bool all_level = sizeof(T) == 4 && P * ((P + 1) / 2) <= kThreads;
        if constexpr (all_level) {
            if (do_far && nslots > 0) {
                using AS = AntShape<P>;
                static_assert(AS::OK, "pencil pairs of a shift exceed the CTA");
                if (ws.ensure(cx.bufs->upcnt, (int64_t)nslots * 4)) { err = "oom upward counters"; return DMK_ERR_OOM; }
                PCK(cudaMemsetAsync(cx.bufs->upcnt.p, 0, (size_t)nslots * 4, st));
                PCK(cudaFuncSetAttribute(k_anterp<P>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)AS::SMEM));
                int per_sm = 0;
                PCK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_anterp<P>, AS::NT, AS::SMEM));
                const int grid = std::min(nslots, std::max(per_sm, 1) * cx.num_sms);
                ::dmk::launch_tick();
                k_anterp<P><<<grid, AS::NT, AS::SMEM, st>>>(tv, reinterpret_cast<const float *>(tb.A), nslots,
                                                            (const int32_t *)cx.tree->slot2box.p, (float *)M,
                                                            (int *)cx.bufs->counter.p + 12, (int *)cx.bufs->upcnt.p);
            }
        }
        const int lmax = tv.nlev - 1;
        for (int l = (tv.nlev == 1 ? 0 : lmax - 1); l >= 0 && do_far && !all_level; --l) {
            int lc = tv.lev_count[l];
            int grid = std::min(lc, maxgrid);
            if (grid <= 0) continue;
            if (ws.ensure(cx.bufs->slab, (int64_t)grid * lay.slab_bytes + 128)) { err = "oom slab"; return DMK_ERR_OOM; }
            ::dmk::launch_tick();
            k_upward<T, P><<<grid, kThreads, lay.smem_bytes, st>>>(tv, tb, tv.lev_start[l], lc, M, lay,
                                                                   (char *)cx.bufs->slab.p,
                                                                   (int *)cx.bufs->counter.p + 6);
        }
        PCK(cudaGetLastError());
    }
    // ---- outgoing expansions of every F_out box; in single precision the
    // incoming expansions then run on the tensor cores (incoming.cu), which
    // read the plane waves plane by plane
    cudaEventRecord(cx.ev[2], st);
    const bool tc_in = incoming_tc<T, P, NF>() && cx.tree->nfin > 0 && do_far;
    const int64_t phi_elems = tc_in ? (int64_t)nslots * NH * N1 * ((N1 + 1) & ~1)
                                    : (int64_t)nslots * N1 * N1 * nz_pad<NF>();
    if (ws.ensure(cx.bufs->Phi, phi_elems * (int64_t)sizeof(C2))) {
        err = "device allocation failed (plane waves)";
        return DMK_ERR_OOM;
    }
    C2 *Phi = (C2 *)cx.bufs->Phi.p;
    if (do_far && !cx.tree->root_leaf && nslots > 0) {
        BufLayout lay = make_layout({P3 * sizeof(T), (size_t)P * P * NH * sizeof(C2), (size_t)P * N1 * NH * sizeof(C2),
                                     (size_t)P * NH * sizeof(T)},
                                    smem_limit);
        if (all_smem<T, P>() && !layout_in_smem(lay)) {
            err = "plane waves: buffers do not fit in shared memory";
            return DMK_ERR_INTERNAL;
        }
        auto kern = tc_in ? k_prox2pw<T, P, NF, true> : k_prox2pw<T, P, NF, false>;
        PCK(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)lay.smem_bytes));
        int grid = std::min(nslots, maxgrid);
        if (ws.ensure(cx.bufs->slab, (int64_t)grid * lay.slab_bytes + 128)) { err = "oom slab"; return DMK_ERR_OOM; }
        ::dmk::launch_tick();
        kern<<<grid, kThreads, lay.smem_bytes, st>>>(tv, tb, nslots, (const int32_t *)cx.tree->slot2box.p, M, Phi,
                                                     lay, (char *)cx.bufs->slab.p);
        PCK(cudaGetLastError());
    }
    // ---- root windowed term, for every root (system)
    {
        const int NW = tb.NW, nhW = tb.nhW, nroots = tv.lev_count[0];
        const size_t scr = (size_t)(2 * P * P * nhW + 2 * P * NW * nhW + NW * NW * nhW);
        const int grid = std::min(nroots, maxgrid);
        if (ws.ensure(cx.bufs->rootscr, (int64_t)grid * scr * sizeof(C2))) { err = "oom root"; return DMK_ERR_OOM; }
        if (do_far) {
            ::dmk::launch_tick();
            k_root<T, P><<<grid, kThreads, 0, st>>>(tv, tb, M, nroots, LamW, (C2 *)cx.bufs->rootscr.p, scr);
            PCK(cudaGetLastError());
        }
    }
    // ---- incoming expansions of every level at once (tensor cores, TMA)
    const T *lam_in = nullptr;
    if (tc_in) {
        const int nfin = cx.tree->nfin;
        const int lstr = (P3 + 3) & ~3;
        if (ws.ensure(cx.bufs->lam_in, (int64_t)nfin * lstr * 4) || ws.ensure(cx.bufs->finc, (int64_t)nfin * 27 * 4) ||
            ws.ensure(cx.bufs->fincnt, (int64_t)nfin * 4)) {
            err = "device allocation failed (incoming expansions)";
            return DMK_ERR_OOM;
        }
        cudaEventRecord(cx.ev[7], st);
        IncomingArgs ia{tv,
                        cx.tables,
                        Phi,
                        nslots,
                        nfin,
                        (const int32_t *)cx.tree->fin2box.p,
                        (int32_t *)cx.bufs->finc.p,
                        (int32_t *)cx.bufs->fincnt.p,
                        (float *)cx.bufs->lam_in.p,
                        (unsigned long long *)cx.bufs->counter.p + 4,
                        (int *)cx.bufs->counter.p + 6,
                        cx.num_sms};
        int rc = run_incoming<T, P, NF>(ia, st, err);
        if (rc) return rc;
        lam_in = (const T *)cx.bufs->lam_in.p;
    } else {
        cudaEventRecord(cx.ev[7], st);
    }
    // ---- local expansions, coarsest level first; leaves evaluate
    {
        // buffer 1 holds the incoming expansion, the p2c scratch (2 P^3) and the
        // evaluation intermediate W (kECH P^2) or the tensor-core operands
        using LS = LocalShape<P, NF>;
        const bool tcore = sizeof(T) == 4 && LS::TC_OK;
        const size_t psi_bytes = std::max({(size_t)2 * N1 * NH * nz_pad<NF>() * sizeof(C2), (size_t)2 * P3 * sizeof(T),
                                           (size_t)kECH * P * P * sizeof(T),
                                           tcore ? (size_t)LS::TC_BUF1 * sizeof(float) : (size_t)0});
        const size_t t1_bytes = std::max((size_t)2 * P * NH * NH * sizeof(C2),
                                         tcore ? (size_t)LS::TC_BUF2 * sizeof(float) : (size_t)0);
        cudaEventRecord(cx.ev[6], st);
        BufLayout lay = make_layout({P3 * sizeof(T), psi_bytes, t1_bytes, (size_t)P * NH * sizeof(T),
                                     (size_t)6 * kECH * P * sizeof(T), (size_t)2 * P * shift_pad<T, P>() * sizeof(T),
                                     P3 * sizeof(T)},
                                    smem_limit - 20480);
        if (all_smem<T, P>() && !layout_in_smem(lay)) {
            err = "local pass: buffers do not fit in shared memory";
            return DMK_ERR_INTERNAL;
        }
        if (tcore && !(lay.in_smem[1] && lay.in_smem[2])) {
            err = "tensor-core operands do not fit in shared memory";
            return DMK_ERR_INTERNAL;
        }
        PCK(cudaFuncSetAttribute(k_local<T, P, NF>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)lay.smem_bytes));
        // per block: the plane-wave arrays of one sibling group (8 octants)
        if (ws.ensure(cx.bufs->psig, (int64_t)cx.num_sms * 8 * N1 * N1 * nz_pad<NF>() * sizeof(C2))) {
            err = "device allocation failed (group translation)";
            return DMK_ERR_OOM;
        }
        for (int l = 0; l < tv.nlev && do_far; ++l) {
            int lc = tv.lev_count[l];
            int grid = std::min((lc + 7) / 8, cx.num_sms);
            if (grid <= 0) continue;
            if (ws.ensure(cx.bufs->slab, (int64_t)grid * lay.slab_bytes + 128)) { err = "oom slab"; return DMK_ERR_OOM; }
            ::dmk::launch_tick();
            k_local<T, P, NF><<<grid, kLThreads, lay.smem_bytes, st>>>(tv, tb, l, tv.lev_start[l], lc, Phi, Lam,
                                                                       LamW, ufar, lay, (char *)cx.bufs->slab.p,
                                                                       (unsigned long long *)cx.bufs->counter.p + 2,
                                                                       (int *)cx.bufs->counter.p + 6,
                                                                       (int *)cx.bufs->counter.p + 32 + l, gfar,
                                                                       (C2 *)cx.bufs->psig.p, lam_in,
                                                                       (const int32_t *)cx.tree->bfin.p,
                                                                       (P3 + 3) & ~3);
        }
        PCK(cudaGetLastError());
    }
    // ---- the far field is done; join the near field
    cudaEventRecord(cx.ev[3], st);
    PCK(cudaStreamWaitEvent(st, cx.join, 0));
    cudaEventRecord(cx.ev[4], st);
    ::dmk::launch_tick();
    k_finalize<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(n, tv.pflag, (const int32_t *)cx.tree->pout.p, ufar,
                                                           unear, gfar, gnear, (const Frame *)cx.tree->frame.p,
                                                           cx.tree->nsys > 1 ? (const int32_t *)cx.tree->psys.p
                                                                             : nullptr,
                                                           cx.mode, cx.pot, cx.grad);
    PCK(cudaGetLastError());
    return 0;
}

template <typename T>
static int run_passes_T(PassCtx &cx, std::string &err) {
    const DevTables<T> &tb = *reinterpret_cast<const DevTables<T> *>(cx.tables);
    if (cx.p == 9 && tb.nf == 6) return run_passes_P<T, 9, 6>(cx, err);
    if (cx.p == 18 && tb.nf == 12) return run_passes_P<T, 18, 12>(cx, err);
    if (cx.p == 19 && tb.nf == 12) return run_passes_P<T, 19, 12>(cx, err);
    if (cx.p == 28 && tb.nf == 19) return run_passes_P<T, 28, 19>(cx, err);
    if (cx.p == 38 && tb.nf == 26) return run_passes_P<T, 38, 26>(cx, err);
    err = "(p, nf) must be one of (9,6), (18,12), (19,12), (28,19), (38,26)";
    return DMK_ERR_UNSUPPORTED;
}

int run_passes(PassCtx &cx, std::string &err) {
    return cx.single ? run_passes_T<float>(cx, err) : run_passes_T<double>(cx, err);
}

}  // namespace dmk
