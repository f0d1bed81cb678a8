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
//               eq. outgoingexpansion2 (Phi_{-m} = conj(Phi_m) for real charges).
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

#include <algorithm>
#include <cstdio>

namespace dmk {

constexpr int kThreads = 256;
constexpr int kCH = 32;  // points per staging chunk in k_upward

template <typename T> struct Cplx;
template <> struct Cplx<float> { using type = float2; };
template <> struct Cplx<double> { using type = double2; };

__device__ __forceinline__ void morton_decode_d(uint64_t m, int &ix, int &iy, int &iz) {
    auto compact = [](uint64_t x) -> int {
        x &= 0x1249249249249249ull;
        x = (x ^ (x >> 2)) & 0x10c30c30c30c30c3ull;
        x = (x ^ (x >> 4)) & 0x100f00f00f00f00full;
        x = (x ^ (x >> 8)) & 0x1f0000ff0000ffull;
        x = (x ^ (x >> 16)) & 0x1f00000000ffffull;
        x = (x ^ (x >> 32)) & 0x1fffffull;
        return (int)x;
    };
    ix = compact(m);
    iy = compact(m >> 1);
    iz = compact(m >> 2);
}

template <typename U>
__device__ __forceinline__ U *buf_ptr(const BufLayout &lay, int i, char *sm, char *slab) {
    return lay.in_smem[i] ? reinterpret_cast<U *>(sm + lay.off[i])
                          : reinterpret_cast<U *>(slab + (size_t)blockIdx.x * lay.slab_bytes + lay.off[i]);
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
template <typename T, int P>
__global__ void __launch_bounds__(kThreads) k_upward(TreeView tv, DevTables<T> tb, int lstart, int lcount, T *M,
                                                     BufLayout lay, char *slab) {
    extern __shared__ __align__(128) char sm[];
    constexpr int P3 = P * P * P;
    constexpr int PS = UpShape<P>::PS, YS = UpShape<P>::YS;
    constexpr int NAG = (P + 3) / 4, NBCG = (P * P + 3) / 4;
    T *acc = buf_ptr<T>(lay, 0, sm, slab);
    // scratch shared by the two phases: staging + Y for the sources of leaf
    // children, then two P^3 buffers for the moment shifts of non-leaf children
    T *scr = buf_ptr<T>(lay, 1, sm, slab);
    T *As = buf_ptr<T>(lay, 2, sm, slab);   // shift matrices A_{-1}, A_{+1}
    T *stg = scr;                           // [3][kCH][PS]
    T *Y = scr + 3 * kCH * PS;              // [kCH][YS]
    T *b0 = scr, *b1 = scr + P3;
    __shared__ int s_lstart[8], s_lpre[9];
    const int tid = threadIdx.x;
    for (int i = tid; i < 2 * P * P; i += kThreads) As[i] = tb.A[i];
    for (int it = blockIdx.x; it < lcount; it += gridDim.x) {
        const int B = lstart + it;
        const bool selfleaf = (tv.bflags[B] & BF_LEAF) != 0;
        if (selfleaf && !(B == 0 && tv.nlev == 1)) continue;
        if (tv.bnsrc[B] == 0) continue;
        for (int i = tid; i < P3; i += kThreads) acc[i] = (T)0;
        const int l = tv.blevel[B];
        int ix, iy, iz;
        morton_decode_d(tv.bkey[B], ix, iy, iz);
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
        {
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
}

// ---------------------------------------------------------------------------
// Outgoing expansions (Step 3, T_prox2pw), parity-split
// ---------------------------------------------------------------------------
template <typename T, int P, int NF>
__global__ void __launch_bounds__(kThreads) k_prox2pw(TreeView tv, DevTables<T> tb, int nslots,
                                                      const int32_t *slot2box, const T *M,
                                                      typename Cplx<T>::type *Phi, BufLayout lay, char *slab) {
    using C2 = typename Cplx<T>::type;
    extern __shared__ __align__(128) char sm[];
    constexpr int P3 = P * P * P, NH = NF + 1, N1 = 2 * NF + 1;
    T *Mb = buf_ptr<T>(lay, 0, sm, slab);
    C2 *T1 = buf_ptr<C2>(lay, 1, sm, slab);  // [a][b][mz]
    C2 *T2 = buf_ptr<C2>(lay, 2, sm, slab);  // [a][my + NF][mz]
    T *hs = buf_ptr<T>(lay, 3, sm, slab);    // [n][m']
    const int tid = threadIdx.x;
    load_hs<T, P, NF>(tb, hs);
    const size_t stride = (size_t)N1 * N1 * NH;
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
            const int my = it / (NH * NH), r = it % (NH * NH), mxp = r / NH, mz = r % NH;
            C2 E{0, 0}, O{0, 0};
            for (int a = 0; a < P; ++a) {
                const C2 t = T2[(a * N1 + my) * NH + mz];
                const T h = hs[a * NH + mxp];
                if (a & 1) cfma(O, h, t); else cfma(E, h, t);
            }
            out[(size_t)(my * N1 + NF + mxp) * NH + mz] = C2{E.x - O.y, E.y + O.x};
            if (mxp > 0) out[(size_t)(my * N1 + NF - mxp) * NH + mz] = C2{E.x + O.y, E.y - O.x};
        }
    }
}

// ---------------------------------------------------------------------------
// Root: windowed kernel W_0 over the unit box (single CTA, global scratch)
// ---------------------------------------------------------------------------
template <typename T, int P>
__global__ void __launch_bounds__(kThreads) k_root(TreeView tv, DevTables<T> tb, const T *Mroot, int has_sources,
                                                   T *LamW, typename Cplx<T>::type *scr) {
    using C2 = typename Cplx<T>::type;
    constexpr int P3 = P * P * P;
    const int n0 = tb.n0, NW = tb.NW, nh = tb.nhW;
    const T *Fr = tb.FWr, *Fi = tb.FWi;
    const int tid = threadIdx.x;
    if (!has_sources) {
        for (int i = tid; i < P3; i += kThreads) LamW[i] = (T)0;
        return;
    }
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

// ---------------------------------------------------------------------------
// Local expansions and leaf evaluation (Step 3), parity-split
// ---------------------------------------------------------------------------
constexpr int kLThreads = 512;
constexpr int kECH = 32;  // targets per evaluation chunk

// One axis of a Chebyshev re-expansion on a P^3 array: out[.., m, ..] =
// sum_{n >= m} A[n][m] in[.., n, ..] along axis AX (0 = z, the fastest index,
// 1 = y, 2 = x).  Each thread owns two rows (P outputs each) in registers and
// reads A from shared memory once per pair of multiply-adds.
template <typename T, int P, int AX, int NT>
__device__ __forceinline__ void shift_pass(const T *__restrict__ A, const T *in, T *out) {
    constexpr int s = AX == 0 ? 1 : (AX == 1 ? P : P * P);
    if constexpr (P > 20) {  // large orders: one output per thread (registers)
        for (int i = threadIdx.x; i < P * P * P; i += NT) {
            const int m = AX == 0 ? i % P : (AX == 1 ? (i / P) % P : i / (P * P));
            const int b = i - m * s;
            T acc = 0;
            for (int n = m; n < P; ++n) acc += A[n * P + m] * in[b + n * s];
            out[i] = acc;
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
        for (int m = 0; m < P; ++m) o0[m] = o1[m] = (T)0;
#pragma unroll
        for (int n = 0; n < P; ++n) {
            const T v0 = in[b0 + n * s], v1 = in[b1 + n * s];
#pragma unroll
            for (int m = 0; m <= n; ++m) {
                const T a = A[n * P + m];
                o0[m] += a * v0;
                if (TWO) o1[m] += a * v1;
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

template <int P, int NF> struct LocalShape {
    static constexpr int NH = NF + 1, N1 = 2 * NF + 1;
    static constexpr int AG = (P + 6) / 7, AC = (P + AG - 1) / AG;  // phase B: a-groups, a per group
    static constexpr int BG = (P + 7) / 8, BC = (P + BG - 1) / BG;  // phase C
    static constexpr int CG = (P + 8) / 9, CC = (P + CG - 1) / CG;  // phase D
};

template <typename T, int P, int NF>
__global__ void __launch_bounds__(kLThreads, 1) k_local(TreeView tv, DevTables<T> tb, int level, int lstart,
                                                        int lcount, const typename Cplx<T>::type *Phi, T *Lam,
                                                        const T *LamW, double *ufar, BufLayout lay, char *slab,
                                                        unsigned long long *flops) {
    using C2 = typename Cplx<T>::type;
    using S = LocalShape<P, NF>;
    constexpr int NH = S::NH, N1 = S::N1, P3 = P * P * P;
    extern __shared__ __align__(128) char sm[];
    T *Ls = buf_ptr<T>(lay, 0, sm, slab);
    C2 *PsE = buf_ptr<C2>(lay, 1, sm, slab);  // [my + NF][mx'][mz]; PsO follows
    C2 *PsO = PsE + N1 * NH * NH;
    C2 *T2 = PsE;                              // [a][b][mz], reuses the Psi buffers
    C2 *T1e = buf_ptr<C2>(lay, 2, sm, slab);  // [a][my'][mz]; T1o follows
    C2 *T1o = T1e + P * NH * NH;
    T *hs = buf_ptr<T>(lay, 3, sm, slab);
    T *ev = buf_ptr<T>(lay, 4, sm, slab);     // [3][kECH][P]
    T *As = buf_ptr<T>(lay, 5, sm, slab);     // shift matrices A_{-1}, A_{+1}
    __shared__ int s_ncol;
    __shared__ int s_cslot[27];
    __shared__ int s_cd[27][3];
    const int tid = threadIdx.x;
    load_hs<T, P, NF>(tb, hs);
    for (int i = tid; i < 2 * P * P; i += kLThreads) As[i] = tb.A[i];
    const size_t pstride = (size_t)N1 * N1 * NH;
    const T invR = (T)(double)(1u << level);
    const T kH = (T)0.86602540378443864676;  // sqrt(3)/2
    for (int it = blockIdx.x; it < lcount; it += gridDim.x) {
        const int B = lstart + it;
        if (tv.bntgt[B] == 0) continue;
        const uint8_t fl = tv.bflags[B];
        __syncthreads();
        // ---- parent's local expansion re-centred on this machine (T_p2c), or the root term
        if (level == 0) {
            for (int i = tid; i < P3; i += kLThreads) Ls[i] = LamW[i];
        } else {
            T *b0 = reinterpret_cast<T *>(PsE);
            T *b1 = reinterpret_cast<T *>(PsO);
            const int Pb = tv.bparent[B];
            const T *Lp = Lam + (size_t)tv.bslot[Pb] * P3;
            for (int i = tid; i < P3; i += kLThreads) b0[i] = Lp[i];
            __syncthreads();
            const int oc = (int)(tv.bkey[B] & 7ull);
            // child coefficient b_m = sum_{n >= m} A_s[n][m] a_n along z, then y, then x
            shift_pass<T, P, 0, kLThreads>(As + ((oc >> 2) & 1) * P * P, b0, b1);
            __syncthreads();
            shift_pass<T, P, 1, kLThreads>(As + ((oc >> 1) & 1) * P * P, b1, b0);
            __syncthreads();
            shift_pass<T, P, 2, kLThreads>(As + (oc & 1) * P * P, b0, Ls);
        }
        __syncthreads();
        // ---- incoming expansion from F_out colleagues -> Chebyshev coefficients
        if (fl & BF_FIN) {
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
            // phase A: Psi = w_l * sum_S omega^(m.delta) Phi_S, folded into even/odd in m_x
            for (int i = tid; i < N1 * NH * NH; i += kLThreads) {
                const int my = i / (NH * NH), r = i % (NH * NH), mxp = r / NH, mz = r % NH;
                const int myv = my - NF;
                const int rxp = mxp % 3, rxm = (3 - rxp) % 3, ry = (myv % 3 + 3) % 3, rz = mz % 3;
                C2 Tp{0, 0}, Up{0, 0}, Dp{0, 0}, Tm{0, 0}, Um{0, 0}, Dm{0, 0};
                const size_t off_p = (size_t)(my * N1 + NF + mxp) * NH + mz;
                const size_t off_m = (size_t)(my * N1 + NF - mxp) * NH + mz;
                for (int j = 0; j < ncol; ++j) {
                    const C2 *ph = Phi + (size_t)s_cslot[j] * pstride;
                    const int kyz = ry * s_cd[j][1] + rz * s_cd[j][2];
                    const int kp = (rxp * s_cd[j][0] + kyz) % 3;
                    const int km = (rxm * s_cd[j][0] + kyz) % 3;
                    const C2 vp = ph[off_p];
                    Tp.x += vp.x; Tp.y += vp.y;
                    const T up = kp ? (T)1 : (T)0, dp = kp == 1 ? (T)1 : (kp == 2 ? (T)-1 : (T)0);
                    cfma(Up, up, vp);
                    cfma(Dp, dp, vp);
                    if (mxp > 0) {
                        const C2 vm = ph[off_m];
                        Tm.x += vm.x; Tm.y += vm.y;
                        const T um = km ? (T)1 : (T)0, dm = km == 1 ? (T)1 : (km == 2 ? (T)-1 : (T)0);
                        cfma(Um, um, vm);
                        cfma(Dm, dm, vm);
                    }
                }
                const T w = tb.w[mxp * mxp + myv * myv + mz * mz] * invR;
                // S0 + omega S1 + omega^2 S2 = T - 1.5 U + i (sqrt3/2) D
                const C2 psp{w * (Tp.x - (T)1.5 * Up.x - kH * Dp.y), w * (Tp.y - (T)1.5 * Up.y + kH * Dp.x)};
                const size_t o = (size_t)(my * NH + mxp) * NH + mz;
                if (mxp > 0) {
                    const C2 psm{w * (Tm.x - (T)1.5 * Um.x - kH * Dm.y), w * (Tm.y - (T)1.5 * Um.y + kH * Dm.x)};
                    PsE[o] = C2{psp.x + psm.x, psp.y + psm.y};
                    PsO[o] = C2{psp.x - psm.x, psp.y - psm.y};
                } else {
                    PsE[o] = psp;
                    PsO[o] = C2{0, 0};
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
                    const C2 ep = PsE[(rp + mxp) * NH + mz], em = PsE[(rm + mxp) * NH + mz];
                    const C2 op = PsO[(rp + mxp) * NH + mz], om = PsO[(rm + mxp) * NH + mz];
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
            if (fl & BF_FIN)
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
        morton_decode_d(tv.bkey[B], ix, iy, iz);
        const double R = level_R(level), s2R = 2.0 / R;
        const double cc[3] = {(ix + 0.5) * R, (iy + 0.5) * R, (iz + 0.5) * R};
        const int s = tv.bstart[B], e = s + tv.bcount[B];
        for (int p0 = s; p0 < e; p0 += kECH) {
            const int np = min(kECH, e - p0);
            for (int t = tid; t < 3 * kECH; t += kLThreads) {
                const int ax = t / kECH, j = t % kECH;
                T *o = ev + (ax * kECH + j) * P;
                if (j < np) {
                    const int kk = p0 + j;
                    const double u = ax == 0 ? tv.ux[kk] : (ax == 1 ? tv.uy[kk] : tv.uz[kk]);
                    const T xi = (T)((u - cc[ax]) * s2R);
                    T t0 = (T)1, t1 = xi;
                    o[0] = (T)1;
                    if (P > 1) o[1] = xi;
#pragma unroll
                    for (int n = 2; n < P; ++n) {
                        T t2 = (T)2 * xi * t1 - t0;
                        o[n] = t2;
                        t0 = t1;
                        t1 = t2;
                    }
                } else {
#pragma unroll
                    for (int n = 0; n < P; ++n) o[n] = (T)0;
                }
            }
            __syncthreads();
            // W[j][ab] = sum_c Lambda[ab][c] T_c(z_j): 4 x 4 register tiles over (ab, j)
            {
                T *W = reinterpret_cast<T *>(PsE);
                const T *tzs = ev + 2 * kECH * P;
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
                // u_j = sum_a T_a(x_j) sum_b T_b(y_j) W[j][a][b]: 16 threads per target
                const int j = tid >> 4, g = tid & 15;
                const T *tx = ev + j * P, *ty = ev + (kECH + j) * P;
                const T *Wj = W + j * (P * P);
                T sum = 0;
                for (int a = g; a < P; a += 16) {
                    T sa = 0;
#pragma unroll
                    for (int b = 0; b < P; ++b) sa += ty[b] * Wj[a * P + b];
                    sum += tx[a] * sa;
                }
#pragma unroll
                for (int o = 8; o > 0; o >>= 1) sum += __shfl_xor_sync(0xffffffffu, sum, o);
                if (g == 0 && j < np && (tv.pflag[p0 + j] & 2)) ufar[p0 + j] = (double)sum;
            }
            __syncthreads();
        }
    }
}

// ---------------------------------------------------------------------------
// Residual near field (Steps 4 and 5)
// ---------------------------------------------------------------------------
// One warp per target leaf, taken from an atomic work counter.  Lanes map to
// (target, source subset) pairs: G lanes share a target and split its sources
// when the leaf holds fewer than 32 targets.  Sources are read straight from
// global memory (all lanes of a group read the same address, served by L1).
// In single precision the coordinates are hi + lo pairs, relative to the leaf
// centres, and the exact dyadic centre offset is added with a TwoSum, so the
// difference of two nearby points keeps full relative precision; the sum over
// a source leaf is compensated (Kahan) and then accumulated in double.
template <typename T> __device__ __forceinline__ T ldexp_t(T x, int e);
template <> __device__ __forceinline__ float ldexp_t<float>(float x, int e) { return ldexpf(x, e); }
template <> __device__ __forceinline__ double ldexp_t<double>(double x, int e) { return ldexp(x, e); }
// centre coordinate (2 i + 1) 2^-(l+1) of cell i at level l, exact
template <typename T> __device__ __forceinline__ T dyadic_centre(int i, int l) {
    return ldexp_t<T>((T)(2 * i + 1), -(l + 1));
}
template <typename T> __device__ __forceinline__ T rsqrt_t(T x);
template <> __device__ __forceinline__ float rsqrt_t<float>(float x) { return rsqrtf(x); }
template <> __device__ __forceinline__ double rsqrt_t<double>(double x) { return rsqrt(x); }

constexpr int kNearThreads = 256;

template <typename T, int QD>
__global__ void __launch_bounds__(kNearThreads) k_near(TreeView tv, int ntl, const int32_t *tleaves,
                                                       const int32_t *nl_off, const int32_t *nl_src,
                                                       const typename Vec4<T>::type *__restrict__ plocal,
                                                       const float4 *__restrict__ plocal_lo, const T *qmono,
                                                       int qdeg, double *unear, int *counter) {
    using V4 = typename Vec4<T>::type;
    constexpr bool kHiLo = sizeof(T) == 4;
    // residual polynomial coefficients in registers (degree QD known at compile time)
    T qc[QD + 1];
#pragma unroll
    for (int d = 0; d <= QD; ++d) qc[d] = qmono[d];
    (void)qdeg;
    const int tid = threadIdx.x, lane = tid & 31;
    // pairs inside the support of the residual kernel (statistics); the
    // counter sits 8 bytes after the work counter
    unsigned inside32 = 0;
    for (;;) {
        int it = 0;
        if (lane == 0) it = atomicAdd(counter, 1);
        it = __shfl_sync(0xffffffffu, it, 0);
        if (it >= ntl) {
#pragma unroll
            unsigned long long inside = inside32;
            for (int o = 16; o > 0; o >>= 1) inside += __shfl_xor_sync(0xffffffffu, inside, o);
            if (lane == 0 && inside) atomicAdd(reinterpret_cast<unsigned long long *>(counter + 2), inside);
            break;
        }
        const int Tb = tleaves[it];
        const int a = tv.blevel[Tb];
        int tx, ty, tz;
        morton_decode_d(tv.bkey[Tb], tx, ty, tz);
        // box centres (2i + 1) 2^-(l+1) are exact in T; so are their differences
        // (at most ~22 significant bits for the level gaps of a balanced tree)
        const T cTx = dyadic_centre<T>(tx, a), cTy = dyadic_centre<T>(ty, a), cTz = dyadic_centre<T>(tz, a);
        const int ts = tv.bstart[Tb], nt = tv.bcount[Tb];
        const int G = nt >= 32 ? 1 : (nt >= 16 ? 2 : (nt >= 8 ? 4 : 8));
        const int per = 32 / G;
        const int l0 = nl_off[it], l1 = nl_off[it + 1];
        for (int t0 = 0; t0 < nt; t0 += per) {
            const int j = t0 + lane / G, g = lane % G;
            const bool valid = j < nt;
            V4 xt;
            float4 xl = make_float4(0.f, 0.f, 0.f, 0.f);
            if (valid) {
                xt = plocal[ts + j];
                if (kHiLo) xl = plocal_lo[ts + j];
            } else {
                xt.x = xt.y = xt.z = xt.w = (T)0;
            }
            double acc = 0.0;
            for (int li = l0; li < l1; ++li) {
                const int Sb = nl_src[li];
                const int b = tv.blevel[Sb];
                int sx, sy, sz;
                morton_decode_d(tv.bkey[Sb], sx, sy, sz);
                // exact dyadic centre difference, added to the target's local coordinate
                const T dcx = cTx - dyadic_centre<T>(sx, b);
                const T dcy = cTy - dyadic_centre<T>(sy, b);
                const T dcz = cTz - dyadic_centre<T>(sz, b);
                T px = xt.x + dcx, py = xt.y + dcy, pz = xt.z + dcz;
                T pxl = (T)0, pyl = (T)0, pzl = (T)0;
                if (kHiLo) {  // TwoSum error terms plus the lo parts
                    T bb = px - xt.x;
                    pxl = ((xt.x - (px - bb)) + (dcx - bb)) + (T)xl.x;
                    bb = py - xt.y;
                    pyl = ((xt.y - (py - bb)) + (dcy - bb)) + (T)xl.y;
                    bb = pz - xt.z;
                    pzl = ((xt.z - (pz - bb)) + (dcz - bb)) + (T)xl.z;
                }
                const T invRb = ldexp_t<T>((T)1, b);
                const T invRb2 = invRb * invRb;
                const T Rb2 = ldexp_t<T>((T)1, -2 * b);
                const int ss = tv.bstart[Sb], ns = tv.bcount[Sb];
                // screening radius: a little above R_b so that rounding in the
                // coarse distance below never drops a pair inside the support
                const T Rb2_screen = Rb2 * (T)1.0009765625;
                T part = 0, comp = 0;
                for (int c0 = 0; c0 < ns; c0 += 32 * G) {
                    // pass 1: coarse distance of 32 sources per lane -> bitmask
                    unsigned mask = 0;
                    if (G == 1 && c0 + 32 <= ns) {  // full chunk, one lane per target
                        const V4 *yp = plocal + ss + c0;
#pragma unroll 8
                        for (int k = 0; k < 32; ++k) {
                            const V4 y = yp[k];
                            const T dx = px - y.x, dy = py - y.y, dz = pz - y.z;
                            if (dx * dx + dy * dy + dz * dz < Rb2_screen) mask |= 1u << k;
                        }
                    } else {
#pragma unroll 8
                        for (int k = 0; k < 32; ++k) {
                            const int jj = c0 + g + G * k;
                            if (jj < ns) {
                                const V4 y = plocal[ss + jj];
                                const T dx = px - y.x, dy = py - y.y, dz = pz - y.z;
                                if (dx * dx + dy * dy + dz * dz < Rb2_screen) mask |= 1u << k;
                            }
                        }
                    }
                    // pass 2: the residual kernel on the pairs inside the support
                    while (mask) {
                        const int k = __ffs(mask) - 1;
                        mask &= mask - 1;
                        const int jj = c0 + g + G * k;
                        const V4 y = plocal[ss + jj];
                        T dx = px - y.x, dy = py - y.y, dz = pz - y.z;
                        if (kHiLo) {
                            const float4 yl = plocal_lo[ss + jj];
                            dx += pxl - (T)yl.x;
                            dy += pyl - (T)yl.y;
                            dz += pzl - (T)yl.z;
                        }
                        const T r2 = dx * dx + dy * dy + dz * dz;
                        const T x = (T)2 * r2 * invRb2 - (T)1;
                        T qv = qc[QD];
#pragma unroll
                        for (int d = QD - 1; d >= 0; --d) qv = qv * x + qc[d];
                        const T rinv = r2 > (T)0 ? rsqrt_t<T>(r2) : (T)0;
                        const T v = rinv - qv * invRb;
                        const T term = (r2 < Rb2) ? y.w * v : (T)0;
                        inside32 += (r2 < Rb2) ? 1u : 0u;
                        const T yk = term - comp;
                        const T tk = part + yk;
                        comp = (tk - part) - yk;
                        part = tk;
                    }
                }
                acc += (double)part - (double)comp;
            }
            for (int o = G >> 1; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
            if (valid && g == 0 && (tv.pflag[ts + j] & 2)) unear[ts + j] = acc;
        }
    }
}

__global__ void k_finalize(int64_t n, const uint8_t *pflag, const int32_t *pout, const double *ufar,
                           const double *unear, const Frame *frame, int mode, double *pot) {
    int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n || !(pflag[k] & 2)) return;
    // mode 0: both parts, 1: far part only, 2: near part only
    double v = (mode == 2 ? 0.0 : ufar[k]) + (mode == 1 ? 0.0 : unear[k]);
    pot[pout[k]] = v / frame->S;
}

// launch k_near with the residual polynomial degree as a template argument
template <typename T, int QD>
static void launch_near_qd(int grid, cudaStream_t st, TreeView tv, int ntl, const int32_t *tleaves,
                           const int32_t *nl_off, const int32_t *nl_src, const typename Vec4<T>::type *plocal,
                           const float4 *plocal_lo, const T *qmono, double *unear, int *counter) {
    k_near<T, QD><<<grid, kNearThreads, 0, st>>>(tv, ntl, tleaves, nl_off, nl_src, plocal, plocal_lo, qmono, QD,
                                                  unear, counter);
}

template <typename T>
static int launch_near(int qdeg, int grid, cudaStream_t st, TreeView tv, int ntl, const int32_t *tleaves,
                       const int32_t *nl_off, const int32_t *nl_src, const typename Vec4<T>::type *plocal,
                       const float4 *plocal_lo, const T *qmono, double *unear, int *counter) {
    switch (qdeg) {
#define DMK_NEAR_CASE(d) \
    case d: launch_near_qd<T, d>(grid, st, tv, ntl, tleaves, nl_off, nl_src, plocal, plocal_lo, qmono, unear, counter); return 0;
        DMK_NEAR_CASE(2) DMK_NEAR_CASE(3) DMK_NEAR_CASE(4) DMK_NEAR_CASE(5) DMK_NEAR_CASE(6) DMK_NEAR_CASE(7)
        DMK_NEAR_CASE(8) DMK_NEAR_CASE(9) DMK_NEAR_CASE(10) DMK_NEAR_CASE(11) DMK_NEAR_CASE(12) DMK_NEAR_CASE(13)
        DMK_NEAR_CASE(14) DMK_NEAR_CASE(15) DMK_NEAR_CASE(16) DMK_NEAR_CASE(17) DMK_NEAR_CASE(18) DMK_NEAR_CASE(19)
        DMK_NEAR_CASE(20) DMK_NEAR_CASE(21) DMK_NEAR_CASE(22) DMK_NEAR_CASE(23) DMK_NEAR_CASE(24) DMK_NEAR_CASE(25)
        DMK_NEAR_CASE(26) DMK_NEAR_CASE(27) DMK_NEAR_CASE(28) DMK_NEAR_CASE(29) DMK_NEAR_CASE(30)
#undef DMK_NEAR_CASE
    default: return 1;
    }
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
        ws.ensure(cx.bufs->LamW, (int64_t)P3 * sizeof(T)) || ws.ensure(cx.bufs->ufar, n * 8) ||
        ws.ensure(cx.bufs->unear, n * 8) || ws.ensure(cx.bufs->counter, 64)) {
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
    PCK(cudaMemsetAsync(cx.bufs->counter.p, 0, 64, st));

    // ---- upward pass (finest level first)
    cudaEventRecord(cx.ev[1], st);
    {
        const size_t scr = std::max((size_t)2 * P3, (size_t)kCH * (3 * UpShape<P>::PS + UpShape<P>::YS)) * sizeof(T);
        BufLayout lay = make_layout({P3 * sizeof(T), scr, (size_t)2 * P * P * sizeof(T)}, smem_limit - 1024);
        PCK(cudaFuncSetAttribute(k_upward<T, P>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)lay.smem_bytes));
        const int lmax = tv.nlev - 1;
        for (int l = (tv.nlev == 1 ? 0 : lmax - 1); l >= 0; --l) {
            int lc = tv.lev_count[l];
            int grid = std::min(lc, maxgrid);
            if (grid <= 0) continue;
            if (ws.ensure(cx.bufs->slab, (int64_t)grid * lay.slab_bytes + 128)) { err = "oom slab"; return DMK_ERR_OOM; }
            ::dmk::launch_tick();
            k_upward<T, P><<<grid, kThreads, lay.smem_bytes, st>>>(tv, tb, tv.lev_start[l], lc, M, lay,
                                                                   (char *)cx.bufs->slab.p);
        }
        PCK(cudaGetLastError());
    }
    // ---- outgoing expansions of every F_out box
    cudaEventRecord(cx.ev[2], st);
    if (ws.ensure(cx.bufs->Phi, (int64_t)nslots * N1 * N1 * NH * sizeof(C2))) {
        err = "device allocation failed (plane waves)";
        return DMK_ERR_OOM;
    }
    C2 *Phi = (C2 *)cx.bufs->Phi.p;
    if (!cx.tree->root_leaf && nslots > 0) {
        BufLayout lay = make_layout({P3 * sizeof(T), (size_t)P * P * NH * sizeof(C2), (size_t)P * N1 * NH * sizeof(C2),
                                     (size_t)P * NH * sizeof(T)},
                                    smem_limit);
        PCK(cudaFuncSetAttribute(k_prox2pw<T, P, NF>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)lay.smem_bytes));
        int grid = std::min(nslots, maxgrid);
        if (ws.ensure(cx.bufs->slab, (int64_t)grid * lay.slab_bytes + 128)) { err = "oom slab"; return DMK_ERR_OOM; }
        ::dmk::launch_tick();
        k_prox2pw<T, P, NF><<<grid, kThreads, lay.smem_bytes, st>>>(
            tv, tb, nslots, (const int32_t *)cx.tree->slot2box.p, M, Phi, lay, (char *)cx.bufs->slab.p);
        PCK(cudaGetLastError());
    }
    // ---- root windowed term
    {
        const int NW = tb.NW, nhW = tb.nhW;
        size_t scr = (size_t)(2 * P * P * nhW + 2 * P * NW * nhW + NW * NW * nhW) * sizeof(C2);
        if (ws.ensure(cx.bufs->rootscr, scr)) { err = "oom root"; return DMK_ERR_OOM; }
        const int has_src = cx.total_sources > 0 ? 1 : 0;
        ::dmk::launch_tick();
        k_root<T, P><<<1, kThreads, 0, st>>>(tv, tb, M, has_src, LamW, (C2 *)cx.bufs->rootscr.p);
        PCK(cudaGetLastError());
    }
    // ---- local expansions, coarsest level first; leaves evaluate
    {
        // buffer 1 holds the incoming expansion, the p2c scratch (2 P^3) and the
        // evaluation intermediate W (kECH P^2)
        const size_t psi_bytes = std::max({(size_t)2 * N1 * NH * NH * sizeof(C2), (size_t)2 * P3 * sizeof(T),
                                           (size_t)kECH * P * P * sizeof(T)});
        cudaEventRecord(cx.ev[6], st);
        BufLayout lay = make_layout({P3 * sizeof(T), psi_bytes, (size_t)2 * P * NH * NH * sizeof(C2),
                                     (size_t)P * NH * sizeof(T), (size_t)3 * kECH * P * sizeof(T),
                                     (size_t)2 * P * P * sizeof(T)},
                                    smem_limit - 2048);
        PCK(cudaFuncSetAttribute(k_local<T, P, NF>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)lay.smem_bytes));
        for (int l = 0; l < tv.nlev; ++l) {
            int lc = tv.lev_count[l];
            int grid = std::min(lc, cx.num_sms * 2);
            if (grid <= 0) continue;
            if (ws.ensure(cx.bufs->slab, (int64_t)grid * lay.slab_bytes + 128)) { err = "oom slab"; return DMK_ERR_OOM; }
            ::dmk::launch_tick();
            k_local<T, P, NF><<<grid, kLThreads, lay.smem_bytes, st>>>(tv, tb, l, tv.lev_start[l], lc, Phi, Lam,
                                                                       LamW, ufar, lay, (char *)cx.bufs->slab.p,
                                                                       (unsigned long long *)cx.bufs->counter.p + 2);
        }
        PCK(cudaGetLastError());
    }
    // ---- residual near field and self corrections
    cudaEventRecord(cx.ev[3], st);
    if (cx.tree->ntleaves > 0) {
        int grid = std::min((cx.tree->ntleaves + 7) / 8, cx.num_sms * 8);
        ::dmk::launch_tick();
        int rc_near = launch_near<T>(tb.qdeg, grid, st, tv, cx.tree->ntleaves, (const int32_t *)cx.tree->tleaves.p,
                                     (const int32_t *)cx.tree->nl_off.p, (const int32_t *)cx.tree->nl_src.p,
                                     (const typename Vec4<T>::type *)cx.tree->plocal.p,
                                     (const float4 *)cx.tree->plocal_lo.p, tb.qmono, unear,
                                     (int *)cx.bufs->counter.p);
        if (rc_near) { err = "residual polynomial degree outside 2..30"; return DMK_ERR_UNSUPPORTED; }
        PCK(cudaGetLastError());
    }
    cudaEventRecord(cx.ev[4], st);
    ::dmk::launch_tick();
    k_finalize<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(n, tv.pflag, (const int32_t *)cx.tree->pout.p, ufar,
                                                           unear, (const Frame *)cx.tree->frame.p, cx.mode,
                                                           cx.pot);
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
