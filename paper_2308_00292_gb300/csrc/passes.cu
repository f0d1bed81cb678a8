// passes.cu -- the upward pass, the plane-wave (dual-space) downward pass and
// the residual near field of the discrete DMK algorithm (Steps 2-5 of Sec. 3.4
// of arXiv 2308.00292), templated on the working precision T and the
// Chebyshev order P.
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
// Kernels:
//   k_upward   level by level, finest first: moments of a non-leaf box from the
//              sources of its leaf children (anterpolation onto the parent grid,
//              eq. proxynd) and from the moments of its non-leaf children (T_c2p,
//              Lemma ctoplemma, exact triangular shift matrices)
//   k_prox2pw  every F_out box: Phi = (F x F x F) M  (T_prox2pw)
//   k_root     the windowed kernel W_0 at the root (eq. windowedkernelft2)
//   k_local    level by level, coarsest first, every box with targets:
//              Lambda = T_p2c(Lambda_parent) (Lemma ptoclemma) plus, for F_in
//              boxes, the incoming expansion of eq. diagonaltranslation formed
//              one m_y slice at a time and converted straight to Chebyshev
//              coefficients (T_pw2poly); leaves then evaluate Lambda at their
//              targets (Step 3 "Evaluate local expansions")
//   k_near     residual kernels R_{L(j)} over the interaction lists (Step 4),
//              including the self correction of Step 5 (r = 0 terms)
#include "passes.h"

#include <algorithm>
#include <cstdio>

namespace dmk {

constexpr int kThreads = 256;
constexpr int kCH = 32;  // points per staging chunk

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

// ---------------------------------------------------------------------------
// Upward pass (Step 2)
// ---------------------------------------------------------------------------
template <typename T, int P>
__global__ void __launch_bounds__(kThreads) k_upward(TreeView tv, DevTables<T> tb, int lstart, int lcount, T *M,
                                                     BufLayout lay, char *slab) {
    extern __shared__ __align__(128) char sm[];
    constexpr int P3 = P * P * P;
    T *acc = buf_ptr<T>(lay, 0, sm, slab);
    T *b0 = buf_ptr<T>(lay, 1, sm, slab);
    T *b1 = buf_ptr<T>(lay, 2, sm, slab);
    T *stg = buf_ptr<T>(lay, 3, sm, slab);  // [3][kCH][P]
    const int tid = threadIdx.x;
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
        int k = 0;
        for (int oc = 0; oc < 8; ++oc) {
            if (!(cm & (1u << oc))) continue;
            const int D = selfleaf ? B : c0 + k;
            ++k;
            if (tv.bnsrc[D] == 0) continue;
            const bool dleaf = selfleaf || (tv.bflags[D] & BF_LEAF);
            if (dleaf) {
                // anterpolation of the leaf's sources onto this box's grid
                const int s = tv.bstart[D], e = s + tv.bcount[D];
                for (int p0 = s; p0 < e; p0 += kCH) {
                    const int np = min(kCH, e - p0);
                    for (int t = tid; t < 3 * kCH; t += kThreads) {
                        const int ax = t / kCH, j = t % kCH;
                        T *o = stg + (ax * kCH + j) * P;
                        if (j < np) {
                            const int kk = p0 + j;
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
                    for (int pr = tid; pr < P * P; pr += kThreads) {
                        const int b = pr / P, c = pr % P;
                        T r[P];
#pragma unroll
                        for (int a = 0; a < P; ++a) r[a] = (T)0;
                        for (int j = 0; j < np; ++j) {
                            const T w = stg[(kCH + j) * P + b] * stg[(2 * kCH + j) * P + c];
                            const T *tx = stg + j * P;
#pragma unroll
                            for (int a = 0; a < P; ++a) r[a] += tx[a] * w;
                        }
#pragma unroll
                        for (int a = 0; a < P; ++a) acc[(a * P + b) * P + c] += r[a];
                    }
                    __syncthreads();
                }
            } else {
                // T_c2p: parent moments from child moments, exact
                const T *Mc = M + (size_t)tv.bslot[D] * P3;
                for (int i = tid; i < P3; i += kThreads) b0[i] = Mc[i];
                __syncthreads();
                const T *Ax = tb.A + (oc & 1) * P * P;
                const T *Ay = tb.A + ((oc >> 1) & 1) * P * P;
                const T *Az = tb.A + ((oc >> 2) & 1) * P * P;
                for (int i = tid; i < P3; i += kThreads) {
                    const int n = i % P, ab = i / P;
                    T s = (T)0;
                    for (int m = 0; m <= n; ++m) s += Az[n * P + m] * b0[ab * P + m];
                    b1[i] = s;
                }
                __syncthreads();
                for (int i = tid; i < P3; i += kThreads) {
                    const int c = i % P, n = (i / P) % P, a = i / (P * P);
                    T s = (T)0;
                    for (int m = 0; m <= n; ++m) s += Ay[n * P + m] * b1[(a * P + m) * P + c];
                    b0[i] = s;
                }
                __syncthreads();
                for (int i = tid; i < P3; i += kThreads) {
                    const int bc = i % (P * P), n = i / (P * P);
                    T s = (T)0;
                    for (int m = 0; m <= n; ++m) s += Ax[n * P + m] * b0[m * P * P + bc];
                    acc[i] += s;
                }
                __syncthreads();
            }
        }
        T *Mo = M + (size_t)tv.bslot[B] * P3;
        for (int i = tid; i < P3; i += kThreads) Mo[i] = acc[i];
        __syncthreads();
    }
}

// ---------------------------------------------------------------------------
// Outgoing expansions (Step 3, T_prox2pw)
// ---------------------------------------------------------------------------
template <typename T, int P>
__global__ void __launch_bounds__(kThreads) k_prox2pw(TreeView tv, DevTables<T> tb, int nslots,
                                                      const int32_t *slot2box, const T *M,
                                                      typename Cplx<T>::type *Phi, BufLayout lay, char *slab) {
    using C2 = typename Cplx<T>::type;
    extern __shared__ __align__(128) char sm[];
    constexpr int P3 = P * P * P;
    const int nf = tb.nf, N1 = tb.N1, nh = tb.nh;
    T *Mb = buf_ptr<T>(lay, 0, sm, slab);
    C2 *T1 = buf_ptr<C2>(lay, 1, sm, slab);   // [a][b][mz]
    C2 *T2 = buf_ptr<C2>(lay, 2, sm, slab);   // [a][mz] for one my
    T *Fs = buf_ptr<T>(lay, 3, sm, slab);     // Fr [N1][P], then Fi
    const int tid = threadIdx.x;
    for (int i = tid; i < N1 * P; i += kThreads) {
        Fs[i] = tb.Fr[i];
        Fs[N1 * P + i] = tb.Fi[i];
    }
    const T *Fr = Fs, *Fi = Fs + N1 * P;
    const size_t stride = (size_t)N1 * N1 * nh;
    for (int slot = blockIdx.x; slot < nslots; slot += gridDim.x) {
        const int B = slot2box[slot];
        if (!(tv.bflags[B] & BF_FOUT)) continue;
        __syncthreads();
        const T *Ms = M + (size_t)slot * P3;
        for (int i = tid; i < P3; i += kThreads) Mb[i] = Ms[i];
        __syncthreads();
        for (int i = tid; i < P * P * nh; i += kThreads) {
            const int mz = i % nh, ab = i / nh;
            const T *fr = Fr + (mz + nf) * P, *fi = Fi + (mz + nf) * P;
            T re = 0, im = 0;
#pragma unroll 6
            for (int c = 0; c < P; ++c) {
                const T m = Mb[ab * P + c];
                re += fr[c] * m;
                im += fi[c] * m;
            }
            T1[i] = C2{re, im};
        }
        __syncthreads();
        C2 *out = Phi + (size_t)slot * stride;
        for (int my = 0; my < N1; ++my) {
            const T *fr = Fr + my * P, *fi = Fi + my * P;
            for (int i = tid; i < P * nh; i += kThreads) {
                const int a = i / nh, mz = i % nh;
                T re = 0, im = 0;
                for (int b = 0; b < P; ++b) {
                    const C2 t = T1[(a * P + b) * nh + mz];
                    re += fr[b] * t.x - fi[b] * t.y;
                    im += fr[b] * t.y + fi[b] * t.x;
                }
                T2[i] = C2{re, im};
            }
            __syncthreads();
            for (int i = tid; i < N1 * nh; i += kThreads) {
                const int mx = i / nh, mz = i % nh;
                const T *gr = Fr + mx * P, *gi = Fi + mx * P;
                T re = 0, im = 0;
                for (int a = 0; a < P; ++a) {
                    const C2 t = T2[a * nh + mz];
                    re += gr[a] * t.x - gi[a] * t.y;
                    im += gr[a] * t.y + gi[a] * t.x;
                }
                out[(size_t)(my * N1 + mx) * nh + mz] = C2{re, im};
            }
            __syncthreads();
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
// Local expansions and leaf evaluation (Step 3)
// ---------------------------------------------------------------------------
template <typename T, int P>
__global__ void __launch_bounds__(kThreads) k_local(TreeView tv, DevTables<T> tb, int level, int lstart, int lcount,
                                                    const typename Cplx<T>::type *Phi, T *Lam, const T *LamW,
                                                    double *ufar, BufLayout lay, char *slab) {
    using C2 = typename Cplx<T>::type;
    extern __shared__ __align__(128) char sm[];
    constexpr int P3 = P * P * P;
    const int nf = tb.nf, N1 = tb.N1, nh = tb.nh;
    T *Ls = buf_ptr<T>(lay, 0, sm, slab);
    C2 *T1 = buf_ptr<C2>(lay, 1, sm, slab);  // [a][my][mz]; also p2c scratch b0
    C2 *T2 = buf_ptr<C2>(lay, 2, sm, slab);  // [a][b][mz]; also p2c scratch b1
    C2 *Ps = buf_ptr<C2>(lay, 3, sm, slab);  // [mx][mz] one my slice of Psi
    T *Fs = buf_ptr<T>(lay, 4, sm, slab);    // Fr [N1][P], Fi
    T *ev = buf_ptr<T>(lay, 5, sm, slab);    // [3][kCH][P]
    __shared__ int s_ncol;
    __shared__ int s_cslot[27];
    __shared__ int s_cd[27][3];
    const int tid = threadIdx.x;
    for (int i = tid; i < N1 * P; i += kThreads) {
        Fs[i] = tb.Fr[i];
        Fs[N1 * P + i] = tb.Fi[i];
    }
    const T *Fr = Fs, *Fi = Fs + N1 * P;
    const size_t pstride = (size_t)N1 * N1 * nh;
    const T invR = (T)(double)(1u << level);
    const T kH = (T)0.86602540378443864676;  // sqrt(3)/2
    for (int it = blockIdx.x; it < lcount; it += gridDim.x) {
        const int B = lstart + it;
        if (tv.bntgt[B] == 0) continue;
        const uint8_t fl = tv.bflags[B];
        __syncthreads();
        // ---- parent's local expansion, re-centred (T_p2c) or the root term
        if (level == 0) {
            for (int i = tid; i < P3; i += kThreads) Ls[i] = LamW[i];
        } else {
            T *b0 = reinterpret_cast<T *>(T1);
            T *b1 = reinterpret_cast<T *>(T2);
            const int Pb = tv.bparent[B];
            const T *Lp = Lam + (size_t)tv.bslot[Pb] * P3;
            for (int i = tid; i < P3; i += kThreads) b0[i] = Lp[i];
            __syncthreads();
            const int oc = (int)(tv.bkey[B] & 7ull);
            const T *Ax = tb.A + (oc & 1) * P * P;
            const T *Ay = tb.A + ((oc >> 1) & 1) * P * P;
            const T *Az = tb.A + ((oc >> 2) & 1) * P * P;
            for (int i = tid; i < P3; i += kThreads) {
                const int m = i % P, ab = i / P;
                T s = 0;
                for (int n = m; n < P; ++n) s += Az[n * P + m] * b0[ab * P + n];
                b1[i] = s;
            }
            __syncthreads();
            for (int i = tid; i < P3; i += kThreads) {
                const int c = i % P, m = (i / P) % P, a = i / (P * P);
                T s = 0;
                for (int n = m; n < P; ++n) s += Ay[n * P + m] * b1[(a * P + n) * P + c];
                b0[i] = s;
            }
            __syncthreads();
            for (int i = tid; i < P3; i += kThreads) {
                const int bc = i % (P * P), m = i / (P * P);
                T s = 0;
                for (int n = m; n < P; ++n) s += Ax[n * P + m] * b0[n * P * P + bc];
                Ls[i] = s;
            }
        }
        __syncthreads();
        // ---- incoming expansion from F_out colleagues -> Chebyshev coefficients
        if (fl & BF_FIN) {
            if (tid == 0) {
                int nc = 0;
                for (int k = 0; k < 27; ++k) {
                    const int S = tv.bcol[(size_t)B * 27 + k];
                    if (S < 0 || !(tv.bflags[S] & BF_FOUT)) continue;
                    s_cslot[nc] = tv.bslot[S];
                    // delta = (c_B - c_S) / R = -(dx, dy, dz)
                    s_cd[nc][0] = 1 - k / 9;
                    s_cd[nc][1] = 1 - (k / 3) % 3;
                    s_cd[nc][2] = 1 - k % 3;
                    ++nc;
                }
                s_ncol = nc;
            }
            __syncthreads();
            const int ncol = s_ncol;
            for (int my = 0; my < N1; ++my) {
                const int myv = my - nf;
                for (int i = tid; i < N1 * nh; i += kThreads) {
                    const int mx = i / nh, mz = i % nh, mxv = mx - nf;
                    T re = 0, im = 0;
                    for (int j = 0; j < ncol; ++j) {
                        int ph = mxv * s_cd[j][0] + myv * s_cd[j][1] + mz * s_cd[j][2];
                        ph = ((ph % 3) + 3) % 3;
                        const C2 v = Phi[(size_t)s_cslot[j] * pstride + (size_t)(my * N1 + mx) * nh + mz];
                        // multiply by exp(2 pi i ph / 3)
                        if (ph == 0) {
                            re += v.x;
                            im += v.y;
                        } else if (ph == 1) {
                            re += (T)-0.5 * v.x - kH * v.y;
                            im += kH * v.x + (T)-0.5 * v.y;
                        } else {
                            re += (T)-0.5 * v.x + kH * v.y;
                            im += -kH * v.x + (T)-0.5 * v.y;
                        }
                    }
                    const T w = tb.w[mxv * mxv + myv * myv + mz * mz] * invR;
                    Ps[i] = C2{re * w, im * w};
                }
                __syncthreads();
                for (int i = tid; i < P * nh; i += kThreads) {
                    const int a = i / nh, mz = i % nh;
                    T re = 0, im = 0;
                    for (int mx = 0; mx < N1; ++mx) {
                        const C2 t = Ps[mx * nh + mz];
                        const T gr = Fr[mx * P + a], gi = Fi[mx * P + a];  // G = gr - i gi
                        re += gr * t.x + gi * t.y;
                        im += gr * t.y - gi * t.x;
                    }
                    T1[(a * N1 + my) * nh + mz] = C2{re, im};
                }
                __syncthreads();
            }
            for (int i = tid; i < P * P * nh; i += kThreads) {
                const int mz = i % nh, b = (i / nh) % P, a = i / (nh * P);
                T re = 0, im = 0;
                for (int my = 0; my < N1; ++my) {
                    const C2 t = T1[(a * N1 + my) * nh + mz];
                    const T gr = Fr[my * P + b], gi = Fi[my * P + b];
                    re += gr * t.x + gi * t.y;
                    im += gr * t.y - gi * t.x;
                }
                T2[i] = C2{re, im};
            }
            __syncthreads();
            for (int i = tid; i < P3; i += kThreads) {
                const int c = i % P, ab = i / P;
                T s = 0;
                for (int mz = 0; mz < nh; ++mz) {
                    const C2 t = T2[ab * nh + mz];
                    const T cz = mz == 0 ? (T)1 : (T)2;
                    s += cz * (Fr[(mz + nf) * P + c] * t.x + Fi[(mz + nf) * P + c] * t.y);
                }
                Ls[i] += s;
            }
            __syncthreads();
        }
        if (!(fl & BF_LEAF)) {
            T *Lo = Lam + (size_t)tv.bslot[B] * P3;
            for (int i = tid; i < P3; i += kThreads) Lo[i] = Ls[i];
            continue;
        }
        // ---- leaf: evaluate the local expansion at its targets
        int ix, iy, iz;
        morton_decode_d(tv.bkey[B], ix, iy, iz);
        const double R = level_R(level), s2R = 2.0 / R;
        const double cc[3] = {(ix + 0.5) * R, (iy + 0.5) * R, (iz + 0.5) * R};
        const int s = tv.bstart[B], e = s + tv.bcount[B];
        for (int p0 = s; p0 < e; p0 += kCH) {
            const int np = min(kCH, e - p0);
            for (int t = tid; t < 3 * kCH; t += kThreads) {
                const int ax = t / kCH, j = t % kCH;
                T *o = ev + (ax * kCH + j) * P;
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
            const int j = tid >> 3, g = tid & 7;
            const T *tx = ev + j * P, *ty = ev + (kCH + j) * P, *tz = ev + (2 * kCH + j) * P;
            T sum = 0;
            for (int a = g; a < P; a += 8) {
                T sa = 0;
                for (int b = 0; b < P; ++b) {
                    const T *row = Ls + (a * P + b) * P;
                    T sbc = 0;
#pragma unroll
                    for (int c = 0; c < P; ++c) sbc += row[c] * tz[c];
                    sa += ty[b] * sbc;
                }
                sum += tx[a] * sa;
            }
            sum += __shfl_xor_sync(0xffffffffu, sum, 4);
            sum += __shfl_xor_sync(0xffffffffu, sum, 2);
            sum += __shfl_xor_sync(0xffffffffu, sum, 1);
            if (g == 0 && j < np && (tv.pflag[p0 + j] & 2)) ufar[p0 + j] = (double)sum;
            __syncthreads();
        }
    }
}

// ---------------------------------------------------------------------------
// Residual near field (Steps 4 and 5)
// ---------------------------------------------------------------------------
template <typename T> __device__ __forceinline__ T rsqrt_t(T x);
template <> __device__ __forceinline__ float rsqrt_t<float>(float x) { return rsqrtf(x); }
template <> __device__ __forceinline__ double rsqrt_t<double>(double x) { return rsqrt(x); }

constexpr int kNearThreads = 128;
constexpr int kNearChunk = 256;

template <typename T>
__global__ void __launch_bounds__(kNearThreads) k_near(TreeView tv, int ntl, const int32_t *tleaves,
                                                       const int32_t *nl_off, const int32_t *nl_src,
                                                       const typename Vec4<T>::type *plocal, const T *qmono,
                                                       int qdeg, double *unear) {
    using V4 = typename Vec4<T>::type;
    __shared__ V4 s_src[kNearChunk];
    __shared__ T s_q[64];
    const int tid = threadIdx.x;
    for (int i = tid; i <= qdeg; i += kNearThreads) s_q[i] = qmono[i];
    for (int it = blockIdx.x; it < ntl; it += gridDim.x) {
        const int Tb = tleaves[it];
        const int a = tv.blevel[Tb];
        int tx, ty, tz;
        morton_decode_d(tv.bkey[Tb], tx, ty, tz);
        const double Ra = level_R(a);
        const double cT[3] = {(tx + 0.5) * Ra, (ty + 0.5) * Ra, (tz + 0.5) * Ra};
        const int ts = tv.bstart[Tb], nt = tv.bcount[Tb];
        const int G = nt > 64 ? 1 : (nt > 32 ? 2 : 4);
        const int per = kNearThreads / G;
        const int l0 = nl_off[it], l1 = nl_off[it + 1];
        for (int t0 = 0; t0 < nt; t0 += per) {
            const int j = t0 + tid / G, g = tid % G;
            const bool valid = j < nt;
            V4 xt;
            if (valid) xt = plocal[ts + j];
            else { xt.x = 0; xt.y = 0; xt.z = 0; xt.w = 0; }
            double acc = 0.0;
            for (int li = l0; li < l1; ++li) {
                const int S = nl_src[li];
                const int b = tv.blevel[S];
                int sx, sy, sz;
                morton_decode_d(tv.bkey[S], sx, sy, sz);
                const double Rb = level_R(b);
                // exact dyadic centre difference
                const T dcx = (T)(cT[0] - (sx + 0.5) * Rb);
                const T dcy = (T)(cT[1] - (sy + 0.5) * Rb);
                const T dcz = (T)(cT[2] - (sz + 0.5) * Rb);
                const T px = xt.x + dcx, py = xt.y + dcy, pz = xt.z + dcz;
                const T invRb = (T)(double)(1u << b);
                const T invRb2 = invRb * invRb;
                const T Rb2 = (T)(Rb * Rb);
                const int ss = tv.bstart[S], ns = tv.bcount[S];
                for (int c0 = 0; c0 < ns; c0 += kNearChunk) {
                    const int nc = min(kNearChunk, ns - c0);
                    __syncthreads();
                    for (int i = tid; i < nc; i += kNearThreads) s_src[i] = plocal[ss + c0 + i];
                    __syncthreads();
                    T part = 0;
                    for (int jj = g; jj < nc; jj += G) {
                        const V4 y = s_src[jj];
                        const T dx = px - y.x, dy = py - y.y, dz = pz - y.z;
                        const T r2 = dx * dx + dy * dy + dz * dz;
                        const T x = (T)2 * r2 * invRb2 - (T)1;
                        T qv = s_q[qdeg];
                        for (int d = qdeg - 1; d >= 0; --d) qv = qv * x + s_q[d];
                        const T rinv = r2 > (T)0 ? rsqrt_t<T>(r2) : (T)0;
                        const T v = rinv - qv * invRb;
                        part += (r2 < Rb2) ? y.w * v : (T)0;
                    }
                    acc += (double)part;
                }
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

template <typename T, int P>
static int run_passes_P(PassCtx &cx, std::string &err) {
    using C2 = typename Cplx<T>::type;
    constexpr int P3 = P * P * P;
    TreeView tv = cx.tree->view();
    const DevTables<T> &tb = *reinterpret_cast<const DevTables<T> *>(cx.tables);
    cudaStream_t st = cx.st;
    Workspace &ws = *cx.ws;
    const int nslots = cx.tree->nslots;
    const int N1 = tb.N1, nh = tb.nh;
    const size_t smem_limit = cx.smem_limit;
    const int64_t n = tv.n;
    const int maxgrid = cx.num_sms * 8;

    if (ws.ensure(cx.bufs->M, (int64_t)nslots * P3 * sizeof(T)) ||
        ws.ensure(cx.bufs->Lam, (int64_t)nslots * P3 * sizeof(T)) ||
        ws.ensure(cx.bufs->LamW, (int64_t)P3 * sizeof(T)) || ws.ensure(cx.bufs->ufar, n * 8) ||
        ws.ensure(cx.bufs->unear, n * 8)) {
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

    // ---- upward pass (finest level first)
    cudaEventRecord(cx.ev[1], st);
    {
        BufLayout lay = make_layout({P3 * sizeof(T), P3 * sizeof(T), P3 * sizeof(T), 3 * kCH * P * sizeof(T)},
                                    smem_limit);
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
    if (ws.ensure(cx.bufs->Phi, (int64_t)nslots * N1 * N1 * nh * sizeof(C2))) {
        err = "device allocation failed (plane waves)";
        return DMK_ERR_OOM;
    }
    C2 *Phi = (C2 *)cx.bufs->Phi.p;
    if (!cx.tree->root_leaf && nslots > 0) {
        BufLayout lay = make_layout({P3 * sizeof(T), (size_t)P * P * nh * sizeof(C2), (size_t)P * nh * sizeof(C2),
                                     (size_t)2 * N1 * P * sizeof(T)},
                                    smem_limit);
        PCK(cudaFuncSetAttribute(k_prox2pw<T, P>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)lay.smem_bytes));
        int grid = std::min(nslots, maxgrid);
        if (ws.ensure(cx.bufs->slab, (int64_t)grid * lay.slab_bytes + 128)) { err = "oom slab"; return DMK_ERR_OOM; }
        ::dmk::launch_tick();
        k_prox2pw<T, P><<<grid, kThreads, lay.smem_bytes, st>>>(tv, tb, nslots, (const int32_t *)cx.tree->slot2box.p,
                                                                M, Phi, lay, (char *)cx.bufs->slab.p);
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
        BufLayout lay = make_layout({P3 * sizeof(T), (size_t)P * N1 * nh * sizeof(C2),
                                     (size_t)P * P * nh * sizeof(C2), (size_t)N1 * nh * sizeof(C2),
                                     (size_t)2 * N1 * P * sizeof(T), 3 * kCH * P * sizeof(T)},
                                    smem_limit - 2048);
        // the p2c scratch aliases the T1 / T2 buffers; they must hold P^3 values each
        PCK(cudaFuncSetAttribute(k_local<T, P>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)lay.smem_bytes));
        for (int l = 0; l < tv.nlev; ++l) {
            int lc = tv.lev_count[l];
            int grid = std::min(lc, maxgrid);
            if (grid <= 0) continue;
            if (ws.ensure(cx.bufs->slab, (int64_t)grid * lay.slab_bytes + 128)) { err = "oom slab"; return DMK_ERR_OOM; }
            ::dmk::launch_tick();
            k_local<T, P><<<grid, kThreads, lay.smem_bytes, st>>>(tv, tb, l, tv.lev_start[l], lc, Phi, Lam, LamW,
                                                                  ufar, lay, (char *)cx.bufs->slab.p);
        }
        PCK(cudaGetLastError());
    }
    // ---- residual near field and self corrections
    cudaEventRecord(cx.ev[3], st);
    if (cx.tree->ntleaves > 0) {
        int grid = std::min(cx.tree->ntleaves, cx.num_sms * 16);
        ::dmk::launch_tick();
        k_near<T><<<grid, kNearThreads, 0, st>>>(tv, cx.tree->ntleaves, (const int32_t *)cx.tree->tleaves.p,
                                                 (const int32_t *)cx.tree->nl_off.p,
                                                 (const int32_t *)cx.tree->nl_src.p,
                                                 (const typename Vec4<T>::type *)cx.tree->plocal.p, tb.qmono, tb.qdeg,
                                                 unear);
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
    switch (cx.p) {
    case 9: return run_passes_P<T, 9>(cx, err);
    case 18: return run_passes_P<T, 18>(cx, err);
    case 28: return run_passes_P<T, 28>(cx, err);
    case 38: return run_passes_P<T, 38>(cx, err);
    default: err = "Chebyshev order must be one of 9, 18, 28, 38 (Table 1)"; return DMK_ERR_UNSUPPORTED;
    }
}

int run_passes(PassCtx &cx, std::string &err) {
    return cx.single ? run_passes_T<float>(cx, err) : run_passes_T<double>(cx, err);
}

}  // namespace dmk
