// incoming.cu -- incoming expansions of the downward pass (Step 3 of Sec. 3.4
// of arXiv 2308.00292) on the fifth-generation tensor cores, single precision.
//
// For every incoming box B (a box with targets and an F_out colleague) of
// every level, in one launch:
//
//   Psi_B(m)  = w_l(m) sum_{S in C(B), F_out(S)} exp(i h_l m . (c_B - c_S)) Phi_S(m)
//                                                      (eq. diagonaltranslation)
//   Lambda_B  = Chebyshev coefficients of Re sum_m exp(i h_l m . (x - c_B)) Psi_B(m)
//                                                      (eqs. incomingexpansion2, localexpansion)
//
// The translation phases are cube roots of unity (h_l R_l = 2 pi / 3), so the
// colleague sum is three partial sums per mode.  The conversion is the
// tensor product of the 1-D matrix G[n][m] = conj(F[m][n]).  G is real and
// even in m for even n and imaginary and odd in m for odd n, so folding Psi
// over the signs of m_x and m_y (and using the Hermitian half spectrum in
// m_z) turns it into eight real arrays Y_c(m'), m' = |m| in [0, NF]^3, one per
// parity class c = (a mod 2, b mod 2, c mod 2) of the output index, and
//
//   Lambda[a][b][c] = sum_{m'} H[a][m'_x] H[b][m'_y] H[c][m'_z] Y_{class(a,b,c)}(m'),
//
// with H[n][m'] = Re F[m'][n] (n even) or Im F[m'][n] (n odd).  The first two
// contractions run as tcgen05.mma kind::tf32 with 3xTF32 operands (x = hi +
// lo).  Each of the two K = 8 steps puts its products hi * hi and its cross
// products lo * hi + hi * lo into TMEM accumulators of their own, and the four
// are added in FP32 when they are read: the tensor core's own accumulation of
// one step into another, or of the small cross terms into the large products,
// lost accuracy against the 1e-6 bar (so did the last contraction's, which is
// why it runs on the CUDA cores in FP32, where it is 2 p^3 (nf + 1) flops of the
// box's 8 p (nf+1)^3 + 4 p^2 (nf+1)^2 + 2 p^3 (nf+1)):
//
//   x: rows (m'_y, class) of one m'_z plane, K = m'_x, N = a (even | odd halves)
//   y: rows (a, class),                      K = m'_y, N = b
//   z: rows (class, a, b), the m'_z sum with FP32 FMAs once every plane is done
//
// The row orders put the eight classes on consecutive rows, so that the warps
// that move a contraction's TMEM result into the next operand (a transpose of
// m'_y and a) store into 32 distinct shared-memory banks.
//
// Warps 0-6 read the plane waves of the colleagues plane by plane with
// coalesced loads, eight colleagues in flight at a time.  Warp 7 issues the
// MMAs (one thread: each tcgen05.mma takes tens of cycles to issue, so the
// issue of plane p overlaps the translation of plane p + 1 instead of holding
// up a translating warp) and asks for the colleagues' plane p + 2 in L2 with
// bulk prefetches.  Two CTAs share an SM so that one CTA's barriers and MMA
// waits overlap the other CTA's work.  All threads of a CTA advance together
// between block barriers, and the box's coefficients leave through a TMA bulk
// store (cp.async.bulk, shared to global).  Every wait is bounded.
#include "incoming.h"
#include "tc.h"

namespace dmk {

namespace {

constexpr long long kWaitCycles = 2000000000ll;  // about 1 s

// TMEM columns of the two groups of accumulators that the x and y contractions
// of consecutive planes alternate between: at column g + 32 (2 s + t) the
// products of K step s, t = 0 hi * hi, t = 1 the cross products
__device__ __forceinline__ uint32_t grp_col(int plane) { return (uint32_t)(128 * (plane & 1)); }

template <int P> struct Par {
    static constexpr int PE = (P + 1) / 2, PO = P / 2;
    __device__ static constexpr int n(int parity) { return parity ? PO : PE; }
    // first row of class c (c = pa + 2 pb + 4 pc) among the rows (class, a, b)
    __device__ static constexpr int zbase(int c) {
        int s = 0;
        for (int k = 0; k < c; ++k) s += n(k & 1) * n((k >> 1) & 1);
        return s;
    }
};

// colleague entries of the incoming boxes: (slot << 5) | k, k = 9 (dx + 1) +
// 3 (dy + 1) + (dz + 1) the colleague's offset, for the F_out colleagues only
__global__ void k_fin_colleagues(TreeView tv, int nfin, const int32_t *fin2box, int32_t *finc, int32_t *fincnt,
                                 unsigned long long *reads) {
    const int f = blockIdx.x * blockDim.x + threadIdx.x;
    if (f >= nfin) return;
    const int B = fin2box[f];
    int n = 0;
    for (int k = 0; k < 27; ++k) {
        const int S = tv.bcol[(size_t)B * 27 + k];
        if (S < 0 || !(tv.bflags[S] & BF_FOUT)) continue;
        finc[(size_t)f * 27 + n++] = (tv.bslot[S] << 5) | k;
    }
    fincnt[f] = n;
    atomicAdd(reads, (unsigned long long)n);
}

template <int P, int NF>
__global__ void __launch_bounds__(kIThreads, 2)
    k_incoming(TreeView tv, DevTables<float> tb, int nfin, const int32_t *fin2box, const int32_t *finc,
               const int32_t *fincnt, const float2 *__restrict__ phi, float *lam_in, int *err) {
    using S = InShape<P, NF>;
    using PR = Par<P>;
    constexpr int NH = S::NH, N1 = S::N1, MXP = S::MXP, CB = S::CB;
    constexpr size_t BOXFL2 = (size_t)NH * N1 * MXP;  // float2 per box of the plane-wave array
    extern __shared__ __align__(1024) char sm[];
    float *Ax = reinterpret_cast<float *>(sm + S::O_AX);   // hi, then lo
    float *Ay = reinterpret_cast<float *>(sm + S::O_AY);   // hi, then lo
    float *T2 = reinterpret_cast<float *>(sm + S::O_T2);   // [row (class, a, b)][m'_z]
    float *Bw = reinterpret_cast<float *>(sm + S::O_BW);   // hi, then lo
    float *Hz = reinterpret_cast<float *>(sm + S::O_HZ);   // [c][m'_z]
    float2 *psi = reinterpret_cast<float2 *>(sm + S::O_PSI);
    float2 *ud = reinterpret_cast<float2 *>(sm + S::O_UD);
    // output staging over both operands, once the box's last x and y
    // contractions have completed
    float *Ls = Ax;
    __shared__ __align__(8) uint64_t bx, by;  // MMA completion per contraction
    __shared__ uint32_t s_tmem;
    __shared__ int s_ncol, s_level, s_slot[27];
    // set by the first wait that gives up: every later wait returns at once
    __shared__ volatile int s_abort;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    bool ok = true;
    auto bwait = [&](uint64_t *bar, uint32_t parity) {
        if (s_abort) return false;
        if (tc::mbar_wait(bar, parity, kWaitCycles)) return true;
        s_abort = 1;
        return false;
    };
    auto hs = [&](int c, int m) -> float {  // H[c][m'] from the plan's F
        return (c & 1) ? tb.Fi[(m + NF) * P + c] : tb.Fr[(m + NF) * P + c];
    };

    // ---- set-up: barriers, TMEM, weights
    if (warp == 0) tc::tmem_alloc(&s_tmem, kITmem);
    if (tid == 0) {
        s_abort = 0;
        tc::mbar_init(&bx, 1);
        tc::mbar_init(&by, 1);
    }
    // B[n][k]: n < 16 the even coefficients 2n, n >= 16 the odd ones 2 (n - 16) + 1;
    // k = m' (zero beyond NF and P)
    for (int i = tid; i < 32 * S::K; i += kIThreads) {
        const int n = i / S::K, k = i % S::K;
        const int c = n < 16 ? 2 * n : 2 * (n - 16) + 1;
        const float v = (c < P && k < NH) ? hs(c, k) : 0.f;
        float h, l;
        tc::split_tf32(v, h, l);
        Bw[tc::kmajor_off(n, k, S::K)] = h;
        Bw[32 * S::K + tc::kmajor_off(n, k, S::K)] = l;
    }
    for (int i = tid; i < P * NH; i += kIThreads) Hz[i] = hs(i / NH, i % NH);
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tmem = s_tmem;

    // modes of a plane owned by this thread: index r = my * N1 + mx
    int moff[S::NMODE], mres[S::NMODE], msq[S::NMODE];
    bool mhas[S::NMODE];
#pragma unroll
    for (int k = 0; k < S::NMODE; ++k) {
        const int r = tid + k * kIWorkers;
        mhas[k] = tid < kIWorkers && r < N1 * N1;
        const int my = mhas[k] ? r / N1 : 0, mx = mhas[k] ? r % N1 : 0;
        moff[k] = my * MXP + mx;
        const int vx = mx - NF, vy = my - NF;
        mres[k] = ((vx % 3) + 3) % 3 + 3 * (((vy % 3) + 3) % 3);
        msq[k] = vx * vx + vy * vy;
    }

    uint32_t nx = 0, ny = 0;  // completed waits per MMA barrier (phase parity)
    const uint32_t id32 = tc::idesc_tf32(128, 32);
    constexpr uint32_t kLbo = 128, kSbo = S::K * 32;
    // the 3xTF32 MMAs of a 128 x 16 operand: K step s puts hi * hi into column
    // d + 64 s and the cross products into d + 64 s + 32
    auto mma3 = [&](uint32_t d, uint32_t aH, uint32_t aL, uint32_t bH, uint32_t bL) {
#pragma unroll
        for (int ks = 0; ks < S::K / 8; ++ks) {
            const uint32_t ko = (uint32_t)ks * 256, dk = d + 64 * ks;
            tc::mma_tf32(dk + 32, tc::sdesc(aL + ko, kLbo, kSbo), tc::sdesc(bH + ko, kLbo, kSbo), id32, false);
            tc::mma_tf32(dk + 32, tc::sdesc(aH + ko, kLbo, kSbo), tc::sdesc(bL + ko, kLbo, kSbo), id32, true);
            tc::mma_tf32(dk, tc::sdesc(aH + ko, kLbo, kSbo), tc::sdesc(bH + ko, kLbo, kSbo), id32, false);
        }
    };
    auto wait_bar = [&](uint64_t *bar, uint32_t &cnt) {
        ok = bwait(bar, cnt & 1u) && ok;
        ++cnt;
    };
    // 8 columns of this lane's four accumulators at c, c + 32, c + 64, c + 96, for
    // two column offsets (the even and odd halves), summed (the large products
    // first); one wait for all eight loads
    auto ld_sum8x2 = [&](uint32_t ta, float (&v0)[8], float (&v1)[8]) {
        float a[8], b[8], c[8], d[8], e[8], f2[8];
        tc::ld_x8(ta, v0);
        tc::ld_x8(ta + 64, a);
        tc::ld_x8(ta + 32, b);
        tc::ld_x8(ta + 96, c);
        tc::ld_x8(ta + 16, v1);
        tc::ld_x8(ta + 16 + 64, d);
        tc::ld_x8(ta + 16 + 32, e);
        tc::ld_x8(ta + 16 + 96, f2);
        tc::ld_wait();
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            v0[i] = (v0[i] + a[i]) + (b[i] + c[i]);
            v1[i] = (v1[i] + d[i]) + (e[i] + f2[i]);
        }
    };
    bool stored = false;  // a bulk store of the staging buffer may still be reading it

    for (int f = blockIdx.x; f < nfin; f += gridDim.x) {
        const int B = fin2box[f];
        if (tid == 0) {
            s_ncol = fincnt[f];
            s_level = tv.blevel[B];
        }
        if (tid < 27) s_slot[tid] = finc[(size_t)f * 27 + tid] >> 5;
        __syncthreads();
        const int ncol = s_ncol, level = s_level;
        constexpr uint32_t kPlaneBytes = (uint32_t)(N1 * MXP * sizeof(float2));  // a multiple of 16
        // warp 7 starts the first two planes of every colleague on their way to L2
        if (warp == 7 && lane < ncol) {
            const float2 *pb = phi + (size_t)s_slot[lane] * BOXFL2;
            tc::prefetch_l2(pb, kPlaneBytes);
            if (NH > 1) tc::prefetch_l2(pb + N1 * MXP, kPlaneBytes);
        }
        // phase of colleague j for the mode residues r = (m_x, m_y, m_z) mod 3: omega^kk,
        // kk = r . delta_j mod 3 with delta = (c_B - c_S) / R, as (cos, sin) of 2 pi kk / 3
        for (int t = tid; t < 27 * ncol; t += kIThreads) {
            const int j = t / 27, r = t % 27, k = finc[(size_t)f * 27 + j] & 31;
            const int dx = (4 - k / 9) % 3, dy = (4 - (k / 3) % 3) % 3, dz = (4 - k % 3) % 3;
            const int kk = ((r % 3) * dx + ((r / 3) % 3) * dy + (r / 9) * dz) % 3;
            constexpr float kH = 0.86602540378443864676f;
            ud[t] = kk == 0 ? make_float2(1.f, 0.f) : make_float2(-0.5f, kk == 1 ? kH : -kH);
        }
        const float *wrow = tb.wl ? tb.wl + (size_t)level * (3 * NF * NF + 1) : tb.w;
        const float wscale = tb.wl ? 1.f : (float)(1u << level);
        // the previous box's coefficients must have left the staging buffer
        if (stored && tid == 0) asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory");
        __syncthreads();

        for (int it = 0; it < NH + 2; ++it) {
            // ---- A. translation of plane it: sum over the colleagues of omega^kk Phi
            float2 Ps[S::NMODE];
#pragma unroll
            for (int k = 0; k < S::NMODE; ++k) Ps[k] = make_float2(0.f, 0.f);
            if (it < NH && tid < kIWorkers) {
                const int rz9 = 9 * (it % 3);
                for (int j0 = 0; j0 < ncol; j0 += CB) {
                    float2 v[CB][S::NMODE];
#pragma unroll
                    for (int jj = 0; jj < CB; ++jj) {
                        const int j = j0 + jj;
                        const float2 *pl =
                            phi + (size_t)s_slot[j < ncol ? j : 0] * BOXFL2 + (size_t)it * (N1 * MXP);
#pragma unroll
                        for (int k = 0; k < S::NMODE; ++k)
                            v[jj][k] = (j < ncol && mhas[k]) ? __ldg(pl + moff[k]) : make_float2(0.f, 0.f);
                    }
#pragma unroll
                    for (int jj = 0; jj < CB; ++jj) {
                        if (j0 + jj >= ncol) break;
                        const float2 *uj = ud + (j0 + jj) * 27 + rz9;
#pragma unroll
                        for (int k = 0; k < S::NMODE; ++k) {
                            const float2 c = uj[mres[k]];
                            Ps[k].x = fmaf(-c.y, v[jj][k].y, fmaf(c.x, v[jj][k].x, Ps[k].x));
                            Ps[k].y = fmaf(c.y, v[jj][k].x, fmaf(c.x, v[jj][k].y, Ps[k].y));
                        }
                    }
                }
            }
            // ---- B. the previous contractions (issued at the end of the last step)
            if (it >= 1 && it <= NH) wait_bar(&bx, nx);  // x of plane it - 1
            if (it >= 2) wait_bar(&by, ny);              // y of plane it - 2
            tc::fence_after_sync();
            // ---- C. Psi of plane it; x result of plane it - 1 -> y operand; y result
            // of plane it - 2 -> the second contraction's plane it - 2
            if (it < NH) {
                const float cz = it == 0 ? 1.f : 2.f;  // m_z < 0 through Hermitian symmetry
#pragma unroll
                for (int k = 0; k < S::NMODE; ++k) {
                    if (!mhas[k]) continue;
                    const float w = cz * wscale * wrow[msq[k] + it * it];
                    psi[tid + k * kIWorkers] = make_float2(w * Ps[k].x, w * Ps[k].y);
                }
            }
            {
                // every warp reads its TMEM lane quadrant q; the two warps of a quadrant
                // split the columns (eight of each parity half each)
                const int q = warp & 3, g = warp >> 2, cls = lane & 7;
                if (it >= 1 && it <= NH) {
                    // x result of plane it - 1: lane row (m'_y = 4 q + l / 8, class l mod 8),
                    // columns a (even a-index in 0..15, odd in 16..31): a-index 8 g .. 8 g + 7
                    const int p = it - 1, myp = 4 * q + (lane >> 3);
                    const uint32_t ta = tmem + ((uint32_t)(32 * q) << 16) + grp_col(p) + (uint32_t)(8 * g);
                    float d0[8], d1[8];
                    ld_sum8x2(ta, d0, d1);
                    const bool odd = (cls & 1) != 0;  // parity of a
#pragma unroll
                    for (int i = 0; i < 8; ++i) {
                        float h, l;
                        tc::split_tf32(odd ? d1[i] : d0[i], h, l);
                        const int o = tc::kmajor_off((8 * g + i) * 8 + cls, myp, S::K);
                        Ay[o] = h;
                        Ay[S::TILE_FL + o] = l;
                    }
                }
                if (it >= 2) {
                    // y result of plane it - 2: lane row (a-index 4 q + l / 8, class l mod 8),
                    // columns b of the class's parity: b-index 8 g .. 8 g + 7
                    const int p = it - 2, ai = 4 * q + (lane >> 3), pa = cls & 1, pb = (cls >> 1) & 1;
                    const uint32_t ta = tmem + ((uint32_t)(32 * q) << 16) + grp_col(p) + (uint32_t)(8 * g);
                    float d0[8], d1[8];
                    ld_sum8x2(ta, d0, d1);
                    const int na = PR::n(pa), nb = PR::n(pb), z0 = PR::zbase(cls) + ai * nb;
                    if (ai < na) {
#pragma unroll
                        for (int i = 0; i < 8; ++i) {
                            const int b = 8 * g + i;
                            if (b >= nb) break;
                            T2[(z0 + b) * NH + p] = pb ? d1[i] : d0[i];
                        }
                    }
                }
            }
            tc::fence_before_sync();
            __syncthreads();
            // ---- E. fold Psi of plane it into the x operand: rows (m'_y, class), K = m'_x.
            // Thread (m'_y, m'_x pair h, parity pc of c) forms the four classes of parity
            // pc at two consecutive m'_x; lane l stores class (s + l) mod 4 at step s, so
            // that the 32 lanes of a store hit eight different bank groups
            if (it < NH) {
                const int pc = lane & 1, hp = (lane >> 1) & 7, myp = 2 * warp + (lane >> 4);
                float yv[4][2];  // [pa + 2 pb][m'_x = 2 hp, 2 hp + 1]
#pragma unroll
                for (int i = 0; i < 2; ++i) {
                    const int mxp = 2 * hp + i;
                    float2 Z[4] = {make_float2(0.f, 0.f), make_float2(0.f, 0.f), make_float2(0.f, 0.f),
                                   make_float2(0.f, 0.f)};  // Z[pa + 2 pb]
                    if (myp < NH && mxp < NH) {
                        const float2 Ppp = psi[(NF + myp) * N1 + NF + mxp], Pmp = psi[(NF + myp) * N1 + NF - mxp];
                        const float2 Ppm = psi[(NF - myp) * N1 + NF + mxp], Pmm = psi[(NF - myp) * N1 + NF - mxp];
                        // fold over the sign of m_x: even (E) and odd (O) parts at +m_y and -m_y;
                        // at m'_x = 0 the even part is the mode itself and the odd part zero
                        float2 Ep = Ppp, Op = make_float2(0.f, 0.f), Em = Ppm, Om = make_float2(0.f, 0.f);
                        if (mxp > 0) {
                            Ep = make_float2(Ppp.x + Pmp.x, Ppp.y + Pmp.y);
                            Op = make_float2(Ppp.x - Pmp.x, Ppp.y - Pmp.y);
                            Em = make_float2(Ppm.x + Pmm.x, Ppm.y + Pmm.y);
                            Om = make_float2(Ppm.x - Pmm.x, Ppm.y - Pmm.y);
                        }
                        // then over the sign of m_y
                        if (myp > 0) {
                            Z[0] = make_float2(Ep.x + Em.x, Ep.y + Em.y);
                            Z[1] = make_float2(Op.x + Om.x, Op.y + Om.y);
                            Z[2] = make_float2(Ep.x - Em.x, Ep.y - Em.y);
                            Z[3] = make_float2(Op.x - Om.x, Op.y - Om.y);
                        } else {
                            Z[0] = Ep;
                            Z[1] = Op;
                        }
                    }
                    // Y = Re (pc = 0) or Im (pc = 1) of (-i)^(pa + pb) Z
                    yv[0][i] = pc ? Z[0].y : Z[0].x;
                    yv[1][i] = pc ? -Z[1].x : Z[1].y;
                    yv[2][i] = pc ? -Z[2].x : Z[2].y;
                    yv[3][i] = pc ? -Z[3].y : -Z[3].x;
                }
                if (myp < 16) {
#pragma unroll
                    for (int st = 0; st < 4; ++st) {
                        const int q4 = (st + (lane >> 1)) & 3;  // the class (pa + 2 pb) of this step
                        float v0 = yv[0][0], v1 = yv[0][1];
#pragma unroll
                        for (int c4 = 1; c4 < 4; ++c4)
                            if (q4 == c4) {
                                v0 = yv[c4][0];
                                v1 = yv[c4][1];
                            }
                        float h0, l0, h1, l1;
                        tc::split_tf32(v0, h0, l0);
                        tc::split_tf32(v1, h1, l1);
                        const int o = tc::kmajor_off(myp * 8 + q4 + 4 * pc, 2 * hp, S::K);
                        *reinterpret_cast<float2 *>(Ax + o) = make_float2(h0, h1);
                        *reinterpret_cast<float2 *>(Ax + S::TILE_FL + o) = make_float2(l0, l1);
                    }
                }
            }
            tc::fence_proxy_async();
            tc::fence_before_sync();
            __syncthreads();
            // ---- G. the contractions of this step, issued by one thread of warp 7 while
            // warps 0-6 go on to translate the next plane; warp 7 first prefetches the
            // colleagues' plane it + 2 into L2
            if (warp == 7 && it + 2 < NH && lane < ncol)
                tc::prefetch_l2(phi + (size_t)s_slot[lane] * BOXFL2 + (size_t)(it + 2) * (N1 * MXP), kPlaneBytes);
            if (warp == 7 && lane == 0) {
                tc::fence_after_sync();
                const uint32_t bH = tc::smem_addr(Bw), bL = bH + 32 * S::K * 4;
                if (it < NH) {
                    const uint32_t aH = tc::smem_addr(Ax), aL = aH + S::TILE_FL * 4;
                    mma3(tmem + grp_col(it), aH, aL, bH, bL);
                    tc::commit(&bx);
                }
                if (it >= 1 && it <= NH) {
                    const uint32_t aH = tc::smem_addr(Ay), aL = aH + S::TILE_FL * 4;
                    mma3(tmem + grp_col(it - 1), aH, aL, bH, bL);
                    tc::commit(&by);
                }
            }
        }
        // ---- the last contraction, over m'_z, in FP32: Lambda[a][b][c] =
        // sum_m' H[c][m'] T2[(class, a, b)][m'], a row per thread and step (the
        // row's values in registers), staged, then stored to global
        for (int row = tid; row < S::NZ; row += kIThreads) {
            int cls = 0;
#pragma unroll
            for (int c = 1; c < 8; ++c)
                if (row >= PR::zbase(c)) cls = c;
            const int pa = cls & 1, pb = (cls >> 1) & 1, pc = cls >> 2;
            const int nb = PR::n(pb), idx = row - PR::zbase(cls), ai = idx / nb, bi = idx % nb;
            float t2[NH];
#pragma unroll
            for (int m = 0; m < NH; ++m) t2[m] = T2[row * NH + m];
            float *out = Ls + ((2 * ai + pa) * P + 2 * bi + pb) * P + pc;
#pragma unroll
            for (int ci = 0; ci < PR::PE; ++ci) {
                if (ci >= PR::n(pc)) break;
                const float *h = Hz + (2 * ci + pc) * NH;
                float acc = 0.f;
#pragma unroll
                for (int m = 0; m < NH; ++m) acc = fmaf(h[m], t2[m], acc);
                out[2 * ci] = acc;
            }
        }
        tc::fence_proxy_async();  // the staged coefficients -> the bulk copy (async proxy)
        __syncthreads();
        if (tid == 0) {
            asm volatile("cp.async.bulk.global.shared::cta.bulk_group [%0], [%1], %2;" ::"l"(lam_in + (size_t)f * S::LSTR),
                         "r"(tc::smem_addr(Ls)), "r"((unsigned)(S::LSTR * 4))
                         : "memory");
            asm volatile("cp.async.bulk.commit_group;" ::: "memory");
            stored = true;
        }
    }
    if (tid == 0 && stored) asm volatile("cp.async.bulk.wait_group 0;" ::: "memory");
    if (!ok) atomicExch(err, 1);
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    if (s_abort && tid == 0) {
        // MMAs that outlived their waits: give them a bounded moment to finish
        // before the TMEM is released
        const long long t0 = clock64();
        while (clock64() - t0 < 20000000ll) {
        }
    }
    __syncthreads();
    if (warp == 0) tc::tmem_dealloc(tmem, kITmem);
}

}  // namespace

template <int P, int NF> int launch_incoming(const IncomingArgs &a, cudaStream_t st, std::string &err) {
    using S = InShape<P, NF>;
    static_assert(S::OK, "shape of the tensor-core incoming pass");
    if (a.nfin <= 0) return 0;
    ::dmk::launch_tick();
    k_fin_colleagues<<<(a.nfin + 127) / 128, 128, 0, st>>>(a.tv, a.nfin, a.fin2box, a.finc, a.fincnt, a.reads);
    cudaError_t e = cudaFuncSetAttribute(k_incoming<P, NF>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)S::BYTES);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_incoming<P, NF>, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
    if (e != cudaSuccess) {
        err = std::string("k_incoming shared memory: ") + cudaGetErrorString(e);
        return DMK_ERR_CUDA;
    }
    const int grid = a.nfin < 2 * a.num_sms ? a.nfin : 2 * a.num_sms;
    const DevTables<float> &tb = *reinterpret_cast<const DevTables<float> *>(a.tables);
    ::dmk::launch_tick();
    k_incoming<P, NF><<<grid, kIThreads, S::BYTES, st>>>(a.tv, tb, a.nfin, a.fin2box, a.finc, a.fincnt,
                                                          (const float2 *)a.phi, a.lam_in, a.err);
    e = cudaGetLastError();
    if (e != cudaSuccess) {
        err = std::string("k_incoming launch: ") + cudaGetErrorString(e);
        return DMK_ERR_CUDA;
    }
    return 0;
}

template int launch_incoming<9, 6>(const IncomingArgs &, cudaStream_t, std::string &);
template int launch_incoming<18, 12>(const IncomingArgs &, cudaStream_t, std::string &);
template int launch_incoming<19, 12>(const IncomingArgs &, cudaStream_t, std::string &);

}  // namespace dmk
