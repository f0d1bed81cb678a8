// near.cu -- the residual near field and the self corrections of the
// discrete DMK algorithm (Steps 4 and 5 of Sec. 3.4 of arXiv 2308.00292), with
// an optional gradient in the target position.
#include "passes.h"
#include "dev_util.h"

#include <algorithm>
#include <type_traits>

namespace dmk {

// ---------------------------------------------------------------------------
// Residual near field (Steps 4 and 5)
// ---------------------------------------------------------------------------
// One warp per target leaf, taken from an atomic work counter.  The leaf's
// points are taken in groups of up to 32 targets; when fewer than 32 targets
// remain, G adjacent lanes share a target and split its candidates.
// For each group:
//   1. the source leaves of the interaction list are read 32 at a time, one
//      per lane, and a leaf whose box lies farther than R_b from the group's
//      bounding box is dropped;
//   2. the sources of the kept leaves form one flat stream, staged in shared
//      memory kNC at a time and moved to the target leaf's frame;
//   3. each lane screens its target against 32 staged sources and marks those
//      closer than R_b; the marked pairs of the warp are compacted into a
//      queue and evaluated 32 at a time, one pair per lane;
//   4. values are summed per target by a segmented warp reduction (a fixed
//      order: the result is deterministic) into per-target accumulators
//      (FP64, or an exact float pair hi + lo in single precision).
// In single precision coordinates are hi + lo pairs relative to the leaf
// centres; the exact dyadic offset between the two leaf centres is added to
// the source with a TwoSum, so differences of nearby points keep their full
// relative precision.
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

constexpr int kNearThreads = 128;
constexpr int kNC = 128;  // staged sources per chunk

// Per-target sums.  The double pass sums in FP64.  The single-precision pass
// keeps a float pair hi + lo made exact by TwoSum: GB300 issues FP64 adds and
// conversions at 1/64 of the FP32 rate, so a double add per run cost more
// than the pairs it sums.  hi + lo carries about 48 bits, as a double sum of
// FP32 runs would.
template <typename T> struct NearAcc { using type = double; };
template <> struct NearAcc<float> { using type = float2; };
__device__ __forceinline__ void acc_zero(double &a) { a = 0.0; }
__device__ __forceinline__ void acc_zero(float2 &a) { a = make_float2(0.f, 0.f); }
__device__ __forceinline__ void acc_add(double &a, double v) { a += v; }
__device__ __forceinline__ void acc_add(float2 &a, float v) {
    const float s = a.x + v, bb = s - a.x;
    a.y += (a.x - (s - bb)) + (v - bb);
    a.x = s;
}
__device__ __forceinline__ double acc_value(double a) { return a; }
__device__ __forceinline__ double acc_value(float2 a) { return (double)a.x + (double)a.y; }

// per-warp shared memory of k_near
template <typename T> struct NearWarp {
    using V4 = typename Vec4<T>::type;
    V4 sh[kNC];        // staged sources: x, y, z in the target leaf's frame (hi) and
                       // |s|^2 - R_b^2 (1 + 2^-9) carrying the leaf level b in its low bits
    float4 sl[kNC];    // single precision: lo parts of x, y, z and the charge
    T sq[kNC];         // double precision: the charge
    V4 th[32];         // the group's targets (hi) and
    float4 tl[32];     // their lo parts
    typename NearAcc<T>::type acc[32];  // per-target sums
    T lox[32], loy[32], loz[32];            // kept source leaves: centre offset,
    int lb_[32];                            // level
    int lss[32], loff[33];                  // first point, offset in the stream
    int fkey[32];                           // per lane: target of its first segment
    T fsum[32];                             // and that segment's sum
    uint16_t q[32 * 32];                    // marked pairs: (target << 7) | staged source
};
// the gradient pass adds the per-target gradient sums
template <typename T> struct NearWarpG : NearWarp<T> {
    typename NearAcc<T>::type gacc[3][32];
};
template <typename T, bool GRAD> using NearWarpT = typename std::conditional<GRAD, NearWarpG<T>, NearWarp<T>>::type;

// the staged threshold |s|^2 - R_b^2 (1 + 2^-9) keeps the level b of the
// source's leaf in its five low mantissa bits (a change of at most 2^-18 of
// its value, well inside the margin); 1 / R_b = 2^b
__device__ __forceinline__ float pack_level(float thr, int b) {
    return __int_as_float((__float_as_int(thr) & ~31) | b);
}
__device__ __forceinline__ double pack_level(double thr, int b) {
    return __longlong_as_double((__double_as_longlong(thr) & ~31ll) | b);
}
__device__ __forceinline__ float inv_radius(float thr) {
    return __int_as_float((127 + (__float_as_int(thr) & 31)) << 23);
}
__device__ __forceinline__ double inv_radius(double thr) {
    return __longlong_as_double((long long)(1023 + (int)(__double_as_longlong(thr) & 31)) << 52);
}
__device__ __forceinline__ int packed_level(float thr) { return __float_as_int(thr) & 31; }
__device__ __forceinline__ int packed_level(double thr) { return (int)(__double_as_longlong(thr) & 31); }
template <typename T> __device__ __forceinline__ T exp_t(T x);
template <> __device__ __forceinline__ float exp_t<float>(float x) { return expf(x); }
template <> __device__ __forceinline__ double exp_t<double>(double x) { return exp(x); }

// screening of 32 staged sources k = u0 + sub + G i against this lane's
// target: bit i set when |t - s|^2 < R_b^2 (1 + 2^-9), with the difference
// formed as (-2 t) . s + (|s|^2 - R_b^2 (1 + 2^-9)) + |t|^2; its cancellation
// error (~1e-6 R_b^2) is far below the 2^-9 margin, so no pair inside the
// support is dropped (the exact test follows in the evaluation)
template <typename T, int G, bool FULL_UNIT>
__device__ __forceinline__ unsigned screen_unit(const typename Vec4<T>::type *sh, int u0, int sub, int fill, T t2x,
                                                T t2y, T t2z, T ntt) {
    unsigned mask = 0;
    const typename Vec4<T>::type *p = sh + u0 + sub;
#pragma unroll 8
    for (int i = 0; i < 32; ++i) {
        if (!FULL_UNIT && u0 + sub + G * i >= fill) break;
        const typename Vec4<T>::type y = p[G * i];
        const T d = fma(t2x, y.x, fma(t2y, y.y, fma(t2z, y.z, y.w)));
        if (d < ntt) mask |= 1u << i;
    }
    return mask;
}

template <typename T, int G>
__device__ __forceinline__ unsigned screen_g(const typename Vec4<T>::type *sh, int u0, int sub, int fill, T t2x,
                                             T t2y, T t2z, T ntt) {
    return u0 + 32 * G <= fill ? screen_unit<T, G, true>(sh, u0, sub, fill, t2x, t2y, t2z, ntt)
                               : screen_unit<T, G, false>(sh, u0, sub, fill, t2x, t2y, t2z, ntt);
}

// YUK: the Yukawa kernel exp(-lam r)/r, whose residual polynomial depends on
// the level (the kernel is not scale invariant): the per-level rows
// [degree, c_0 .. c_qdeg] (stride qdeg + 2) sit in shared memory after the
// warps' areas, and the degrees are run-time values (one instantiation per
// precision)
template <typename T, int QD, bool GRAD, bool YUK>
__global__ void __launch_bounds__(kNearThreads, 6) k_near(TreeView tv, int ntl, const int32_t *tleaves,
                                                       const int32_t *nl_off, const int32_t *nl_src,
                                                       const typename Vec4<T>::type *__restrict__ plocal,
                                                       const float4 *__restrict__ plocal_lo, const T *qmono,
                                                       int qdeg, int nlev, T lam, double *unear, double *gnear,
                                                       int *counter) {
    using V4 = typename Vec4<T>::type;
    constexpr bool kHiLo = sizeof(T) == 4;
    constexpr unsigned FULL = 0xffffffffu;
    extern __shared__ __align__(32) char nsm[];
    NearWarpT<T, GRAD> &W = reinterpret_cast<NearWarpT<T, GRAD> *>(nsm)[threadIdx.x >> 5];
    // residual polynomial coefficients in registers (degree QD known at compile time)
    T qc[QD + 1];
    T *s_q = reinterpret_cast<T *>(nsm + (kNearThreads / 32) * sizeof(NearWarpT<T, GRAD>));
    if constexpr (YUK) {
        for (int i = threadIdx.x; i < nlev * (qdeg + 2); i += kNearThreads) s_q[i] = qmono[i];
        __syncthreads();
    } else {
#pragma unroll
        for (int d = 0; d <= QD; ++d) qc[d] = qmono[d];
    }
    (void)lam;
    const int lane = threadIdx.x & 31;
    const T kBig = (T)1e30;
    // pairs inside the support of the residual kernel (statistics); the
    // counter sits 8 bytes after the work counter
    unsigned inside32 = 0;
    // pairs screened (staged sources times the group's targets), counted at
    // counter + 10 as 64 bits
    unsigned long long screened = 0;
    for (;;) {
        int it = 0;
        if (lane == 0) it = atomicAdd(counter, 1);
        it = __shfl_sync(FULL, it, 0);
        if (it >= ntl) {
            unsigned long long inside = inside32;
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) inside += __shfl_xor_sync(FULL, inside, o);
            if (lane == 0 && inside) atomicAdd(reinterpret_cast<unsigned long long *>(counter + 2), inside);
            if (lane == 0 && screened) atomicAdd(reinterpret_cast<unsigned long long *>(counter + 10), screened);
            break;
        }
        const int Tb = tleaves[it];
        const int a = tv.blevel[Tb];
        int tx, ty, tz;
        box_decode_d(tv.bkey[Tb], a, tx, ty, tz);
        // box centres (2i + 1) 2^-(l+1) are exact in T; so are their differences
        // (at most ~22 significant bits for the level gaps of a balanced tree)
        const T cTx = dyadic_centre<T>(tx, a), cTy = dyadic_centre<T>(ty, a), cTz = dyadic_centre<T>(tz, a);
        const int ts = tv.bstart[Tb], nt = tv.bcount[Tb];
        const int l0 = nl_off[it], l1 = nl_off[it + 1];
        for (int j0 = 0, per = 32; j0 < nt; j0 += per) {
            // lanes per target from the targets still to do: the last group of a
            // leaf shares lanes instead of leaving them idle
            const int rem = nt - j0;
            const int G = rem >= 32 ? 1 : (rem >= 16 ? 2 : (rem >= 8 ? 4 : 8));
            per = 32 / G;
            const int t = lane / G, sub = lane % G;
            const int ng = min(per, rem);
            // the group's targets and their bounding box
            T bl[3] = {kBig, kBig, kBig}, bh[3] = {-kBig, -kBig, -kBig};
            if (lane < ng) {
                const V4 v = plocal[ts + j0 + lane];
                W.th[lane] = v;
                if (kHiLo) W.tl[lane] = plocal_lo[ts + j0 + lane];
                bl[0] = bh[0] = v.x;
                bl[1] = bh[1] = v.y;
                bl[2] = bh[2] = v.z;
            }
            acc_zero(W.acc[lane]);
            if constexpr (GRAD)
                for (int d = 0; d < 3; ++d) acc_zero(W.gacc[d][lane]);
#pragma unroll
            for (int o = 16; o > 0; o >>= 1)
#pragma unroll
                for (int d = 0; d < 3; ++d) {
                    bl[d] = min(bl[d], __shfl_xor_sync(FULL, bl[d], o));
                    bh[d] = max(bh[d], __shfl_xor_sync(FULL, bh[d], o));
                }
            __syncwarp();
            const bool tvalid = t < ng;
            const V4 xt = W.th[tvalid ? t : 0];
            const T t2x = (T)-2 * xt.x, t2y = (T)-2 * xt.y, t2z = (T)-2 * xt.z;
            const T ntt = -(xt.x * xt.x + xt.y * xt.y + xt.z * xt.z);
            for (int lb = l0; lb < l1; lb += 32) {
                // 1. up to 32 source leaves, one per lane; drop those out of reach
                const int li = lb + lane;
                bool keep = false;
                int ns = 0, ss = 0;
                T ox = 0, oy = 0, oz = 0;
                int b = 0;
                if (li < l1) {
                    const int Sb = nl_src[li];
                    b = tv.blevel[Sb];
                    int sx, sy, sz;
                    box_decode_d(tv.bkey[Sb], b, sx, sy, sz);
                    ox = dyadic_centre<T>(sx, b) - cTx;
                    oy = dyadic_centre<T>(sy, b) - cTy;
                    oz = dyadic_centre<T>(sz, b) - cTz;
                    const T Rb = ldexp_t<T>((T)1, -b), hb = (T)0.5 * Rb;
                    ss = tv.bstart[Sb];
                    ns = tv.bcount[Sb];
                    // distance between the leaf's box and the group's bounding box
                    const T gx = max((T)0, max(bl[0] - (ox + hb), (ox - hb) - bh[0]));
                    const T gy = max((T)0, max(bl[1] - (oy + hb), (oy - hb) - bh[1]));
                    const T gz = max((T)0, max(bl[2] - (oz + hb), (oz - hb) - bh[2]));
                    keep = ns > 0 && gx * gx + gy * gy + gz * gz <= Rb * Rb * (T)1.0078125;
                }
                const unsigned kb = __ballot_sync(FULL, keep);
                const int nk = __popc(kb);
                if (nk == 0) continue;
                const int slot = __popc(kb & ((1u << lane) - 1u));
                int cum = keep ? ns : 0;
#pragma unroll
                for (int o = 1; o < 32; o <<= 1) {
                    const int v = __shfl_up_sync(FULL, cum, o);
                    if (lane >= o) cum += v;
                }
                if (keep) {
                    W.lox[slot] = ox;
                    W.loy[slot] = oy;
                    W.loz[slot] = oz;
                    W.lb_[slot] = b;
                    W.lss[slot] = ss;
                    W.loff[slot + 1] = cum;
                }
                if (lane == 0) W.loff[0] = 0;
                const int stream = __shfl_sync(FULL, cum, 31);
                __syncwarp();
                int lf = 0;  // leaf of this lane's next stream position (positions only grow)
                const unsigned lt_mask = (1u << lane) - 1u;
                for (int cur = 0; cur < stream;) {
                    // 2. stage up to kNC sources of the stream in the target leaf's
                    // frame, 32 positions at a time, keeping only sources closer than
                    // R_b (1 + 2^-10) to the group's bounding box: the others cannot
                    // reach any of its targets
                    int fill = 0;
                    while (fill <= kNC - 32 && cur < stream) {
                        const int pos = cur + lane;
                        bool keep = false;
                        V4 hv;
                        float4 lv = make_float4(0.f, 0.f, 0.f, 0.f);
                        T qsrc = 0;
                        if (pos < stream) {
                            while (W.loff[lf + 1] <= pos) ++lf;
                            const int src = W.lss[lf] + pos - W.loff[lf];
                            const V4 y = plocal[src];
                            const T ax = W.lox[lf], ay = W.loy[lf], az = W.loz[lf];
                            const int lev = W.lb_[lf];
                            hv.x = y.x + ax;
                            hv.y = y.y + ay;
                            hv.z = y.z + az;
                            const T Rb2 = ldexp_t<T>((T)1.001953125, -2 * lev);  // R_b^2 (1 + 2^-9)
                            const T gx = max((T)0, max(bl[0] - hv.x, hv.x - bh[0]));
                            const T gy = max((T)0, max(bl[1] - hv.y, hv.y - bh[1]));
                            const T gz = max((T)0, max(bl[2] - hv.z, hv.z - bh[2]));
                            keep = gx * gx + gy * gy + gz * gz < Rb2;
                            hv.w = pack_level(hv.x * hv.x + hv.y * hv.y + hv.z * hv.z - Rb2, lev);
                            if (kHiLo) {  // TwoSum error terms plus the lo parts
                                const float4 yl = plocal_lo[src];
                                T bb = hv.x - y.x;
                                lv.x = (float)(((y.x - (hv.x - bb)) + (ax - bb)) + (T)yl.x);
                                bb = hv.y - y.y;
                                lv.y = (float)(((y.y - (hv.y - bb)) + (ay - bb)) + (T)yl.y);
                                bb = hv.z - y.z;
                                lv.z = (float)(((y.z - (hv.z - bb)) + (az - bb)) + (T)yl.z);
                                lv.w = (float)y.w;
                            } else {
                                qsrc = y.w;
                            }
                        }
                        const unsigned km = __ballot_sync(FULL, keep);
                        if (keep) {
                            const int k = fill + __popc(km & lt_mask);
                            W.sh[k] = hv;
                            if (kHiLo) W.sl[k] = lv;
                            else W.sq[k] = qsrc;
                        }
                        fill += __popc(km);
                        cur += 32;
                    }
                    __syncwarp();
                    if (fill == 0) continue;
                    screened += (unsigned long long)fill * (unsigned)ng;
                    // 3. screening, 32 candidates per lane: k = u0 + sub + G i
                    for (int u0 = 0; u0 < fill; u0 += 32 * G) {
                        unsigned mask = 0;
                        if (tvalid) {
                            switch (G) {
                            case 1: mask = screen_g<T, 1>(W.sh, u0, sub, fill, t2x, t2y, t2z, ntt); break;
                            case 2: mask = screen_g<T, 2>(W.sh, u0, sub, fill, t2x, t2y, t2z, ntt); break;
                            case 4: mask = screen_g<T, 4>(W.sh, u0, sub, fill, t2x, t2y, t2z, ntt); break;
                            default: mask = screen_g<T, 8>(W.sh, u0, sub, fill, t2x, t2y, t2z, ntt); break;
                            }
                        }
                        // compaction: the warp's marked pairs, in lane order (targets ascending)
                        const int cnt = __popc(mask);
                        int pre = cnt;
#pragma unroll
                        for (int o = 1; o < 32; o <<= 1) {
                            const int v = __shfl_up_sync(FULL, pre, o);
                            if (lane >= o) pre += v;
                        }
                        const int total = __shfl_sync(FULL, pre, 31);
                        int o = pre - cnt;
                        while (mask) {
                            const int i = __ffs(mask) - 1;
                            mask &= mask - 1;
                            W.q[o++] = (uint16_t)((t << 7) | (u0 + sub + G * i));
                        }
                        __syncwarp();
                        if (total == 0) continue;
                        // the residual kernel: lane L takes the marked pairs [L n, (L + 1) n)
                        // in order, so it meets each target in one run; a run that starts
                        // inside the lane's block belongs to this lane alone and goes to
                        // the target's sum directly, the run at the block start may be
                        // shared with earlier lanes and is combined below in lane order
                        const int nper = (total + 31) >> 5;
                        const int e0 = min(lane * nper, total), e1 = min(e0 + nper, total);
                        int cur = -1, first = -1;
                        T part = 0, fpart = 0;
                        T pg[3] = {0, 0, 0}, fpg[3] = {0, 0, 0};  // gradient runs
                        V4 x = W.th[0];
                        float4 xl = make_float4(0.f, 0.f, 0.f, 0.f);
                        for (int e = e0; e < e1; ++e) {
                            const int ent = W.q[e], tt = ent >> 7, k = ent & 127;
                            if (tt != cur) {  // a new run: flush the previous one, load the target
                                if (cur >= 0) {
                                    if (first < 0) {
                                        first = cur;
                                        fpart = part;
                                        if constexpr (GRAD) fpg[0] = pg[0], fpg[1] = pg[1], fpg[2] = pg[2];
                                    } else {
                                        acc_add(W.acc[cur], part);
                                        if constexpr (GRAD)
                                            for (int d = 0; d < 3; ++d) acc_add(W.gacc[d][cur], pg[d]);
                                    }
                                }
                                cur = tt;
                                part = 0;
                                pg[0] = pg[1] = pg[2] = 0;
                                x = W.th[tt];
                                if (kHiLo) xl = W.tl[tt];
                            }
                            const V4 y = W.sh[k];
                            T dx = x.x - y.x, dy = x.y - y.y, dz = x.z - y.z;
                            T qj;
                            if (kHiLo) {
                                const float4 yl = W.sl[k];
                                dx += (T)xl.x - (T)yl.x;
                                dy += (T)xl.y - (T)yl.y;
                                dz += (T)xl.z - (T)yl.z;
                                qj = (T)yl.w;
                            } else {
                                qj = W.sq[k];
                            }
                            const T iR = inv_radius(y.w), iR2 = iR * iR;
                            const T r2 = dx * dx + dy * dy + dz * dz;
                            const T xx = (T)2 * r2 * iR2 - (T)1;  // r < R_b  <=>  xx < 1
                            T qv, dq = 0;
                            if constexpr (YUK) {
                                const T *qr = s_q + packed_level(y.w) * (qdeg + 2);
                                const int dg = (int)qr[0];
                                qv = qr[1 + dg];
                                for (int d = dg - 1; d >= 0; --d) qv = qv * xx + qr[1 + d];
                            } else {
                                qv = qc[QD];
#pragma unroll
                                for (int d = QD - 1; d >= 0; --d) {
                                    if constexpr (GRAD) dq = dq * xx + qv;
                                    qv = qv * xx + qc[d];
                                }
                            }
                            const T rinv = r2 > (T)0 ? rsqrt_t<T>(r2) : (T)0;
                            const bool in = xx < (T)1;
                            T kern = rinv;
                            if constexpr (YUK) kern = exp_t<T>(-lam * r2 * rinv) * rinv;
                            const T val = in ? qj * (kern - qv * iR) : (T)0;
                            inside32 += in ? 1u : 0u;
                            part += val;
                            if constexpr (GRAD) {
                                // grad_x R(|x - y|) = -(x - y) (1/r^3 + 4 q'(xx) / R^3), xx = 2 r^2/R^2 - 1
                                const T gf = in ? -qj * (rinv * rinv * rinv + (T)4 * dq * iR * iR2) : (T)0;
                                pg[0] += gf * dx;
                                pg[1] += gf * dy;
                                pg[2] += gf * dz;
                            }
                        }
                        if (cur >= 0) {
                            if (first < 0) {
                                first = cur;
                                fpart = part;
                                if constexpr (GRAD) fpg[0] = pg[0], fpg[1] = pg[1], fpg[2] = pg[2];
                            } else {
                                acc_add(W.acc[cur], part);
                                if constexpr (GRAD)
                                    for (int d = 0; d < 3; ++d) acc_add(W.gacc[d][cur], pg[d]);
                            }
                        }
                        // first runs: a segmented sum over lanes with the same target
                        // (lanes without pairs carry no key)
                        int key = first >= 0 ? first : -1 - lane;
                        T v = fpart;
#pragma unroll
                        for (int d = 1; d < 32; d <<= 1) {
                            const T vu = __shfl_up_sync(FULL, v, d);
                            const int ku = __shfl_up_sync(FULL, key, d);
                            if constexpr (GRAD) {
#pragma unroll
                                for (int c = 0; c < 3; ++c) {
                                    const T gu = __shfl_up_sync(FULL, fpg[c], d);
                                    if (lane >= d && ku == key) fpg[c] += gu;
                                }
                            }
                            if (lane >= d && ku == key) v += vu;
                        }
                        const int kn = __shfl_down_sync(FULL, key, 1);
                        __syncwarp();
                        if (first >= 0 && (lane == 31 || kn != key)) {
                            acc_add(W.acc[key], v);
                            if constexpr (GRAD)
                                for (int d = 0; d < 3; ++d) acc_add(W.gacc[d][key], fpg[d]);
                        }
                        __syncwarp();
                    }
                    __syncwarp();
                }
            }
            if (lane < ng && (tv.pflag[ts + j0 + lane] & 2)) {
                unear[ts + j0 + lane] = acc_value(W.acc[lane]);
                if constexpr (GRAD)
                    for (int d = 0; d < 3; ++d)
                        gnear[3 * (size_t)(ts + j0 + lane) + d] = acc_value(W.gacc[d][lane]);
            }
            __syncwarp();
        }
    }
}

// launch k_near with the residual polynomial degree as a template argument;
// returns 1 for a degree outside 2..30, 2 for a failed launch, 3 for an
// unsupported combination (the Yukawa kernel with gradients)
template <typename T, int QD, bool GRAD, bool YUK>
static cudaError_t launch_near_qd(int grid, cudaStream_t st, const NearArgs &a) {
    const size_t smem = (size_t)(kNearThreads / 32) * sizeof(NearWarpT<T, GRAD>) +
                        (YUK ? (size_t)a.nlev * (a.qdeg + 2) * sizeof(T) : 0);
    cudaError_t e =
        cudaFuncSetAttribute(k_near<T, QD, GRAD, YUK>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    k_near<T, QD, GRAD, YUK><<<grid, kNearThreads, smem, st>>>(
        a.tv, a.ntl, a.tleaves, a.nl_off, a.nl_src, (const typename Vec4<T>::type *)a.plocal, a.plocal_lo,
        (const T *)a.qmono, a.qdeg, a.nlev, (T)a.lam, a.unear, a.gnear, a.counter);
    return cudaGetLastError();
}

template <typename T, bool GRAD>
static int launch_near_t(int grid, cudaStream_t st, const NearArgs &a) {
    switch (a.qdeg) {
#define DMK_NEAR_CASE(d) \
    case d: \
        return launch_near_qd<T, d, GRAD, false>(grid, st, a) == cudaSuccess ? 0 : 2;
        DMK_NEAR_CASE(2) DMK_NEAR_CASE(3) DMK_NEAR_CASE(4) DMK_NEAR_CASE(5) DMK_NEAR_CASE(6) DMK_NEAR_CASE(7)
        DMK_NEAR_CASE(8) DMK_NEAR_CASE(9) DMK_NEAR_CASE(10) DMK_NEAR_CASE(11) DMK_NEAR_CASE(12) DMK_NEAR_CASE(13)
        DMK_NEAR_CASE(14) DMK_NEAR_CASE(15) DMK_NEAR_CASE(16) DMK_NEAR_CASE(17) DMK_NEAR_CASE(18) DMK_NEAR_CASE(19)
        DMK_NEAR_CASE(20) DMK_NEAR_CASE(21) DMK_NEAR_CASE(22) DMK_NEAR_CASE(23) DMK_NEAR_CASE(24) DMK_NEAR_CASE(25)
        DMK_NEAR_CASE(26) DMK_NEAR_CASE(27) DMK_NEAR_CASE(28) DMK_NEAR_CASE(29) DMK_NEAR_CASE(30)
#undef DMK_NEAR_CASE
    default: return 1;
    }
}

int launch_near(bool single, const NearArgs &a, int num_sms, cudaStream_t st) {
    // one warp per target leaf and no persistent blocks: short blocks let the
    // concurrent far-field kernels take SMs as they free up
    const int wpb = kNearThreads / 32;
    const int grid = (a.ntl + wpb - 1) / wpb;
    (void)num_sms;
    if (grid <= 0) return 0;
    ::dmk::launch_tick();
    const bool grad = a.gnear != nullptr;
    if (a.yukawa) {
        if (grad || a.nlev < 1 || a.nlev > kMaxLevel + 1) return 3;
        if (a.qdeg < 2 || a.qdeg > kMaxYukawaDegree) return 1;
        const cudaError_t e = single ? launch_near_qd<float, 2, false, true>(grid, st, a)
                                     : launch_near_qd<double, 2, false, true>(grid, st, a);
        return e == cudaSuccess ? 0 : 2;
    }
    if (single) return grad ? launch_near_t<float, true>(grid, st, a) : launch_near_t<float, false>(grid, st, a);
    return grad ? launch_near_t<double, true>(grid, st, a) : launch_near_t<double, false>(grid, st, a);
}

}  // namespace dmk
