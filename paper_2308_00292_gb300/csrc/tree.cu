// tree.cu -- device construction of the level-restricted adaptive oct-tree
// (Sec. 3.2 and Step 0 of Sec. 3.4 of arXiv 2308.00292).
//
// Pipeline (all on the device; the host only reads per-level box counts):
//   1. bounding box of all points -> unit-box map u = (x - lo) / S
//   2. 63-bit Morton keys of the finest (level-21) cells, stable radix sort
//   3. level-synchronous top-down build: a box is split when it holds more than
//      n_s points that do not all share one finest cell, or when the level
//      restriction forced it; children are emitted in Morton order, so every
//      level is a sorted array of cells and lookups are binary searches
//   4. level restriction: a leaf at level a that shares a boundary point with
//      a non-leaf box at level a+1 is forced to split; the tree is rebuilt
//      until no leaf is forced (the smallest balanced refinement)
//   5. colleagues (same-level boxes sharing a boundary point, Sec. 3.2),
//      flags F_leaf / F_out / F_in (Step 0), expansion slots, and the
//      residual-kernel interaction list of every target leaf (Step 4).
//
// A batch of independent systems is built as one forest: every system is
// mapped to its own unit box, and the system index s prefixes every key.  A
// point key is (s << 3 kb) | Morton(kb-bit cells); a box key at level l is
// (s << 3 l) | Morton(level-l cell), so the children's keys (key << 3 | octant)
// keep the prefix, every level stays sorted by (system, cell), and lookups
// never cross systems.  The roots (level 0) are the systems, in order.  With
// one system s = 0, kb = 21 and the keys are plain Morton codes.
#include "tree.h"

#include <algorithm>
#include <cfloat>
#include <cstdio>
#include <cstdlib>

namespace dmk {

// ------------------------------------------------------------------ morton
__host__ __device__ __forceinline__ uint64_t spread3(uint64_t x) {
    x &= 0x1fffffull;
    x = (x | (x << 32)) & 0x1f00000000ffffull;
    x = (x | (x << 16)) & 0x1f0000ff0000ffull;
    x = (x | (x << 8)) & 0x100f00f00f00f00full;
    x = (x | (x << 4)) & 0x10c30c30c30c30c3ull;
    x = (x | (x << 2)) & 0x1249249249249249ull;
    return x;
}
__host__ __device__ __forceinline__ uint32_t compact3(uint64_t x) {
    x &= 0x1249249249249249ull;
    x = (x ^ (x >> 2)) & 0x10c30c30c30c30c3ull;
    x = (x ^ (x >> 4)) & 0x100f00f00f00f00full;
    x = (x ^ (x >> 8)) & 0x1f0000ff0000ffull;
    x = (x ^ (x >> 16)) & 0x1f00000000ffffull;
    x = (x ^ (x >> 32)) & 0x1fffffull;
    return (uint32_t)x;
}
__host__ __device__ __forceinline__ uint64_t morton_encode(uint32_t ix, uint32_t iy, uint32_t iz) {
    return spread3(ix) | (spread3(iy) << 1) | (spread3(iz) << 2);
}
__host__ __device__ __forceinline__ void morton_decode(uint64_t m, int &ix, int &iy, int &iz) {
    ix = (int)compact3(m);
    iy = (int)compact3(m >> 1);
    iz = (int)compact3(m >> 2);
}

uint64_t host_morton_encode(uint32_t ix, uint32_t iy, uint32_t iz) { return morton_encode(ix, iy, iz); }

// key of (level, cell) unique over levels: Morton code with a leading one bit
__device__ __forceinline__ uint64_t cell_key(int level, uint64_t m) { return m | (1ull << (3 * level)); }

// the Morton cell and the system of a box key at level l
__device__ __forceinline__ uint64_t key_cell(uint64_t key, int l) { return key & ((1ull << (3 * l)) - 1ull); }
__device__ __forceinline__ uint64_t key_sys(uint64_t key, int l) { return key >> (3 * l); }

// entry of the forced-split set: the cell key of (level, cell) below bit
// 3 kb, the system above it
__device__ __forceinline__ uint64_t forced_key(int level, uint64_t m, uint64_t sys, int kb) {
    return cell_key(level, m) | (sys << (3 * kb));
}

// ------------------------------------------------------------------ hash set
__device__ __forceinline__ uint32_t hash64(uint64_t k) {
    k ^= k >> 33;
    k *= 0xff51afd7ed558ccdull;
    k ^= k >> 33;
    k *= 0xc4ceb9fe1a85ec53ull;
    k ^= k >> 33;
    return (uint32_t)k;
}
__device__ bool hset_insert(uint64_t *tab, uint32_t cap, uint64_t key, int *overflow) {
    uint32_t h = hash64(key) & (cap - 1);
    for (uint32_t probe = 0; probe < cap; ++probe) {
        unsigned long long prev = atomicCAS((unsigned long long *)&tab[h], 0ull, (unsigned long long)key);
        if (prev == 0ull) return true;
        if (prev == key) return false;
        h = (h + 1) & (cap - 1);
    }
    atomicExch(overflow, 1);
    return false;
}
__device__ bool hset_contains(const uint64_t *tab, uint32_t cap, uint64_t key) {
    uint32_t h = hash64(key) & (cap - 1);
    for (uint32_t probe = 0; probe < cap; ++probe) {
        uint64_t v = tab[h];
        if (v == key) return true;
        if (v == 0ull) return false;
        h = (h + 1) & (cap - 1);
    }
    return false;
}

// ------------------------------------------------------------------ 1. bbox
__global__ void k_bbox_partial(const double *src, int64_t ns, const double *tgt, int64_t nt, double *part,
                               int *bad) {
    double mn[3] = {INFINITY, INFINITY, INFINITY}, mx[3] = {-INFINITY, -INFINITY, -INFINITY};
    int64_t n = ns + nt;
    int nonfinite = 0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const double *x = i < ns ? src + 3 * i : tgt + 3 * (i - ns);
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            double v = x[d];
            if (!isfinite(v)) nonfinite = 1;
            mn[d] = fmin(mn[d], v);
            mx[d] = fmax(mx[d], v);
        }
    }
    if (nonfinite) atomicExch(bad, 1);
    __shared__ double s[6][256];
    for (int d = 0; d < 3; ++d) {
        s[d][threadIdx.x] = mn[d];
        s[3 + d][threadIdx.x] = mx[d];
    }
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if ((int)threadIdx.x < o)
            for (int d = 0; d < 3; ++d) {
                s[d][threadIdx.x] = fmin(s[d][threadIdx.x], s[d][threadIdx.x + o]);
                s[3 + d][threadIdx.x] = fmax(s[3 + d][threadIdx.x], s[3 + d][threadIdx.x + o]);
            }
        __syncthreads();
    }
    if (threadIdx.x == 0)
        for (int d = 0; d < 6; ++d) part[blockIdx.x * 6 + d] = s[d][0];
}

__global__ void k_bbox_final(const double *part, int nblk, Frame *frame) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    double mn[3] = {INFINITY, INFINITY, INFINITY}, mx[3] = {-INFINITY, -INFINITY, -INFINITY};
    for (int b = 0; b < nblk; ++b)
        for (int d = 0; d < 3; ++d) {
            mn[d] = fmin(mn[d], part[b * 6 + d]);
            mx[d] = fmax(mx[d], part[b * 6 + 3 + d]);
        }
    double S = 0.0;
    for (int d = 0; d < 3; ++d) S = fmax(S, mx[d] - mn[d]);
    if (!(S > 0.0)) S = 1.0;
    for (int d = 0; d < 3; ++d) frame->lo[d] = mn[d];
    frame->S = S;
    frame->rS = 1.0 / S;
}

// one block per system of a batch: the bounding box of its points -> frame[s]
__global__ void k_bbox_sys(const double *src, const int64_t *off, Frame *frame, int *bad) {
    const int sy = blockIdx.x;
    const int64_t a = off[sy], b = off[sy + 1];
    double mn[3] = {INFINITY, INFINITY, INFINITY}, mx[3] = {-INFINITY, -INFINITY, -INFINITY};
    int nonfinite = 0;
    for (int64_t i = a + threadIdx.x; i < b; i += blockDim.x) {
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            const double v = src[3 * i + d];
            if (!isfinite(v)) nonfinite = 1;
            mn[d] = fmin(mn[d], v);
            mx[d] = fmax(mx[d], v);
        }
    }
    if (nonfinite) atomicExch(bad, 1);
    __shared__ double s[6][256];
    for (int d = 0; d < 3; ++d) {
        s[d][threadIdx.x] = mn[d];
        s[3 + d][threadIdx.x] = mx[d];
    }
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if ((int)threadIdx.x < o)
            for (int d = 0; d < 3; ++d) {
                s[d][threadIdx.x] = fmin(s[d][threadIdx.x], s[d][threadIdx.x + o]);
                s[3 + d][threadIdx.x] = fmax(s[3 + d][threadIdx.x], s[3 + d][threadIdx.x + o]);
            }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        double S = 0.0;
        for (int d = 0; d < 3; ++d) S = fmax(S, s[3 + d][0] - s[d][0]);
        if (!(S > 0.0)) S = 1.0;
        for (int d = 0; d < 3; ++d) frame[sy].lo[d] = b > a ? s[d][0] : 0.0;
        frame[sy].S = S;
        frame[sy].rS = 1.0 / S;
    }
}

// ------------------------------------------------------------------ 2. keys
// (x - lo) / S correctly rounded, as one IEEE subtraction and one IEEE
// division would give, without the division: with rS = RN(1 / S), the product
// a rS is within two ulps of a / S; a Newton step on the exact remainder
// a - q S (one FMA) brings it within one ulp, and a second step then yields
// the correctly rounded quotient (Markstein, IBM J. Res. Dev. 34(1), 1990:
// q + (a - q S) RN(1/S), rounded once, is RN(a / S) when q is within an ulp).
// GB300 runs FP64 at 1/62 of its FP32 rate, and the division was most of the
// key kernel's time.
__device__ __forceinline__ double unit_coord(double x, double lo, double S, double rS) {
    const double a = __dsub_rn(x, lo);
    if (!(rS >= DBL_MIN && rS <= DBL_MAX)) return __ddiv_rn(a, S);  // 1 / S subnormal or infinite
    double q = __dmul_rn(a, rS);
    q = __fma_rn(__fma_rn(-q, S, a), rS, q);
    return __fma_rn(__fma_rn(-q, S, a), rS, q);
}
// cell of u in [0, 1] at kb bits (exact scaling by 2^kb)
__device__ __forceinline__ uint32_t fine_cell(double u, int kb) {
    const double top = (double)(1u << kb);
    double f = floor(u * top);
    if (f > top - 1.0) f = top - 1.0;
    if (f < 0.0) f = 0.0;
    return (uint32_t)f;
}

// system of input point i (off: nsys + 1 ascending offsets; NULL = one system)
__device__ __forceinline__ int point_sys(const int64_t *off, int nsys, int64_t i) {
    if (!off) return 0;
    int lo = 0, hi = nsys - 1;  // last s with off[s] <= i
    while (lo < hi) {
        const int m = (lo + hi + 1) >> 1;
        if (off[m] <= i) lo = m; else hi = m - 1;
    }
    return lo;
}

// unit-box coordinates of every point (kept in input order for the gather:
// the map costs three FP64 divisions, done once) and its key
__global__ void k_make_keys(const double *src, int64_t ns, const double *tgt, int64_t n, const Frame *frame,
                            const int64_t *off, int nsys, int kb, uint64_t *keys, uint32_t *idx, double *u) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const double *x = i < ns ? src + 3 * i : tgt + 3 * (i - ns);
    const int sy = point_sys(off, nsys, i);
    const Frame f = frame[sy];
    const double u0 = unit_coord(x[0], f.lo[0], f.S, f.rS), u1 = unit_coord(x[1], f.lo[1], f.S, f.rS),
                 u2 = unit_coord(x[2], f.lo[2], f.S, f.rS);
    u[3 * i] = u0;
    u[3 * i + 1] = u1;
    u[3 * i + 2] = u2;
    uint32_t c0 = fine_cell(u0, kb);
    uint32_t c1 = fine_cell(u1, kb);
    uint32_t c2 = fine_cell(u2, kb);
    keys[i] = morton_encode(c0, c1, c2) | ((uint64_t)sy << (3 * kb));
    idx[i] = (uint32_t)i;
}

__global__ void k_gather_points(const double *u, const double *charges, int64_t ns, int64_t n, int same,
                                const uint64_t *skeys, int kb, const uint32_t *idx, double *ux, double *uy,
                                double *uz, double *q, uint8_t *pflag, int32_t *pout, int32_t *psys) {
    int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    int64_t i = idx[k];
    if (psys) psys[k] = (int)(skeys[k] >> (3 * kb));
    ux[k] = u[3 * i];
    uy[k] = u[3 * i + 1];
    uz[k] = u[3 * i + 2];
    if (same) {
        q[k] = charges[i];
        pflag[k] = 3;
        pout[k] = (int32_t)i;
    } else if (i < ns) {
        q[k] = charges[i];
        pflag[k] = 1;
        pout[k] = -1;
    } else {
        q[k] = 0.0;
        pflag[k] = 2;
        pout[k] = (int32_t)(i - ns);
    }
}

// ------------------------------------------------------------------ 3. levels
struct LevelArgs {
    const uint64_t *keys;  // sorted point keys
    uint64_t *bkey;
    int8_t *blevel;
    int32_t *bstart, *bcount, *bparent, *bchild0;
    uint8_t *bcmask;
    int32_t *off9, *cnt, *excl;
    const uint64_t *forced;
    uint32_t fcap;
    int kb;  // bits per axis of the point keys
};

// the roots of a batch: box s is system s (points off[s] .. off[s + 1])
__global__ void k_roots(int nsys, const int64_t *off, uint64_t *bkey, int8_t *blevel, int32_t *bstart,
                        int32_t *bcount, int32_t *bparent) {
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= nsys) return;
    bkey[s] = (uint64_t)s;
    blevel[s] = 0;
    bstart[s] = (int32_t)off[s];
    bcount[s] = (int32_t)(off[s + 1] - off[s]);
    bparent[s] = -1;
}

// eight threads per box: thread j > 0 finds by binary search the first point
// of octant j in the box's sorted range, so the searches run side by side
__global__ void k_level_split(LevelArgs a, int level, int lstart, int lcount, int leaf_cap, int max_level) {
    const int64_t gi = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int i = (int)(gi >> 3), j = (int)(gi & 7);
    const bool valid = i < lcount;
    int32_t s = 0, e = 0;
    bool split = false;
    if (valid) {
        const int b = lstart + i;
        s = a.bstart[b];
        e = s + a.bcount[b];
        if (level < max_level) {
            const uint64_t k = a.bkey[b];
            if (e - s > leaf_cap && a.keys[s] != a.keys[e - 1]) split = true;
            else if (hset_contains(a.forced, a.fcap, forced_key(level, key_cell(k, level), key_sys(k, level), a.kb)))
                split = true;
        }
    }
    int32_t l = s;  // first index with octant >= j (j = 0: the box's start)
    if (split && j > 0) {
        const int shift = 3 * (a.kb - 1 - level);
        int32_t h = e;
        while (l < h) {
            const int32_t m = (l + h) >> 1;
            if ((int)((a.keys[m] >> shift) & 7ull) < j) l = m + 1; else h = m;
        }
    }
    // octant j is non-empty when the next boundary lies beyond this one
    int32_t next = __shfl_down_sync(0xffffffffu, l, 1, 8);
    if (j == 7) next = e;
    const unsigned ne = __ballot_sync(0xffffffffu, split && next > l);
    if (!valid) return;
    int32_t *off = a.off9 + (int64_t)i * 9;
    if (split) {
        off[j] = l;
        if (j == 7) off[8] = e;
    }
    if (j == 0) a.cnt[i] = __popc((ne >> (threadIdx.x & 24)) & 0xffu);
}

__global__ void k_level_emit(LevelArgs a, int level, int lstart, int lcount, int next_start) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= lcount) return;
    int b = lstart + i;
    if (a.cnt[i] == 0) {
        a.bchild0[b] = -1;
        a.bcmask[b] = 0;
        return;
    }
    const int32_t *off = a.off9 + (int64_t)i * 9;
    int base = next_start + a.excl[i];
    a.bchild0[b] = base;
    uint8_t mask = 0;
    int k = 0;
    uint64_t pk = a.bkey[b] << 3;
    for (int oc = 0; oc < 8; ++oc) {
        if (off[oc + 1] <= off[oc]) continue;
        int nb = base + k++;
        a.bkey[nb] = pk | (uint64_t)oc;
        a.blevel[nb] = (int8_t)(level + 1);
        a.bstart[nb] = off[oc];
        a.bcount[nb] = off[oc + 1] - off[oc];
        a.bparent[nb] = b;
        mask |= (uint8_t)(1u << oc);
    }
    a.bcmask[b] = mask;
}

__device__ __forceinline__ int find_box(const uint64_t *bkey, int lstart, int lcount, uint64_t key) {
    int l = lstart, h = lstart + lcount - 1;
    while (l <= h) {
        int m = (l + h) >> 1;
        uint64_t v = bkey[m];
        if (v == key) return m;
        if (v < key) l = m + 1; else h = m - 1;
    }
    return -1;
}

struct LevelTable {
    int start[kMaxLevel + 2];
    int count[kMaxLevel + 2];
    int nlev;
};

// ------------------------------------------------------------------ 4. balance
__global__ void k_balance(const uint64_t *bkey, const int8_t *blevel, const uint8_t *bcmask, int nb, LevelTable lt,
                          uint64_t *forced, uint32_t fcap, int kb, int *changed, int *overflow) {
    int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= nb) return;
    if (bcmask[b] != 0) return;  // not a leaf
    int l = blevel[b];
    if (l + 1 >= lt.nlev) return;
    int ix, iy, iz;
    const uint64_t cell = key_cell(bkey[b], l), sy = key_sys(bkey[b], l);
    morton_decode(cell, ix, iy, iz);
    const uint64_t pre1 = sy << (3 * (l + 1));
    int lim = 1 << (l + 1);
    int ns = lt.start[l + 1], nc = lt.count[l + 1];
    for (int jx = 2 * ix - 1; jx <= 2 * ix + 2; ++jx) {
        if (jx < 0 || jx >= lim) continue;
        for (int jy = 2 * iy - 1; jy <= 2 * iy + 2; ++jy) {
            if (jy < 0 || jy >= lim) continue;
            for (int jz = 2 * iz - 1; jz <= 2 * iz + 2; ++jz) {
                if (jz < 0 || jz >= lim) continue;
                bool inside = (jx >> 1) == ix && (jy >> 1) == iy && (jz >> 1) == iz;
                if (inside) continue;
                int c = find_box(bkey, ns, nc, pre1 | morton_encode(jx, jy, jz));
                if (c >= 0 && bcmask[c] != 0) {
                    hset_insert(forced, fcap, forced_key(l, cell, sy, kb), overflow);
                    atomicExch(changed, 1);
                    return;
                }
            }
        }
    }
}

// The level restriction completed on cell sets, without rebuilding the tree:
// S = the forced set = every box that splits (the first tree's non-leaf boxes,
// then the forced ones).  A cell n at level l is a box if its parent is in S
// and it holds points; a box n that is not in S but shares a boundary point
// with a member of S one level finer must split.  Every round pushes from all
// of S (new boxes may neighbour old members); the forced set grows
// monotonically to the same least fixpoint as check-and-rebuild rounds.
__global__ void k_collect_nonleaf(const uint64_t *bkey, const int8_t *blevel, const uint8_t *bcmask, int nb,
                                  uint64_t *forced, uint32_t fcap, int kb, uint64_t *slist, int *count, int lcap,
                                  int *overflow) {
    int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= nb || bcmask[b] == 0) return;
    const int l = blevel[b];
    const uint64_t key = forced_key(l, key_cell(bkey[b], l), key_sys(bkey[b], l), kb);
    if (hset_insert(forced, fcap, key, overflow)) {
        const int k = atomicAdd(count, 1);
        if (k < lcap) slist[k] = key; else atomicExch(overflow, 1);
    }
}

// whether cell m at level l of system sy holds points (sorted point keys with
// kb bits per axis; sy < 2^(63 - 3 kb))
__device__ __forceinline__ bool cell_nonempty(const uint64_t *keys, int64_t n, int kb, int l, uint64_t sy,
                                              uint64_t m) {
    const int shift = 3 * (kb - l);
    const uint64_t pre = (sy << (3 * l)) | m;  // the cell's key prefix
    const uint64_t lo = pre << shift;
    int64_t a = 0, b = n;
    while (a < b) {
        const int64_t mid = (a + b) >> 1;
        if (keys[mid] < lo) a = mid + 1; else b = mid;
    }
    return a < n && (keys[a] >> shift) == pre;
}

__global__ void k_push_balance(const uint64_t *keys, int64_t n, int max_level, int kb, uint64_t *forced,
                               uint32_t fcap, uint64_t *slist, int ns, int *count, int lcap, int *changed,
                               int *overflow) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= ns) return;
    const uint64_t sk = slist[i];
    const uint64_t sys = sk >> (3 * kb), ck = sk & ((1ull << (3 * kb)) - 1ull);
    const int ls = (63 - __clzll((long long)ck)) / 3;
    if (ls < 1 || ls >= max_level) return;  // a cell at the deepest level never splits
    int sx, sy, sz;
    morton_decode(ck ^ (1ull << (3 * ls)), sx, sy, sz);
    const int l = ls - 1, lim = 1 << l;
    const int px = sx >> 1, py = sy >> 1, pz = sz >> 1;
    // level-l cells sharing a boundary point with s: 2 i - 1 <= s <= 2 i + 2 per axis
    for (int ix = (sx - 1) >> 1; ix <= (sx + 1) >> 1; ++ix) {
        if (ix < 0 || ix >= lim) continue;
        for (int iy = (sy - 1) >> 1; iy <= (sy + 1) >> 1; ++iy) {
            if (iy < 0 || iy >= lim) continue;
            for (int iz = (sz - 1) >> 1; iz <= (sz + 1) >> 1; ++iz) {
                if (iz < 0 || iz >= lim) continue;
                if (ix == px && iy == py && iz == pz) continue;
                const uint64_t m = morton_encode(ix, iy, iz);
                const uint64_t key = forced_key(l, m, sys, kb);
                if (hset_contains(forced, fcap, key)) continue;
                if (l > 0 && !hset_contains(forced, fcap, forced_key(l - 1, m >> 3, sys, kb))) continue;
                if (!cell_nonempty(keys, n, kb, l, sys, m)) continue;
                if (hset_insert(forced, fcap, key, overflow)) {
                    const int k = atomicAdd(count, 1);
                    if (k < lcap) slist[k] = key; else atomicExch(overflow, 1);
                    atomicExch(changed, 1);
                }
            }
        }
    }
}

// ------------------------------------------------------------------ 5. finish
__global__ void k_box_finish(int nb, const uint64_t *bkey, const int8_t *blevel, const int32_t *bstart,
                             const int32_t *bcount, const uint8_t *bcmask, const int32_t *psrc, const int32_t *ptgt,
                             LevelTable lt, int32_t *bnsrc, int32_t *bntgt, int32_t *bcol, uint8_t *bflags,
                             int32_t *isleaf_i32, int32_t *isnonleaf_i32, int *nleaf) {
    int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= nb) return;
    int32_t s = bstart[b], e = s + bcount[b];
    bnsrc[b] = psrc ? psrc[e] - psrc[s] : e - s;
    bntgt[b] = ptgt ? ptgt[e] - ptgt[s] : e - s;
    int l = blevel[b];
    int ix, iy, iz;
    morton_decode(key_cell(bkey[b], l), ix, iy, iz);
    const uint64_t pre = key_sys(bkey[b], l) << (3 * l);
    int lim = 1 << l;
    int k = 0;
    for (int dx = -1; dx <= 1; ++dx)
        for (int dy = -1; dy <= 1; ++dy)
            for (int dz = -1; dz <= 1; ++dz, ++k) {
                int jx = ix + dx, jy = iy + dy, jz = iz + dz;
                int c = -1;
                if (jx >= 0 && jy >= 0 && jz >= 0 && jx < lim && jy < lim && jz < lim)
                    c = (dx == 0 && dy == 0 && dz == 0) ? b
                                                         : find_box(bkey, lt.start[l], lt.count[l],
                                                                    pre | morton_encode(jx, jy, jz));
                bcol[(int64_t)b * 27 + k] = c;
            }
    bool leaf = bcmask[b] == 0;
    bflags[b] = leaf ? BF_LEAF : 0;
    isleaf_i32[b] = leaf ? 1 : 0;
    // expansion slots: every non-leaf box, and every root (a root that is a
    // leaf anterpolates its own sources for the windowed term W_0)
    isnonleaf_i32[b] = (leaf && l > 0) ? 0 : 1;
    if (leaf) atomicAdd(nleaf, 1);
}

__global__ void k_box_flags(int nb, const int32_t *bnsrc, const int32_t *bntgt, const int32_t *bcol, uint8_t *bflags) {
    int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= nb) return;
    // F_out: non-leaf with sources
    uint8_t f = bflags[b];
    if (!(f & BF_LEAF) && bnsrc[b] > 0) f |= BF_FOUT;
    bflags[b] = f;
}

__global__ void k_box_flags_in(int nb, const int32_t *bnsrc, const int32_t *bntgt, const int32_t *bcol,
                               uint8_t *bflags) {
    int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= nb) return;
    if (bntgt[b] == 0) return;
    bool fin = false;
    for (int k = 0; k < 27 && !fin; ++k) {
        int c = bcol[(int64_t)b * 27 + k];
        if (c >= 0 && (bflags[c] & BF_FOUT)) fin = true;
    }
    if (fin) bflags[b] |= BF_FIN;
}

// 1 for an incoming box (F_in with targets), else 0
__global__ void k_is_fin(int nb, const uint8_t *bflags, const int32_t *bntgt, int32_t *isfin) {
    int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= nb) return;
    isfin[b] = ((bflags[b] & BF_FIN) && bntgt[b] > 0) ? 1 : 0;
}

// bfin[b] = index of b among the incoming boxes (box order) or -1; fin2box inverts it
__global__ void k_fin_index(int nb, const int32_t *isfin, int32_t *bfin, int32_t *fin2box) {
    int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= nb) return;
    const int f = isfin[b] ? bfin[b] : -1;  // bfin holds the exclusive scan of isfin
    bfin[b] = f;
    if (f >= 0) fin2box[f] = b;
}

__global__ void k_slots(int nb, const int32_t *isslot, const int32_t *excl, int32_t *bslot) {
    int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= nb) return;
    bslot[b] = isslot[b] ? excl[b] : -1;
}

__global__ void k_slot2box(int nb, const int32_t *bslot, int32_t *slot2box) {
    int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= nb) return;
    int s = bslot[b];
    if (s >= 0) slot2box[s] = b;
}

// leaf index and leaf-local coordinates of every point; in single precision
// the coordinates are split into hi + lo parts (double-float) so that
// differences of nearby points keep their relative precision
template <typename T>
__global__ void k_point_local(int nb, const uint64_t *bkey, const int8_t *blevel, const int32_t *bstart,
                              const int32_t *bcount, const uint8_t *bflags, const double *ux, const double *uy,
                              const double *uz, const double *q, const uint8_t *pflag, int32_t *pleaf,
                              typename Vec4<T>::type *plocal, float4 *plocal_lo) {
    // one warp per box (leaves hold tens of points)
    int b = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (b >= nb || !(bflags[b] & BF_LEAF)) return;
    int l = blevel[b];
    int ix, iy, iz;
    morton_decode(key_cell(bkey[b], l), ix, iy, iz);
    double R = level_R(l);
    double cx = (ix + 0.5) * R, cy = (iy + 0.5) * R, cz = (iz + 0.5) * R;
    int32_t s = bstart[b], e = s + bcount[b];
    for (int32_t k = s + (threadIdx.x & 31); k < e; k += 32) {
        pleaf[k] = b;
        typename Vec4<T>::type v;
        const double dx = ux[k] - cx, dy = uy[k] - cy, dz = uz[k] - cz;
        v.x = (T)dx;
        v.y = (T)dy;
        v.z = (T)dz;
        v.w = (pflag[k] & 1) ? (T)q[k] : (T)0;
        plocal[k] = v;
        if (plocal_lo) {
            float4 lo;
            lo.x = (float)(dx - (double)v.x);
            lo.y = (float)(dy - (double)v.y);
            lo.z = (float)(dz - (double)v.z);
            lo.w = 0.f;
            plocal_lo[k] = lo;
        }
    }
}

// residual-kernel interaction lists (target-centric form of Step 4):
// source leaf S (level b) acts on target leaf T (level a) when S is a leaf
// colleague of T's level-b ancestor (b <= a), or S is a leaf at level a+1
// touching T (T is then a coarse neighbour of S); pairs can only interact if
// the boxes are closer than R_b, the support of R_b.
// Is the gap between box A (level la, cell a*) and box B (level lb, cell b*)
// below R_lb?  Exact integer arithmetic in units of 2^-L, L = max(la, lb) + 1:
// the centres are (2 i + 1) 2^(L - l - 1), the half sides 2^(L - l - 1) and
// R_lb = 2^(L - lb) units (coordinates below 2^22, squares below 2^46).
__device__ __forceinline__ bool box_within(int la, int ax, int ay, int az, int lb, int bx, int by, int bz) {
    const int L = (la > lb ? la : lb) + 1, sa = L - la - 1, sb = L - lb - 1;
    const long long half = (1ll << sa) + (1ll << sb);
    long long d2 = 0;
    const int ia[3] = {ax, ay, az}, ib[3] = {bx, by, bz};
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        const long long ca = (2ll * ia[d] + 1) << sa, cb = (2ll * ib[d] + 1) << sb;
        const long long g = (ca > cb ? ca - cb : cb - ca) - half;
        if (g > 0) d2 += g * g;
    }
    return d2 < (1ll << (2 * (L - lb)));
}

// FILL = false: count every list (cnt, pairs) and write it to tmp, kNearCap
// entries per target leaf (cap_over is set if a list is longer); FILL = true:
// write the lists at their offsets
constexpr int kNearCap = 128;
template <bool FILL>
__global__ void k_near_lists(int ntl, const int32_t *tleaves, const uint64_t *bkey, const int8_t *blevel,
                             const int32_t *bparent, const int32_t *bchild0, const uint8_t *bcmask,
                             const uint8_t *bflags, const int32_t *bnsrc, const int32_t *bntgt, const int32_t *bcol,
                             int32_t *cnt, const int32_t *off, int32_t *list, unsigned long long *pairs,
                             int32_t *tmp, int *cap_over) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= ntl) return;
    int T = tleaves[i];
    int a = blevel[T];
    int tx, ty, tz;
    morton_decode(key_cell(bkey[T], a), tx, ty, tz);
    int n = 0;
    int32_t *out = FILL ? list + off[i] : tmp + (size_t)i * kNearCap;
    long long np = 0;
    int B = T;
    for (int b = a; b >= 0; --b) {
        for (int k = 0; k < 27; ++k) {
            int C = bcol[(int64_t)B * 27 + k];
            if (C < 0 || !(bflags[C] & BF_LEAF) || bnsrc[C] == 0) continue;
            int cx, cy, cz;
            morton_decode(key_cell(bkey[C], b), cx, cy, cz);
            if (!box_within(a, tx, ty, tz, b, cx, cy, cz)) continue;
            if (FILL || n < kNearCap) out[n] = C;
            np += bnsrc[C];
            ++n;
        }
        B = bparent[B];
        if (B < 0) break;
    }
    for (int k = 0; k < 27; ++k) {
        int C = bcol[(int64_t)T * 27 + k];
        if (C < 0 || (bflags[C] & BF_LEAF)) continue;
        int c0 = bchild0[C];
        uint8_t m = bcmask[C];
        int kk = 0;
        for (int oc = 0; oc < 8; ++oc) {
            if (!(m & (1u << oc))) continue;
            int D = c0 + kk++;
            if (!(bflags[D] & BF_LEAF) || bnsrc[D] == 0) continue;
            int dx, dy, dz;
            morton_decode(key_cell(bkey[D], a + 1), dx, dy, dz);
            if (!box_within(a, tx, ty, tz, a + 1, dx, dy, dz)) continue;
            if (FILL || n < kNearCap) out[n] = D;
            np += bnsrc[D];
            ++n;
        }
    }
    if (!FILL) {
        cnt[i] = n;
        if (n > kNearCap) atomicExch(cap_over, 1);
        atomicAdd(pairs, (unsigned long long)(np * (long long)bntgt[T]));
    }
}

// the counted lists, copied from the fixed-capacity scratch to their offsets
__global__ void k_compact_lists(int ntl, const int32_t *tmp, const int32_t *off, int32_t *list) {
    const int i = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (i >= ntl) return;
    const int o = off[i], n = off[i + 1] - o;
    for (int k = threadIdx.x & 31; k < n; k += 32) list[o + k] = tmp[(size_t)i * kNearCap + k];
}

__global__ void k_list_target_leaves(int nb, const uint8_t *bflags, const int32_t *bntgt, const int32_t *excl,
                                     const int32_t *is, int32_t *tleaves) {
    int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= nb) return;
    if (is[b]) tleaves[excl[b]] = b;
}
__global__ void k_is_target_leaf(int nb, const uint8_t *bflags, const int32_t *bntgt, int32_t *is) {
    int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= nb) return;
    is[b] = ((bflags[b] & BF_LEAF) && bntgt[b] > 0) ? 1 : 0;
}
__global__ void k_flag_prefix_src(int64_t n, const uint8_t *pflag, int32_t *fs, int32_t *ft) {
    int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    fs[k] = pflag[k] & 1;
    ft[k] = (pflag[k] >> 1) & 1;
}
__global__ void k_set_last(int32_t *arr, int64_t n, const int32_t *total) { arr[n] = *total; }

__global__ void k_leaf_export(int nb, const uint64_t *bkey, const int8_t *blevel, const int32_t *bstart,
                              const int32_t *bcount, const uint8_t *bflags, const uint32_t *idx, int32_t *lev_out,
                              int64_t *cell_out) {
    int b = blockIdx.x;
    if (b >= nb || !(bflags[b] & BF_LEAF)) return;
    int32_t s = bstart[b], e = s + bcount[b];
    for (int32_t k = s + threadIdx.x; k < e; k += blockDim.x) {
        uint32_t i = idx[k];
        lev_out[i] = blevel[b];
        cell_out[i] = (int64_t)key_cell(bkey[b], blevel[b]);
    }
}

// ------------------------------------------------------------------ driver
#define CK(x)                                                               \
    do {                                                                    \
        cudaError_t e_ = (x);                                               \
        if (e_ != cudaSuccess) {                                            \
            err = std::string(#x) + ": " + cudaGetErrorString(e_);          \
            return DMK_ERR_CUDA_I;                                          \
        }                                                                   \
    } while (0)

static inline unsigned nblk(int64_t n, int t) { return (unsigned)((n + t - 1) / t); }

int TreeBuilder::grow_boxes(int64_t need, cudaStream_t st, std::string &err, size_t keep) {
    if (need <= box_cap) return 0;
    int64_t cap = std::max<int64_t>(need, box_cap * 2);
    cap = std::max<int64_t>(cap, 4096);
    // the arrays a level split writes keep their first `keep` boxes (the
    // levels built so far, copied device to device); the others are filled
    // after the boxes are complete, so their contents need not survive
    int rc = 0;
    rc |= ws.grow_keep(bkey, cap * sizeof(uint64_t), keep * sizeof(uint64_t), st);
    rc |= ws.grow_keep(blevel, cap, keep, st);
    rc |= ws.grow_keep(bstart, cap * 4, keep * 4, st);
    rc |= ws.grow_keep(bcount, cap * 4, keep * 4, st);
    rc |= ws.grow_keep(bparent, cap * 4, keep * 4, st);
    rc |= ws.grow_keep(bchild0, cap * 4, keep * 4, st);
    rc |= ws.grow_keep(bcmask, cap, keep, st);
    rc |= ws.ensure(bflags, cap);
    rc |= ws.ensure(bnsrc, cap * 4);
    rc |= ws.ensure(bntgt, cap * 4);
    rc |= ws.ensure(bcol, cap * 27 * 4);
    rc |= ws.ensure(bslot, cap * 4);
    rc |= ws.ensure(bscr0, cap * 4);
    rc |= ws.ensure(bscr1, cap * 4);
    rc |= ws.ensure(bscr2, (cap + 1) * 4);
    if (rc & 2) { err = "device-to-device copy of the box arrays failed"; return DMK_ERR_CUDA_I; }
    if (rc) { err = "device allocation failed (boxes)"; return DMK_ERR_OOM_I; }
    box_cap = cap;
    return 0;
}

int forest_key_bits(int nsys) {
    int sb = 0;
    while (sb < 40 && (1ll << sb) < (long long)nsys) ++sb;
    return std::min(kMortonBits, (63 - sb) / 3);
}

int TreeBuilder::build(const double *src, int64_t ns, const double *charges, const double *tgt, int64_t nt, bool same,
                       int leaf_cap, int max_level, int point_prec, cudaStream_t st, std::string &err,
                       int nsys_in, const int64_t *h_off) {
    n = same ? ns : ns + nt;
    this->same = same;
    const int64_t N = n;
    const bool forest = h_off != nullptr;
    if (forest && !same) { err = "a batch of systems needs targets equal to sources"; return DMK_ERR_INVALID_ARG_I; }
    nsys = forest ? nsys_in : 1;
    kb = forest ? forest_key_bits(nsys) : kMortonBits;
    max_level = std::min(max_level, kb);
    // ---- 1. bounding box (of every system)
    const int bb_blocks = 256;
    if (ws.ensure(bbox_part, bb_blocks * 6 * sizeof(double)) || ws.ensure(frame, (int64_t)nsys * sizeof(Frame)) ||
        ws.ensure(flags, 16 * sizeof(int)) || (forest && ws.ensure(sysoff, (int64_t)(nsys + 1) * 8)) ||
        (forest && ws.ensure(psys, N * 4))) {
        err = "device allocation failed";
        return DMK_ERR_OOM_I;
    }
    int *d_flags = (int *)flags.p;  // [0] bad input, [1] changed, [2] overflow, [3] total
    CK(cudaMemsetAsync(d_flags, 0, 16 * sizeof(int), st));
    const int64_t *d_off = forest ? (const int64_t *)sysoff.p : nullptr;
    if (forest) {
        CK(cudaMemcpyAsync(sysoff.p, h_off, (size_t)(nsys + 1) * 8, cudaMemcpyHostToDevice, st));
        ::dmk::launch_tick();
        k_bbox_sys<<<nsys, 256, 0, st>>>(src, d_off, (Frame *)frame.p, d_flags);
    } else {
        ::dmk::launch_tick();
        k_bbox_partial<<<bb_blocks, 256, 0, st>>>(src, ns, same ? nullptr : tgt, same ? 0 : nt,
                                                  (double *)bbox_part.p, d_flags);
        ::dmk::launch_tick();
        k_bbox_final<<<1, 32, 0, st>>>((double *)bbox_part.p, bb_blocks, (Frame *)frame.p);
    }
    CK(cudaGetLastError());
    // ---- 2. keys and sort
    if (ws.ensure(keys, N * 8) || ws.ensure(keys2, N * 8) || ws.ensure(idx, N * 4) || ws.ensure(idx2, N * 4) ||
        ws.ensure(sort_tmp, radix_tmp_bytes(N)) || ws.ensure(ux, N * 8) || ws.ensure(uy, N * 8) ||
        ws.ensure(uz, N * 8) || ws.ensure(utmp, N * 24) || ws.ensure(q, N * 8) || ws.ensure(pflag, N) ||
        ws.ensure(pout, N * 4) ||
        ws.ensure(pleaf, N * 4) || ws.ensure(plocal, N * (point_prec ? 16 : 32)) ||
        ws.ensure(plocal_lo, point_prec ? N * 16 : 16) ||
        ws.ensure(pscan0, (N + 1) * 4) || ws.ensure(pscan1, (N + 1) * 4) ||
        ws.ensure(scan_tmp, scan_tmp_bytes(std::max<int64_t>(N + 1, 1 << 20)))) {
        err = "device allocation failed (points)";
        return DMK_ERR_OOM_I;
    }
    ::dmk::launch_tick();
    k_make_keys<<<nblk(N, 256), 256, 0, st>>>(src, ns, same ? nullptr : tgt, N, (const Frame *)frame.p, d_off,
                                              nsys, kb, (uint64_t *)keys.p, (uint32_t *)idx.p, (double *)utmp.p);
    uint64_t *skeys;
    uint32_t *sidx;
    radix_sort_pairs((uint64_t *)keys.p, (uint32_t *)idx.p, (uint64_t *)keys2.p, (uint32_t *)idx2.p, N, 63,
                     sort_tmp.p, sort_tmp.bytes, st, &skeys, &sidx);
    sorted_keys = skeys;
    sorted_idx = sidx;
    ::dmk::launch_tick();
    k_gather_points<<<nblk(N, 256), 256, 0, st>>>((const double *)utmp.p, charges, ns, N, same ? 1 : 0, skeys, kb,
                                                  sidx, (double *)ux.p, (double *)uy.p, (double *)uz.p,
                                                  (double *)q.p, (uint8_t *)pflag.p, (int32_t *)pout.p,
                                                  forest ? (int32_t *)psys.p : nullptr);
    CK(cudaGetLastError());
    int h_bad = 0;
    CK(cudaMemcpyAsync(&h_bad, d_flags, sizeof(int), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    if (h_bad) {
        err = "non-finite coordinate in sources or targets";
        return DMK_ERR_INVALID_ARG_I;
    }
    CK(cudaMemcpy(&h_frame, frame.p, sizeof(Frame), cudaMemcpyDeviceToHost));

    // ---- 3/4. build, check level restriction, rebuild
    const uint32_t fcap = 1u << 20;
    if (ws.ensure(forced, fcap * sizeof(uint64_t))) { err = "device allocation failed"; return DMK_ERR_OOM_I; }
    CK(cudaMemsetAsync(forced.p, 0, fcap * sizeof(uint64_t), st));
    int64_t est = std::max<int64_t>(4096, 16 * (N / std::max(leaf_cap, 1) + 64) + 2 * (int64_t)nsys);
    // diagnostic: a smaller first capacity, so that the box arrays grow while
    // the levels are built (the estimate above leaves that path to rare trees)
    if (const char *e = std::getenv("DMK_TREE_INITIAL_BOXES")) {
        const long long v = std::atoll(e);
        if (v > 0 && box_cap == 0) est = std::max<int64_t>(4096, v);
    }
    if (int rc = grow_boxes(est, st, err)) return rc;
    rounds = 0;
    bool pushed = false;  // the forced set has been completed on the cell sets
    for (int rebuilds = 0;; ++rebuilds) {
        if (rebuilds > 64) { err = "level restriction did not converge"; return DMK_ERR_INTERNAL_I; }
        // roots
        if (forest) {
            ::dmk::launch_tick();
            k_roots<<<nblk(nsys, 128), 128, 0, st>>>(nsys, d_off, (uint64_t *)bkey.p, (int8_t *)blevel.p,
                                                      (int32_t *)bstart.p, (int32_t *)bcount.p, (int32_t *)bparent.p);
        } else {
            uint64_t zero64 = 0;
            int8_t zero8 = 0;
            int32_t zero32 = 0, n32 = (int32_t)N, m1 = -1;
            CK(cudaMemcpyAsync(bkey.p, &zero64, 8, cudaMemcpyHostToDevice, st));
            CK(cudaMemcpyAsync(blevel.p, &zero8, 1, cudaMemcpyHostToDevice, st));
            CK(cudaMemcpyAsync(bstart.p, &zero32, 4, cudaMemcpyHostToDevice, st));
            CK(cudaMemcpyAsync(bcount.p, &n32, 4, cudaMemcpyHostToDevice, st));
            CK(cudaMemcpyAsync(bparent.p, &m1, 4, cudaMemcpyHostToDevice, st));
        }
        lt_start[0] = 0;
        lt_count[0] = nsys;
        nlev = 1;
        int nbox = nsys;
        for (int l = 0; l < max_level; ++l) {
            int lc = lt_count[l];
            if (ws.ensure(lvl_off9, (int64_t)lc * 9 * 4) || ws.ensure(lvl_cnt, (int64_t)lc * 4) ||
                ws.ensure(lvl_excl, (int64_t)lc * 4)) {
                err = "device allocation failed";
                return DMK_ERR_OOM_I;
            }
            LevelArgs la{(const uint64_t *)skeys, (uint64_t *)bkey.p, (int8_t *)blevel.p, (int32_t *)bstart.p,
                         (int32_t *)bcount.p, (int32_t *)bparent.p, (int32_t *)bchild0.p, (uint8_t *)bcmask.p,
                         (int32_t *)lvl_off9.p, (int32_t *)lvl_cnt.p, (int32_t *)lvl_excl.p,
                         (const uint64_t *)forced.p, fcap, kb};
            ::dmk::launch_tick();
            k_level_split<<<nblk((int64_t)lc * 8, 128), 128, 0, st>>>(la, l, lt_start[l], lc, leaf_cap, max_level);
            scan_exclusive_i32((int32_t *)lvl_cnt.p, (int32_t *)lvl_excl.p, lc, d_flags + 3, scan_tmp.p,
                               scan_tmp.bytes, st);
            int total = 0;
            CK(cudaMemcpyAsync(&total, d_flags + 3, 4, cudaMemcpyDeviceToHost, st));
            CK(cudaStreamSynchronize(st));
            if (total > 0 && nbox + total > box_cap) {
                // grow the box arrays, keeping the levels built so far (device to device)
                const int64_t need = (int64_t)(nbox + total) * 2;
                if (int rc = grow_boxes(need, st, err, (size_t)nbox)) return rc;
                la.bkey = (uint64_t *)bkey.p;
                la.blevel = (int8_t *)blevel.p;
                la.bstart = (int32_t *)bstart.p;
                la.bcount = (int32_t *)bcount.p;
                la.bparent = (int32_t *)bparent.p;
                la.bchild0 = (int32_t *)bchild0.p;
                la.bcmask = (uint8_t *)bcmask.p;
            }
            ::dmk::launch_tick();
            k_level_emit<<<nblk(lc, 128), 128, 0, st>>>(la, l, lt_start[l], lc, nbox);
            CK(cudaGetLastError());
            if (total == 0) break;
            lt_start[l + 1] = nbox;
            lt_count[l + 1] = total;
            nbox += total;
            nlev = l + 2;
        }
        // boxes of the deepest level are leaves
        {
            int l = nlev - 1;
            CK(cudaMemsetAsync((int32_t *)bchild0.p + lt_start[l], 0xff, (size_t)lt_count[l] * 4, st));
            CK(cudaMemsetAsync((uint8_t *)bcmask.p + lt_start[l], 0, (size_t)lt_count[l], st));
        }
        nb = nbox;
        LevelTable lt;
        for (int l = 0; l < kMaxLevel + 2; ++l) {
            lt.start[l] = l < nlev ? lt_start[l] : 0;
            lt.count[l] = l < nlev ? lt_count[l] : 0;
        }
        lt.nlev = nlev;
        if (!pushed) {
            // complete the level restriction on the cell sets, then rebuild once
            pushed = true;
            const int lcap = (int)fcap;
            if (ws.ensure(slist, (int64_t)lcap * 8)) { err = "device allocation failed"; return DMK_ERR_OOM_I; }
            CK(cudaMemsetAsync(d_flags + 1, 0, 3 * sizeof(int), st));  // changed, overflow, count
            ::dmk::launch_tick();
            k_collect_nonleaf<<<nblk(nb, 128), 128, 0, st>>>((const uint64_t *)bkey.p, (const int8_t *)blevel.p,
                                                             (const uint8_t *)bcmask.p, nb, (uint64_t *)forced.p,
                                                             fcap, kb, (uint64_t *)slist.p, d_flags + 3, lcap,
                                                             d_flags + 2);
            int any = 0;
            for (int pr = 0;; ++pr) {
                int hc[3];
                CK(cudaMemcpyAsync(hc, d_flags + 1, 3 * sizeof(int), cudaMemcpyDeviceToHost, st));
                CK(cudaStreamSynchronize(st));
                if (hc[1]) { err = "forced-split table overflow"; return DMK_ERR_INTERNAL_I; }
                if ((pr > 0 && !hc[0]) || hc[2] == 0) break;
                if (pr > 64) { err = "level restriction did not converge"; return DMK_ERR_INTERNAL_I; }
                any |= hc[0];
                ++rounds;
                CK(cudaMemsetAsync(d_flags + 1, 0, sizeof(int), st));
                ::dmk::launch_tick();
                k_push_balance<<<nblk(hc[2], 128), 128, 0, st>>>(skeys, N, max_level, kb, (uint64_t *)forced.p,
                                                                 fcap, (uint64_t *)slist.p, hc[2], d_flags + 3, lcap,
                                                                 d_flags + 1, d_flags + 2);
            }
            if (any) continue;  // rebuild with the completed forced set
        }
        CK(cudaMemsetAsync(d_flags + 1, 0, 2 * sizeof(int), st));
        ::dmk::launch_tick();
        k_balance<<<nblk(nb, 128), 128, 0, st>>>((const uint64_t *)bkey.p, (const int8_t *)blevel.p,
                                                 (const uint8_t *)bcmask.p, nb, lt, (uint64_t *)forced.p, fcap, kb,
                                                 d_flags + 1, d_flags + 2);
        int hf[2];
        CK(cudaMemcpyAsync(hf, d_flags + 1, 2 * sizeof(int), cudaMemcpyDeviceToHost, st));
        CK(cudaStreamSynchronize(st));
        if (hf[1]) { err = "forced-split table overflow"; return DMK_ERR_INTERNAL_I; }
        if (!hf[0]) break;
    }

    // ---- 5. counts, colleagues, flags, slots
    LevelTable lt;
    for (int l = 0; l < kMaxLevel + 2; ++l) {
        lt.start[l] = l < nlev ? lt_start[l] : 0;
        lt.count[l] = l < nlev ? lt_count[l] : 0;
    }
    lt.nlev = nlev;
    const int32_t *psrc = nullptr, *ptgt = nullptr;
    if (!same) {
        ::dmk::launch_tick();
        k_flag_prefix_src<<<nblk(N, 256), 256, 0, st>>>(N, (const uint8_t *)pflag.p, (int32_t *)pscan0.p,
                                                        (int32_t *)pscan1.p);
        // exclusive scans in place into the (n+1)-long arrays
        scan_exclusive_i32((int32_t *)pscan0.p, (int32_t *)pscan0.p, N, d_flags + 4, scan_tmp.p, scan_tmp.bytes, st);
        ::dmk::launch_tick();
        k_set_last<<<1, 1, 0, st>>>((int32_t *)pscan0.p, N, d_flags + 4);
        scan_exclusive_i32((int32_t *)pscan1.p, (int32_t *)pscan1.p, N, d_flags + 5, scan_tmp.p, scan_tmp.bytes, st);
        ::dmk::launch_tick();
        k_set_last<<<1, 1, 0, st>>>((int32_t *)pscan1.p, N, d_flags + 5);
        psrc = (const int32_t *)pscan0.p;
        ptgt = (const int32_t *)pscan1.p;
    }
    int32_t *isleaf = (int32_t *)bscr0.p, *isslot = (int32_t *)bscr1.p, *excl = (int32_t *)bscr2.p;
    CK(cudaMemsetAsync(d_flags + 9, 0, sizeof(int), st));
    ::dmk::launch_tick();
    k_box_finish<<<nblk(nb, 128), 128, 0, st>>>(nb, (const uint64_t *)bkey.p, (const int8_t *)blevel.p,
                                                (const int32_t *)bstart.p, (const int32_t *)bcount.p,
                                                (const uint8_t *)bcmask.p, psrc, ptgt, lt, (int32_t *)bnsrc.p,
                                                (int32_t *)bntgt.p, (int32_t *)bcol.p, (uint8_t *)bflags.p, isleaf,
                                                isslot, d_flags + 9);
    ::dmk::launch_tick();
    k_box_flags<<<nblk(nb, 128), 128, 0, st>>>(nb, (const int32_t *)bnsrc.p, (const int32_t *)bntgt.p,
                                               (const int32_t *)bcol.p, (uint8_t *)bflags.p);
    ::dmk::launch_tick();
    k_box_flags_in<<<nblk(nb, 128), 128, 0, st>>>(nb, (const int32_t *)bnsrc.p, (const int32_t *)bntgt.p,
                                                  (const int32_t *)bcol.p, (uint8_t *)bflags.p);
    scan_exclusive_i32(isslot, excl, nb, d_flags + 6, scan_tmp.p, scan_tmp.bytes, st);
    root_leaf = (nlev == 1);
    ::dmk::launch_tick();
    k_slots<<<nblk(nb, 128), 128, 0, st>>>(nb, isslot, excl, (int32_t *)bslot.p);
    // the incoming boxes (isleaf's contents are no longer needed: it is reused)
    if (ws.ensure(bfin, (int64_t)nb * 4) || ws.ensure(fin2box, (int64_t)nb * 4)) {
        err = "device allocation failed";
        return DMK_ERR_OOM_I;
    }
    ::dmk::launch_tick();
    k_is_fin<<<nblk(nb, 128), 128, 0, st>>>(nb, (const uint8_t *)bflags.p, (const int32_t *)bntgt.p, isleaf);
    // exclusive scan into bfin, then each thread turns its own entry into the index
    scan_exclusive_i32(isleaf, (int32_t *)bfin.p, nb, d_flags + 10, scan_tmp.p, scan_tmp.bytes, st);
    ::dmk::launch_tick();
    k_fin_index<<<nblk(nb, 128), 128, 0, st>>>(nb, isleaf, (int32_t *)bfin.p, (int32_t *)fin2box.p);
    CK(cudaGetLastError());
    int hs[5] = {0, 0, 0, 0, 0};  // slots, -, -, leaves, incoming boxes
    CK(cudaMemcpyAsync(hs, d_flags + 6, 5 * sizeof(int), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    nslots = hs[0];
    nleaves = hs[3];
    nfin = hs[4];
    if (ws.ensure(slot2box, (int64_t)std::max(nslots, 1) * 4)) { err = "device allocation failed"; return DMK_ERR_OOM_I; }
    ::dmk::launch_tick();
    k_slot2box<<<nblk(nb, 128), 128, 0, st>>>(nb, (const int32_t *)bslot.p, (int32_t *)slot2box.p);

    // leaf index and local coordinates of every point
    if (point_prec)
        { ::dmk::launch_tick();
        k_point_local<float><<<nblk(nb, 4), 128, 0, st>>>(nb, (const uint64_t *)bkey.p, (const int8_t *)blevel.p,
                                                 (const int32_t *)bstart.p, (const int32_t *)bcount.p,
                                                 (const uint8_t *)bflags.p, (const double *)ux.p,
                                                 (const double *)uy.p, (const double *)uz.p, (const double *)q.p,
                                                 (const uint8_t *)pflag.p, (int32_t *)pleaf.p,
                                                 (float4 *)plocal.p, (float4 *)plocal_lo.p);
        }
    else
        { ::dmk::launch_tick();
        k_point_local<double><<<nblk(nb, 4), 128, 0, st>>>(nb, (const uint64_t *)bkey.p, (const int8_t *)blevel.p,
                                                  (const int32_t *)bstart.p, (const int32_t *)bcount.p,
                                                  (const uint8_t *)bflags.p, (const double *)ux.p,
                                                  (const double *)uy.p, (const double *)uz.p, (const double *)q.p,
                                                  (const uint8_t *)pflag.p, (int32_t *)pleaf.p,
                                                  (double4_32a *)plocal.p, nullptr);
        }

    // ---- octant ranges of the leaves (near-field refinement)

    // ---- near-field lists over target leaves
    int32_t *istl = isleaf;  // reuse: 1 for target leaves
    ::dmk::launch_tick();
    k_is_target_leaf<<<nblk(nb, 128), 128, 0, st>>>(nb, (const uint8_t *)bflags.p, (const int32_t *)bntgt.p, istl);
    scan_exclusive_i32(istl, excl, nb, d_flags + 7, scan_tmp.p, scan_tmp.bytes, st);
    CK(cudaMemcpyAsync(&ntleaves, d_flags + 7, 4, cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    if (ws.ensure(tleaves, (int64_t)std::max(ntleaves, 1) * 4) ||
        ws.ensure(nl_cnt, (int64_t)(ntleaves + 1) * 4) || ws.ensure(nl_off, (int64_t)(ntleaves + 1) * 4) ||
        ws.ensure(pairs, 8) || ws.ensure(nl_tmp, (int64_t)std::max(ntleaves, 1) * kNearCap * 4)) {
        err = "device allocation failed";
        return DMK_ERR_OOM_I;
    }
    ::dmk::launch_tick();
    k_list_target_leaves<<<nblk(nb, 128), 128, 0, st>>>(nb, (const uint8_t *)bflags.p, (const int32_t *)bntgt.p,
                                                         excl, istl, (int32_t *)tleaves.p);
    CK(cudaMemsetAsync(pairs.p, 0, 8, st));
    CK(cudaMemsetAsync(d_flags + 9, 0, sizeof(int), st));  // a list longer than the scratch capacity
    if (ntleaves > 0) {
        ::dmk::launch_tick();
        k_near_lists<false><<<nblk(ntleaves, 128), 128, 0, st>>>(
            ntleaves, (const int32_t *)tleaves.p, (const uint64_t *)bkey.p, (const int8_t *)blevel.p,
            (const int32_t *)bparent.p, (const int32_t *)bchild0.p, (const uint8_t *)bcmask.p,
            (const uint8_t *)bflags.p, (const int32_t *)bnsrc.p, (const int32_t *)bntgt.p, (const int32_t *)bcol.p,
            (int32_t *)nl_cnt.p, nullptr, nullptr, (unsigned long long *)pairs.p, (int32_t *)nl_tmp.p,
            d_flags + 9);
        scan_exclusive_i32((int32_t *)nl_cnt.p, (int32_t *)nl_off.p, ntleaves, d_flags + 8, scan_tmp.p,
                           scan_tmp.bytes, st);
        ::dmk::launch_tick();
        k_set_last<<<1, 1, 0, st>>>((int32_t *)nl_off.p, ntleaves, d_flags + 8);
    }
    int ntot = 0, over = 0;
    CK(cudaMemcpyAsync(&ntot, d_flags + 8, 4, cudaMemcpyDeviceToHost, st));
    CK(cudaMemcpyAsync(&over, d_flags + 9, 4, cudaMemcpyDeviceToHost, st));
    unsigned long long hp = 0;
    CK(cudaMemcpyAsync(&hp, pairs.p, 8, cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    if (ntleaves == 0) ntot = 0;
    near_pairs = (int64_t)hp;
    if (ws.ensure(nl_src, (int64_t)std::max(ntot, 1) * 4)) { err = "device allocation failed"; return DMK_ERR_OOM_I; }
    if (ntleaves > 0 && !over) {
        // every list fitted the scratch: copy them to their offsets
        ::dmk::launch_tick();
        k_compact_lists<<<nblk(ntleaves, 4), 128, 0, st>>>(ntleaves, (const int32_t *)nl_tmp.p,
                                                           (const int32_t *)nl_off.p, (int32_t *)nl_src.p);
    } else if (ntleaves > 0) {
        // some list is longer than the scratch: traverse again, writing at the offsets
        ::dmk::launch_tick();
        k_near_lists<true><<<nblk(ntleaves, 128), 128, 0, st>>>(
            ntleaves, (const int32_t *)tleaves.p, (const uint64_t *)bkey.p, (const int8_t *)blevel.p,
            (const int32_t *)bparent.p, (const int32_t *)bchild0.p, (const uint8_t *)bcmask.p,
            (const uint8_t *)bflags.p, (const int32_t *)bnsrc.p, (const int32_t *)bntgt.p, (const int32_t *)bcol.p,
            nullptr, (const int32_t *)nl_off.p, (int32_t *)nl_src.p, nullptr, nullptr, nullptr);
    }
    CK(cudaGetLastError());
    near_list_len = ntot;
    return 0;
}

TreeView TreeBuilder::view() const {
    TreeView v;
    v.n = n;
    v.ux = (const double *)ux.p;
    v.uy = (const double *)uy.p;
    v.uz = (const double *)uz.p;
    v.q = (const double *)q.p;
    v.pflag = (const uint8_t *)pflag.p;
    v.nb = nb;
    v.bkey = (const uint64_t *)bkey.p;
    v.blevel = (const int8_t *)blevel.p;
    v.bstart = (const int32_t *)bstart.p;
    v.bcount = (const int32_t *)bcount.p;
    v.bparent = (const int32_t *)bparent.p;
    v.bchild0 = (const int32_t *)bchild0.p;
    v.bcmask = (const uint8_t *)bcmask.p;
    v.bflags = (const uint8_t *)bflags.p;
    v.bnsrc = (const int32_t *)bnsrc.p;
    v.bntgt = (const int32_t *)bntgt.p;
    v.bcol = (const int32_t *)bcol.p;
    v.bslot = (const int32_t *)bslot.p;
    for (int l = 0; l < kMaxLevel + 2; ++l) {
        v.lev_start[l] = l < nlev ? lt_start[l] : 0;
        v.lev_count[l] = l < nlev ? lt_count[l] : 0;
    }
    v.nlev = nlev;
    return v;
}

int TreeBuilder::export_leaves(int32_t *lev, int64_t *cell, cudaStream_t st, std::string &err) {
    DBuf dl, dc;
    if (ws.ensure(dl, n * 4) || ws.ensure(dc, n * 8)) { err = "device allocation failed"; return DMK_ERR_OOM_I; }
    ::dmk::launch_tick();
    k_leaf_export<<<nb, 128, 0, st>>>(nb, (const uint64_t *)bkey.p, (const int8_t *)blevel.p,
                                      (const int32_t *)bstart.p, (const int32_t *)bcount.p,
                                      (const uint8_t *)bflags.p, sorted_idx, (int32_t *)dl.p, (int64_t *)dc.p);
    CK(cudaMemcpyAsync(lev, dl.p, n * 4, cudaMemcpyDeviceToHost, st));
    CK(cudaMemcpyAsync(cell, dc.p, n * 8, cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    ws.release(dl);
    ws.release(dc);
    return 0;
}

}  // namespace dmk
