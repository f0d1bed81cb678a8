// tree.h -- device buffers and the tree builder of libdmk (internal).
#pragma once

#include <algorithm>

#include "dmk.h"
#include "dmk_internal.h"

namespace dmk {

enum {
    DMK_ERR_INVALID_ARG_I = DMK_ERR_INVALID_ARG,
    DMK_ERR_OOM_I = DMK_ERR_OOM,
    DMK_ERR_CUDA_I = DMK_ERR_CUDA,
    DMK_ERR_INTERNAL_I = DMK_ERR_INTERNAL,
};

// A device allocation that grows on demand (contents are not preserved).
struct DBuf {
    void *p = nullptr;
    size_t bytes = 0;
    DBuf() = default;
    DBuf(const DBuf &) = delete;
    DBuf &operator=(const DBuf &) = delete;
    ~DBuf() {
        if (p) cudaFree(p);
    }
};

struct Workspace {
    size_t live = 0;
    // returns 0 on success
    int ensure(DBuf &b, int64_t bytes) {
        if (bytes <= 0) bytes = 16;
        if (b.p && (int64_t)b.bytes >= bytes) return 0;
        if (b.p) {
            cudaFree(b.p);
            live -= b.bytes;
            b.p = nullptr;
            b.bytes = 0;
        }
        size_t want = (size_t)bytes;
        if (cudaMalloc(&b.p, want) != cudaSuccess) {
            cudaGetLastError();
            b.p = nullptr;
            return 1;
        }
        b.bytes = want;
        live += want;
        return 0;
    }
    // grows b to at least bytes keeping its first keep bytes: a new buffer,
    // a device-to-device copy on st, then the old buffer is freed once the
    // copy is done; returns 0 on success, 1 when allocation fails, 2 when the
    // copy fails (b then keeps its old buffer)
    int grow_keep(DBuf &b, int64_t bytes, size_t keep, cudaStream_t st) {
        if (b.p && (int64_t)b.bytes >= bytes) return 0;
        DBuf nb;
        if (ensure(nb, bytes)) return 1;
        keep = std::min(keep, b.bytes);
        if (keep && (cudaMemcpyAsync(nb.p, b.p, keep, cudaMemcpyDeviceToDevice, st) != cudaSuccess ||
                     cudaStreamSynchronize(st) != cudaSuccess)) {
            release(nb);
            return 2;
        }
        release(b);
        b.p = nb.p;
        b.bytes = nb.bytes;
        nb.p = nullptr;
        nb.bytes = 0;
        return 0;
    }
    void release(DBuf &b) {
        if (b.p) {
            cudaFree(b.p);
            live -= b.bytes;
        }
        b.p = nullptr;
        b.bytes = 0;
    }
};

struct Frame {
    double lo[3];
    double S;
    double rS;  // 1 / S, correctly rounded
};

template <typename T> struct Vec4;
template <> struct Vec4<float> { using type = float4; };
template <> struct Vec4<double> { using type = double4_32a; };

uint64_t host_morton_encode(uint32_t ix, uint32_t iy, uint32_t iz);

// bits per axis of the point keys of a forest of nsys systems (the system
// index takes the bits above them in a 63-bit key)
int forest_key_bits(int nsys);

class TreeBuilder {
public:
    explicit TreeBuilder(Workspace &w) : ws(w) {}
    // Build the tree of the union of sources and targets (targets ignored
    // when same).  point_prec: 1 -> float4 leaf-local coordinates, 0 -> double4.
    // A batch (h_off != NULL, host array of nsys + 1 ascending offsets into
    // src, targets equal to sources) is built as a forest with one root per
    // system, each system in its own unit box.
    int build(const double *src, int64_t ns, const double *charges, const double *tgt, int64_t nt, bool same,
              int leaf_cap, int max_level, int point_prec, cudaStream_t st, std::string &err, int nsys = 1,
              const int64_t *h_off = nullptr);
    TreeView view() const;
    int export_leaves(int32_t *lev, int64_t *cell, cudaStream_t st, std::string &err);

    Workspace &ws;
    int64_t n = 0;
    bool same = true;
    int nb = 0, nlev = 0, nslots = 0, nleaves = 0, ntleaves = 0, rounds = 0, near_list_len = 0;
    int nfin = 0;  // boxes with targets and an F_out colleague (the incoming boxes)
    int nsys = 1, kb = kMortonBits;  // systems (roots) and bits per axis of the point keys
    bool root_leaf = false;
    int64_t near_pairs = 0;
    int lt_start[kMaxLevel + 2] = {0}, lt_count[kMaxLevel + 2] = {0};
    Frame h_frame{};
    const uint64_t *sorted_keys = nullptr;
    const uint32_t *sorted_idx = nullptr;

    // points (sorted)
    DBuf keys, keys2, idx, idx2, sort_tmp, ux, uy, uz, utmp, q, pflag, pout, pleaf, plocal, plocal_lo, pscan0,
        pscan1, scan_tmp;
    DBuf bbox_part, frame, flags, forced, slist, sysoff, psys;  // frame: one per system
    // boxes
    int64_t box_cap = 0;
    DBuf bkey, blevel, bstart, bcount, bparent, bchild0, bcmask, bflags, bnsrc, bntgt, bcol, bslot;
    DBuf bscr0, bscr1, bscr2, slot2box;
    // incoming boxes in box order: bfin[box] = its index among them or -1,
    // fin2box[index] = the box
    DBuf bfin, fin2box;
    DBuf lvl_off9, lvl_cnt, lvl_excl;
    // near-field lists
    DBuf tleaves, nl_cnt, nl_off, nl_src, nl_tmp, pairs;

private:
    int grow_boxes(int64_t need, cudaStream_t st, std::string &err, size_t keep = 0);
};

}  // namespace dmk
