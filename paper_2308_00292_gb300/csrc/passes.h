// passes.h -- launch context of the DMK passes (internal).
#pragma once

#include "tree.h"

namespace dmk {

// Placement of a kernel's per-CTA buffers: in shared memory while they fit,
// otherwise in a per-CTA slab of global scratch.
struct BufLayout {
    int n;
    size_t off[8];
    unsigned char in_smem[8];
    size_t smem_bytes, slab_bytes;
};

struct PassBufs {
    DBuf M, Lam, LamW, Phi, ufar, unear, slab, rootscr, counter;
};

struct PassCtx {
    TreeBuilder *tree;
    PassBufs *bufs;
    Workspace *ws;
    const void *tables;   // DevTables<float> or DevTables<double>
    bool single;          // working precision float
    int p;
    int mode;             // 0 all, 1 far only, 2 near only
    int64_t total_sources;
    double *pot;
    cudaStream_t st;
    cudaEvent_t ev[7];  // 0 start, 1 upward, 2 plane waves, 6 local, 3 near, 4 finalize, 5 end
    size_t smem_limit;
    int num_sms;
};

int run_passes(PassCtx &cx, std::string &err);

}  // namespace dmk
