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
    DBuf M, Lam, LamW, Phi, ufar, unear, gfar, gnear, slab, rootscr, counter, psig;
    DBuf lam_in, finc, fincnt;  // the tensor-core incoming pass: coefficients, colleague lists
    DBuf upcnt;                 // the single-precision upward pass: arrivals per expansion slot
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
    double *grad;         // gradients of the potentials (n_tgt x 3), or null
    cudaStream_t st;
    cudaEvent_t ev[8];  // 0 start, 1 upward, 2 plane waves, 7 incoming, 6 local, 3 far done, 4 finalize, 5 end
    cudaStream_t side;  // the near field's stream, forked after the tree and joined before finalize
    cudaEvent_t fork, join, nev[2];  // nev: start and end of the near field on side
    size_t smem_limit;
    int num_sms;
};

int run_passes(PassCtx &cx, std::string &err);

// The residual near field (near.cu): unear (and gnear, if not null) of every
// point of the ntl target leaves.  Returns 0, 1 for a polynomial degree outside
// 2..30, 2 for a failed launch.
struct NearArgs {
    TreeView tv;
    int ntl;
    const int32_t *tleaves, *nl_off, *nl_src;
    const void *plocal;         // float4 or double4 leaf-local points
    const float4 *plocal_lo;    // single precision: lo parts
    const void *qmono;          // residual polynomial, monomial coefficients (float or double);
                                // per level [nlev][qdeg + 1] for the Yukawa kernel
    int qdeg;
    double *unear, *gnear;
    int *counter;
    bool yukawa;                // kernel exp(-lam r)/r with per-level polynomials
    double lam;                 // unit-box lambda (Yukawa)
    int nlev;                   // levels of the per-level table
};
int launch_near(bool single, const NearArgs &a, int num_sms, cudaStream_t st);

}  // namespace dmk
