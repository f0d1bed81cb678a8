// log2d.h -- the 2D Laplace kernel log r (internal).
#pragma once

#include <string>

#include "dmk_internal.h"
#include "tree.h"

namespace dmk {

// Plan tables of the 2D pass on the device (FP64).
struct Log2dDev {
    int p, nf, N1, n0, NW, gdeg;
    const double *A;          // [2][p][p]: T_n((xi + s) / 2) = sum_m A_s[n][m] T_m(xi), s = -1, +1
    const double *Fr, *Fi;    // [N1][p]: moments -> plane waves, theta = pi / 3
    const double *FWr, *FWi;  // [NW][p]: the same for the root window
    const double *w;          // [2 nf^2 + 1]: translation weights (every level)
    const double *wW;         // [2 n0^2 + 1]: root window weights
    const double *g;          // [gdeg + 1]: G(t) in x = 2 t - 1, monomials if gmono else Chebyshev
    // the table-driven log of the residual kernel (Tang's method), [256] each:
    const double *lgF;        // F_k ~ 1 / (1 + (k + 1/2) / 256)
    const double *lgL;        // -(1/2) log F_k
    const double *lgE;        // g[0] - (j/2) log 2 (j = 1 ... 255: t = m 2^-j)
    int gmono;
    double G0;                // G(0)
    // the mixed-precision near field (FP32 pairs, FP64 sums of the lanes)
    int mixed;
    const float *gcf;         // [4 gcn4]: G in Chebyshev polynomials of x, FP32, degree
    int gcdeg, gcn4;          // gcdeg, zero above it (16-byte aligned)
};

struct Log2dBufs {
    DBuf x3, t3, mom, loc, phi, ufar, unear, qco, qtot;
    DBuf cnt;    // pairs inside the support evaluated by the near field (u64)
    DBuf qpart;  // partial sums of the total charge
};

// One evaluation: sources [ns][2], charges [ns], targets [nt][2] (targets ==
// sources with nt == ns: every source is a target), potentials [nt]; all
// device pointers, work on stream st; near_ev[0] and near_ev[1] (either may be
// null) are recorded on st before and after the near field.  Returns a DMK_* code.
int run_log2d(const Log2dDev &d, TreeBuilder &tree, Workspace &ws, Log2dBufs &bf, const double *src, int64_t ns,
              const double *charges, const double *tgt, int64_t nt, int leaf_cap, int max_level, double *pot,
              cudaStream_t st, const cudaEvent_t near_ev[2], std::string &err);

}  // namespace dmk
