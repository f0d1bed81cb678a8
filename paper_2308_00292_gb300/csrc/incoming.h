// incoming.h -- incoming expansions of the downward pass on the tensor cores
// (internal): shapes of the single-precision kernel and its launcher.
#pragma once

#include <string>

#include "passes.h"

namespace dmk {

constexpr int kIThreads = 256;  // threads of a CTA; two CTAs share an SM
constexpr int kIWorkers = 224;  // warps 0-6 translate; warp 7 issues the MMAs and prefetches
constexpr int kITmem = 256;     // TMEM columns of a CTA

// Shapes of the tensor-core incoming pass for Chebyshev order P and Fourier
// half-width NF.  Plane waves are stored plane by plane (m_z outermost):
// Phi[slot][m_z][m_y][m_x], m_x padded to MXP.
template <int P, int NF> struct InShape {
    static constexpr int NH = NF + 1, N1 = 2 * NF + 1, MXP = (N1 + 1) & ~1;
    static constexpr int PE = (P + 1) / 2, PO = P / 2;  // even / odd Chebyshev indices
    static constexpr int K = 16;                        // contraction length: m' = 0..NF, padded
    static constexpr int NZ = 2 * P * P;                // rows (class, a, b) of the last contraction
    static constexpr int TILE_FL = 128 * K;             // one part (hi or lo) of a 128 x 16 operand
    static constexpr int NMODE = (N1 * N1 + kIWorkers - 1) / kIWorkers;  // plane modes per translating thread
    static constexpr int CB = 8;                        // colleagues whose loads are in flight together
    static constexpr int LSTR = (P * P * P + 3) & ~3;   // floats per box of the output
    static constexpr size_t O_AX = 0;                                     // [hi, lo]
    static constexpr size_t O_AY = O_AX + (size_t)2 * TILE_FL * 4;        // [hi, lo]
    static constexpr size_t O_T2 = O_AY + (size_t)2 * TILE_FL * 4;        // [NZ][NH] second contraction
    static constexpr size_t O_BW = O_T2 + ((size_t)NZ * NH * 4 + 127) / 128 * 128;  // [hi, lo] 32 x 16
    static constexpr size_t O_HZ = O_BW + (size_t)2 * 32 * K * 4;         // [P][NH] the last contraction's H
    static constexpr size_t O_PSI = O_HZ + ((size_t)P * NH * 4 + 127) / 128 * 128;
    static constexpr size_t O_UD = O_PSI + ((size_t)N1 * N1 * 8 + 127) / 128 * 128;
    static constexpr size_t BYTES = O_UD + ((size_t)27 * 27 * 8 + 127) / 128 * 128;
    static constexpr bool OK = NH <= 16 && PE <= 16 && 2 * BYTES <= 224 * 1024 &&
                               (size_t)LSTR * 4 <= (size_t)4 * TILE_FL * 4;  // output staged over both operands
};

// Incoming expansions Lambda_in of the nfin incoming boxes (all levels), in
// single precision, written to lam_in[f * LSTR ...] for incoming box f.
struct IncomingArgs {
    TreeView tv;
    const void *tables;        // DevTables<float>
    const void *phi;           // plane-major plane waves (float2), nslots x NH x N1 x MXP
    int nslots;
    int nfin;
    const int32_t *fin2box;
    int32_t *finc, *fincnt;    // scratch: nfin x 27 colleague entries, nfin counts
    float *lam_in;             // nfin x LSTR
    unsigned long long *reads; // colleague plane-wave arrays read (sum over incoming boxes)
    int *err;                  // set when a bounded wait gives up
    int num_sms;
};

template <int P, int NF> int launch_incoming(const IncomingArgs &a, cudaStream_t st, std::string &err);

}  // namespace dmk
