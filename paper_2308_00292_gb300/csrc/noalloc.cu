// noalloc.cu -- dmk_direct_noalloc: an evaluation entry point that performs
// no device allocation.
//
// Who needs it: code that must not allocate device memory while it runs --
// an application that hands all device memory to its own pool and does not
// allow libraries to grow their footprint, or a latency-critical loop that
// cannot afford the device-wide synchronisation an allocation may cause.  dmk_eval
// cannot serve them: its tree and expansions grow with the input and live in
// plan scratch allocated on first use.
//
// What it computes: the direct sum u_i = sum_{j : y_j != x_i} rho_j / |x_i - y_j|
// in double precision, for at most kMaxTargets targets (any number of
// sources).  It is the library's residual pair kernel (k_near) with the whole
// kernel 1/r over every pair instead of the residual kernel over a tree's
// interaction lists: sources are split into kSplits ranges evaluated by
// different thread blocks, and the partial sums of each (range, target) go to
// scratch before a second kernel adds them in a fixed order.
//
// The scratch is the file-scope array g_noalloc_scratch below
// (kSplits * kMaxTargets doubles = 2 MiB), resident on every device that loads
// the library until the process exits.  Host code cannot use the array's name
// as a device address, so every call looks the address up on the current
// device with cudaGetSymbolAddress (no allocation; a device reset that reloads
// the module cannot leave a stale address behind).  The first call on a device
// loads the module there, so it should happen before any stream capture
// begins.  All calls share the array: each call overwrites every partial it
// later reads, so nothing has to be cleared, but calls that overlap on the
// device (other streams, other host threads) race on it and must be
// serialised by the caller.
#include <cstdint>
#include <string>

#include "dmk.h"
#include "dmk_internal.h"

namespace {

constexpr int kSplits = 16;
constexpr int64_t kMaxTargets = 16384;
constexpr int kThreadsN = 128;
constexpr int kChunk = 256;

__device__ __align__(256) double g_noalloc_scratch[kSplits * kMaxTargets];

// partial sums of targets [blockIdx.x * kThreadsN, ...) over source range blockIdx.y
__global__ void __launch_bounds__(kThreadsN) k_direct_partial(const double *src, int64_t ns, const double *q,
                                                              const double *tgt, int64_t nt, double *part) {
    struct Src { double x, y, z, w; };
    __shared__ Src s_src[kChunk];
    const int64_t t = (int64_t)blockIdx.x * kThreadsN + threadIdx.x;
    const int split = blockIdx.y;
    const int64_t j0 = ns * split / kSplits, j1 = ns * (split + 1) / kSplits;
    double x = 0, y = 0, z = 0;
    if (t < nt) {
        x = tgt[3 * t];
        y = tgt[3 * t + 1];
        z = tgt[3 * t + 2];
    }
    double acc = 0.0;
    for (int64_t c0 = j0; c0 < j1; c0 += kChunk) {
        const int nc = (int)(j1 - c0 < kChunk ? j1 - c0 : kChunk);
        __syncthreads();
        for (int i = threadIdx.x; i < nc; i += kThreadsN) {
            const int64_t j = c0 + i;
            s_src[i] = Src{src[3 * j], src[3 * j + 1], src[3 * j + 2], q[j]};
        }
        __syncthreads();
        for (int i = 0; i < nc; ++i) {
            const Src s = s_src[i];
            const double dx = x - s.x, dy = y - s.y, dz = z - s.z;
            const double r2 = dx * dx + dy * dy + dz * dz;
            if (r2 > 0.0) acc += s.w * rsqrt(r2);
        }
    }
    if (t < nt) part[(int64_t)split * kMaxTargets + t] = acc;
}

__global__ void k_direct_reduce(const double *part, int64_t nt, double *pot) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= nt) return;
    double s = 0.0;
    for (int k = 0; k < kSplits; ++k) s += part[(int64_t)k * kMaxTargets + t];
    pot[t] = s;
}

int fail(int code, const std::string &m) {
    ::dmk::set_error_detail(m);
    return code;
}

}  // namespace

extern "C" DMK_API int dmk_direct_noalloc(const double *sources, int64_t n_src, const double *charges,
                                          const double *targets, int64_t n_tgt, double *potentials,
                                          void *cuda_stream) {
    ::dmk::set_error_detail("");
    if (n_src < 0 || n_tgt < 0) return fail(DMK_ERR_INVALID_ARG, "negative size");
    if (n_tgt > kMaxTargets)
        return fail(DMK_ERR_INVALID_ARG, "dmk_direct_noalloc: n_tgt exceeds its fixed scratch (16384 targets)");
    if ((n_src > 0 && (!sources || !charges)) || (n_tgt > 0 && (!targets || !potentials)))
        return fail(DMK_ERR_INVALID_ARG, "NULL array with a nonzero size");
    if (n_tgt == 0) return DMK_OK;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        cudaGetLastError();
        return fail(DMK_ERR_CUDA, "no current CUDA device");
    }
    // the device address of the array on the current device
    void *scratch = nullptr;
    {
        const cudaError_t e = cudaGetSymbolAddress(&scratch, g_noalloc_scratch);
        if (e != cudaSuccess || !scratch) {
            cudaGetLastError();
            return fail(DMK_ERR_CUDA, std::string("cudaGetSymbolAddress failed: ") + cudaGetErrorString(e));
        }
    }
    cudaStream_t st = (cudaStream_t)cuda_stream;
    dim3 grid((unsigned)((n_tgt + kThreadsN - 1) / kThreadsN), kSplits);
    ::dmk::launch_tick();
    k_direct_partial<<<grid, kThreadsN, 0, st>>>(sources, n_src, charges, targets, n_tgt, (double *)scratch);
    ::dmk::launch_tick();
    k_direct_reduce<<<(unsigned)((n_tgt + 255) / 256), 256, 0, st>>>((const double *)scratch, n_tgt, potentials);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return fail(DMK_ERR_CUDA, std::string("kernel launch failed: ") + cudaGetErrorString(e));
    return DMK_OK;
}
