// api.cu -- the C ABI of libdmk (include/dmk.h): plan construction (Step 1 of
// Sec. 3.4), one evaluation pass (Steps 0 and 2-5), statistics and tree export.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <memory>
#include <new>
#include <string>

#include "dmk.h"
#include "log2d.h"
#include "passes.h"

namespace dmk {
std::atomic<long long> g_launches{0};
}

namespace {
thread_local std::string g_detail;
}

namespace dmk {
// lets entry points defined in other translation units report a detail
void set_error_detail(const std::string &m) { g_detail = m; }
}

namespace {

int fail(int code, const std::string &msg) {
    g_detail = msg;
    return code;
}
}  // namespace

// plans carry this word while they live; an entry point handed anything
// else (a destroyed or foreign handle) refuses it instead of reading through it
constexpr uint64_t kPlanMagic = 0x646d6b2d706c616eull;

struct dmk_plan_s {
    uint64_t magic = kPlanMagic;
    int kernel = 0, dim = 3;
    double eps = 0;
    dmk_opts opts{};
    dmk::Tables tb;
    bool host_only = false;
    int device = 0;
    int precision = 0;
    int leaf_cap = 280, max_level = 20;
    int qdeg = 0;
    int gdeg_f32 = 0;           // DMK_LOG2D: degree of G's series on the FP32 near field
    double lambda = 0.0;        // Yukawa parameter (input units), 0 for Laplace
    dmk::YukawaTables yt;       // Yukawa tables at the last unit-box lambda
    dmk::Workspace ws;
    dmk::DBuf ytab;             // their device copy (working precision)
    dmk::DBuf tab;  // device tables (working precision)
    dmk::DevTables<double> dt_d{};
    dmk::DevTables<float> dt_f{};
    // the 2D Laplace kernel log r
    dmk::Log2dTables t2;
    dmk::DBuf tab2;
    dmk::Log2dDev d2{};
    dmk::Log2dBufs b2;
    std::unique_ptr<dmk::TreeBuilder> tree;
    dmk::PassBufs bufs;
    dmk::DBuf h_src, h_q, h_tgt, h_pot;  // device copies for dmk_eval_host
    dmk_eval_stats stats{};
    cudaEvent_t ev[8] = {};
    // the near field runs on an internal low-priority stream, concurrently with
    // the far field on the caller's stream: its short blocks fill the SMs that
    // the per-level far-field launches leave idle
    cudaStream_t side = nullptr;
    cudaEvent_t fork = nullptr, join = nullptr, nev[2] = {};
    bool events = false;
    size_t smem_limit = 0;
    int num_sms = 0;
    ~dmk_plan_s() {
        magic = 0;
        if (events) {
            for (auto &e : ev) cudaEventDestroy(e);
            for (auto &e : nev) cudaEventDestroy(e);
            cudaEventDestroy(fork);
            cudaEventDestroy(join);
        }
        if (side) cudaStreamDestroy(side);
    }
};

namespace {

// a live plan handle: a destroyed or foreign pointer is refused, not used
bool bad_plan(const dmk_plan_s *plan) { return !plan || plan->magic != kPlanMagic; }

template <typename T>
int upload_tables(dmk_plan_s *pl, dmk::DevTables<T> &dt) {
    const dmk::Tables &tb = pl->tb;
    const int p = tb.p, nf = tb.nf, N1 = 2 * nf + 1, n0 = tb.n0, NW = 2 * n0 + 1;
    std::vector<T> h;
    auto push = [&](const std::vector<double> &v) {
        size_t off = h.size();
        for (double x : v) h.push_back((T)x);
        while (h.size() % 32) h.push_back((T)0);
        return off;
    };
    std::vector<double> A2(tb.A[0]);
    A2.insert(A2.end(), tb.A[1].begin(), tb.A[1].end());
    size_t oA = push(A2), oFr = push(tb.Fr), oFi = push(tb.Fi), oFWr = push(tb.FWr), oFWi = push(tb.FWi);
    size_t ow = push(tb.w), owW = push(tb.wW), oq = push(tb.qmono);
    if (pl->ws.ensure(pl->tab, (int64_t)h.size() * sizeof(T))) return fail(DMK_ERR_OOM, "device allocation failed (tables)");
    if (cudaMemcpy(pl->tab.p, h.data(), h.size() * sizeof(T), cudaMemcpyHostToDevice) != cudaSuccess)
        return fail(DMK_ERR_CUDA, "copying the plan tables to the device failed");
    const T *base = (const T *)pl->tab.p;
    dt.p = p;
    dt.nf = nf;
    dt.N1 = N1;
    dt.nh = nf + 1;
    dt.n0 = n0;
    dt.NW = NW;
    dt.nhW = n0 + 1;
    dt.qdeg = (int)tb.qmono.size() - 1;
    dt.A = base + oA;
    dt.Fr = base + oFr;
    dt.Fi = base + oFi;
    dt.FWr = base + oFWr;
    dt.FWi = base + oFWi;
    dt.w = base + ow;
    dt.wW = base + owW;
    dt.qmono = base + oq;
    return DMK_OK;
}

// per-evaluation tables of the Yukawa kernel at the unit-box lambda S
template <typename T>
int upload_yukawa(dmk_plan_s *pl, dmk::DevTables<T> &dt, double lam_unit, int nlev) {
    if (pl->yt.lam != lam_unit || pl->yt.nlev < nlev) {
        std::string err;
        if (dmk::build_yukawa_tables(pl->tb, lam_unit, nlev, pl->yt, err) != 0)
            return fail(DMK_ERR_UNSUPPORTED, err);
        std::vector<T> h;
        auto push = [&](const std::vector<double> &v) {
            size_t off = h.size();
            for (double x : v) h.push_back((T)x);
            while (h.size() % 32) h.push_back((T)0);
            return off;
        };
        const size_t ow = push(pl->yt.wl), oW = push(pl->yt.wW), oq = push(pl->yt.qmono);
        if (pl->ws.ensure(pl->ytab, (int64_t)h.size() * sizeof(T)))
            return fail(DMK_ERR_OOM, "device allocation failed (Yukawa tables)");
        if (cudaMemcpy(pl->ytab.p, h.data(), h.size() * sizeof(T), cudaMemcpyHostToDevice) != cudaSuccess)
            return fail(DMK_ERR_CUDA, "copying the Yukawa tables to the device failed");
        const T *base = (const T *)pl->ytab.p;
        dt.wl = base + ow;
        dt.wW = base + oW;
        dt.ql = base + oq;
        dt.lam = (T)lam_unit;
        dt.qdeg = pl->yt.qdeg;
    }
    return DMK_OK;
}

// The degree at which the FP32 near field of a DMK_LOG2D plan cuts G's
// Chebyshev series: where the tail stays below 1e-2 eps max(1, |G|) (FP32
// cannot resolve more), at least 3.
static int log2d_f32_degree(const std::vector<double> &gc, double eps) {
    double gmax = 1.0;
    for (int j = 0; j <= 256; ++j) {
        const double x = -1.0 + j / 128.0;
        double b1 = 0.0, b2 = 0.0;
        for (int k = (int)gc.size() - 1; k >= 1; --k) {
            const double b0 = 2.0 * x * b1 - b2 + gc[k];
            b2 = b1;
            b1 = b0;
        }
        gmax = std::max(gmax, std::fabs(x * b1 - b2 + gc[0]));
    }
    int d = (int)gc.size() - 1;
    for (double tail = 0.0; d > 3 && tail + std::fabs(gc[d]) <= 1e-2 * eps * gmax; --d) tail += std::fabs(gc[d]);
    return d;
}

int upload_log2d(dmk_plan_s *pl) {
    const dmk::Tables &tb = pl->tb;
    std::vector<double> h;
    auto push = [&](const std::vector<double> &v) {
        size_t off = h.size();
        h.insert(h.end(), v.begin(), v.end());
        while (h.size() % 32) h.push_back(0.0);
        return off;
    };
    std::vector<double> A2(tb.A[0]);
    A2.insert(A2.end(), tb.A[1].begin(), tb.A[1].end());
    const std::vector<double> &gv = pl->t2.gmono.empty() ? pl->t2.g : pl->t2.gmono;
    // Tang's table-driven log for the residual kernel: t = m 2^e, m in [1, 2),
    // log m = -log F_k + log1p(m F_k - 1) for the leading 8 fraction bits k of m.
    // F_k is any double near 1 / (1 + (k + 1/2) / 256); -log F_k is taken for the
    // stored F_k, in extended precision and rounded once.
    std::vector<double> lgF(256), lgL(256), lgE(256);
    for (int k = 0; k < 256; ++k) {
        lgF[k] = 1.0 / (1.0 + (k + 0.5) / 256.0);
        lgL[k] = (double)(-0.5L * std::log((long double)lgF[k]));
        lgE[k] = (double)((long double)gv[0] - 0.5L * (long double)k * std::log(2.0L));
    }
    const size_t oA = push(A2), oFr = push(tb.Fr), oFi = push(tb.Fi), oFWr = push(pl->t2.FWr),
                 oFWi = push(pl->t2.FWi), ow = push(pl->t2.w), owW = push(pl->t2.wW), og = push(gv),
                 olF = push(lgF), olL = push(lgL), olE = push(lgE);
    // The Chebyshev coefficients of G for the FP32 near field (degree
    // gdeg_f32), rounded to FP32, zero-padded at the top to groups of four (zero
    // leading coefficients leave Clenshaw's recurrence unchanged), packed two
    // to a double slot.
    const std::vector<double> &gc = pl->t2.g;
    const int gdeg_f = pl->gdeg_f32;
    std::vector<float> gcf((gdeg_f / 4 + 1) * 4, 0.0f);
    for (int k = 0; k <= gdeg_f; ++k) gcf[k] = (float)gc[k];
    std::vector<double> gcf_words(gcf.size() / 2, 0.0);
    memcpy(gcf_words.data(), gcf.data(), gcf.size() * sizeof(float));
    const size_t ogc = push(gcf_words);
    if (pl->ws.ensure(pl->tab2, (int64_t)h.size() * 8)) return fail(DMK_ERR_OOM, "device allocation failed (tables)");
    if (cudaMemcpy(pl->tab2.p, h.data(), h.size() * 8, cudaMemcpyHostToDevice) != cudaSuccess)
        return fail(DMK_ERR_CUDA, "copying the plan tables to the device failed");
    const double *base = (const double *)pl->tab2.p;
    dmk::Log2dDev &d = pl->d2;
    d.p = tb.p;
    d.nf = tb.nf;
    d.N1 = 2 * tb.nf + 1;
    d.n0 = pl->t2.n0;
    d.NW = 2 * pl->t2.n0 + 1;
    d.gdeg = (int)pl->t2.g.size() - 1;
    d.gmono = pl->t2.gmono.empty() ? 0 : 1;
    d.A = base + oA;
    d.Fr = base + oFr;
    d.Fi = base + oFi;
    d.FWr = base + oFWr;
    d.FWi = base + oFWi;
    d.w = base + ow;
    d.wW = base + owW;
    d.g = base + og;
    d.lgF = base + olF;
    d.lgL = base + olL;
    d.lgE = base + olE;
    d.G0 = pl->t2.G0;
    d.mixed = pl->precision == DMK_MIXED ? 1 : 0;
    d.gcf = (const float *)(base + ogc);
    d.gcdeg = gdeg_f;
    d.gcn4 = (int)gcf.size() / 4;
    return DMK_OK;
}

// one evaluation of the 2D pass (after the empty cases and cudaSetDevice)
int eval_log2d(dmk_plan_s *pl, const double *src, int64_t ns, const double *q, const double *tgt, int64_t nt,
               double *pot, cudaStream_t st) {
    if (!pl->tree) pl->tree.reset(new dmk::TreeBuilder(pl->ws));
    std::string err;
    const long long launches0 = dmk::g_launches.load();
    cudaEventRecord(pl->ev[0], st);
    int rc = dmk::run_log2d(pl->d2, *pl->tree, pl->ws, pl->b2, src, ns, q, tgt, nt, pl->leaf_cap, pl->max_level,
                            pot, st, pl->nev, err);
    if (rc) return fail(rc, "2D pass: " + err);
    cudaEventRecord(pl->ev[5], st);
    cudaError_t ce = cudaStreamSynchronize(st);
    if (ce != cudaSuccess) return fail(DMK_ERR_CUDA, std::string("device execution failed: ") + cudaGetErrorString(ce));
    ce = cudaGetLastError();
    if (ce != cudaSuccess) return fail(DMK_ERR_CUDA, std::string("kernel launch failed: ") + cudaGetErrorString(ce));
    dmk_eval_stats &s = pl->stats;
    s = dmk_eval_stats{};
    s.n_points = pl->tree->n;
    s.n_levels = pl->tree->nlev;
    s.n_boxes = pl->tree->nb;
    s.n_leaves = pl->tree->nleaves;
    s.near_pairs = pl->tree->near_pairs;
    s.balance_rounds = pl->tree->rounds;
    s.n_fin = pl->tree->nfin;
    float t05 = 0, tn = 0;
    cudaEventElapsedTime(&t05, pl->ev[0], pl->ev[5]);
    s.t_total_ms = t05;
    if (cudaEventElapsedTime(&tn, pl->nev[0], pl->nev[1]) == cudaSuccess) s.t_near_ms = tn;
    else cudaGetLastError();
    s.n_launches = dmk::g_launches.load() - launches0;
    if (pl->tree->ntleaves > 0 && pl->b2.cnt.p) {
        // every candidate pair is screened; the device counts those inside the support
        unsigned long long inside = 0;
        if (cudaMemcpy(&inside, pl->b2.cnt.p, 8, cudaMemcpyDeviceToHost) != cudaSuccess)
            return fail(DMK_ERR_CUDA, "reading the near-field counter failed");
        s.near_pairs_inside = (int64_t)inside;
        s.near_pairs_screened = s.near_pairs;
    }
    return DMK_OK;
}

bool valid_p(int p) { return p == 0 || p == 9 || p == 18 || p == 19 || p == 28 || p == 38; }

int eval_device(dmk_plan_s *pl, const double *src, int64_t ns, const double *q, const double *tgt, int64_t nt,
                double *pot, double *grad, cudaStream_t st, int nsys = 1, const int64_t *h_off = nullptr) {
    if (nt == 0) return DMK_OK;
    if (cudaSetDevice(pl->device) != cudaSuccess) return fail(DMK_ERR_CUDA, "cudaSetDevice failed");
    if (ns == 0) {
        if (cudaMemsetAsync(pot, 0, (size_t)nt * sizeof(double), st) != cudaSuccess ||
            (grad && cudaMemsetAsync(grad, 0, (size_t)nt * 3 * sizeof(double), st) != cudaSuccess) ||
            cudaStreamSynchronize(st) != cudaSuccess)
            return fail(DMK_ERR_CUDA, "clearing the potentials failed");
        pl->stats = dmk_eval_stats{};
        return DMK_OK;
    }
    const bool same = (tgt == src && nt == ns);
    const int64_t n = same ? ns : ns + nt;
    if (n >= (int64_t)INT32_MAX / 2) return fail(DMK_ERR_UNSUPPORTED, "more than 2^30 points");
    if (pl->kernel == DMK_LOG2D) {
        if (grad) return fail(DMK_ERR_UNSUPPORTED, "the 2D kernel has no gradient pass");
        if (nsys > 1) return fail(DMK_ERR_UNSUPPORTED, "the 2D kernel has no batched pass");
        return eval_log2d(pl, src, ns, q, tgt, nt, pot, st);
    }
    if (!pl->tree) pl->tree.reset(new dmk::TreeBuilder(pl->ws));
    std::string err;
    const bool single = pl->precision == DMK_MIXED;
    const long long launches0 = dmk::g_launches.load();
    cudaEventRecord(pl->ev[0], st);
    int rc = pl->tree->build(src, ns, q, same ? nullptr : tgt, same ? 0 : nt, same, pl->leaf_cap, pl->max_level,
                             single ? 1 : 0, st, err, nsys, h_off);
    if (rc) return fail(rc, "tree: " + err);
    if (pl->kernel == DMK_YUKAWA) {
        if (nsys > 1) return fail(DMK_ERR_UNSUPPORTED, "Yukawa batches: every system has its own lambda S");
        if (grad) return fail(DMK_ERR_UNSUPPORTED, "the Yukawa kernel has no gradient pass");
        // exp(-lambda |x - y|) = exp(-(lambda S) |u - v|) in the unit box
        const double lam_unit = pl->lambda * pl->tree->h_frame.S;
        rc = single ? upload_yukawa<float>(pl, pl->dt_f, lam_unit, pl->tree->nlev)
                    : upload_yukawa<double>(pl, pl->dt_d, lam_unit, pl->tree->nlev);
        if (rc) return rc;
    }
    dmk::PassCtx cx{};
    cx.tree = pl->tree.get();
    cx.bufs = &pl->bufs;
    cx.ws = &pl->ws;
    cx.tables = single ? (const void *)&pl->dt_f : (const void *)&pl->dt_d;
    cx.single = single;
    cx.p = pl->tb.p;
    cx.mode = (pl->opts.flags & DMK_FLAG_FAR_ONLY) ? 1 : ((pl->opts.flags & DMK_FLAG_NEAR_ONLY) ? 2 : 0);
    cx.total_sources = ns;
    cx.pot = pot;
    cx.grad = grad;
    cx.st = st;
    for (int i = 0; i < 8; ++i) cx.ev[i] = pl->ev[i];
    cx.side = pl->side;
    cx.fork = pl->fork;
    cx.join = pl->join;
    cx.nev[0] = pl->nev[0];
    cx.nev[1] = pl->nev[1];
    cx.smem_limit = pl->smem_limit;
    cx.num_sms = pl->num_sms;
    rc = dmk::run_passes(cx, err);
    if (rc) {
        // a pass that failed to launch may leave near-field work queued
        cudaStreamSynchronize(pl->side);
        return fail(rc, "passes: " + err);
    }
    cudaEventRecord(pl->ev[5], st);
    cudaError_t ce = cudaStreamSynchronize(st);
    if (ce != cudaSuccess) return fail(DMK_ERR_CUDA, std::string("device execution failed: ") + cudaGetErrorString(ce));
    ce = cudaGetLastError();
    if (ce != cudaSuccess) return fail(DMK_ERR_CUDA, std::string("kernel launch failed: ") + cudaGetErrorString(ce));
    dmk_eval_stats &s = pl->stats;
    s = dmk_eval_stats{};
    s.n_points = n;
    s.n_levels = pl->tree->nlev;
    s.n_boxes = pl->tree->nb;
    s.n_leaves = pl->tree->nleaves;
    s.near_pairs = pl->tree->near_pairs;
    s.balance_rounds = pl->tree->rounds;
    s.n_fout = pl->tree->root_leaf ? 0 : pl->tree->nslots;
    s.n_fin = pl->tree->nfin;
    float t01 = 0, t12 = 0, t23 = 0, t34 = 0, t05 = 0;
    cudaEventElapsedTime(&t01, pl->ev[0], pl->ev[1]);
    cudaEventElapsedTime(&t12, pl->ev[1], pl->ev[2]);
    cudaEventElapsedTime(&t23, pl->ev[2], pl->ev[3]);
    cudaEventElapsedTime(&t34, pl->ev[3], pl->ev[4]);
    cudaEventElapsedTime(&t05, pl->ev[0], pl->ev[5]);
    s.t_tree_ms = t01;
    s.t_upward_ms = t12;
    s.t_downward_ms = t23;
    s.t_near_ms = t34;
    s.t_total_ms = t05;
    float t63 = 0, tn = 0, t76 = 0;
    cudaEventElapsedTime(&t63, pl->ev[6], pl->ev[3]);
    s.t_local_ms = t63;
    if (cudaEventElapsedTime(&t76, pl->ev[7], pl->ev[6]) == cudaSuccess) s.t_incoming_ms = t76;
    else cudaGetLastError();
    float t27 = 0;
    if (cudaEventElapsedTime(&t27, pl->ev[2], pl->ev[7]) == cudaSuccess) s.t_planewave_ms = t27;
    else cudaGetLastError();
    // the near field ran on the side stream, overlapping the far field
    if (cudaEventElapsedTime(&tn, pl->nev[0], pl->nev[1]) == cudaSuccess) s.t_near_ms = tn;
    else cudaGetLastError();
    s.n_launches = dmk::g_launches.load() - launches0;
    if (pl->bufs.counter.p) {
        // device words: [0] near work queue, [8] near pairs inside R_L,
        // [16] local-pass flops, [24] a tensor-core or TMA wait that gave up,
        // [32] colleague arrays read by the incoming pass, [40] pairs screened
        // by the near field
        unsigned char w[48] = {0};
        if (cudaMemcpy(w, pl->bufs.counter.p, sizeof(w), cudaMemcpyDeviceToHost) != cudaSuccess)
            return fail(DMK_ERR_CUDA, "reading the device status words failed");
        unsigned long long inside = 0, f = 0, reads = 0;
        int timeout = 0;
        memcpy(&inside, w + 8, 8);
        memcpy(&f, w + 16, 8);
        memcpy(&timeout, w + 24, 4);
        memcpy(&reads, w + 32, 8);
        unsigned long long screened = 0;
        memcpy(&screened, w + 40, 8);
        if (pl->tree->ntleaves > 0) {
            s.near_pairs_inside = (int64_t)inside;
            s.near_pairs_screened = (int64_t)screened;
        }
        s.local_flops = (int64_t)f;
        if (s.t_incoming_ms > 0.f || reads > 0) {
            const int64_t P = pl->tb.p, NH = pl->tb.nf + 1, N1 = 2 * pl->tb.nf + 1;
            s.incoming_reads = (int64_t)reads;
            s.incoming_flops = 8 * N1 * N1 * NH * (int64_t)reads +
                               s.n_fin * (8 * P * NH * NH * NH + 4 * P * P * NH * NH + 2 * P * P * P * NH);
        }
        if (timeout) return fail(DMK_ERR_TIMEOUT, "a tensor-core completion wait gave up (local pass)");
    }
    return DMK_OK;
}

}  // namespace

extern "C" {

const char *dmk_error_string(int code) {
    switch (code) {
    case DMK_OK: return "success";
    case DMK_ERR_INVALID_ARG: return "invalid argument";
    case DMK_ERR_UNSUPPORTED: return "unsupported kernel, dimension or option";
    case DMK_ERR_OOM: return "out of memory";
    case DMK_ERR_CUDA: return "CUDA error";
    case DMK_ERR_TIMEOUT: return "device wait timed out";
    case DMK_ERR_DEPTH: return "tree depth limit exceeded";
    case DMK_ERR_INTERNAL: return "internal error";
    default: return "unknown status code";
    }
}

const char *dmk_last_error_detail(void) { return g_detail.c_str(); }

int dmk_plan(dmk_kernel kernel, int dim, double eps, const dmk_opts *opts, dmk_plan_t *out) {
    g_detail.clear();
    if (!out) return fail(DMK_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    if (!(eps >= 1e-12 && eps <= 1e-2)) return fail(DMK_ERR_INVALID_ARG, "eps must lie in [1e-12, 1e-2]");
    if (kernel != DMK_LAPLACE && kernel != DMK_YUKAWA && kernel != DMK_LOG2D)
        return fail(DMK_ERR_UNSUPPORTED, "only DMK_LAPLACE, DMK_YUKAWA (3D) and DMK_LOG2D (2D) are implemented");
    if (dim != (kernel == DMK_LOG2D ? 2 : 3))
        return fail(DMK_ERR_UNSUPPORTED, "DMK_LAPLACE and DMK_YUKAWA are 3D kernels, DMK_LOG2D a 2D one");
    dmk_opts o{};
    if (opts) o = *opts;
    if (kernel == DMK_YUKAWA && !(o.kernel_param > 0.0 && std::isfinite(o.kernel_param)))
        return fail(DMK_ERR_INVALID_ARG, "DMK_YUKAWA needs kernel_param = lambda > 0");
    if (o.leaf_cap < 0 || o.precision < 0 || o.precision > 1 || o.max_level < 0 || o.max_level > dmk::kMaxLevel ||
        o.nf < 0 || o.nf > dmk::kMaxNf || !valid_p(o.p) || (o.flags & ~7))
        return fail(DMK_ERR_INVALID_ARG, "option out of range");
    if ((o.flags & DMK_FLAG_FAR_ONLY) && (o.flags & DMK_FLAG_NEAR_ONLY))
        return fail(DMK_ERR_INVALID_ARG, "DMK_FLAG_FAR_ONLY and DMK_FLAG_NEAR_ONLY are exclusive");
    if (kernel == DMK_LOG2D && (o.flags & (DMK_FLAG_FAR_ONLY | DMK_FLAG_NEAR_ONLY)))
        return fail(DMK_ERR_UNSUPPORTED, "the 2D pass evaluates both parts");
    std::unique_ptr<dmk_plan_s> pl(new (std::nothrow) dmk_plan_s());
    if (!pl) return fail(DMK_ERR_OOM, "host allocation failed");
    pl->kernel = kernel;
    pl->lambda = kernel == DMK_YUKAWA ? o.kernel_param : 0.0;
    pl->dim = dim;
    pl->eps = eps;
    pl->opts = o;
    pl->precision = o.precision;
    // the paper's leaf capacities: 280 / 800 in 3D, 120 / 160 in 2D (Sec. 5.1)
    if (kernel == DMK_LOG2D)
        pl->leaf_cap = o.leaf_cap > 0 ? o.leaf_cap : (eps >= 1e-6 * (1 - 1e-12) ? 120 : 160);
    else
        pl->leaf_cap = o.leaf_cap > 0 ? o.leaf_cap : (eps >= 1e-6 * (1 - 1e-12) ? 280 : 800);
    pl->max_level = o.max_level > 0 ? o.max_level : dmk::kMaxLevel;
    std::string err;
    // Single precision cannot deliver eps below ~1e-7.  At the 1e-6 row of
    // Table 1 the method error of p = 18 alone reaches ~0.5-1e-6 on clustered
    // clouds, so the mixed path takes p = 19 to leave room for its rounding.
    if (o.precision == DMK_MIXED && eps < 1e-7) return fail(DMK_ERR_UNSUPPORTED, "DMK_MIXED needs eps >= 1e-7");
    int p_req = o.p;
    if (p_req == 0 && o.precision == DMK_MIXED && kernel != DMK_LOG2D && eps < 1e-3 * (1 - 1e-12)) p_req = 19;
    // the Yukawa kernel at the 1e-6 row: p = 18 leaves its far field at ~1.0 eps
    // (lambda S = 10, uniform points), p = 19 at ~0.8 eps
    if (p_req == 0 && kernel == DMK_YUKAWA && eps < 1e-3 * (1 - 1e-12) && eps >= 1e-6 * (1 - 1e-12)) p_req = 19;
    // log r in 2D at the 1e-6 row: p = 18 leaves uniform disks at up to 1.08 eps
    // (3000 points, the oracle), p = 19 at 0.74 eps
    if (p_req == 0 && kernel == DMK_LOG2D && eps < 1e-3 * (1 - 1e-12) && eps >= 1e-6 * (1 - 1e-12)) p_req = 19;
    if (dmk::build_tables(eps, p_req, o.nf, pl->tb, err) != 0) return fail(DMK_ERR_UNSUPPORTED, err);
    pl->qdeg = (int)pl->tb.qmono.size() - 1;
    if (kernel == DMK_LOG2D) {
        if (dmk::build_log2d_tables(pl->tb, pl->t2, err) != 0) return fail(DMK_ERR_UNSUPPORTED, err);
        if (pl->t2.g.size() > 64) return fail(DMK_ERR_INTERNAL, "2D residual polynomial degree above 63");
        pl->gdeg_f32 = log2d_f32_degree(pl->t2.g, eps);
    }
    if (pl->qdeg >= 64) return fail(DMK_ERR_INTERNAL, "residual polynomial degree above 63");
    pl->host_only = (o.flags & DMK_FLAG_HOST_ONLY) != 0;
    if (!pl->host_only) {
        if (cudaGetDevice(&pl->device) != cudaSuccess) {
            cudaGetLastError();
            return fail(DMK_ERR_CUDA, "no CUDA device available");
        }
        int smem = 0, sms = 0;
        if (cudaDeviceGetAttribute(&smem, cudaDevAttrMaxSharedMemoryPerBlockOptin, pl->device) != cudaSuccess ||
            cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, pl->device) != cudaSuccess) {
            cudaGetLastError();
            return fail(DMK_ERR_CUDA, "querying the device failed");
        }
        pl->smem_limit = (size_t)smem;
        pl->num_sms = sms;
        for (auto &e : pl->ev)
            if (cudaEventCreate(&e) != cudaSuccess) return fail(DMK_ERR_CUDA, "cudaEventCreate failed");
        for (auto &e : pl->nev)
            if (cudaEventCreate(&e) != cudaSuccess) return fail(DMK_ERR_CUDA, "cudaEventCreate failed");
        if (cudaEventCreateWithFlags(&pl->fork, cudaEventDisableTiming) != cudaSuccess ||
            cudaEventCreateWithFlags(&pl->join, cudaEventDisableTiming) != cudaSuccess)
            return fail(DMK_ERR_CUDA, "cudaEventCreate failed");
        pl->events = true;
        int least = 0, greatest = 0;
        if (cudaDeviceGetStreamPriorityRange(&least, &greatest) != cudaSuccess) {
            cudaGetLastError();
            least = 0;
        }
        if (cudaStreamCreateWithPriority(&pl->side, cudaStreamNonBlocking, least) != cudaSuccess)
            return fail(DMK_ERR_CUDA, "cudaStreamCreate failed");
        int rc = kernel == DMK_LOG2D           ? upload_log2d(pl.get())
                 : pl->precision == DMK_MIXED ? upload_tables<float>(pl.get(), pl->dt_f)
                                              : upload_tables<double>(pl.get(), pl->dt_d);
        if (rc) return rc;
    }
    *out = pl.release();
    return DMK_OK;
}

int dmk_plan_destroy(dmk_plan_t plan) {
    if (!plan) return DMK_OK;
    if (bad_plan(plan)) return fail(DMK_ERR_INVALID_ARG, "not a live plan handle");
    delete plan;
    return DMK_OK;
}

int dmk_eval(dmk_plan_t plan, const double *sources, int64_t n_src, const double *charges, const double *targets,
             int64_t n_tgt, double *potentials, void *cuda_stream) {
    g_detail.clear();
    if (bad_plan(plan)) return fail(DMK_ERR_INVALID_ARG, "plan is NULL or not a live plan handle");
    if (plan->host_only) return fail(DMK_ERR_INVALID_ARG, "plan was built with DMK_FLAG_HOST_ONLY");
    if (n_src < 0 || n_tgt < 0) return fail(DMK_ERR_INVALID_ARG, "negative size");
    if ((n_src > 0 && (!sources || !charges)) || (n_tgt > 0 && (!targets || !potentials)))
        return fail(DMK_ERR_INVALID_ARG, "NULL array with a nonzero size");
    return eval_device(plan, sources, n_src, charges, targets, n_tgt, potentials, nullptr,
                       (cudaStream_t)cuda_stream);
}

int dmk_eval_grad(dmk_plan_t plan, const double *sources, int64_t n_src, const double *charges,
                  const double *targets, int64_t n_tgt, double *potentials, double *gradients, void *cuda_stream) {
    g_detail.clear();
    if (bad_plan(plan)) return fail(DMK_ERR_INVALID_ARG, "plan is NULL or not a live plan handle");
    if (plan->host_only) return fail(DMK_ERR_INVALID_ARG, "plan was built with DMK_FLAG_HOST_ONLY");
    if (n_src < 0 || n_tgt < 0) return fail(DMK_ERR_INVALID_ARG, "negative size");
    if ((n_src > 0 && (!sources || !charges)) || (n_tgt > 0 && (!targets || !potentials || !gradients)))
        return fail(DMK_ERR_INVALID_ARG, "NULL array with a nonzero size");
    return eval_device(plan, sources, n_src, charges, targets, n_tgt, potentials, gradients,
                       (cudaStream_t)cuda_stream);
}

int dmk_eval_batch(dmk_plan_t plan, const double *points, const double *charges, const int64_t *offsets,
                   int n_systems, double *potentials, void *cuda_stream) {
    g_detail.clear();
    if (bad_plan(plan)) return fail(DMK_ERR_INVALID_ARG, "plan is NULL or not a live plan handle");
    if (plan->host_only) return fail(DMK_ERR_INVALID_ARG, "plan was built with DMK_FLAG_HOST_ONLY");
    if (!offsets || n_systems < 1 || n_systems > (1 << 24))
        return fail(DMK_ERR_INVALID_ARG, "n_systems must lie in 1..2^24 with an offsets array");
    if (offsets[0] != 0) return fail(DMK_ERR_INVALID_ARG, "offsets[0] must be 0");
    for (int s = 0; s < n_systems; ++s)
        if (offsets[s + 1] < offsets[s]) return fail(DMK_ERR_INVALID_ARG, "offsets must not decrease");
    const int64_t total = offsets[n_systems];
    if (total == 0) return DMK_OK;
    if (!points || !charges || !potentials) return fail(DMK_ERR_INVALID_ARG, "NULL array with a nonzero size");
    return eval_device(plan, points, total, charges, points, total, potentials, nullptr, (cudaStream_t)cuda_stream,
                       n_systems, offsets);
}

int dmk_eval_host(dmk_plan_t plan, const double *sources, int64_t n_src, const double *charges,
                  const double *targets, int64_t n_tgt, double *potentials, void *cuda_stream) {
    g_detail.clear();
    if (bad_plan(plan)) return fail(DMK_ERR_INVALID_ARG, "plan is NULL or not a live plan handle");
    if (plan->host_only) return fail(DMK_ERR_INVALID_ARG, "plan was built with DMK_FLAG_HOST_ONLY");
    if (n_src < 0 || n_tgt < 0) return fail(DMK_ERR_INVALID_ARG, "negative size");
    if ((n_src > 0 && (!sources || !charges)) || (n_tgt > 0 && (!targets || !potentials)))
        return fail(DMK_ERR_INVALID_ARG, "NULL array with a nonzero size");
    if (n_tgt == 0) return DMK_OK;
    cudaStream_t st = (cudaStream_t)cuda_stream;
    if (cudaSetDevice(plan->device) != cudaSuccess) return fail(DMK_ERR_CUDA, "cudaSetDevice failed");
    const bool same = (targets == sources && n_tgt == n_src);
    dmk::Workspace &ws = plan->ws;
    const int64_t bpp = 8 * plan->dim;  // bytes per point
    if (ws.ensure(plan->h_src, std::max<int64_t>(n_src, 1) * bpp) || ws.ensure(plan->h_q, std::max<int64_t>(n_src, 1) * 8) ||
        ws.ensure(plan->h_pot, n_tgt * 8) || (!same && ws.ensure(plan->h_tgt, n_tgt * bpp)))
        return fail(DMK_ERR_OOM, "device allocation failed (host-call buffers)");
    if (n_src > 0 &&
        (cudaMemcpyAsync(plan->h_src.p, sources, (size_t)(n_src * bpp), cudaMemcpyHostToDevice, st) != cudaSuccess ||
         cudaMemcpyAsync(plan->h_q.p, charges, (size_t)n_src * 8, cudaMemcpyHostToDevice, st) != cudaSuccess))
        return fail(DMK_ERR_CUDA, "host-to-device copy failed");
    if (!same && cudaMemcpyAsync(plan->h_tgt.p, targets, (size_t)(n_tgt * bpp), cudaMemcpyHostToDevice, st) != cudaSuccess)
        return fail(DMK_ERR_CUDA, "host-to-device copy failed");
    const double *dsrc = (const double *)plan->h_src.p;
    const double *dtgt = same ? dsrc : (const double *)plan->h_tgt.p;
    int rc = eval_device(plan, dsrc, n_src, (const double *)plan->h_q.p, dtgt, n_tgt, (double *)plan->h_pot.p,
                         nullptr, st);
    if (rc) return rc;
    if (cudaMemcpyAsync(potentials, plan->h_pot.p, (size_t)n_tgt * 8, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
        return fail(DMK_ERR_CUDA, "device-to-host copy failed");
    return DMK_OK;
}

}  // extern "C"

namespace {
// out[i][d] = w1[i] g1[i][d] + w2[i] g2[i][d], either term absent when its
// weight pointer is null
__global__ void k_adjoint_combine(int64_t n, const double *w1, const double *g1, const double *w2,
                                  const double *g2, double *out) {
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= 3 * n) return;
    const int64_t i = k / 3;
    double v = 0.0;
    if (w1) v += w1[i] * g1[k];
    if (w2) v += w2[i] * g2[k];
    out[k] = v;
}
}  // namespace

extern "C" {

int dmk_adjoint_combine(int64_t n, const double *w1, const double *g1, const double *w2, const double *g2,
                        double *out, void *cuda_stream) {
    g_detail.clear();
    if (n < 0) return fail(DMK_ERR_INVALID_ARG, "negative size");
    if (n == 0) return DMK_OK;
    if (!out || (w1 && !g1) || (w2 && !g2)) return fail(DMK_ERR_INVALID_ARG, "NULL array with a nonzero size");
    if (n > ((int64_t)1 << 40)) return fail(DMK_ERR_INVALID_ARG, "n too large");
    ::dmk::launch_tick();
    k_adjoint_combine<<<(unsigned)((3 * n + 255) / 256), 256, 0, (cudaStream_t)cuda_stream>>>(n, w1, g1, w2, g2,
                                                                                             out);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return fail(DMK_ERR_CUDA, std::string("launch failed: ") + cudaGetErrorString(e));
    return DMK_OK;
}

}  // extern "C"

namespace {
// time plan evaluations at each candidate leaf capacity; keep the fastest
template <typename Eval>
int tune_leaf_cap(dmk_plan_s *plan, const int *candidates, int n_candidates, int reps, int *best_leaf_cap,
                  float *times_ms, Eval eval) {
    // the default candidates bracket the balance point of Sec. 5.1.1: the near
    // field grows linearly with the cap, the far field with the number of boxes
    static const int kDefault[] = {64, 100, 140, 200, 280, 400, 560};
    const int *cand = candidates ? candidates : kDefault;
    const int nc = candidates ? n_candidates : (int)(sizeof(kDefault) / sizeof(kDefault[0]));
    if (nc <= 0 || nc > 64) return fail(DMK_ERR_INVALID_ARG, "n_candidates must lie in 1..64");
    for (int i = 0; i < nc; ++i)
        if (cand[i] <= 0 || cand[i] > (1 << 20)) return fail(DMK_ERR_INVALID_ARG, "leaf cap out of range");
    if (reps < 0 || reps > 100) return fail(DMK_ERR_INVALID_ARG, "reps must lie in 0..100");
    if (reps == 0) reps = 3;
    const int keep = plan->leaf_cap;
    int best = -1;
    float best_ms = 0;
    for (int i = 0; i < nc; ++i) {
        plan->leaf_cap = cand[i];
        // one untimed evaluation grows the scratch for this tree shape
        float t = 0;
        for (int r = 0; r <= reps; ++r) {
            const int rc = eval();
            if (rc) {
                plan->leaf_cap = keep;
                return rc;
            }
            if (r == 1 || (r > 1 && plan->stats.t_total_ms < t)) t = plan->stats.t_total_ms;
        }
        if (times_ms) times_ms[i] = t;
        if (best < 0 || t < best_ms) {
            best = i;
            best_ms = t;
        }
    }
    plan->leaf_cap = cand[best];
    if (best_leaf_cap) *best_leaf_cap = cand[best];
    return DMK_OK;
}
}  // namespace

extern "C" {

int dmk_tune_leaf_cap(dmk_plan_t plan, const double *sources, int64_t n_src, const double *charges,
                      const double *targets, int64_t n_tgt, const int *candidates, int n_candidates, int reps,
                      int *best_leaf_cap, float *times_ms, void *cuda_stream) {
    g_detail.clear();
    if (bad_plan(plan)) return fail(DMK_ERR_INVALID_ARG, "plan is NULL or not a live plan handle");
    if (plan->host_only) return fail(DMK_ERR_INVALID_ARG, "plan was built with DMK_FLAG_HOST_ONLY");
    if (n_src < 0 || n_tgt < 0) return fail(DMK_ERR_INVALID_ARG, "negative size");
    if ((n_src > 0 && (!sources || !charges)) || (n_tgt > 0 && !targets))
        return fail(DMK_ERR_INVALID_ARG, "NULL array with a nonzero size");
    if (plan->ws.ensure(plan->h_pot, std::max<int64_t>(n_tgt, 1) * 8))
        return fail(DMK_ERR_OOM, "device allocation failed (tuning)");
    double *pot = (double *)plan->h_pot.p;
    cudaStream_t st = (cudaStream_t)cuda_stream;
    return tune_leaf_cap(plan, candidates, n_candidates, reps, best_leaf_cap, times_ms, [&]() {
        return eval_device(plan, sources, n_src, charges, targets, n_tgt, pot, nullptr, st);
    });
}

int dmk_tune_leaf_cap_batch(dmk_plan_t plan, const double *points, const double *charges, const int64_t *offsets,
                            int n_systems, const int *candidates, int n_candidates, int reps, int *best_leaf_cap,
                            float *times_ms, void *cuda_stream) {
    g_detail.clear();
    if (bad_plan(plan)) return fail(DMK_ERR_INVALID_ARG, "plan is NULL or not a live plan handle");
    if (plan->host_only) return fail(DMK_ERR_INVALID_ARG, "plan was built with DMK_FLAG_HOST_ONLY");
    if (!offsets || n_systems < 1 || n_systems > (1 << 24) || offsets[0] != 0)
        return fail(DMK_ERR_INVALID_ARG, "n_systems must lie in 1..2^24 with offsets from 0");
    for (int s = 0; s < n_systems; ++s)
        if (offsets[s + 1] < offsets[s]) return fail(DMK_ERR_INVALID_ARG, "offsets must not decrease");
    const int64_t total = offsets[n_systems];
    if (total > 0 && (!points || !charges)) return fail(DMK_ERR_INVALID_ARG, "NULL array with a nonzero size");
    if (plan->ws.ensure(plan->h_pot, std::max<int64_t>(total, 1) * 8))
        return fail(DMK_ERR_OOM, "device allocation failed (tuning)");
    double *pot = (double *)plan->h_pot.p;
    cudaStream_t st = (cudaStream_t)cuda_stream;
    return tune_leaf_cap(plan, candidates, n_candidates, reps, best_leaf_cap, times_ms, [&]() {
        return total == 0 ? (int)DMK_OK
                          : eval_device(plan, points, total, charges, points, total, pot, nullptr, st, n_systems,
                                        offsets);
    });
}

int dmk_plan_get_params(dmk_plan_t plan, dmk_plan_params *out) {
    if (bad_plan(plan) || !out) return fail(DMK_ERR_INVALID_ARG, "NULL argument or not a live plan handle");
    out->eps = plan->eps;
    out->c = plan->tb.c;
    out->p = plan->tb.p;
    out->nf = plan->tb.nf;
    out->n0 = plan->kernel == DMK_LOG2D ? plan->t2.n0 : plan->tb.n0;
    out->leaf_cap = plan->leaf_cap;
    out->max_level = plan->max_level;
    out->precision = plan->precision;
    out->q_degree = plan->kernel == DMK_LOG2D ? (int)plan->t2.g.size() - 1 : plan->qdeg;
    out->psi0_over_c0 = plan->tb.psi0_over_c0;
    out->q_degree_f32 = plan->kernel == DMK_LOG2D ? plan->gdeg_f32 : out->q_degree;
    return DMK_OK;
}

int dmk_plan_get_table(dmk_plan_t plan, int which, double *out, int64_t n, int64_t *len) {
    if (bad_plan(plan) || !len) return fail(DMK_ERR_INVALID_ARG, "NULL argument or not a live plan handle");
    std::vector<double> v;
    if (plan->kernel == DMK_LOG2D && which >= 1) {
        switch (which) {
        case 1: v = plan->t2.w; break;
        case 2:
            v.push_back(plan->t2.hW);
            v.insert(v.end(), plan->t2.wW.begin(), plan->t2.wW.end());
            break;
        case 3: v = plan->t2.g; break;
        case 4: v.push_back(plan->t2.G0); break;
        default: return fail(DMK_ERR_INVALID_ARG, "unknown table");
        }
        which = -1;
    }
    switch (which) {
    case -1: break;
    case 0: v = plan->tb.psi_grid; break;
    case 1: v = plan->tb.w; break;
    case 2:
        v.push_back(plan->tb.hW);
        v.insert(v.end(), plan->tb.wW.begin(), plan->tb.wW.end());
        break;
    case 3: v = plan->tb.qcheb; break;
    default: return fail(DMK_ERR_INVALID_ARG, "unknown table");
    }
    *len = (int64_t)v.size();
    if (out) {
        if (n < (int64_t)v.size()) return fail(DMK_ERR_INVALID_ARG, "output too small");
        std::memcpy(out, v.data(), v.size() * sizeof(double));
    }
    return DMK_OK;
}

int dmk_plan_get_yukawa_table(dmk_plan_t plan, double lambda_unit, int level, int which, double *out, int64_t n,
                              int64_t *len) {
    if (bad_plan(plan) || !len) return fail(DMK_ERR_INVALID_ARG, "NULL argument or not a live plan handle");
    if (plan->kernel != DMK_YUKAWA) return fail(DMK_ERR_INVALID_ARG, "not a DMK_YUKAWA plan");
    if (!(lambda_unit > 0.0) || level < 0 || level > dmk::kMaxLevel || which < 0 || which > 2)
        return fail(DMK_ERR_INVALID_ARG, "argument out of range");
    dmk::YukawaTables yt;
    std::string err;
    if (dmk::build_yukawa_tables(plan->tb, lambda_unit, level + 1, yt, err) != 0)
        return fail(DMK_ERR_UNSUPPORTED, err);
    const int ns = 3 * plan->tb.nf * plan->tb.nf + 1;
    std::vector<double> v;
    if (which == 0) v.assign(yt.wl.begin() + (size_t)level * ns, yt.wl.begin() + (size_t)(level + 1) * ns);
    else if (which == 1) v = yt.wW;
    else {
        // the level's own degree, without its header
        const size_t row = (size_t)level * (yt.qdeg + 2);
        const int dg = (int)yt.qmono[row];
        v.assign(yt.qmono.begin() + row + 1, yt.qmono.begin() + row + 2 + dg);
    }
    *len = (int64_t)v.size();
    if (out) {
        if (n < (int64_t)v.size()) return fail(DMK_ERR_INVALID_ARG, "output too small");
        std::memcpy(out, v.data(), v.size() * sizeof(double));
    }
    return DMK_OK;
}

int dmk_get_stats(dmk_plan_t plan, dmk_eval_stats *out) {
    if (bad_plan(plan) || !out) return fail(DMK_ERR_INVALID_ARG, "NULL argument or not a live plan handle");
    *out = plan->stats;
    return DMK_OK;
}

int dmk_get_tree(dmk_plan_t plan, int32_t *leaf_level, int64_t *leaf_cell, int64_t n_points) {
    if (bad_plan(plan) || !leaf_level || !leaf_cell)
        return fail(DMK_ERR_INVALID_ARG, "NULL argument or not a live plan handle");
    if (!plan->tree || plan->tree->n != n_points)
        return fail(DMK_ERR_INVALID_ARG, "n_points does not match the last evaluation");
    std::string err;
    int rc = plan->tree->export_leaves(leaf_level, leaf_cell, 0, err);
    if (rc) return fail(rc, err);
    return DMK_OK;
}

}  // extern "C"
