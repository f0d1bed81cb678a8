/*
 * dmk.h -- C ABI of libdmk, a GB300 (sm_103a) implementation of the discrete
 * evaluation pass of the dual-space multilevel kernel-splitting (DMK) method
 * of Jiang & Greengard, arXiv 2308.00292.
 *
 * The library computes, for targets x_i and sources y_j with charges rho_j,
 *
 *     u_i = sum_{j : y_j != x_i} K(x_i - y_j) rho_j            (eq. discretesum)
 *
 * with K(r) = 1/r, the 3D Laplace kernel without the 1/(4 pi) factor
 * (eq. laplacesum); coincident source/target pairs contribute zero, as in the
 * self-interaction remark of Sec. 3.1.  The requested precision eps is the
 * "prescribed precision" of Sec. 3.4 (Step 0 comment); the error is measured
 * as the relative l2 norm over all targets.
 *
 * Every computation runs in CUDA kernels on the device; there is no CPU
 * fallback.  All functions return a dmk_status code; on failure
 * dmk_last_error_detail() gives a thread-local description.
 */
#ifndef DMK_H
#define DMK_H

#include <stdint.h>

#if defined(__GNUC__)
#define DMK_API __attribute__((visibility("default")))
#else
#define DMK_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ------------------------------------------------------ */
typedef enum {
    DMK_OK = 0,
    DMK_ERR_INVALID_ARG = 1,  /* null pointer, negative size, non-finite
                                 coordinate, eps outside [1e-12, 1e-2], ... */
    DMK_ERR_UNSUPPORTED = 2,  /* kernel / dimension / option not implemented */
    DMK_ERR_OOM = 3,          /* device or host allocation failed */
    DMK_ERR_CUDA = 4,         /* a CUDA runtime call failed (no device, ...) */
    DMK_ERR_TIMEOUT = 5,      /* a bounded device-side wait expired */
    DMK_ERR_DEPTH = 6,        /* the tree would exceed the maximum depth */
    DMK_ERR_INTERNAL = 7      /* internal consistency check failed */
} dmk_status;

/* ---- kernels and precision ---------------------------------------------- */
typedef enum {
    DMK_LAPLACE = 0,       /* 1/r in 3D (Sec. 3) */
    DMK_YUKAWA = 1,        /* exp(-lambda r)/r in 3D, lambda = opts.kernel_param > 0,
                              split in Fourier space (Sec. 3.7); no batches, no
                              gradients */
    DMK_LOG2D = 2,         /* log r in 2D (dim 2), the Fourier-space splitting of
                              Sec. 3.7 at lambda = 0; both parts (no FAR_ONLY /
                              NEAR_ONLY), no batches, no gradients; DMK_MIXED
                              (eps >= 1e-7) evaluates the residual pairs in single
                              precision from hi/lo coordinates and keeps the far
                              field and the sums in double;
                              dmk_eval and dmk_eval_host take n x 2 coordinates;
                              potentials sum rho_j log |x_i - y_j| over y_j != x_i */
    DMK_SQRTLAPLACE = 3    /* reserved: 1/r^2 in 3D (Sec. 4) */
} dmk_kernel;

typedef enum {
    DMK_FP64 = 0,   /* every step in double precision */
    DMK_MIXED = 1   /* transforms, expansions and residual sums in single
                       precision; potentials accumulated in double */
} dmk_precision;

/* Flags for dmk_opts.flags. */
enum {
    DMK_FLAG_FAR_ONLY = 1,    /* return only the far part (windowed + difference
                                 kernels, eqs. farpotential): a diagnostic; the
                                 near-field pass is skipped */
    DMK_FLAG_NEAR_ONLY = 2,   /* return only the residual-kernel part and the
                                 self corrections (eq. nearpotential, Step 5); the
                                 far-field passes are skipped */
    DMK_FLAG_HOST_ONLY = 4    /* dmk_plan: build the host-side tables only and
                                 touch no device (for inspecting the plan); such
                                 a plan cannot be evaluated */
};

/* Options; a zero-initialised struct selects the defaults. */
typedef struct {
    int leaf_cap;        /* n_s: a box with more points is subdivided
                            (default 280 at eps >= 1e-6, 800 below, Sec. 5.1.1) */
    int precision;       /* dmk_precision (default DMK_FP64) */
    double kernel_param; /* DMK_YUKAWA: lambda > 0, in the units of the points */
    int flags;           /* DMK_FLAG_* */
    int max_level;       /* deepest tree level, 1..20 (default 20) */
    int p;               /* override: Chebyshev order per dimension (Table 1) */
    int nf;              /* override: Fourier modes m in [-nf, nf]^3 (Table 1) */
} dmk_opts;

typedef struct dmk_plan_s *dmk_plan_t;

/*
 * dmk_plan -- choose the method parameters for eps and build the plan tables
 * (Step 1 "Precomputation" of Sec. 3.4): c, p and N1 = 2 nf + 1 from Table 1,
 * the PSWF psi_0^c (App. A.5), the 1-D Chebyshev / plane-wave operators, the
 * diagonal-translation weights (eqs. diagonaltranslation, wlmdef) and the
 * windowed root kernel weights (Sec. 3.6, eq. windowedkernelft2), and copy
 * them to the current CUDA device.
 *
 *   kernel  DMK_LAPLACE or DMK_YUKAWA with dim 3, or DMK_LOG2D with dim 2
 *           (else DMK_ERR_UNSUPPORTED);
 *   eps     in [1e-12, 1e-2] (else DMK_ERR_INVALID_ARG);
 *   opts    may be NULL (defaults);
 *   out     receives the plan; the caller releases it with dmk_plan_destroy.
 */
DMK_API int dmk_plan(dmk_kernel kernel, int dim, double eps, const dmk_opts *opts, dmk_plan_t *out);

/*
 * dmk_eval -- one evaluation pass (Steps 0, 2-5 of Sec. 3.4) on device data.
 *
 *   sources     device pointer, n_src x 3 doubles, row-major (x, y, z per point);
 *               n_src x 2 (x, y) for a DMK_LOG2D plan
 *   n_src       number of sources (>= 0)
 *   charges     device pointer, n_src doubles
 *   targets     device pointer, n_tgt x 3 doubles; may be the same pointer as
 *               sources (with n_tgt == n_src), in which case every source is
 *               also a target and its own term is excluded
 *   n_tgt       number of targets (>= 0)
 *   potentials  device pointer, n_tgt doubles, caller-allocated, overwritten
 *   cuda_stream cudaStream_t to run on (NULL = legacy default stream)
 *
 * Inputs may lie anywhere in R^3 (they are mapped to the unit box and the
 * potentials scaled back, Sec. 3.1).  The library never writes the inputs and
 * never frees caller memory; its scratch (tree, expansions) belongs to the
 * plan, grows on demand and is reused by later calls.  A plan must not be
 * used by two calls at the same time.  The call synchronises cuda_stream
 * before it returns.  On error the potentials are unspecified.
 *
 * Environment: DMK_TREE_INITIAL_BOXES=n gives a new plan's tree a first box
 * capacity of max(n, 4096) instead of the estimate 16 (N / n_s + 64); a
 * diagnostic that makes the box arrays grow while the levels are built.
 */
DMK_API int dmk_eval(dmk_plan_t plan,
             const double *sources, int64_t n_src, const double *charges,
             const double *targets, int64_t n_tgt, double *potentials,
             void *cuda_stream);

/*
 * dmk_eval_host -- dmk_eval on host arrays: copies the inputs to the device,
 * evaluates, and copies the potentials back (same argument meaning, host
 * pointers; pinned host memory makes the copies faster).  The device copies
 * live in the plan's scratch.
 */
DMK_API int dmk_eval_host(dmk_plan_t plan,
                  const double *sources, int64_t n_src, const double *charges,
                  const double *targets, int64_t n_tgt, double *potentials,
                  void *cuda_stream);

/*
 * dmk_eval_batch -- dmk_eval of many independent systems in one pass.  System s
 * holds the points offsets[s] .. offsets[s + 1] - 1; they are its sources and
 * its targets (every point's own term excluded), and no system sees another's
 * charges.  Each system is mapped to its own unit box (Sec. 3.1), so a level-l
 * box has side 2^-l in every system and all systems share the plan's tables;
 * the tree is one forest with a root per system, and every kernel processes
 * the boxes of all systems of a level together.
 *
 *   points      device pointer, total x 3 doubles, row-major, the systems one
 *               after another (total = offsets[n_systems])
 *   charges     device pointer, total doubles
 *   offsets     HOST pointer, n_systems + 1 ascending int64 offsets,
 *               offsets[0] = 0; empty systems are allowed
 *   n_systems   1 .. 2^24
 *   potentials  device pointer, total doubles, caller-allocated, overwritten
 *   cuda_stream as in dmk_eval
 *
 * The system index takes the top bits of the 63-bit point keys: with n_systems
 * up to 2^k the tree depth is limited to (63 - k) / 3 levels (17 levels for
 * 4096 systems).  Statistics (dmk_get_stats) cover the whole batch;
 * dmk_get_tree reports each point's leaf cell within its own system.
 */
DMK_API int dmk_eval_batch(dmk_plan_t plan,
                           const double *points, const double *charges, const int64_t *offsets, int n_systems,
                           double *potentials, void *cuda_stream);

/*
 * dmk_eval_grad -- dmk_eval plus the gradient of the potential at every target,
 * grad u(x_i) = sum_{j : y_j != x_i} rho_j (y_j - x_i) / |x_i - y_j|^3, from the same
 * pass differentiated: the Chebyshev local expansions through T_n' = n U_{n-1}
 * (Sec. 2.1) and the residual kernel through R_L'(r) (x - y) / r (Sec. 3.6).  The
 * negated gradient times a target's charge is the force on it; the gradient
 * with respect to a source follows from evaluating with the roles swapped.
 *
 *   arguments   as in dmk_eval
 *   gradients   device pointer, n_tgt x 3 doubles, row-major (d/dx, d/dy, d/dz of
 *               u at target i), caller-allocated, overwritten
 *
 * The gradients carry the method's error relative to their own size (about eps
 * for the FP64 path); the flags DMK_FLAG_FAR_ONLY / NEAR_ONLY apply to them too.
 */
DMK_API int dmk_eval_grad(dmk_plan_t plan,
                          const double *sources, int64_t n_src, const double *charges,
                          const double *targets, int64_t n_tgt, double *potentials, double *gradients,
                          void *cuda_stream);

/*
 * dmk_adjoint_combine -- the chain-rule products of the adjoint pass:
 * out_i = w1_i g1_i + w2_i g2_i for rows g of three doubles.  The paper gives no
 * gradients; the adjoint follows from the symmetry of the kernel (eq.
 * discretesum with K(x - y) = K(y - x)): for L(u), u_i = sum_j K(x_i - y_j) rho_j,
 * the gradient with respect to source y_j is rho_j grad v(y_j), v the potential
 * of the charges dL/du placed at the targets, and the gradient with respect to
 * target x_i is (dL/du_i) grad u(x_i); both are such products, and where
 * sources and targets coincide they add.  dmk_eval_grad supplies grad v and
 * grad u.
 *
 *   n         rows (>= 0)
 *   w1, g1    device pointers: n weights and n x 3 gradients (row-major); both
 *             NULL to omit the term
 *   w2, g2    the same for the second term
 *   out       device pointer, n x 3 doubles, caller-allocated, overwritten (may
 *             alias g1 or g2)
 *   stream    asynchronous with respect to the host; runs on cuda_stream
 */
DMK_API int dmk_adjoint_combine(int64_t n, const double *w1, const double *g1, const double *w2,
                                const double *g2, double *out, void *cuda_stream);

/*
 * dmk_direct_noalloc -- the direct sum u_i = sum_{j : y_j != x_i} rho_j / |x_i - y_j|
 * in double precision, performing no device allocation.  The paper has no
 * counterpart: this entry point exists for callers that cannot allocate while
 * they run -- applications that give all device memory to their own pool,
 * loops that cannot absorb the synchronisation an allocation can cause -- and
 * that therefore cannot use dmk_eval, whose scratch grows with the input.
 *
 *   arguments   as in dmk_eval (device pointers, row-major points); targets
 *               may equal sources; coincident pairs contribute zero
 *   limits      n_tgt <= 16384 (larger -> DMK_ERR_INVALID_ARG), any n_src;
 *               cost O(n_src * n_tgt)
 *   scratch     a fixed 2 MiB device array inside the library, shared by all
 *               calls: calls that overlap on the device race and must be
 *               serialised by the caller.  Every call looks up the array's
 *               address on the current device (no allocation); the first call
 *               on a device loads the library's module there, so make it before
 *               any stream capture.
 *   stream      asynchronous with respect to the host; runs on cuda_stream
 */
DMK_API int dmk_direct_noalloc(const double *sources, int64_t n_src, const double *charges,
                               const double *targets, int64_t n_tgt, double *potentials,
                               void *cuda_stream);

/*
 * dmk_tune_leaf_cap -- choose the plan's leaf capacity n_s by timing.  The
 * accuracy of the method is set by p and nf (Table 1) and does not depend on
 * n_s; n_s only moves work between the residual near field, which grows
 * linearly with it, and the far field, which grows with the number of boxes
 * (the balance discussed in Sec. 5.1.1).  The best n_s depends on the point
 * distribution and the hardware, so it is measured: for every candidate the
 * plan evaluates the given problem reps + 1 times (the first untimed) and
 * keeps the smallest device time of one evaluation; the fastest candidate
 * becomes the plan's leaf capacity for later calls.
 *
 *   sources ... n_tgt  a representative problem, as in dmk_eval (device pointers)
 *   candidates    leaf capacities to try (each 1..2^20), or NULL for the
 *                 default list 64, 100, 140, 200, 280, 400, 560
 *   n_candidates  entries of candidates (1..64; ignored when it is NULL)
 *   reps          timed evaluations per candidate (0 = 3, at most 100)
 *   best_leaf_cap receives the chosen capacity (may be NULL)
 *   times_ms      receives one time per candidate, in milliseconds (may be NULL)
 *   cuda_stream   as in dmk_eval
 *
 * On error the plan keeps its previous leaf capacity.  The potentials are
 * computed into the plan's scratch and discarded.
 */
DMK_API int dmk_tune_leaf_cap(dmk_plan_t plan,
                              const double *sources, int64_t n_src, const double *charges,
                              const double *targets, int64_t n_tgt,
                              const int *candidates, int n_candidates, int reps,
                              int *best_leaf_cap, float *times_ms, void *cuda_stream);

/* dmk_tune_leaf_cap for a batch of systems (arguments as in dmk_eval_batch,
 * the rest as in dmk_tune_leaf_cap): the capacity that evaluates the whole
 * batch fastest. */
DMK_API int dmk_tune_leaf_cap_batch(dmk_plan_t plan,
                                    const double *points, const double *charges, const int64_t *offsets,
                                    int n_systems, const int *candidates, int n_candidates, int reps,
                                    int *best_leaf_cap, float *times_ms, void *cuda_stream);

/* Release a plan and all its device memory.  NULL is accepted.  Every call
 * that takes a plan checks that it is a live handle (a marker word that
 * dmk_plan sets and dmk_plan_destroy clears) and returns DMK_ERR_INVALID_ARG
 * for anything else, without reading further; a handle whose memory was
 * already freed cannot be detected reliably. */
DMK_API int dmk_plan_destroy(dmk_plan_t plan);

/* Static description of a status code. */
DMK_API const char *dmk_error_string(int code);

/* Thread-local detail of the last failure in this thread ("" if none). */
DMK_API const char *dmk_last_error_detail(void);

/* ---- introspection (diagnostics and tests) -------------------------------- */

/* Method parameters chosen by dmk_plan. */
typedef struct {
    double eps, c;          /* precision, PSWF bandwidth */
    int p, nf, n0;          /* Chebyshev order, difference / root Fourier half-widths */
    int leaf_cap, max_level, precision;
    int q_degree;           /* degree of the residual-kernel polynomial in r^2
                               (DMK_LOG2D: of G, R_l(r) = log(r / R_l) + G(r^2 / R_l^2)) */
    double psi0_over_c0;    /* psi(0)/c_0: the self term at R = 1 */
    int q_degree_f32;       /* DMK_LOG2D: the degree at which the single-precision
                               near field (DMK_MIXED) cuts G's Chebyshev series, where
                               its tail falls below 1e-2 eps max(1, |G|); q_degree
                               for the 3D kernels */
} dmk_plan_params;

DMK_API int dmk_plan_get_params(dmk_plan_t plan, dmk_plan_params *out);

/* Copy a host-side plan table into out (capacity n doubles); returns the
 * table's length through *len.  which:
 *   0  psi_0^c on the grid x_k = k / 64, k = 0..256, normalised psi(0) = 1
 *   1  translation weights w(s), s = |m|^2 = 0..3 nf^2, at box side R = 1
 *   2  root weights wW(s), s = 0..3 n0^2, and (first) the root spacing hW
 *   3  residual polynomial: Chebyshev coefficients of q(t) = Phi(sqrt t)/sqrt t
 *      on t in [0, 1]
 * A DMK_LOG2D plan answers 1-3 with its 2D tables: 1 the weights w(s),
 * s = 0..2 nf^2 (the same at every level), 2 hW and wW(s), s = 0..2 n0^2,
 * 3 the Chebyshev coefficients (in 2 t - 1) of G with the residual
 * R_l(r) = log(r / R_l) + G(r^2 / R_l^2); and 4: G(0). */
DMK_API int dmk_plan_get_table(dmk_plan_t plan, int which, double *out, int64_t n, int64_t *len);

/* Yukawa tables of a DMK_YUKAWA plan at a unit-box lambda (the library uses
 * lambda S, S the largest extent of the points): which
 *   0  translation weights w_l(s), s = |m|^2 = 0..3 nf^2, of the given level
 *      (eqs. yukawaPSWFkernels, wlmdef: (h_l / 2 pi)^3 Dhat_l(h_l |m|))
 *   1  root weights wW(s), s = 0..3 n0^2 (windowed kernel, eq. windowedkernelft2
 *      with the transform of exp(-lambda r)/r truncated at R_t)
 *   2  residual polynomial of the given level, monomials in 2 t - 1 with
 *      t = r^2 / R_l^2 (degree <= 62): the mollified kernel is S_l(r) = q_l(t) / R_l
 * Works on host-only plans (no device).  Arguments as in dmk_plan_get_table. */
DMK_API int dmk_plan_get_yukawa_table(dmk_plan_t plan, double lambda_unit, int level, int which, double *out,
                                      int64_t n, int64_t *len);

/* Statistics of the last dmk_eval. */
typedef struct {
    int64_t n_points;       /* points in the tree (union of sources and targets) */
    int32_t n_levels;       /* L_max + 1 */
    int64_t n_boxes, n_leaves, n_fout;
    int64_t n_fin;          /* incoming boxes: boxes with targets and an F_out colleague */
    int64_t near_pairs;     /* candidate source-target pairs of the residual sum */
    int32_t balance_rounds; /* rebuilds needed by the level restriction */
    float t_tree_ms, t_upward_ms, t_downward_ms, t_near_ms, t_total_ms;
    int64_t n_launches;     /* kernels of this library launched by the call */
    int64_t near_pairs_inside; /* candidate pairs closer than the residual support R_L */
    int64_t local_flops;    /* algorithmic flops of the local-expansion pass (p2c,
                               translation, plane waves to Chebyshev, leaf evaluation) */
    float t_local_ms;       /* device time of the local-expansion pass alone */
    float t_incoming_ms;    /* device time of the tensor-core incoming pass (translation and
                               plane waves to Chebyshev for every level), 0 when the
                               local-expansion pass forms the incoming expansions itself */
    int64_t incoming_reads; /* colleague plane-wave arrays read by the incoming pass */
    int64_t incoming_flops; /* its algorithmic flops: translation 8 N1^2 (nf + 1) per
                               colleague array, and the three parity-split contractions
                               8 p (nf+1)^3 + 4 p^2 (nf+1)^2 + 2 p^3 (nf+1) per incoming box */
    float t_planewave_ms;   /* device time of the outgoing plane waves and the root term */
    int64_t near_pairs_screened; /* pairs whose distance the near field tested: the sources
                                    left after culling against each target group's bounding
                                    box, times the group's targets (3D); every candidate
                                    pair (2D log r, where t_near_ms times the near field on
                                    the evaluation's stream) */
} dmk_eval_stats;

DMK_API int dmk_get_stats(dmk_plan_t plan, dmk_eval_stats *out);

/* Tree of the last dmk_eval, for parity checks.  For every point of the
 * (source u target) set, in input order (sources, then targets when they are
 * a separate array): leaf_level[i] and leaf_cell[i], the Morton interleave of
 * the leaf's cell indices at its level (bit 3b + d = bit b of axis d).  Host
 * arrays of n_points entries (see dmk_get_stats). */
DMK_API int dmk_get_tree(dmk_plan_t plan, int32_t *leaf_level, int64_t *leaf_cell, int64_t n_points);

#ifdef __cplusplus
}
#endif

#endif /* DMK_H */
