/*
 * dmk_oracle.h -- plain FP64 CPU oracle for the discrete DMK evaluation pass
 * (Jiang & Greengard, "A dual-space multilevel kernel-splitting framework for
 * discrete and continuous convolution", arXiv 2308.00292).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the
 * benchmark's CPU-baseline leg may load this library.  It shares no code with
 * the CUDA path (no headers, helpers, tables or constant generators) and is
 * deliberately slow and literal: every step follows the paper's description
 * (Sec. 3.4, Steps 0-5) with plain loops in double precision.
 *
 * Kernel: the 3D Laplace kernel 1/r without the 1/(4 pi) factor (eq. laplacesum),
 * or the Yukawa kernel exp(-lambda r) / r (Sec. 3.7, oracle_params.lambda > 0);
 * coincident source/target pairs contribute zero (Sec. 3.1 self-interaction
 * remark).
 *
 * Two kernel splittings are implemented:
 *   ORACLE_PSWF     -- the prolate-spheroidal splitting of Sec. 3.6 (eq. newkernels),
 *                      parameters from Table 1;
 *   ORACLE_GAUSSIAN -- the Gaussian (Ewald) telescoping splitting of Sec. 3.2
 *                      (eqs. mlks, kerneldef, differencekernelft), used as an
 *                      independent cross-check of the whole pass.
 *
 * Unit-box mapping (the definition both the oracle and the CUDA path follow,
 * each in its own code): lo_d = min over all points of coordinate d,
 * S = max_d (max_d - lo_d) (S = 1 if that is 0), u = (x - lo) / S in IEEE
 * double (one subtraction, one division, no fused operations).  The finest
 * Morton cell of a point is min(2^21 - 1, floor(u * 2^21)) per axis.
 * Potentials in original units are the unit-box potentials divided by S.
 */
#ifndef DMK_ORACLE_H
#define DMK_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum { ORACLE_PSWF = 0, ORACLE_GAUSSIAN = 1 };

/* Method parameters for a requested precision.  Any field passed in as > 0
 * overrides the default chosen from eps (Table 1 for the PSWF splitting). */
typedef struct {
    int splitting;     /* ORACLE_PSWF or ORACLE_GAUSSIAN */
    double eps;        /* requested precision */
    int leaf_cap;      /* n_s: a box with more points than this is split */
    int p;             /* Chebyshev order per dimension */
    int nf;            /* difference-kernel Fourier modes m in [-nf, nf]^3 */
    int n0;            /* windowed root kernel modes m in [-n0, n0]^3 */
    double c;          /* PSWF bandwidth c (PSWF only) */
    double delta;      /* Gaussian: sigma_l = R_l / delta */
    double gauss_b;    /* Gaussian: window parameter b of Lemma trunc_lemma */
    int max_level;     /* deepest level a box may have (<= 21) */
    int nthreads;      /* OpenMP threads (0 = runtime default) */
    double lambda;     /* Yukawa kernel exp(-lambda r) / r when > 0 (input units;
                          oracle_kernel takes it in unit-box units); 0: 1 / r */
} oracle_params;

/* Fill defaults from eps / splitting; fields already > 0 are kept. */
void oracle_default_params(oracle_params *prm);

/* O1: u_i = sum_{j : y_j != x_i} rho_j / |x_i - y_j| with compensated
 * (Neumaier) summation.  Coordinates row-major [n][3]. */
void oracle_direct(const double *src, const double *rho, int64_t ns,
                   const double *tgt, int64_t nt, double *pot, int nthreads);

/* O1 for the Yukawa kernel exp(-lambda r) / r (Sec. 3.7), same conventions. */
void oracle_direct_yukawa(const double *src, const double *rho, int64_t ns,
                          const double *tgt, int64_t nt, double lambda, double *pot, int nthreads);

/* O2: the plain DMK pass.  tgt may be the same pointer as src (with nt == ns),
 * in which case every point is both a source and a target.  pot_far / pot_near
 * (may be NULL) receive the far part (windowed + difference kernels, from the
 * local expansions) and the near part (residual kernels + self corrections).
 * Returns 0 on success, < 0 on failure. */
int oracle_dmk(const oracle_params *prm,
               const double *src, const double *rho, int64_t ns,
               const double *tgt, int64_t nt,
               double *pot, double *pot_far, double *pot_near);

/* O1 gradient in the target position: grad[3 i + d] = d/dx_d of u(x_i). */
void oracle_direct_grad(const double *src, const double *rho, int64_t ns,
                        const double *tgt, int64_t nt, double *grad, int nthreads);

/* O2 gradient: the plain DMK pass with the derivative of the local expansions
 * (Chebyshev derivatives T_n' = n U_{n-1}) and of the residual kernel
 * (R_L'(r) (x - y) / r) at every target; grad (and the optional far / near
 * parts) hold nt x 3 doubles; pot may be NULL. */
int oracle_dmk_grad(const oracle_params *prm,
                    const double *src, const double *rho, int64_t ns,
                    const double *tgt, int64_t nt,
                    double *pot, double *grad, double *grad_far, double *grad_near);

/* Tree export for parity checks.  Returns the number of boxes (>= 1) or < 0.
 * For every point of the (source u target) set, in the order sources then
 * (if tgt != src) targets: leaf_level[i], leaf_cell[i] = Morton interleave of
 * the leaf's (ix, iy, iz) at its level (bit 3b+0 = x bit b, +1 = y, +2 = z).
 * If box_level / box_cell / box_leaf are non-NULL (capacity max_boxes) every
 * box is listed, ordered by level then cell. */
int64_t oracle_tree(const oracle_params *prm,
                    const double *src, int64_t ns, const double *tgt, int64_t nt,
                    int32_t *leaf_level, int64_t *leaf_cell,
                    int32_t *box_level, int64_t *box_cell, int32_t *box_leaf,
                    int64_t max_boxes);

/* ---- pieces exposed for the pin tests ---------------------------------- */
/* psi_0^c(x) normalised so that psi(0) = 1 (any real x). */
void oracle_pswf(double c, const double *x, int64_t n, double *out);
/* lambda_0, c_0 = int_0^1 psi, c_2 = int_0^1 x^2 psi, chi_0 (all for psi(0)=1). */
void oracle_pswf_constants(double c, double *lambda0, double *c0, double *c2,
                           double *chi0);
/* Kernel pieces of a splitting at level l (box side R_l = 2^-l):
 * what: 0 = mollified S_l(r) (r = 0 gives the limit), 1 = residual R_l(r),
 *       2 = D_l(r) = S_{l+1} - S_l, 3 = Dhat_l(k), 4 = What_0(k). */
void oracle_kernel(const oracle_params *prm, int what, int level,
                   const double *r, int64_t n, double *out);
/* Fourier spacing of the difference kernel at level l and of the root term. */
double oracle_h(const oracle_params *prm, int level);
double oracle_hW(const oracle_params *prm);


/* ---- the 2D Laplace kernel log r (Sec. 3.7 at lambda = 0, in the plane) ----
 * u_i = sum_{j : y_j != x_i} rho_j log |x_i - y_j|; coordinates row-major
 * [n][2]; the PSWF splitting (c, p, nf from Table 1 as in 3D, n0 from the
 * 2D root window) or, as an independent cross-check, the Gaussian one
 * (sigma_l = R_l / delta, residual -E_1(r^2 / sigma_l^2) / 2 in closed form).  The unit-box map
 * is the 3D one on two coordinates; pot is in input units (it includes
 * log S times the charge of the sources not coincident with the target),
 * pot_far / pot_near (may be NULL) are the unit-box far and near parts. */
void oracle_direct_log2d(const double *src, const double *rho, int64_t ns,
                         const double *tgt, int64_t nt, double *pot, int nthreads);
int oracle_dmk_log2d(const oracle_params *prm,
                     const double *src, const double *rho, int64_t ns,
                     const double *tgt, int64_t nt,
                     double *pot, double *pot_far, double *pot_near);
/* Kernel pieces in the unit box at level l: what 0 = S_l(0), the mollified
 * kernel at r = 0 (r ignored); 1 = residual R_l(r); 3 = Dhat_l(k);
 * 4 = What_0(k). */
void oracle_kernel_log2d(const oracle_params *prm, int what, int level,
                         const double *r, int64_t n, double *out);
/* The quad-tree of the points src [ns][2] (every point a source and a target):
 * per point its leaf's level and cell (ix, iy).  Returns the box count or < 0. */
int64_t oracle_tree_log2d(const oracle_params *prm, const double *src, int64_t ns,
                          int32_t *leaf_level, int64_t *leaf_ix, int64_t *leaf_iy);
/* Root spacing h_W and mode count n0 of the 2D window. */
double oracle_hW_log2d(const oracle_params *prm);
int oracle_n0_log2d(const oracle_params *prm);

#ifdef __cplusplus
}
#endif
#endif
