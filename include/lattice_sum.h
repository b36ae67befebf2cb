/*
 * lattice_sum.h -- C ABI of the GB300 (sm_103a) lattice-sum library.
 *
 * Grid-based summation of Newton potentials 1/|x - a| over 3D lattices with
 * defects in canonical / Tucker tensor form, after Khoromskaia & Khoromskij,
 * "Tucker tensor method for fast grid-based summation of long-range
 * potentials on 3D lattices with defects" (arXiv 1411.1994):
 *
 *   lattice_sum_create        -- Sec. 3.2, Thm 3.1(A), Eq. (EwaldTensorGl):
 *                                reference canonical vectors on the doubled
 *                                grid (Eq. master_pot) and their 1D shift-sums
 *                                over the sites of each rectangular block;
 *   lattice_sum_add_defects   -- Sec. 4.1, Eq. (Can_LatticeSum_full), and
 *                                Sec. 4.4 classes (A)/(D): vacancies,
 *                                impurities, clusters and off-lattice charges
 *                                appended as shifted rank-R canonical terms;
 *   lattice_sum_rhosvd_reduce -- Def. 4.1, Sec. 4.3 (Eq. SideMTuckS, an eps
 *                                threshold instead of a fixed rank) and
 *                                Thm A.1(c),(d): orthogonalise the side
 *                                matrices, truncate by discarded singular
 *                                values, project, contract the Tucker core;
 *   lattice_sum_eval_slab     -- Eq. (Tucker_singePot): values of the Tucker
 *                                tensor on z-slabs by n-mode products.
 *
 * Conventions shared by every call
 * --------------------------------
 *  - Cubic box [box_lo, box_hi]^3 with an N^3 grid, mesh h = (box_hi -
 *    box_lo) / N. Collocation points are cell centres x_i = box_lo + (i+1/2)h;
 *    charges sit on grid vertices box_lo + m h, m in [0, N] (a site is
 *    snapped to the nearest vertex, m = floor((pos - box_lo)/h + 1/2)).
 *  - Reference vectors live on the doubled grid: g_q[j] = w_q^(1/3)
 *    exp(-t_q^2 ((j - N + 1/2) h)^2), j = 0..2N-1, with the sinc nodes
 *    t_q = sinh(q s_h)/t_scale, w_0 = s_h/(t_scale sqrt(pi)),
 *    w_q = 2 s_h cosh(q s_h)/(t_scale sqrt(pi)), q = 0..R-1 (s_h = sinc_step)
 *    for the Newton kernel 1/r. For the Yukawa kernel exp(-kappa r)/r
 *    (kappa > 0; Sec. 2.3, Eq. LalpYukawa, read as exp(-kappa r)/r =
 *    (2/sqrt(pi)) int exp(-kappa^2/(4 t^2)) exp(-r^2 t^2) dt) every weight is
 *    multiplied by exp(-kappa^2/(4 t_q^2)) and the nodes are q = 1..R (the
 *    node t = 0 has weight 0); row q - 1 of the reference vectors holds node q.
 *    The Slater and dipole kernels: see LS_KERNEL_*.
 *  - A window of a centre at vertex m is (W_m g_q)[i] = g_q[i - m + N].
 *  - Return value: LS_OK (0) or a negative LS_ERR_* code; the message is
 *    available from lattice_sum_last_error(ctx). A call made in the wrong
 *    order returns LS_ERR_STATE and changes nothing.
 *  - Ownership: the library owns every device buffer it allocates (reference
 *    vectors, side matrices, Tucker factors); they live until
 *    lattice_sum_destroy. Host inputs are read during the call only.
 *  - Streams: all device work is enqueued on the stream given to
 *    lattice_sum_create (a cudaStream_t passed as void*; NULL = legacy
 *    default stream). Calls return without waiting for the device, except
 *    lattice_sum_rhosvd_reduce (which reads the truncation ranks back) and
 *    lattice_sum_read (a synchronous copy to host memory).
 *  - Every kernel is hand-written for sm_103a; there is no CPU fallback. If
 *    no usable GPU is present the calls return LS_ERR_CUDA.
 */
#ifndef LATTICE_SUM_H
#define LATTICE_SUM_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* status codes */
#define LS_OK               0
#define LS_ERR_ARG         -1   /* invalid argument (sizes, pointers, ranges) */
#define LS_ERR_OOM         -2   /* device allocation failed                    */
#define LS_ERR_CUDA        -3   /* a CUDA call or kernel launch failed         */
#define LS_ERR_NOCONVERGE  -4   /* the eigen-solver hit its sweep limit        */
#define LS_ERR_STATE       -5   /* call out of order                           */
#define LS_ERR_TIMEOUT     -6   /* a bounded device-side wait gave up          */

/* arithmetic of the reduction and evaluation steps */
#define LS_FP64   0   /* contractions (projection, core, slabs) in FP64 DFMA             */
#define LS_MIXED  1   /* the same orthogonalisation (FP64 Gram, eigen-solver, CholeskyQR) */
                      /* with the projection, the core contraction and the slab         */
                      /* products on tcgen05 tensor cores: each operand row is scaled    */
                      /* by a power of two and split into two exact 6-bit digits and a  */
                      /* rest of two BF16 parts; digit products accumulate exactly in    */
                      /* FP32 TMEM accumulators (13 MMAs per k16 step, K chunks of       */
                      /* 1024 summed in FP64): about 2^-30 of sum |a_k b_k|              */

/* defect kinds */
#define LS_DEFECT_SITES 0  /* sites block[site : site+extent) get charge `charge`     */
                           /* (0 = vacancy, Z' = impurity; extent 3,3,3 = a cluster)   */
#define LS_DEFECT_POINT 1  /* an extra charge `charge` at position `pos` (off-lattice) */

/* output types of lattice_sum_eval_slab */
#define LS_OUT_F64 0
#define LS_OUT_F32 1

/* what lattice_sum_read copies */
#define LS_READ_GENVEC   0  /* double [R][2N]  reference vectors g_q                    */
#define LS_READ_COLUMNS  1  /* double [C_l][N] canonical vectors of mode l (unit length */
                            /*                 after rhosvd_reduce, raw before)          */
#define LS_READ_NORMS    2  /* double [C_l]    norms of the raw canonical vectors        */
#define LS_READ_TERMS    3  /* int32  [T][3]   column of each term in each mode          */
#define LS_READ_XI       4  /* double [T]      term weights (charges; after reduce: the  */
                            /*                 charges times the three vector norms)     */
#define LS_READ_SIGMA    5  /* double [C_l]    singular values of mode l, descending     */
#define LS_READ_BASIS    6  /* double [r_l][N] orthonormal Tucker vectors of mode l      */
#define LS_READ_PROJ     7  /* double [r_l][C_l] projections Z_l^T a_c                   */
#define LS_READ_CORE     8  /* double [r1][r2][r3] Tucker core (r3 fastest)              */
#define LS_READ_TUCKER_REF 9 /* double [r_ref][2N] reference Tucker vectors (Tucker-       */
                            /*                 reference contexts)                       */

typedef struct ls_ctx ls_ctx;

typedef struct {
    int64_t N;          /* grid points per axis of the box (>= 2)                       */
    double  box_lo;     /* box [box_lo, box_hi] on every axis                           */
    double  box_hi;
    int32_t R;          /* canonical rank of the reference tensor (1..64)               */
    double  sinc_step;  /* sinc quadrature step s_h (> 0)                                */
    double  t_scale;    /* substitution scale s in t = sinh(u)/s (> 0); see             */
                        /* lattice_sum_fit_t_scale                                       */
    int32_t precision;  /* LS_FP64 or LS_MIXED                                           */
    int32_t flags;      /* LS_FLAG_GALERKIN, LS_FLAG_SVD_GRAM or LS_FLAG_SVD_ONESIDED, OR-ed */
    double  kappa;      /* kernel parameter (see kernel); finite, >= 0, and small       */
                        /* enough that kappa^2/(4 t_1^2) <= 600 (t_1 = sinh(s_h)/t_scale) */
    int32_t kernel;     /* LS_KERNEL_YUKAWA: exp(-kappa r)/r, the Newton 1/r at kappa=0 */
                        /* LS_KERNEL_SLATER: exp(-kappa r), kappa > 0                    */
                        /* LS_KERNEL_DIPOLE: 1/r^3, kappa = 0                            */
    double  ref_eps;    /* LS_FLAG_TUCKER_REF: threshold of the reference Tucker tensor  */
                        /* (0 < ref_eps < 1); ignored otherwise                          */
} ls_params;

/* kernel families (Sec. 2.3), each a Laplace-Gauss integral
 * p(r) = int_0^inf a(t) exp(-r^2 t^2) dt discretised by the same sinc rule:
 *   YUKAWA a = (2/sqrt(pi)) exp(-kappa^2/(4 t^2))       (Eq. LalpYukawa, LalpNewt)
 *   SLATER a = (kappa/sqrt(pi)) t^-2 exp(-kappa^2/(4 t^2)) (Eq. LalpSlater, t -> t^2)
 *   DIPOLE a = (4/sqrt(pi)) t^2                          (Eq. LalpPoly, n = 3/2)
 * with weights w_q = s_h a(t_q) cosh(q s_h)/t_scale (halved at q = 0). Only the
 * Newton kernel has a(0) > 0 and uses q = 0..R-1; the others q = 1..R. */
/* flags: reference vectors as cell averages, (1/h) int over [(j-N)h, (j-N+1)h] of
 * exp(-t_q^2 x^2) times w_q^(1/3), i.e. Eq. (galten) with piecewise-constant basis
 * functions divided by the cell volume, instead of collocation at cell centres */
#define LS_FLAG_GALERKIN 1
/* flags: how lattice_sum_rhosvd_reduce finds the singular values of the side
 * matrices (Def. 4.1). LS_FLAG_SVD_ONESIDED: without squaring them (the
 * default of LS_FP64 contexts; see lattice_sum_rhosvd_reduce), good down to
 * about u sigma_1. LS_FLAG_SVD_GRAM: from the eigenvalues of the FP64 Gram
 * matrix (the default of LS_MIXED contexts), good to about sqrt(8 u T) sigma_1,
 * which suffices for eps >= 1e-6. At most one of the two. */
#define LS_FLAG_SVD_GRAM 2
#define LS_FLAG_SVD_ONESIDED 4
/* flags: the Tucker-reference variant (Thm 3.1(B), Sec. 4.1, Thm 4.3). The
 * reference tensor is the rank-r_ref Tucker tensor T = sum b_m t_m1 (x) t_m2
 * (x) t_m3 on the doubled grid, the RHOSVD of the canonical reference tensor
 * at ref_eps; every block and defect is a Tucker term (assembled or windowed
 * reference Tucker vectors, core = charge times b), and lattice_sum_rhosvd_-
 * reduce is the generalized RHOSVD of that sum of Tucker tensors (Thm 4.3):
 * the agglomerated side matrix of mode l concatenates every term's r_ref
 * vectors, each term's block scaled to unit Frobenius norm (the scale moved
 * into its core, so that every side matrix has spectral norm <= 1, as the
 * bound needs); its truncated SVD (non-squaring route) gives Z_l, and the
 * core is the projection of the sum itself. info->xi_norm then holds
 * |B_hat| = (sum_s ||B_s||^2)^(1/2) and info->bound_abs the Thm 4.3 bound
 * |B_hat| sum_l d_l. Not with LS_FLAG_SVD_GRAM. */
#define LS_FLAG_TUCKER_REF 8
/* LS_FLAG_CACHE_GENVEC: keep the reference vectors g_q (Sec. 2.2: computed once and
 * stored for repeated use) in a process-wide device cache keyed by everything they
 * depend on (device, N, the grid step, R, sinc step, t-scale, kernel family, kappa,
 * collocated or Galerkin entries; the doubles compared bit for bit). A context created
 * with the flag copies them from the cache (device to device) when the key is present
 * and adds them when it is not. The cache holds up to 8 entries (the oldest is freed
 * first) until lattice_sum_cache_clear or process exit. Results do not change: the
 * cached vectors are the bytes the kernel wrote. */
#define LS_FLAG_CACHE_GENVEC 16

#define LS_KERNEL_YUKAWA 0
#define LS_KERNEL_SLATER 1
#define LS_KERNEL_DIPOLE 2

typedef struct {
    int64_t L[3];        /* sites per axis (>= 1)                                        */
    double  origin[3];   /* position of site (0,0,0)                                     */
    double  spacing[3];  /* site spacing per axis                                        */
    double  charge;      /* charge of every site                                         */
} ls_block;

typedef struct {
    int32_t kind;        /* LS_DEFECT_SITES or LS_DEFECT_POINT                           */
    int32_t block;       /* block index (SITES)                                          */
    int64_t site[3];     /* first site (SITES)                                           */
    int64_t extent[3];   /* sites per axis (SITES; >= 1)                                 */
    double  pos[3];      /* position (POINT)                                             */
    double  charge;      /* new charge of the sites (SITES) / added charge (POINT)       */
} ls_defect;

typedef struct {
    int32_t r[3];               /* Tucker ranks                                          */
    int32_t C[3];               /* distinct canonical vectors per mode                   */
    int64_t T;                  /* canonical terms R_total                               */
    double  sigma_discarded[3]; /* (sum_{k>r} sigma_k^2)^(1/2) per mode                  */
    double  sigma_total[3];     /* (sum_k sigma_k^2)^(1/2) per mode                      */
    double  xi_norm;            /* ||xi||_2 with the vector norms folded in              */
    double  bound_abs;          /* Thm A.1(d) bound xi_norm * sum_l d_l, with           */
                                /* d_l^2 = sigma_discarded[l]^2 + C_l * floor_l: the     */
                                /* eigenvalues of the FP64 Gram matrix are resolved to   */
                                /* C_l * floor_l, floor_l = 8 u T (u = 2^-53)             */
    int32_t sweeps[3];          /* eigen-solver sweeps per mode                          */
    int64_t rotations[3];       /* Jacobi rotations applied per mode (all sweeps)        */
    int32_t pivots[3];          /* columns kept by the pivoted Cholesky pre-compression  */
} ls_tucker_info;

/*
 * lattice_sum_fit_t_scale -- choose the scale s of the sinc substitution.
 * Sec. 2.1 (Eqs. laplace, hM, sinc_conv): the rank-R expansion reproduces
 * 1/r only on a range [r_min, r_max]; this host routine picks s to minimise
 * the maximum relative error |r sum_q w_q exp(-t_q^2 r^2) - 1| over that
 * range (log-scan then golden section). Pure host arithmetic, done once per
 * (R, sinc_step, range) and stored by the caller, as the paper stores its
 * reference vectors. Writes s and the error reached; LS_ERR_ARG on bad input.
 */
int lattice_sum_fit_t_scale(int32_t R, double sinc_step, double r_min, double r_max,
                            double* t_scale_out, double* max_rel_err_out);

/*
 * lattice_sum_fit_t_scale_kernel -- the same fit for a kernel family and
 * parameter (LS_KERNEL_YUKAWA with kappa = 0 is lattice_sum_fit_t_scale).
 * The error minimised is max_r |sum_q w_q exp(-t_q^2 r^2) - p(r)| / m(r) with
 * m(r) = 1/r (Yukawa family: the relative error for the Newton kernel, and
 * relative to the unscreened 1/r otherwise; Eq. sinc_conv bounds the absolute
 * error), 1 (Slater, which is 1 at r = 0) or 1/r^3 (dipole: the relative
 * error). LS_ERR_ARG on bad input (an unknown kernel, kappa < 0 or not
 * finite, kappa = 0 for Slater or kappa != 0 for the dipole).
 */
int lattice_sum_fit_t_scale_kernel(int32_t R, double sinc_step, int32_t kernel, double kappa, double r_min,
                                   double r_max, double* t_scale_out, double* max_rel_err_out);

/*
 * lattice_sum_create -- reference vectors and assembled lattice sums.
 * Thm 3.1(A): for each block, mode l and rank index q the canonical vector
 * v[i] = sum_k g_q[i - m_k + N] over the block's L_l snapped site vertices
 * m_k. `blocks` (host, nblocks >= 1 entries) are copied. `stream` is a
 * cudaStream_t or NULL. On success *out holds a new context.
 * Errors: LS_ERR_ARG (bad sizes, a site outside the box, an unknown kernel,
 * a kappa the kernel does not take or too large for the sinc rule), LS_ERR_OOM,
 * LS_ERR_CUDA.
 */
int lattice_sum_create(ls_ctx** out, const ls_params* params, const ls_block* blocks,
                       int32_t nblocks, void* stream);

/*
 * lattice_sum_add_defects -- append defects as canonical terms.
 * Eq. (Can_LatticeSum_full): each defect adds R terms xi * (x)_l
 * (sum over its windows of W_m g_q); xi = charge - block charge (SITES) or
 * charge (POINT). Vectors shared by several defects are stored once
 * (distinct window sets per mode). May be called several times before
 * lattice_sum_rhosvd_reduce. `defects` is host memory with n entries.
 * Errors: LS_ERR_ARG (block index, site range, position outside the box),
 * LS_ERR_STATE (after the reduction), LS_ERR_OOM, LS_ERR_CUDA.
 */
int lattice_sum_add_defects(ls_ctx* ctx, const ls_defect* defects, int64_t n);

/*
 * lattice_sum_rhosvd_reduce -- RHOSVD rank reduction to Tucker form.
 * Def. 4.1 / Thm A.1: per mode, the side matrix of unit canonical vectors
 * (a vector shared by k terms enters with weight sqrt(k), which leaves
 * A A^T unchanged) is orthogonalised via its FP64 Gram matrix G: a pivoted
 * Cholesky G ~ L L^T keeps pivot columns until the remaining trace is below
 * 1e-4 eps^2 T (that remainder joins the discarded tail and the bound); the
 * k x k matrix H = L^T L is diagonalised by a block Jacobi iteration (FP32
 * rotations with the diagonal kept to about 48 bits) and an FP64-grade
 * re-projection H' = U^T H U: on LS_MIXED contexts the iteration stops at an
 * off-diagonal ratio of 1e-4 and the diagonal of H' gives the eigenvalues;
 * with LS_FLAG_SVD_GRAM on an LS_FP64 context a second iteration on H' runs
 * to off-diagonal ratios of 1e-10; the basis Y = A_w L U diag(1/lambda) is
 * orthonormalised by CholeskyQR (first pass: the inverse-square-root series
 * where Y Y^T is within 0.1 of I, else a Cholesky factorisation, FP32 in one
 * CTA's shared memory while r fits there (about 238), FP64 on a cooperative
 * grid above; second pass: the series in FP64-grade arithmetic).
 * r_l is the smallest rank whose discarded singular values satisfy
 * (sum_{k>r} s_k^2)^(1/2) <= eps (sum_k s_k^2)^(1/2). The projections
 * P_l = Z_l^T A_l and the core
 * mu = sum_nu xi_nu P1[:,c1] (x) P2[:,c2] (x) P3[:,c3] follow.
 * That is the Gram route (LS_FLAG_SVD_GRAM; LS_MIXED contexts). It squares
 * the singular values: they are resolved to about sqrt(8 u T) sigma_1.
 * The non-squaring route (LS_FLAG_SVD_ONESIDED; LS_FP64 contexts): the Gram
 * route gives a basis Q1 of every direction 1e3 times above the Gram noise;
 * the residual rows E = A_w - (A_w Q1^T) Q1 give, by the same route, a basis
 * Q2 of the rest of the range, orthogonal to Q1; one-sided (Hestenes) Jacobi
 * in FP64 on the rows of B = [Q1; Q2] A_w^T gives the singular values and the
 * rotation M without forming B B^T; the eps rule (with E's energy outside Q2
 * in the tail) picks r and Z = M_r [Q1; Q2]. Singular values are then good
 * to about u sigma_1 and the Tucker result agrees with a dense SVD's to FP64
 * rounding over the conditioning of the truncation (sigma_1 / gap).
 * `forced_ranks` (host, 3 entries or NULL) overrides the eps rule (each
 * clipped to C_l and, on the Gram route, to the eigenvalues of the FP64 Gram
 * matrix above its rounding noise 8 u T; on the non-squaring route, to the
 * dimension of Q). Fills *info (may be NULL). Synchronises the stream.
 * Errors: LS_ERR_ARG (eps <= 0 and no forced ranks), LS_ERR_STATE (called
 * twice), LS_ERR_NOCONVERGE, LS_ERR_TIMEOUT, LS_ERR_OOM, LS_ERR_CUDA.
 */
int lattice_sum_rhosvd_reduce(ls_ctx* ctx, double eps, const int32_t* forced_ranks,
                              ls_tucker_info* info);

/*
 * lattice_sum_batch_reduce -- the batched form: RHOSVD of n independent
 * contexts (each created and given its defects as usual) in one call.
 * Every context is reduced as lattice_sum_rhosvd_reduce(ctx, eps) would
 * reduce it; what changes is the schedule. The pivoted Cholesky, the two
 * Jacobi runs and the CholeskyQR factorisation of all 3n modes run as one
 * launch each on the stream of ctxs[0] (one thread-block cluster or CTA
 * group per mode); the per-context products run on each context's own
 * stream, ordered against the shared launches by events. `infos` (host, n entries,
 * may be NULL) receives each context's ls_tucker_info. Synchronises all the
 * streams. Errors: LS_ERR_ARG (NULL or repeated context, eps <= 0),
 * LS_ERR_STATE (a context already reduced), and the errors of
 * lattice_sum_rhosvd_reduce; the message is on the failing context and on
 * lattice_sum_last_error(NULL).
 */
int lattice_sum_batch_reduce(ls_ctx* const* ctxs, int32_t n, double eps, ls_tucker_info* infos);

/*
 * lattice_sum_gemm_nt -- D = A B^T for device FP64 matrices (A: M x K, B:
 * N x K, D: M x N, all row-major), in the arithmetic the reduction uses for
 * its dense FP64 products (Gram matrices, CholeskyQR, FP64 projection): each
 * row scaled by a power of two and written as eight exact base-128 digits,
 * digit products summed exactly per level in FP32 on tcgen05 tensor cores,
 * levels recombined in integer and FP64 arithmetic. The error is about
 * 2^-53 sum_k |a_mk| |b_nk|, as for an FP64 dot product. Exposed so that the
 * arithmetic can be checked on its own. `stream` is a cudaStream_t or NULL;
 * the call synchronises it. Errors: LS_ERR_ARG, LS_ERR_OOM, LS_ERR_CUDA,
 * LS_ERR_TIMEOUT.
 */
int lattice_sum_gemm_nt(const double* A, const double* B, int64_t M, int64_t N, int64_t K, double* D,
                        void* stream);

/*
 * lattice_sum_jacobi_eig -- one run of the reduction's block Jacobi on a
 * symmetric k x k device matrix H (row-major FP64; the upper triangle is
 * read), as the truncation step runs it (Thm 2.1 needs the eigen-
 * decomposition of each compressed Gram matrix).
 * - Arithmetic: the diagonal as an FP32 hi/lo pair, the off-diagonal part
 *   and the accumulated rotation in FP32. A pair rotates while
 *   |e_pq| > abs_floor and e_pq^2 > tol^2 |d_p d_q|. abs_floor should be
 *   above the FP32 noise of E (the reduction passes its resolution floor),
 *   or pairs of tiny eigenvalues never settle.
 * - Outputs: D (device, k) receives the diagonal after convergence, V
 *   (device, k x k row-major) the accumulated rotation I + F, whose columns
 *   are the eigenvectors; *sweeps (may be NULL) the sweeps taken.
 * - form 1: one thread-block cluster with the matrix in shared memory
 *   (k up to a device-dependent limit: 208 on GB300). form 2: one cooperative
 *   grid with the matrix in global memory (any k). On the same input both
 *   forms give the same D and V.
 * - max_sweeps: the sweep limit (1..60; 0 = 60), after which the call
 *   returns LS_ERR_NOCONVERGE.
 * - Synchronises `stream` (a cudaStream_t or NULL).
 * - Errors: LS_ERR_ARG, LS_ERR_OOM, LS_ERR_CUDA, LS_ERR_NOCONVERGE,
 *   LS_ERR_TIMEOUT.
 */
int lattice_sum_jacobi_eig(const double* H, int32_t k, double tol, double abs_floor, int32_t form,
                           int32_t max_sweeps, double* D, double* V, int32_t* sweeps, void* stream);

/*
 * lattice_sum_svd_rows -- the one-sided (Hestenes) Jacobi of the non-squaring
 * route on its own, exposed so that it can be checked against a dense SVD:
 * the m rows of B (device, m x C, row-major FP64; not modified) are rotated
 * in pairs, in FP64, until every pair is orthogonal to within tol
 * (|b_p . b_q| <= tol ||b_p|| ||b_q||; 8 u sqrt(C) in the reduction) or a
 * sweep's largest such cosine is below 1e-9. Def. 4.1 needs the singular
 * values of each side matrix; no product B B^T is formed, so each value keeps
 * the relative accuracy of its row (Demmel & Veselic 1992).
 * - Outputs: sig2 (device, m) the squared row norms after convergence (the
 *   squared singular values of B, unsorted); M (device, m x m row-major) the
 *   accumulated rotation, so that M B has those orthogonal rows (the rows of M
 *   are the left singular vectors of B); *sweeps (may be NULL) the sweeps
 *   taken; rotations (host, 64 entries, may be NULL) the rotations per sweep.
 * - max_sweeps: the sweep limit (1..60; 0 = 60), after which the call
 *   returns LS_ERR_NOCONVERGE.
 * - Synchronises `stream` (a cudaStream_t or NULL).
 * - Errors: LS_ERR_ARG, LS_ERR_OOM, LS_ERR_CUDA, LS_ERR_NOCONVERGE,
 *   LS_ERR_TIMEOUT.
 */
int lattice_sum_svd_rows(const double* B, int32_t m, int32_t C, double tol, int32_t max_sweeps, double* sig2,
                         double* M, int32_t* sweeps, int64_t* rotations, void* stream);

/*
 * Failure-path hooks (no counterpart in the paper): they let tests drive the
 * library's error paths without faulting the GPU.
 *
 * lattice_sum_test_fail_alloc -- the n-th device allocation of a context
 * from now (n = 0: the next one) reports cudaErrorMemoryAllocation, so that
 * the call making it returns LS_ERR_OOM; n < 0 switches the injection off.
 * Process-wide, one shot. A context whose call failed can still be destroyed.
 *
 * lattice_sum_test_bounded_wait -- runs the bounded group barrier that the
 * cooperative kernels use between their rounds, in a two-CTA grid with
 * spin_limit polls (each with a short sleep): with absent = 0 both CTAs
 * arrive and the call returns LS_OK; with absent = 1 the second CTA leaves
 * without arriving, the first one's wait runs out and the call returns
 * LS_ERR_TIMEOUT, the kernel having ended normally (the context stays
 * usable). Synchronises `stream`. Errors: LS_ERR_ARG, LS_ERR_OOM, LS_ERR_CUDA.
 */
int lattice_sum_test_fail_alloc(int64_t n);
int lattice_sum_test_bounded_wait(int32_t absent, int64_t spin_limit, void* stream);

/*
 * lattice_sum_gemm_nt_mixed -- D = A B^T for device FP64 matrices (A: M x K,
 * B: N x K, row-major; K <= 4096 with FP32 output, any K with FP64 output:
 * chunks of 4096 added in FP64) in the arithmetic of the mixed slab
 * evaluation. Each operand row is scaled by a power of two to (-64, 64) and
 * written as d0 + d1 2^-7 + t1 + t2: d0, d1 nearest integers in [-64, 64],
 * t1 and t2 11-bit rests, all stored exactly as FP16 (times 2^9). The form
 * is good to 2^-36 of the row's scale.
 * On tcgen05 tensor cores the level-0 products d0 d0 and the level-1
 * products (d0 d1 + d1 d0) 2^-7 accumulate EXACTLY in FP32 (integers below
 * 2^24 in their units; above K = 2048 d0 d1 and d1 d0 take an accumulator
 * each). The eight products below them go to a third
 * accumulator, whose rounding (the tensor cores' adds truncate) sits below
 * 2^-14 of the result.
 * Error: about 2^-32 of max_k|a_mk| max_k|b_nk| per term, from the dropped
 * d1 t2 and t2 d1 products, plus the third accumulator's drift (its adds
 * truncate): on random data 2^-38 K^1.5 of max|a| max|b| or less.
 * D (device, M x N row-major) is LS_OUT_F32 (the exact sum rounded once) or
 * LS_OUT_F64 per `out_dtype`. `tile_n` picks the output tile width (32, 64,
 * 128; 0 = by size). `stream` is a cudaStream_t or NULL; the call
 * synchronises it. Errors: LS_ERR_ARG, LS_ERR_OOM, LS_ERR_CUDA,
 * LS_ERR_TIMEOUT.
 */
int lattice_sum_gemm_nt_mixed(const double* A, const double* B, int64_t M, int64_t N, int64_t K, void* D,
                              int32_t out_dtype, int32_t tile_n, void* stream);

/*
 * lattice_sum_eval_slab -- Tucker tensor values on z-slabs.
 * Eq. (Tucker_singePot): for each z index i3, M = B x3 Z3[:, i3] and
 * out[s][i1][i2] = sum_{a,b} Z1[a][i1] M[a][b] Z2[b][i2] (i2 fastest).
 * `z_index` is host memory (nslab entries in [0, N)); `out_dev` is device
 * memory of nslab * N * N elements of `out_dtype` (LS_OUT_F64/LS_OUT_F32),
 * owned by the caller. LS_FP64 contexts: FP64 products, asynchronous on the
 * context's stream. LS_MIXED contexts: the three products on tcgen05 tensor
 * cores in the arithmetic of lattice_sum_gemm_nt_mixed, with
 * the core and the side matrices in that form kept in the context after the
 * first call; the call synchronises the stream to read the kernels' status.
 * Errors: LS_ERR_ARG, LS_ERR_STATE (before the reduction), LS_ERR_OOM,
 * LS_ERR_CUDA.
 */
int lattice_sum_eval_slab(ls_ctx* ctx, const int64_t* z_index, int32_t nslab, void* out_dev,
                          int32_t out_dtype);

/*
 * lattice_sum_tune_eval -- lattice_sum_eval_slab (same arguments, same
 * result) on an LS_MIXED context, with the output tile width of its three
 * tensor-core products (M = B x3 Z3 rows, T = M Z2^T, S = Z1 T^T, Eq.
 * Tucker_singePot) chosen by measurement: in the first chunk of slabs each
 * product runs at widths 32, 64 and 128 (one warm-up and two runs timed by
 * CUDA events), and the fastest width is kept, process-wide, for products of
 * that shape; later evaluations (any context) use it. Every width gives the
 * same result bit for bit. `report` (host, `cap` bytes; may be NULL with
 * cap 0) receives a JSON object: per product its shape, the three times in
 * ms and the width kept. Synchronises the stream. Errors: as
 * lattice_sum_eval_slab; LS_ERR_ARG on an LS_FP64 context or a report
 * buffer that is too small.
 */
int lattice_sum_tune_eval(ls_ctx* ctx, const int64_t* z_index, int32_t nslab, void* out_dev, int32_t out_dtype,
                          char* report, int64_t cap);

/*
 * lattice_sum_als_refine -- ALS refinement of the reduced Tucker tensor,
 * Thm A.1(a)-(b): the best rank-(r1, r2, r3) Tucker approximation maximises
 * the core norm ||mu|| over orthonormal bases, and alternating maximisation
 * from the RHOSVD start finds it. One step for mode l, the other two bases
 * fixed: Y_l <- the r_l leading left singular vectors of the N x r_m r_n
 * matrix B_l = sum_nu xi_nu a_l,nu (x) (Y_m^T a_m,nu) (x) (Y_n^T a_n,nu).
 * B_l lies in the range of the mode-l side matrix, so the step works in the
 * orthonormal basis Q_l of that range which the non-squaring route keeps:
 * B_l = Q_l^T S_l, S_l = (Q_l A_l^T) W_l (m_l x r_m r_n; W_l the terms
 * grouped by their mode-l vector, as the core's first step), and its leading
 * left singular vectors come from one-sided Jacobi on the rows of S_l (no
 * squaring). `sweeps` (0..100) sweeps over the modes l = 1, 2, 3; then the
 * projections and the core are recomputed (Thm A.1(c)). Ranks do not
 * change. history (host, sweeps + 1 entries, may be NULL): ||mu|| at the
 * start and after each sweep (non-decreasing: ||A - A_r||^2 = ||A||^2 -
 * ||mu||^2). info (may be NULL): the reduction's report (its bound still
 * holds), with sweeps[] = the ALS sweeps. Needs a context reduced on the
 * non-squaring route (LS_FP64, or LS_FLAG_SVD_ONESIDED). Synchronises the
 * stream. Errors: LS_ERR_ARG, LS_ERR_STATE, LS_ERR_OOM, LS_ERR_CUDA,
 * LS_ERR_NOCONVERGE, LS_ERR_TIMEOUT.
 */
int lattice_sum_als_refine(ls_ctx* ctx, int32_t sweeps, double* history, ls_tucker_info* info);

/*
 * lattice_sum_galerkin -- the Galerkin matrix of the reduced potential in a
 * rank-one basis, Eq. (nuc_pot): for basis functions G_k = g_k^1 (x) g_k^2
 * (x) g_k^3 sampled at the grid's cell centres,
 *   V[k][m] = <G_k (.) G_m, T> = sum_abc B_abc M1_a M2_b M3_c,
 *   M_l = Z_l^T (g_k^l (.) g_m^l)     (1D Hadamard and scalar products),
 * the grid inner product (times h^3 it is the midpoint rule for the integral
 * of v g_k g_m). basis[l] (host array of 3 device pointers) holds double
 * [nb][N], row k = g_k^l; V (device, nb x nb, row-major) receives the
 * symmetric matrix. The products run in the FP64-grade tensor-core arithmetic
 * of lattice_sum_gemm_nt. Synchronises the stream.
 * Errors: LS_ERR_ARG, LS_ERR_STATE (before the reduction), LS_ERR_OOM,
 * LS_ERR_CUDA, LS_ERR_TIMEOUT.
 */
int lattice_sum_galerkin(ls_ctx* ctx, const double* const* basis, int32_t nb, double* V);

/*
 * lattice_sum_get_factors -- device pointers of the Tucker factors (valid
 * until lattice_sum_destroy; library-owned): Z[l] = double [r_l][N]
 * (orthonormal rows), core = double [r1][r2][r3]; ranks[3] receives r_l.
 * Errors: LS_ERR_STATE before the reduction, LS_ERR_ARG on NULL pointers.
 */
int lattice_sum_get_factors(ls_ctx* ctx, const double** Z, const double** core, int32_t* ranks);

/*
 * lattice_sum_read -- synchronous copy of an internal array to host memory,
 * for checking and checkpointing. `what` is an LS_READ_* code, `mode` the
 * mode (0..2) where the array is per mode, `dst` host memory of `bytes`
 * bytes; the layouts are listed with the LS_READ_* codes. `*needed_bytes`
 * (may be NULL) receives the size of the array. LS_ERR_ARG when `bytes` is
 * too small (nothing copied), LS_ERR_STATE when the array does not exist yet.
 */
int lattice_sum_read(ls_ctx* ctx, int32_t what, int32_t mode, void* dst, int64_t bytes,
                     int64_t* needed_bytes);

/*
 * lattice_sum_profile -- tracing. enable != 0 clears the trace and starts
 * recording: every step of every context then records a pair of CUDA
 * events on its stream around its kernels (per step name: genvec,
 * assemble, norms, gram, jacobi, select, basis, cholqr2, project, core,
 * eval), and the library counts its kernel launches and host<->device
 * bytes. enable == 0 stops recording (the trace is kept). Process-wide.
 */
int lattice_sum_profile(int32_t enable);

/*
 * lattice_sum_profile_report -- waits for the recorded events and writes a
 * NUL-terminated JSON object into `buf` (host, `cap` bytes):
 *   {"steps": {"<name>": {"launches": n, "kernels": k, "ms": t}, ...},
 *    "kernel_launches": K, "h2d_bytes": B, "d2h_bytes": B}
 * `ms` is the summed event time of the step, `launches` how often the step
 * ran and `kernels` how many kernels it launched. `*needed_bytes` (may be
 * NULL) receives the length + 1. LS_ERR_ARG when `cap` is too small.
 */
int lattice_sum_profile_report(char* buf, int64_t cap, int64_t* needed_bytes);

/*
 * lattice_sum_eval_slab_noalloc -- slab evaluation that allocates nothing.
 * No counterpart in the paper: this is an interface for callers that cannot
 * allocate device memory when they evaluate (for example a host application
 * that reserves all of its device memory in one arena at start-up and forbids
 * later allocations, or a latency-critical loop that must not wait on the
 * driver's allocator). It computes what lattice_sum_eval_slab computes, with
 * the same FP64 kernels, from Tucker factors the caller passes in:
 *   Z0, Z1, Z2 -- device, double [r_l][N] (e.g. from lattice_sum_get_factors
 *                 or a checkpoint), core -- device, double [r0][r1][r2],
 *   ranks      -- host, 3 entries, z_index -- host, nslab entries in [0, N),
 *   out_dev    -- device, nslab * N * N elements of out_dtype (caller-owned),
 *   stream     -- cudaStream_t or NULL.
 * Its scratch is one file-scope __device__ array of 32 MiB (64 KiB of slab
 * indices, the rest for the two per-slab products), which every GPU that loads
 * this library holds until the process exits. A slab needs
 * 8 * (r0 * r1 + r0 * N) bytes of it; larger requests return LS_ERR_ARG and
 * compute nothing; more slabs than fit at once are processed in chunks. The
 * call makes no cudaMalloc, cudaFree or other allocating call, and no host-to-
 * device copy: the slab indices reach the array as kernel arguments. The first
 * call on each device looks up the array's device address (cudaGetSymbolAddress)
 * with that device current, and looks it up again when the device's context has
 * been re-created (cudaDeviceReset); make that first call before any stream
 * capture on the device begins. All calls share the one array, and it keeps
 * the last call's contents (every element a call reads was written earlier in
 * the same call, so nothing needs clearing): calls whose kernels overlap on the
 * GPU (other streams, other host threads) race on it, so serialise them.
 * Errors are read with lattice_sum_last_error(NULL). Asynchronous on `stream`.
 */
int lattice_sum_eval_slab_noalloc(const double* Z0, const double* Z1, const double* Z2, const double* core,
                                  const int32_t* ranks, int64_t N, const int64_t* z_index, int32_t nslab,
                                  void* out_dev, int32_t out_dtype, void* stream);

/* Frees every device buffer of the context (stream-ordered) and the context. */
void lattice_sum_destroy(ls_ctx* ctx);

/* lattice_sum_cache_clear -- frees the entries of the reference-vector cache
 * (LS_FLAG_CACHE_GENVEC) on every device and returns how many there were (>= 0),
 * or LS_ERR_CUDA. It synchronises the device of each entry (cudaFree); contexts keep
 * their own copies and are not affected. Not to be called while another thread
 * creates a context with the flag. */
int lattice_sum_cache_clear(void);

/* Message of the last failed call on ctx ("" if none); ctx may be NULL for
 * failures of lattice_sum_create. The string lives until the next call. */
const char* lattice_sum_last_error(const ls_ctx* ctx);

#ifdef __cplusplus
}
#endif
#endif /* LATTICE_SUM_H */
