// Internal declarations shared by the CUDA translation units of the
// lattice-sum library (not part of the public C ABI in include/lattice_sum.h).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "lattice_sum.h"

namespace ls {

// ---------------------------------------------------------------------------
// error flags raised by device code (bounded waits, failed pivots)
// ---------------------------------------------------------------------------
enum DeviceFlag : int {
    FLAG_OK = 0,
    FLAG_TIMEOUT = 1,      // a bounded spin-wait gave up
    FLAG_NOT_SPD = 2,      // Cholesky met a non-positive pivot
    FLAG_NOCONVERGE = 3,   // Jacobi sweep limit reached
};

// Scratch words used by device-side grid barriers and status reporting.
struct DevStatus {
    unsigned int bar_count;
    unsigned int bar_gen;
    int flag;
    int sweeps;
    unsigned int sweep_active[64];
    unsigned int arrive;        // arrivals at a counting barrier (only grows)
    int done;                   // the pivoted Cholesky: the stopping rule ended the factorisation
};

// ---------------------------------------------------------------------------
// tracing: every kernel launch site bumps this counter (ls_api.cu owns it)
// ---------------------------------------------------------------------------
void count_kernels(int n);
// host<->device bytes copied by the library (the e2e accounting)
void count_h2d(int64_t n);
void count_d2h(int64_t n);

// An NVTX range for the lifetime of the object (ABI calls and pipeline steps): a
// timeline tool (Nsight Systems, ncu's NVTX filters) shows them by name; without a
// tool attached the calls return at once.
struct NvtxRange {
    explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange&) = delete;
    NvtxRange& operator=(const NvtxRange&) = delete;
};

// Records a CUDA-event pair around a step on a stream while tracing is on
// (lattice_sum_profile); the pairs are reported by name. Every step is also an
// NVTX range.
struct Scope {
    const char* name;
    cudaStream_t st;
    cudaEvent_t a = nullptr;
    long long k0 = 0;
    Scope(const char* n, cudaStream_t s);
    ~Scope();
    Scope(const Scope&) = delete;
    Scope& operator=(const Scope&) = delete;
};

// Launch-configuration queries cached per kernel (ls_eval.cu): the kernel's dynamic shared
// memory limit is raised only when a launch needs more than before, and its resident
// blocks per SM are asked of the driver once per (threads, shared memory).
cudaError_t grow_smem(const void* kernel, size_t bytes);
cudaError_t blocks_per_sm(const void* kernel, int threads, size_t smem, int* out);

// Asynchronous host-to-device upload through pinned staging (ls_eval.cu): `src` may be
// reused as soon as the call returns.
cudaError_t upload_h2d(void* dst, const void* src, size_t bytes, cudaStream_t st);

// message returned by lattice_sum_last_error(NULL) (calls without a context)
void set_global_error(const char* msg);

// ---------------------------------------------------------------------------
// launchers implemented in ls_f64.cu (all enqueue on `st`, return cudaError)
// ---------------------------------------------------------------------------

// G0: g[q][j] = w_q^(1/3) exp(-t_q^2 ((j - N + 1/2) h)^2), q < R, j < 2N, for the kernel family
// (LS_KERNEL_*) and its parameter kappa: weights w = h a(t) cosh(u)/s from the family's
// Laplace-Gauss density a(t); nodes from q = 1 except for the Newton kernel.
// galerkin: each entry the average of the Gaussian over its cell [(j - N) h, (j - N + 1) h].
cudaError_t launch_genvec(double* g, int R, int64_t N, double h, double sinc_step, double t_scale,
                          int kernel, double kappa, bool galerkin, cudaStream_t st);

// G1/G2: out[c][i] = sum_{k<wcnt[c]} g[colq[c]][i - win[woff[c]+k] + N],
// for columns c in [c0, c0 + ncols); out has row stride N.
cudaError_t launch_assemble(const double* g, int64_t N, const int32_t* colq, const int32_t* woff,
                            const int32_t* wcnt, const int32_t* win, int64_t c0, int64_t ncols,
                            double* out, cudaStream_t st);

// norms[c] = ||a_c||; a_c /= norms[c] in place (rows of a, stride N).
cudaError_t launch_norm_columns(double* a, int64_t C, int64_t N, double* norms, cudaStream_t st);

// Cholesky A = L L^T in place (lower; A is r x r row-major, its upper part is
// overwritten) and Li = L^{-1} (lower, zeros above) for several matrices in
// one cooperative launch. st: zeroed status per job; a non-positive pivot
// raises FLAG_NOT_SPD (the pivot is replaced by 1 so the launch completes).
// gate (device, may be NULL): the job is skipped, Li left as it is, when
// *gate < kSeriesGate (the caller's series has written Li instead).
constexpr double kSeriesGate = 0.1;
struct CholJob {
    double* A; double* Li; DevStatus* st; int r; const double* gate = nullptr;
};
cudaError_t launch_chol_inv_multi(const CholJob* jobs, int njobs, int num_sms, cudaStream_t st);

// Cholesky A = L L^T and Li = L^{-1} in FP32 arithmetic, one CTA per matrix
// with the matrix in shared memory (r <= chol32_max_r()): A is read (lower
// part, FP64) and left unchanged, Li (r x r FP64, zeros above) is written.
// A non-positive pivot raises FLAG_NOT_SPD in st (the pivot is replaced by 1).
cudaError_t launch_chol32_multi(const CholJob* jobs, int njobs, cudaStream_t st);
int chol32_max_r();

// Block Jacobi of symmetric k x k matrices (ls_eig.cu): diagonal as an FP32
// hi/lo pair, off-diagonal part and the accumulated rotation I + F in FP32.
// Reads H (row-major, upper triangle),
// writes the diagonal after convergence to outD[a * ldd] and I + F
// (add_identity) or F to outF (k x k, row-major, eigenvectors in columns).
// st->sweeps (on entry: sweeps already recorded, 0 for a fresh status) is
// advanced by the sweeps taken, sweep_active[] records the rotations of
// each sweep; FLAG_NOCONVERGE after max_sweeps. A pair rotates when
// |e_pq| > abs_floor, max(d_p, d_q) >= tau and e_pq^2 > tol^2 |d_p d_q|.
struct DfJob {
    const double* H; int k; double* outD; int64_t ldd; double* outF; int add_identity; DevStatus* st;
    double abs_floor; double tau; double tol;
};
// Pairs of 8-index blocks per round, one inner sweep per 16 x 16 subproblem,
// dense tile rotations: m - 1 synchronisations a sweep for m blocks. One
// thread-block cluster per matrix, in shared memory, for k <= jacobi_blk_max_k():
int jacobi_blk_max_k();
cudaError_t launch_jacobi_blk(const DfJob* jobs, int njobs, int max_sweeps, cudaStream_t st);
// The block form in one cooperative grid with the matrices in global memory
// (any k; the same rounds, criteria and arithmetic; one confirming sweep more).
cudaError_t launch_jacobi_gblk(const DfJob* jobs, int njobs, int max_sweeps, int num_sms, cudaStream_t st);

// V = I (C x C).
cudaError_t launch_identity(double* V, int64_t C, cudaStream_t st);

// Parallel cyclic Jacobi on up to three symmetric matrices at once (one
// cooperative launch, CTAs split between the jobs). Each job: G (C x C, only
// the upper triangle is used; in place -> eigenvalues on the diagonal), V
// (C x C, starts as I -> eigenvectors in columns), snap (>= 6 * (C/2+1)
// doubles of scratch), st (zeroed status; sweeps used, or a negative count if
// the limit was hit). Rotations with |a_pq| below abs_floor, below
// tol * sqrt(|a_pp a_qq|), or with both a_pp and a_qq below tau are skipped.
struct JacobiJob {
    double* G; double* V; double* snap; DevStatus* st; int64_t C; double abs_floor; double tau;
};
cudaError_t launch_jacobi_multi(const JacobiJob* jobs, int njobs, int max_sweeps, double tol, int num_sms,
                                cudaStream_t st);

// Sort eigenvalues (diag of G) descending: perm[k], lam[k]; select the rank
// (forced if forced > 0, then clipped to the eigenvalues above `resolution`)
// and write out[0] = r, out[1] = discarded^2, out[2] = total (as doubles);
// also inv_sqrt_lam[k] = 1/sqrt(lam[k]) and lam[k] <- sqrt(max(lam[k], 0)).
// *extra (device, may be NULL) is energy outside the problem that belongs to
// the discarded tail (and to the total). n jobs, one CTA each, in one launch
// per 16 jobs.
struct SortSelectJob {
    const double* G; int64_t C; int forced; const double* extra; int32_t* perm; double* lam; double* inv_sqrt_lam;
    double* out;
    int64_t dstride = 0;      // stride between the C values read from G (0: C + 1, the diagonal)
    double resolution = -1.0; // this job's resolution (< 0: the launch's)
};
cudaError_t launch_sort_select(int n, const SortSelectJob* jobs, double eps, double resolution, cudaStream_t st);

// Pivoted Cholesky G P = L L^T (greedy diagonal pivoting) of C x C PSD
// matrices, stopped when the trace of the remaining Schur complement is
// <= delta or after kmax columns. Each job: G (C x C; the grid form overwrites
// it with the Schur complement), L (C x kmax, row-major, column t = t-th pivot
// step), d (C scratch), cand (kPcholCand doubles of scratch; its last element
// receives the final residual trace), piv (kmax), st (zeroed; st->sweeps
// receives the number k of columns).
constexpr int kPcholCand = 6 * 1024 + 8;
struct PcholJob {
    const double* G; double* L; double* d; double* cand; int* piv; DevStatus* st; int64_t C; int kmax; double delta;
    double* Lp = nullptr;   // the grid form: C x panel, the last panel's columns (zero past its last pivot)
};
// One panel of the grid form: each job continues at column st->sweeps (G
// holding the Schur complement G - L[:, :k] L[:, :k]^T) and takes up to
// `panel` pivots; d_report (2 njobs ints, may be NULL) receives each job's
// (columns so far, done).
cudaError_t launch_pchol_panel(const PcholJob* jobs, int panel, int njobs, int num_sms, int* d_report, cudaStream_t st);

// The same factorisation held in shared memory by one thread-block cluster per
// matrix (ls_pchol.cu; same jobs and outputs): usable when
// pchol_cluster_size(C, kmax) > 0 for every job.
int pchol_cluster_size(int C, int kmax);
cudaError_t launch_pchol_cluster(const PcholJob* jobs, int njobs, cudaStream_t st);
// The panel of the grid form held by one cluster per matrix (ls_pchol.cu; same jobs,
// outputs and report): usable when pchol_cpanel_fits(max C, panel).
bool pchol_cpanel_fits(int64_t Cmax, int panel);
cudaError_t launch_pchol_cpanel(const PcholJob* jobs, int panel, int njobs, int* d_report, cudaStream_t st);
// xin[t] = xi[t] * n0[tc[3t]] * n1[tc[3t+1]] * n2[tc[3t+2]].
cudaError_t launch_fold_norms(const double* xi, const int32_t* tcol, int64_t T, const double* n0,
                              const double* n1, const double* n2, double* xin, cudaStream_t st);

// out = in^T for a rows x cols row-major matrix.
cudaError_t launch_transpose(const double* in, int64_t rows, int64_t cols, double* out, cudaStream_t st);

// Core (FP64): B[i][j][k] = sum_t xin[t] P0[i][c0] P1[j][c1] P2[k][c2] in two
// exact steps: terms grouped by c0 (perm/off: terms sorted by c0, CSR
// offsets) give W[c0][j*r2+k] = sum_{t in group} xin P1[j][c1] P2[k][c2]
// (P1t, P2t are the transposed projections), then B_(0) = P0 W, in chunks of
// w_cols groups (W holds w_cols * r1 * r2 doubles).
cudaError_t launch_core_f64(const double* P0, const double* P1t, const double* P2t, const int32_t* C, const int32_t* r,
                            const int32_t* tcol, const double* xin, const int32_t* perm, const int32_t* off,
                            double* W, int64_t w_cols, double* B, cudaStream_t st);

// The grouped first step of launch_core_f64 alone, for the groups [cbeg, cbeg + ncols):
// W[c - cbeg][j*r2+k] = sum_{t in group c} xin[t] P1t[c1(t)][j] P2t[c2(t)][k] with
// c1 = tcol[3t+1], c2 = tcol[3t+2] (the ALS refinement passes the term columns with the
// mode of the update first).
cudaError_t launch_core_step1_f64(const double* P1t, const double* P2t, int r1, int r2, const int32_t* tcol,
                                  const double* xin, const int32_t* perm, const int32_t* off, int cbeg, int ncols,
                                  double* W, cudaStream_t st);

// Slab evaluation (FP64 arithmetic): out[s][x][y] for nslab z indices.
// work holds >= r0*r1*nslab + r0*N*nslab doubles.
cudaError_t launch_eval_f64(const double* const Z[3], const int32_t* r, const double* B, int64_t N,
                            const int32_t* zidx, int nslab, double* work, void* out, int out_f32,
                            cudaStream_t st);

// One-sided (Hestenes) Jacobi in FP64 (ls_osj.cu): rows of B (m x C, row stride ldb) are
// rotated in pairs, in place, until every pair is orthogonal to within tol (|b_p . b_q| <=
// tol ||b_p|| ||b_q||); M (m x m, row-major) receives the accumulated rotation (rows: the
// left singular vectors of the original B as combinations of its rows' index), sig2 (m)
// the squared row norms (the squared singular values, unsorted). st: zeroed status;
// st->sweeps receives the sweeps taken, sweep_active[] the rotations of each sweep; cmax
// (64 zeroed words) the largest |cos| of each sweep as float bits. The iteration stops
// after a sweep with no rotation or with every |cos| below 1e-9; FLAG_NOCONVERGE after
// max_sweeps (<= 60). Up to three matrices per cooperative launch.
struct OsjJob {
    double* B; int64_t ldb; int C; double* M; int m; double* sig2; DevStatus* st; double tol; unsigned* cmax;
};
cudaError_t launch_osj(const OsjJob* jobs, int njobs, int max_sweeps, int num_sms, cudaStream_t st);
// E[c][n] = w[c] A[c][n] - D[c][n] (w may be NULL: 1), rows x N.
cudaError_t launch_resid_rows(const double* A, const double* w, const double* D, int64_t rows, int64_t N, double* E,
                              cudaStream_t st);
// Y[e] -= D[e], e < n.
cudaError_t launch_sub(double* Y, const double* D, int64_t n, cudaStream_t st);
// out[j][:] = M[perm[j]][:] times scale[j] (scale may be NULL: 1), rows of length len, j < r.
cudaError_t launch_gather_rows(const double* M, int64_t len, const int32_t* perm, int r, const double* scale,
                               double* out, cudaStream_t st);
// Blocks of w rows (length N) of A: nrm[j] = Frobenius norm of block j, out block j =
// sqrt(mult[j]) / nrm[j] times it (zero where nrm[j] = 0).
cudaError_t launch_block_frob(const double* A, int w, int64_t N, int nblocks, const double* mult, double* nrm,
                              double* out, cudaStream_t st);
// The bounded group barrier of the cooperative kernels with `limit` polls, in a two-CTA grid
// whose second CTA arrives (absent = 0) or does not (absent = 1): the failure-path probe.
cudaError_t launch_wait_probe(DevStatus* st, int absent, long long limit, cudaStream_t stream);
// *out = sum_e x[e]^2, e < n (device).
cudaError_t launch_sum_squares(const double* x, int64_t n, double* out, cudaStream_t st);
// *out = sum_e x[e]^3, e < n (device).
cudaError_t launch_sum_cubes(const double* x, int64_t n, double* out, cudaStream_t st);

// Galerkin matrix steps (ls_galerkin.cu), Eq. (nuc_pot): H[p][i] = g[k_p][i] g[m_p][i] for
// the pairs (k_p, m_p) (g: nb rows of length N); and, per pair, v_p = sum_a M0[p][a]
// sum_b Y[p][a r1 + b] M1[p][b], stored at V[k][m] and V[m][k] (V: nb x nb).
cudaError_t launch_hadamard_pairs(const double* g, int64_t N, const int2* pairs, int np, double* H, cudaStream_t st);
cudaError_t launch_galerkin_contract(const double* Y, const double* M0, const double* M1, int r0, int r1,
                                     const int2* pairs, int np, int nb, double* V, cudaStream_t st);

}  // namespace ls
