// FP64-grade tensor-core (tcgen05) products: exact slices; see ls_tc.cu.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>

namespace ls {

// FP64-grade products on tcgen05 tensor cores: every operand row in eight
// exact base-128 digits, digit products accumulated exactly per level in TMEM,
// recombined in integer and FP64 arithmetic (error about 2^-53 of
// sum |a_k||b_k|, as an FP64 dot product). `flag` (device int) receives
// FLAG_TIMEOUT if a bounded wait gives up; no host synchronisation.
// Each takes n <= 3 products (one per mode) and runs them in one launch.
// G_l = diag(w_l) A_l A_l^T diag(w_l)  (A_l: C_l rows of length N; w may be NULL). Where
// upper[l] is nonzero, only the 128 x 64 tiles that reach the diagonal or lie above it are
// formed (for readers of G[min(i,j)][max(i,j)]); the entries strictly below are not written.
int x64_gram(int n, const double* const a[], const int64_t C[], int64_t N, const double* const w[], double* const G[],
             int* flag, cudaStream_t st, std::string* err, const int* upper = nullptr);
// P_l = Z_l A_l^T  (Z_l: r_l x N, A_l: C_l x N, P_l: r_l x C_l).
// S_l -= L_l[:, k0_l : k0_l + kb_l] L_l[:, k0_l : k0_l + kb_l]^T (the Schur complement after a
// panel of the pivoted Cholesky) on the upper triangle of S_l and the tiles that cross its
// diagonal (read S[min(i,j)][max(i,j)]): L_l C_l x kmax_l row-major, S_l C_l x C_l; kb_l = 0
// skips job l
// skips job l if the device flag skip[l] (when skip is given) is nonzero when the product runs
int x64_syrk_sub(int n, const double* const L[], const int64_t kmax[], const int k0[], const int kb[],
                 const int64_t C[], double* const S[], int* flag, cudaStream_t st, std::string* err,
                 const int* const skip[] = nullptr);
int x64_project(int n, const double* const Z[], const int r[], const double* const a[], const int64_t C[], int64_t N,
                double* const P[], int* flag, cudaStream_t st, std::string* err);
// dst_l = T_l src_l  (T_l: r_l x r_l, src_l and dst_l: r_l x N).
int x64_apply(int n, const double* const T[], const int r[], const double* const src[], int64_t N,
              double* const dst[], int* flag, cudaStream_t st, std::string* err);
// Y_l[m][x] = isl_l[m] sum_c V_l[c][perm_l[m]] w_l[c] a_l[c][x]  (V_l: C_l x ldv_l;
// a_l: C_l x N; Y_l: r_l x N): the basis vectors from the eigenvectors of the
// compressed Gram matrix.
int x64_basis(int n, const double* const V[], const int64_t ldv[], const int32_t* const perm[],
              const double* const w[], const double* const isl[], const double* const a[], const int64_t C[],
              int64_t N, const int r[], double* const Y[], int* flag, cudaStream_t st, std::string* err);
// Vg_l[c][j] = sum_i L_l[c][i] U_l[i][j] / sqrt(H_l[j][j])  (0 where H_jj <= 0; L_l: C_l rows of
// stride kmax_l; U_l, H_l: k_l x k_l; Vg_l: C_l x k_l).
int x64_pchol_vectors(int n, const double* const L[], const int64_t kmax[], const int k[], const int64_t C[],
                      const double* const U[], const double* const H[], double* const Vg[], int* flag,
                      cudaStream_t st, std::string* err);
// H_l = L_l^T L_l over the first k_l columns of L_l (C_l rows of stride kmax_l; H_l: k_l x k_l).
int x64_pchol_gram(int n, const double* const L[], const int64_t kmax[], const int k[], const int64_t C[],
                   double* const H[], int* flag, cudaStream_t st, std::string* err);
// out_l = op(A_l) op(B_l) (+ add_l) for k_l x k_l row-major matrices (ta/tb: 1 = transpose;
// add may be null). skip (if given): device flags, product l not formed when *skip[l] != 0
// as it runs.
int x64_small(int n, const double* const A[], const int ta[], const double* const B[], const int tb[],
              const int k[], double* const out[], const double* const add[], int* flag, cudaStream_t st,
              std::string* err, const int* const skip[] = nullptr);
// T_l = S_l^{-1/2} by the series I - Delta/2 + 3/8 Delta^2 - 5/16 Delta^3 (Delta = S_l - I);
// D2_l receives Delta^2 (scratch of the caller). With gate (device doubles, one per
// matrix): gate_l = ||Delta_l||_F, and T_l (and D2_l) are formed only where gate_l <
// kSeriesGate (elsewhere a Cholesky pass gated on the same value writes T_l).
int x64_lowdin(int n, const double* const S[], const int k[], double* const D2[], double* const T[], int* flag,
               cudaStream_t st, std::string* err, double* const gate[] = nullptr);
// A strided FP64 operand: entry (i, k) = p[i * si + k * sk], i < rows, k < cols, row i scaled
// by rs[i] when rs (device) is given. A row-major matrix is {p, rows, cols, cols, 1}; its
// transpose is {p, cols_of_p, rows_of_p, 1, cols_of_p}.
struct X64Mat {
    const double* p;
    int64_t rows, cols, si, sk;
    const double* rs;
};
// D_l = X_l Y_l^T (X_l: rows_x x K, Y_l: rows_y x K; D_l: rows_x x rows_y, row stride ld_l).
int x64_nt(int n, const X64Mat X[], const X64Mat Y[], double* const D[], const int64_t ld[], int* flag,
           cudaStream_t st, std::string* err);
// D = A B^T (row-major, device memory), synchronised, with the status checked.
int x64_gemm_nt(const double* A, const double* B, int64_t M, int64_t N, int64_t K, double* D, cudaStream_t st,
                std::string* err);

}  // namespace ls
