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
// G_l = diag(w_l) A_l A_l^T diag(w_l)  (A_l: C_l rows of length N; w may be NULL).
int x64_gram(int n, const double* const a[], const int64_t C[], int64_t N, const double* const w[], double* const G[],
             int* flag, cudaStream_t st, std::string* err);
// P_l = Z_l A_l^T  (Z_l: r_l x N, A_l: C_l x N, P_l: r_l x C_l).
int x64_project(int n, const double* const Z[], const int r[], const double* const a[], const int64_t C[], int64_t N,
                double* const P[], int* flag, cudaStream_t st, std::string* err);
// dst_l = T_l src_l  (T_l: r_l x r_l, src_l and dst_l: r_l x N).
int x64_apply(int n, const double* const T[], const int r[], const double* const src[], int64_t N,
              double* const dst[], int* flag, cudaStream_t st, std::string* err);
// D = A B^T (row-major, device memory), synchronised, with the status checked.
int x64_gemm_nt(const double* A, const double* B, int64_t M, int64_t N, int64_t K, double* D, cudaStream_t st,
                std::string* err);

}  // namespace ls
