// Tensor-core (tcgen05) kernels of the mixed-precision path.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>

namespace ls {

// Core contraction on tcgen05 tensor cores (BF16x3 split products, FP32
// accumulation in TMEM): B[i][j][k] = sum_t xin[t] P0[i][c0] P1[j][c1] P2[k][c2].
int tc_core(const double* P0, const double* P1, const double* P2, const int32_t* C, const int32_t* r,
            const int32_t* tcol, const double* xin, const int32_t* perm, const int32_t* off, int64_t T, double* B,
            int num_sms, cudaStream_t st, std::string* err);

// Projection on tcgen05 tensor cores: P[k][c] = sum_i Z[k][i] a[c][i].
int tc_project(const double* Z, int r, const double* a, int64_t C, int64_t N, double* P, cudaStream_t st,
               std::string* err);

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
