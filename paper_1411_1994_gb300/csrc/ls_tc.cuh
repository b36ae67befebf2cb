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

// Slab evaluation on tcgen05 tensor cores.
int tc_eval(const double* const Z[3], const int32_t* r, const double* B, int64_t N, const int32_t* zidx,
            int nslab, double* work, void* out, int out_f32, int num_sms, cudaStream_t st, std::string* err);

}  // namespace ls
