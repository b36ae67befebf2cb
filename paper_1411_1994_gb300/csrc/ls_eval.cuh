// Slab evaluation on tcgen05 tensor cores (two exact digits + two tails operand
// form in FP16, exact accumulation of the two leading levels); see ls_eval.cu.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>

namespace ls {

// An operand in digit + tail form: FP16 parts[p][b][i][k] (p = 0: digit d0, 1: d1
// 2^-7, 2, 3: tails; all times 2^9), `batch` stacked matrices of `rows` rows of
// `kpad` (a multiple of 32) entries, and the row exponents e[b][i].
struct DtOp {
    uint16_t* p = nullptr;
    int* e = nullptr;
    int64_t rows = 0, kpad = 0, batch = 1;
    bool ok() const { return p && e; }
};

enum DtOutMode : int { DT_F32 = 0, DT_F64 = 1, DT_PAIR = 2 };

// Output of a product: D[z][m][n] at p[z * zs + n * ldn + m] (m contiguous) as FP32,
// FP64 or an unevaluated FP32 pair (float2 hi, lo).
struct DtOut {
    void* p;
    int64_t ldn, zs;
    int mode;
};

// tile_n: output tile width (32, 64 or 128; 0 picks by N).
struct DtOpts {
    int tile_n = 0;
};

// Operands of one reduced tensor kept between evaluations.
struct DtEvalCache;
void dt_eval_free(DtEvalCache* c);

// S_s[x][y] = sum_{a,b,c} B[a][b][c] Z0[a][x] Z1[b][y] Z2[c][zidx[s]] for the
// nslab slabs (zidx: device int32), into out (nslab x N x N, FP32 if out_f32
// else FP64). Builds *cache on first use. Synchronises to read the kernels'
// status flag. Ranks up to 2048.
int dt_eval(DtEvalCache** cache, const double* const Z[3], const int32_t* r, const double* B, int64_t N,
            const int32_t* zidx, int nslab, void* out, int out_f32, const DtOpts& opt, cudaStream_t st,
            std::string* err);

// D = A B^T (A: M x K, B: N x K, D: M x N row-major; device memory; K <= 2048) by
// the same product, synchronised, with the status checked.
int dt_gemm_nt(const double* A, const double* B, int64_t M, int64_t N, int64_t K, void* D, int out_f32,
               const DtOpts& opt, cudaStream_t st, std::string* err);

}  // namespace ls
