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
// FP64 (optionally added to p) or an unevaluated FP32 pair (float2 hi, lo).
struct DtOut {
    void* p;
    int64_t ldn, zs;
    int mode;
    int accumulate = 0;   // DT_F64 only: p += D
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
// status flag. Ranks up to 4096. With tune_report, the first chunk's three
// products are each timed at every tile width and the fastest width is kept for
// their shapes (later products of those shapes use it); the timings are appended
// to *tune_report as JSON members.
int dt_eval(DtEvalCache** cache, const double* const Z[3], const int32_t* r, const double* B, int64_t N,
            const int32_t* zidx, int nslab, void* out, int out_f32, const DtOpts& opt, cudaStream_t st,
            std::string* err, std::string* tune_report = nullptr);

// D = A B^T (A: M x K, B: N x K, D: M x N row-major; device memory) by the same
// product, synchronised, with the status checked. K above 4096 runs in exact chunks
// added in FP64 (FP64 output only).
int dt_gemm_nt(const double* A, const double* B, int64_t M, int64_t N, int64_t K, void* D, int out_f32,
               const DtOpts& opt, cudaStream_t st, std::string* err);

// Core contraction of the reduced tensor (Thm A.1(c)) in the same arithmetic:
//   B[i][j][k] = sum_t xin[t] P0[i][c0(t)] P1[j][c1(t)] P2[k][c2(t)].
// Terms come grouped by mode-0 column (perm, off: host arrays, CSR offsets over
// C[0] groups). Step 1 is one grouped product with a K range per group:
//   W[g][j][k] = sum_{t in g} xin[t] P1[j][c1(t)] P2[k][c2(t)],
// kept as FP32 pairs. Step 2 is B_(0) = P0 W, over chunks of at most 2048
// groups added in FP64. P_l: r_l x C_l row-major; tcol: [T][3] device; xin:
// device; B: device, r0 x r1 x r2. Asynchronous; `flag` receives FLAG_TIMEOUT
// if a bounded wait gives up.
int dt_core(const double* P0, const double* P1, const double* P2, const int32_t* C, const int32_t* r,
            const int32_t* tcol, const double* xin, const int32_t* perm, const int32_t* off, int64_t T, double* Bc,
            int* flag, cudaStream_t st, std::string* err);

}  // namespace ls
