// FP64-grade products on tcgen05 tensor cores for sm_103a (the exact-slice
// scheme below): the reduction's dense FP64 contractions (weighted Gram
// matrices, Def. 4.1 / Thm 2.1; CholeskyQR products; the projection P = Z A^T,
// Thm A.1(c)). One tile of 128 x 64 outputs per CTA, operands in 64B-swizzled
// shared memory by TMA through two stages of k-blocks of 32 (plain loads; no
// multicast), one thread issuing tcgen05.mma for the CTA, four epilogue warps
// reading the accumulators back with tcgen05.ld. Every mbarrier wait is
// bounded: on timeout the kernel raises a flag, drains the copies it issued,
// frees its TMEM and returns.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cudaTypedefs.h>

#include <string.h>

#include <algorithm>
#include <mutex>
#include <string>
#include <vector>

#include "lattice_sum.h"
#include "ls_common.cuh"
#include "ls_tc.cuh"
#include "ls_tcgen05.cuh"

namespace ls {

namespace {

using namespace tc5;

constexpr int TBM = 128, TBN = 64, TBK = 32;
constexpr int TILE_A = TBM * TBK * 2;          // bytes of one bf16 A tile (8 KB)
constexpr int TILE_B = TBN * TBK * 2;          // 4 KB

enum OutMode : int { OUT_F64 = 0, OUT_F32 = 1 };

struct TcOut {
    void* p;            // D
    int64_t ld;         // row stride (elements)
    int64_t zs;         // batch stride (elements)
    int mode;
    int accumulate;     // F64 only: D += result
    int negate;         // F64 only: the result enters with a minus sign
};

// ---------------------------------------------------------------------------
// FP64-grade products on the tensor cores: exact slices
//
// Each operand row is scaled by 2^-E (its largest entry then below 1/2 in
// magnitude) and written as eight balanced base-128 digits d_i in [-64, 64]:
// x = 2^E sum_i d_i 128^-(i+1), to 2^-57 of 2^E. The digits are integers,
// exact in BF16. Products d_i d_j (|.| <= 2^12) of one level l = i + j (at
// most eight pairs) summed over K <= 512 stay below 2^24, so each level
// accumulates EXACTLY in its own FP32 TMEM accumulator; the 36 pairs with
// l <= 7 are all that lie above 2^-56 of the result. The epilogue recombines
// the exact level sums by integer Horner steps (levels 0-3 and 4-7), converts
// once to FP64 and applies 2^(E_a + E_b): a product is good to about 2^-53 of
// sum_k |a_k| |b_k|, as an FP64 dot product is, while the arithmetic runs on
// the tensor cores. A stage of 8 slices x (128 + 64) rows x 32 k takes 96 KB of
// shared memory, so that the next k-block loads while the MMAs of this one run;
// the eight accumulators fill TMEM's 512 columns.
// ---------------------------------------------------------------------------
constexpr int XSL = 8;                              // slices (digits)
constexpr int XKCHUNK = 512;                        // K per exact accumulation
constexpr int XSTAGE = XSL * (TILE_A + TILE_B);     // 96 KB
constexpr int XNST = 2;                             // stages
constexpr int XTMEM = XSL * TBN;                    // 512 columns
// warp 0 TMA, warp 1 MMA + TMEM, warps 2-9 epilogue: two warps a TMEM lane quarter, each
// holding the running FP64 sums of half the tile's columns in registers across the K-chunks
constexpr int X64_THREADS = 320;
constexpr int X64_EPI_COLS = TBN / 2;

struct X64Job {
    CUtensorMap a, b;     // (k, row, slice): the eight digit matrices of each operand
    int M, N, nkb;        // k-blocks of 64 over all of K
    int tiles_n, b0;      // tiles along N; first block of the job
    int transposed;       // D stored at out.p[n * out.ld + m]
    int upper;            // only tiles that reach the diagonal or above it (a symmetric D's upper part)
    const int* skip;      // if given and nonzero when the CTA starts: nothing to do
    const int* ea;
    const int* eb;
    TcOut out;
};
constexpr int kX64MaxJobs = 3;
struct X64Group {
    X64Job j[kX64MaxJobs];
    int n;
};

// RN((hi 2^28 + lo) 2^s) for |hi|, |lo| < 2^46: the recombined level sums as a double,
// rounded once to nearest-even like fma((double)hi, 2^-35, (double)lo 2^-63) scaled by
// 2^(s + 63), but built on the integer pipe (the bit length, a shift of the 128-bit sum,
// the round bit and sticky bits, the exponent field): FP64 instructions run at a small
// fraction of the integer rate on this GPU, and the epilogue converts every output entry
// of every K-chunk. Results outside the normal range take the FP64 formula.
__device__ __forceinline__ double rn_scaled(long long hi, long long lo, int s) {
    const __int128 X = ((__int128)hi << 28) + (__int128)lo;
    if (X == 0) return 0.0;
    const bool neg = X < 0;
    const unsigned __int128 A = neg ? (unsigned __int128)(-X) : (unsigned __int128)X;
    const unsigned long long ah = (unsigned long long)(A >> 64), al = (unsigned long long)A;
    const int nb = ah ? 128 - __clzll((long long)ah) : 64 - __clzll((long long)al);   // bit length, <= 75
    int e = nb - 1 + s;                                                                 // unbiased exponent
    unsigned long long m;                                                               // 53 significant bits
    if (nb <= 53) {
        m = al << (53 - nb);
    } else {
        const int sh = nb - 53;   // 1 .. 22
        m = (al >> sh) | (sh < 64 ? (ah << (64 - sh)) : 0ull);
        const unsigned long long rem = al & ((1ull << sh) - 1), half = 1ull << (sh - 1);
        if (rem > half || (rem == half && (m & 1ull))) {
            if (++m == (1ull << 53)) {
                m >>= 1;
                ++e;
            }
        }
    }
    if (e < -1022 || e > 1023) return ldexp(fma((double)hi, 0x1p-35, (double)lo * 0x1p-63), s + 63);
    const unsigned long long bits =
        (neg ? 0x8000000000000000ull : 0ull) | ((unsigned long long)(e + 1023) << 52) | (m & 0xfffffffffffffull);
    return __longlong_as_double((long long)bits);
}

// One 128 x 64 output tile of one job per CTA, all of K: the K-chunks of 512 run in
// turn on the same eight accumulators (the MMA warp waits until the epilogue has drained
// them). The epilogue adds each chunk's recombined value to a running FP64 sum in
// registers (the first chunk starting from the output where it accumulates) and writes
// the tile, which only this CTA writes, once: the same additions in the same order as
// adding every chunk into the output in turn.
__global__ void __launch_bounds__(X64_THREADS, 1) k_x64_gemm(const __grid_constant__ X64Group G, int* flag) {
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    unsigned char* smem = (unsigned char*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    uint64_t* full = (uint64_t*)(smem + XNST * XSTAGE);   // [XNST]
    uint64_t* empty = full + XNST;                       // [XNST]
    uint64_t* accum = empty + XNST;   // accumulators of a chunk complete
    uint64_t* drained = accum + 1;    // epilogue has read them
    uint32_t* tmem_slot = (uint32_t*)(drained + 1);
    int ji = 0;
    while (ji + 1 < G.n && (int)blockIdx.x >= G.j[ji + 1].b0) ++ji;
    const X64Job& J = G.j[ji];
    const int tile = (int)blockIdx.x - J.b0;
    const int tm = tile / J.tiles_n, tn = tile - tm * J.tiles_n;
    const int n0 = tn * TBN, m0 = tm * TBM;
    if (J.upper && m0 >= n0 + TBN) return;   // strictly below the diagonal: not wanted
    if (J.skip && *(volatile const int*)J.skip) return;
    const int kbc = XKCHUNK / TBK;
    const int nchunk = (J.nkb + kbc - 1) / kbc;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

    if (threadIdx.x == 0) {
        for (int s = 0; s < XNST; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], 1);
        }
        mbar_init(accum, 1);
        mbar_init(drained, (X64_THREADS - 64) / 32);   // one arrival per epilogue warp
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                     "r"(XTMEM));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    const uint32_t tmem = *tmem_slot;

    if (warp == 0 && lane == 0) {
        // TMA producer: a ring of XNST stages, each refilled once the MMAs that read it are done
        int issued = 0;
        for (int kb = 0; kb < J.nkb; ++kb) {
            const int s = kb % XNST, u = kb / XNST;
            if (u > 0 && !mbar_wait(&empty[s], (u - 1) & 1, flag)) break;
            const int kx = kb * TBK;
            unsigned char* st = smem + s * XSTAGE;
            mbar_expect_tx(&full[s], XSTAGE);
#pragma unroll
            for (int i = 0; i < XSL; ++i) tma_load_3d(st + i * TILE_A, &J.a, kx, m0, i, &full[s]);
#pragma unroll
            for (int j = 0; j < XSL; ++j) tma_load_3d(st + XSL * TILE_A + j * TILE_B, &J.b, kx, n0, j, &full[s]);
            issued = kb + 1;
        }
        // every issued stage must have landed before the CTA may exit
        for (int j = issued > XNST ? issued - XNST : 0; j < issued; ++j) mbar_drain(&full[j % XNST], (j / XNST) & 1);
    } else if (warp == 1 && lane == 0) {
        // MMA issuer: pair (i, j) into the accumulator of level i + j; a chunk starts from zero
        const uint32_t idesc = idesc_bf16(TBM, TBN);
        bool ok = true;
        for (int c = 0; c < nchunk && ok; ++c) {
            if (c > 0 && !mbar_wait(drained, (c - 1) & 1, flag)) break;
            asm volatile("tcgen05.fence::after_thread_sync;");
            const int kbe = min(J.nkb, (c + 1) * kbc);
            for (int kb = c * kbc; kb < kbe; ++kb) {
                const int s = kb % XNST;
                if (!mbar_wait(&full[s], (kb / XNST) & 1, flag)) { ok = false; break; }
                asm volatile("tcgen05.fence::after_thread_sync;");
                const uint32_t base = smem_u32(smem + s * XSTAGE);
                const bool first_kb = kb == c * kbc;
#pragma unroll
                for (int kk = 0; kk < TBK / 16; ++kk) {
                    const uint64_t o = (uint64_t)((kk * 32) >> 4);   // 16 bf16 = 32 bytes along K
#pragma unroll
                    for (int l = 0; l < XSL; ++l)
#pragma unroll
                        for (int i = 0; i <= l; ++i) {
                            const uint64_t a = smem_desc_sw64(base + i * TILE_A) + o;
                            const uint64_t b = smem_desc_sw64(base + XSL * TILE_A + (l - i) * TILE_B) + o;
                            mma_bf16(tmem + (uint32_t)(l * TBN), a, b, idesc, (!first_kb || kk || i) ? 1u : 0u);
                        }
                }
                mma_commit(&empty[s]);
            }
            mma_commit(accum);
        }
    } else if (warp >= 2) {
        const int q = warp & 3, c0 = ((warp - 2) >> 2) * X64_EPI_COLS;
        const int row = m0 + 32 * q + lane;
        const int er = row < J.M ? J.ea[row] : 0;
        const uint32_t lanes = (uint32_t)(32 * q) << 16;
        double acc[X64_EPI_COLS];
        bool all = true;
        for (int c = 0; c < nchunk; ++c) {
            if (!mbar_wait(accum, c & 1, flag)) { all = false; break; }
            asm volatile("tcgen05.fence::after_thread_sync;");
#pragma unroll
            for (int g = 0; g < X64_EPI_COLS / 8; ++g) {
                const int cc = c0 + 8 * g;
                // the eight levels of eight columns: eight loads, one wait
                uint32_t S[XSL][8];
#pragma unroll
                for (int l = 0; l < XSL; ++l) tmem_ld8_issue(tmem + lanes + (uint32_t)(l * TBN + cc), S[l]);
                tmem_wait_ld();
#pragma unroll
                for (int l = 0; l < XSL; ++l) reg_after_wait8(S[l]);
                if (row >= J.M) continue;
#pragma unroll
                for (int jj = 0; jj < 8; ++jj) {
                    const int col = n0 + cc + jj;
                    if (col >= J.N) continue;
                    // exact level sums (integers below 2^24), recombined by Horner steps in int64
                    long long hi = 0, lo = 0;
#pragma unroll
                    for (int l = 0; l < 4; ++l) hi = hi * 128 + (long long)__float2int_rn(__uint_as_float(S[l][jj]));
#pragma unroll
                    for (int l = 4; l < 8; ++l) lo = lo * 128 + (long long)__float2int_rn(__uint_as_float(S[l][jj]));
                    // sum_l S_l 2^(-7(l+2)) = (hi 2^28 + lo) 2^-63, times 2^(E_a + E_b)
                    const double v0 = rn_scaled(hi, lo, er + J.eb[col] - 63);
                    const double v = J.out.negate ? -v0 : v0;
                    double& a = acc[8 * g + jj];
                    if (c > 0) {
                        a = a + v;
                    } else if (J.out.accumulate) {
                        const double* o = (const double*)J.out.p +
                                          (J.transposed ? (int64_t)col * J.out.ld + row : (int64_t)row * J.out.ld + col);
                        a = *o + v;
                    } else {
                        a = v;
                    }
                }
            }
            asm volatile("tcgen05.fence::before_thread_sync;");
            __syncwarp();
            if (lane == 0) asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(drained)) : "memory");
        }
        if (all && row < J.M) {
#pragma unroll
            for (int i = 0; i < X64_EPI_COLS; ++i) {
                const int col = n0 + c0 + i;
                if (col >= J.N) continue;
                double* o = (double*)J.out.p + (J.transposed ? (int64_t)col * J.out.ld + row : (int64_t)row * J.out.ld + col);
                *o = acc[i];
            }
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    if (warp == 1) {
        asm volatile("tcgen05.fence::after_thread_sync;");
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(XTMEM));
    }
}

struct X64Ptrs {
    __nv_bfloat16* p[XSL];
};

// The digits of one entry from V = round(x 2^(56 - E)) (|V| < 2^55): balanced base-128
// digits taken from the least significant by integer steps (V - d is a multiple of 128,
// so the arithmetic shift is an exact division); one FP64 multiply and one conversion an
// entry, the rest on the integer pipe.
__device__ __forceinline__ void x64_digits(double x_scaled, int64_t at, const X64Ptrs& d) {
    long long V = __double2ll_rn(x_scaled);
#pragma unroll
    for (int i = XSL - 1; i > 0; --i) {
        int r = (int)(V & 127);
        if (r >= 64) r -= 128;
        d.p[i][at] = __int2bfloat16_rn(r);
        V = (V - r) >> 7;
    }
    d.p[0][at] = __int2bfloat16_rn((int)V);
}
// |x| as an integer: non-negative doubles order like their bit patterns
__device__ __forceinline__ unsigned long long abs_bits(double x) {
    return (unsigned long long)__double_as_longlong(x) & 0x7fffffffffffffffull;
}

// Operands of one or more products, split in one launch: source j contributes rows
// i < rows of x(i, k) = src[i*si + k*sk] (k < cols), scaled by rs[i] if given; its
// CTAs start at cta0. One CTA per row. E = exponent with max_k |x| in
// [2^(E-2), 2^(E-1)), so that x 2^-E lies in (-1/2, 1/2) and its digits in [-64, 64];
// zero digits past cols. A transposed source is read with si = 1, sk = its row stride.
struct X64Split {
    const double* src;
    int64_t rows, cols, si, sk;
    const double* rs;
    X64Ptrs d;
    int* e;
    int64_t kpad, cta0;
};
constexpr int kX64MaxSplits = 6;
struct X64SplitGroup {
    X64Split s[kX64MaxSplits];
    int n;
};

__global__ void __launch_bounds__(128) k_split_x64(const __grid_constant__ X64SplitGroup G) {
    __shared__ unsigned long long s_mb[4];
    int j = 0;
    while (j + 1 < G.n && (int64_t)blockIdx.x >= G.s[j + 1].cta0) ++j;
    const X64Split& S = G.s[j];
    const int64_t i = blockIdx.x - S.cta0;
    const double* x = S.src + i * S.si;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    unsigned long long mb = 0;
    for (int64_t k = threadIdx.x; k < S.cols; k += blockDim.x) mb = max(mb, abs_bits(x[k * S.sk]));
    for (int o = 16; o; o >>= 1) mb = max(mb, __shfl_xor_sync(0xffffffffu, mb, o));
    if (lane == 0) s_mb[warp] = mb;
    __syncthreads();
    mb = max(max(s_mb[0], s_mb[1]), max(s_mb[2], s_mb[3]));
    const double sc = S.rs ? fabs(S.rs[i]) : 1.0;
    const double mx = sc * __longlong_as_double((long long)mb);
    const int E = mx > 0.0 ? ilogb(mx) + 2 : 0;
    if (threadIdx.x == 0) S.e[i] = E;
    const double f = (S.rs ? S.rs[i] : 1.0) * ldexp(1.0, 56 - E);
    for (int64_t k = threadIdx.x; k < S.kpad; k += blockDim.x)
        x64_digits(k < S.cols ? x[k * S.sk] * f : 0.0, i * S.kpad + k, S.d);
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
// rows x kpad bf16 matrices, `batch` of them back to back; box = box_rows x 32 (64-byte swizzle)
bool make_map(CUtensorMap* m, const void* base, int64_t rows, int64_t kpad, int64_t batch, int box_rows) {
    auto fn = encode_fn();
    if (!fn) return false;
    cuuint64_t dims[3] = {(cuuint64_t)kpad, (cuuint64_t)rows, (cuuint64_t)batch};
    cuuint64_t strides[2] = {(cuuint64_t)(kpad * 2), (cuuint64_t)(rows * kpad * 2)};
    cuuint32_t box[3] = {(cuuint32_t)TBK, (cuuint32_t)box_rows, 1};
    cuuint32_t es[3] = {1, 1, 1};
    CUresult r = fn(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, const_cast<void*>(base), dims, strides, box, es,
                    CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_64B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                    CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS;
}

int64_t pad64(int64_t x) { return (x + 63) / 64 * 64; }

// an operand in exact-slice form: eight digit matrices (rows x kpad) and a row exponent
struct X64Op {
    X64Ptrs d{};
    int* e = nullptr;
    int64_t rows = 0, kpad = 0;
    bool ok() const {
        for (int i = 0; i < XSL; ++i)
            if (!d.p[i]) return false;
        return e != nullptr;
    }
};

X64Op x64_alloc(Arena& ar, int64_t rows, int64_t kpad) {
    X64Op x;
    // one allocation for the eight slices
    __nv_bfloat16* base = ar.get<__nv_bfloat16>((int64_t)XSL * rows * kpad);
    for (int i = 0; i < XSL; ++i) x.d.p[i] = base ? base + (int64_t)i * rows * kpad : nullptr;
    x.e = ar.get<int>(rows);
    x.rows = rows;
    x.kpad = kpad;
    return x;
}


// Operand splits collected and launched together (flushed when full or on demand)
struct SplitBatch {
    cudaStream_t st;
    X64SplitGroup g{};
    int64_t ctas = 0;
    cudaError_t err = cudaSuccess;
    explicit SplitBatch(cudaStream_t s) : st(s) { g.n = 0; }
    // rows of x(i, k) = src[i*si + k*sk] times rs[i] (if given) into d
    void add(const double* src, int64_t rows, int64_t cols, int64_t si, int64_t sk, const double* rs, const X64Op& d) {
        if (rows <= 0) return;
        if (g.n == kX64MaxSplits) flush();
        g.s[g.n++] = X64Split{src, rows, cols, si, sk, rs, d.d, d.e, d.kpad, ctas};
        ctas += rows;
    }
    cudaError_t flush() {
        if (g.n > 0 && err == cudaSuccess) {
            k_split_x64<<<(unsigned)ctas, 128, 0, st>>>(g);
            count_kernels(1);
            err = cudaGetLastError();
        }
        g.n = 0;
        ctas = 0;
        return err;
    }
};

// one product of a group: D (+)= A B^T, A: M x kpad, B: N x kpad (exact-slice form)
struct X64Spec {
    const X64Op* A;
    const X64Op* B;
    int64_t M, N;
    TcOut out;
    int transposed;
    int upper;   // compute only the tiles that reach the diagonal or above it
    const int* skip = nullptr;   // device flag: the product is not wanted when it is nonzero
};

// up to kX64MaxJobs products in one launch; out.mode must be OUT_F64
int gemm_x64(const X64Spec* sp, int n, int* flag, cudaStream_t st, std::string* err) {
    if (n < 1) return LS_OK;
    if (n > kX64MaxJobs) return tc_err(err, "x64 gemm: too many products", LS_ERR_ARG);
    X64Group g;
    memset(&g, 0, sizeof g);
    int blocks = 0;
    for (int i = 0; i < n; ++i) {
        const X64Spec& s0 = sp[i];
        const int64_t kpad = s0.A->kpad;
        if (kpad % TBK != 0 || s0.B->kpad != kpad || s0.out.mode != OUT_F64)
            return tc_err(err, "x64 gemm: bad operands", LS_ERR_ARG);
        X64Job& J = g.j[i];
        // the slices of an operand lie rows x kpad apart in one allocation: one map each
        if (s0.M > s0.A->rows || s0.N > s0.B->rows ||
            !make_map(&J.a, s0.A->d.p[0], s0.A->rows, kpad, XSL, TBM) || !make_map(&J.b, s0.B->d.p[0], s0.B->rows, kpad, XSL, TBN))
            return tc_err(err, "x64 gemm: cuTensorMapEncodeTiled failed");
        J.M = (int)s0.M;
        J.N = (int)s0.N;
        J.nkb = (int)(kpad / TBK);
        J.tiles_n = (int)((s0.N + TBN - 1) / TBN);
        J.b0 = blocks;
        J.transposed = s0.transposed;
        J.upper = s0.upper;
        J.skip = s0.skip;
        J.ea = s0.A->e;
        J.eb = s0.B->e;
        J.out = s0.out;
        blocks += (int)((s0.M + TBM - 1) / TBM) * J.tiles_n;
    }
    g.n = n;
    if (blocks == 0) return LS_OK;
    const size_t smem = XNST * XSTAGE + 1024 + 256;
    static std::once_flag attr_once;
    static cudaError_t attr_err = cudaSuccess;
    std::call_once(attr_once, [&] {
        attr_err = cudaFuncSetAttribute(k_x64_gemm, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    });
    if (attr_err != cudaSuccess) return tc_err(err, "x64 gemm: cannot reserve shared memory");
    k_x64_gemm<<<blocks, X64_THREADS, smem, st>>>(g, flag);
    count_kernels(1);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return tc_err(err, std::string("x64 gemm launch: ") + cudaGetErrorString(e));
    return LS_OK;
}


}  // namespace

// FP64-grade products on the tensor cores (exact slices) -------------------
// G_l = diag(w_l) A_l A_l^T diag(w_l), A_l: C_l rows of length N
int x64_gram(int n, const double* const a[], const int64_t C[], int64_t N, const double* const w[], double* const G[],
             int* flag, cudaStream_t st, std::string* err, const int* upper) {
    Arena ar(st);
    SplitBatch sb(st);
    std::vector<X64Op> xs(n);
    std::vector<X64Spec> sp(n);
    for (int l = 0; l < n; ++l) {
        xs[l] = x64_alloc(ar, C[l], pad64(N));
        if (!xs[l].ok()) return tc_err(err, "x64_gram: out of memory", LS_ERR_OOM);
        sb.add(a[l], C[l], N, N, 1, w ? w[l] : nullptr, xs[l]);
    }
    if (sb.flush() != cudaSuccess) return tc_err(err, "x64_gram: split failed");
    for (int l = 0; l < n; ++l)
        sp[l] = X64Spec{&xs[l], &xs[l], C[l], C[l], TcOut{G[l], C[l], 0, OUT_F64, 0}, 0, upper ? upper[l] : 0};
    return gemm_x64(sp.data(), n, flag, st, err);
}

// S_l -= L_l[:, k0_l : k0_l + kb_l] L_l[:, k0_l : k0_l + kb_l]^T on the tiles of S_l that
// reach its diagonal or lie above it (S_l symmetric: its readers take S[min(i,j)][max(i,j)]):
// L_l C_l x kmax_l (rows), S_l C_l x C_l; jobs with kb_l = 0 are skipped, and so are those
// whose device flag skip[l] (if given) is nonzero when the product runs
int x64_syrk_sub(int n, const double* const L[], const int64_t kmax[], const int k0[], const int kb[],
                 const int64_t C[], double* const S[], int* flag, cudaStream_t st, std::string* err,
                 const int* const skip[]) {
    for (int l0 = 0; l0 < n; l0 += kX64MaxJobs) {
        Arena ar(st);
        SplitBatch sb(st);
        std::vector<X64Op> xs;
        std::vector<X64Spec> sp;
        xs.reserve(kX64MaxJobs);
        for (int l = l0; l < std::min(n, l0 + kX64MaxJobs); ++l) {
            if (kb[l] <= 0) continue;
            xs.push_back(x64_alloc(ar, C[l], pad64(kb[l])));
            if (!xs.back().ok()) return tc_err(err, "x64_syrk_sub: out of memory", LS_ERR_OOM);
            sb.add(L[l] + k0[l], C[l], kb[l], kmax[l], 1, nullptr, xs.back());
        }
        if (xs.empty()) continue;
        if (sb.flush() != cudaSuccess) return tc_err(err, "x64_syrk_sub: split failed");
        int i = 0;
        for (int l = l0; l < std::min(n, l0 + kX64MaxJobs); ++l) {
            if (kb[l] <= 0) continue;
            sp.push_back(X64Spec{&xs[i], &xs[i], C[l], C[l], TcOut{S[l], C[l], 0, OUT_F64, 1, 1}, 0, 1,
                                 skip ? skip[l] : nullptr});
            ++i;
        }
        const int rc = gemm_x64(sp.data(), (int)sp.size(), flag, st, err);
        if (rc != LS_OK) return rc;
    }
    return LS_OK;
}

// P_l = Z_l A_l^T: Z_l r_l x N, A_l C_l x N (rows), P_l r_l x C_l
int x64_project(int n, const double* const Z[], const int r[], const double* const a[], const int64_t C[], int64_t N,
                double* const P[], int* flag, cudaStream_t st, std::string* err) {
    Arena ar(st);
    SplitBatch sb(st);
    const int64_t kp = pad64(N);
    std::vector<X64Op> zs(n), as(n);
    std::vector<X64Spec> sp(n);
    for (int l = 0; l < n; ++l) {
        zs[l] = x64_alloc(ar, r[l], kp);
        as[l] = x64_alloc(ar, C[l], kp);
        if (!zs[l].ok() || !as[l].ok()) return tc_err(err, "x64_project: out of memory", LS_ERR_OOM);
        sb.add(Z[l], r[l], N, N, 1, nullptr, zs[l]);
        sb.add(a[l], C[l], N, N, 1, nullptr, as[l]);
        sp[l] = X64Spec{&zs[l], &as[l], r[l], C[l], TcOut{P[l], C[l], 0, OUT_F64, 0}, 0};
    }
    if (sb.flush() != cudaSuccess) return tc_err(err, "x64_project: split failed");
    return gemm_x64(sp.data(), n, flag, st, err);
}

// dst_l = T_l src_l: T_l r_l x r_l, src_l and dst_l r_l x N (rows). Computed as
// dst^T = src^T T^T (src read transposed by the split) with a transposed store: each
// epilogue warp writes 32 consecutive entries of a row of dst.
int x64_apply(int n, const double* const T[], const int r[], const double* const src[], int64_t N,
              double* const dst[], int* flag, cudaStream_t st, std::string* err) {
    Arena ar(st);
    SplitBatch sb(st);
    std::vector<X64Op> ss(n), ts(n);
    std::vector<X64Spec> sp(n);
    for (int l = 0; l < n; ++l) {
        const int64_t kp = pad64(r[l]);
        ss[l] = x64_alloc(ar, N, kp);
        ts[l] = x64_alloc(ar, r[l], kp);
        if (!ss[l].ok() || !ts[l].ok()) return tc_err(err, "x64_apply: out of memory", LS_ERR_OOM);
        sb.add(src[l], N, r[l], 1, N, nullptr, ss[l]);
        sb.add(T[l], r[l], r[l], r[l], 1, nullptr, ts[l]);
        sp[l] = X64Spec{&ss[l], &ts[l], N, r[l], TcOut{dst[l], N, 0, OUT_F64, 0}, 1};
    }
    if (sb.flush() != cudaSuccess) return tc_err(err, "x64_apply: split failed");
    return gemm_x64(sp.data(), n, flag, st, err);
}

// Y_l[m][x] = isl[m] sum_c V_l[c][perm[m]] w[c] a_l[c][x]  (the basis step): the row
// factor A~[m][c] = isl[m] V[c][perm[m]] w[c] is formed first, a_l is transposed, and
// the product is taken as Y^T = a_l^T A~^T with a transposed store.
__global__ void k_basis_rows(const double* __restrict__ V, int64_t ldv, const int32_t* __restrict__ perm,
                             const double* __restrict__ w, const double* __restrict__ isl, int64_t C, int r,
                             double* __restrict__ At) {
    const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e >= (int64_t)r * C) return;
    const int m = (int)(e / C);
    const int64_t c = e - (int64_t)m * C;
    At[e] = V[c * ldv + perm[m]] * w[c] * isl[m];
}

int x64_basis(int n, const double* const V[], const int64_t ldv[], const int32_t* const perm[],
              const double* const w[], const double* const isl[], const double* const a[], const int64_t C[],
              int64_t N, const int r[], double* const Y[], int* flag, cudaStream_t st, std::string* err) {
    Arena ar(st);
    SplitBatch sb(st);
    std::vector<X64Op> as(n), ys(n);
    std::vector<X64Spec> sp(n);
    for (int l = 0; l < n; ++l) {
        const int64_t kp = pad64(C[l]);
        double* At = ar.get<double>((int64_t)r[l] * C[l]);
        as[l] = x64_alloc(ar, N, kp);
        ys[l] = x64_alloc(ar, r[l], kp);
        if (!At || !as[l].ok() || !ys[l].ok()) return tc_err(err, "x64_basis: out of memory", LS_ERR_OOM);
        const int64_t ne = (int64_t)r[l] * C[l];
        k_basis_rows<<<(unsigned)((ne + 255) / 256), 256, 0, st>>>(V[l], ldv[l], perm[l], w[l], isl[l], C[l], r[l], At);
        count_kernels(1);
        if (cudaGetLastError() != cudaSuccess) return tc_err(err, "x64_basis: launch failed");
        sb.add(a[l], N, C[l], 1, N, nullptr, as[l]);      // a_l^T, read transposed
        sb.add(At, r[l], C[l], C[l], 1, nullptr, ys[l]);
        sp[l] = X64Spec{&as[l], &ys[l], N, r[l], TcOut{Y[l], N, 0, OUT_F64, 0}, 1};
    }
    if (sb.flush() != cudaSuccess) return tc_err(err, "x64_basis: split failed");
    return gemm_x64(sp.data(), n, flag, st, err);
}

// rs[j] = 1/sqrt(H[j][j]) where positive, else 0
__global__ void k_diag_rsqrt(const double* __restrict__ H, int k, double* __restrict__ rs) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= k) return;
    const double h = H[(int64_t)j * k + j];
    rs[j] = h > 0.0 ? 1.0 / sqrt(h) : 0.0;
}

// Vg_l[c][j] = sum_i L_l[c][i] U_l[i][j] / sqrt(H_l[j][j])  (C_l x k_l, row stride k_l; L_l has
// row stride kmax_l): eigenvectors of the compressed Gram matrix, as Vg^T = (U^T scaled) L^T
// with a transposed store.
int x64_pchol_vectors(int n, const double* const L[], const int64_t kmax[], const int k[], const int64_t C[],
                      const double* const U[], const double* const H[], double* const Vg[], int* flag,
                      cudaStream_t st, std::string* err) {
    Arena ar(st);
    SplitBatch sb(st);
    std::vector<X64Op> us(n), ls(n);
    std::vector<X64Spec> sp(n);
    for (int l = 0; l < n; ++l) {
        const int64_t kp = pad64(k[l]);
        double* rs = ar.get<double>(k[l]);
        us[l] = x64_alloc(ar, k[l], kp);
        ls[l] = x64_alloc(ar, C[l], kp);
        if (!rs || !us[l].ok() || !ls[l].ok()) return tc_err(err, "x64_pchol_vectors: out of memory", LS_ERR_OOM);
        k_diag_rsqrt<<<(k[l] + 127) / 128, 128, 0, st>>>(H[l], k[l], rs);
        count_kernels(1);
        if (cudaGetLastError() != cudaSuccess) return tc_err(err, "x64_pchol_vectors: launch failed");
        sb.add(U[l], k[l], k[l], 1, k[l], rs, us[l]);          // U^T, read transposed, rows scaled
        sb.add(L[l], C[l], k[l], kmax[l], 1, nullptr, ls[l]);
        sp[l] = X64Spec{&us[l], &ls[l], k[l], C[l], TcOut{Vg[l], k[l], 0, OUT_F64, 0}, 1};
    }
    if (sb.flush() != cudaSuccess) return tc_err(err, "x64_pchol_vectors: split failed");
    return gemm_x64(sp.data(), n, flag, st, err);
}

// H_l = L_l^T L_l over the first k_l columns of L_l (C_l rows of stride kmax_l): the
// compressed Gram matrix after the pivoted Cholesky, as X X^T with X = L^T read transposed.
int x64_pchol_gram(int n, const double* const L[], const int64_t kmax[], const int k[], const int64_t C[],
                   double* const H[], int* flag, cudaStream_t st, std::string* err) {
    for (int g0 = 0; g0 < n; g0 += kX64MaxJobs) {
        const int ng = std::min(kX64MaxJobs, n - g0);
        Arena ar(st);
        SplitBatch sb(st);
        std::vector<X64Op> ls(ng);
        std::vector<X64Spec> sp(ng);
        for (int i = 0; i < ng; ++i) {
            const int l = g0 + i;
            ls[i] = x64_alloc(ar, k[l], pad64(C[l]));
            if (!ls[i].ok()) return tc_err(err, "x64_pchol_gram: out of memory", LS_ERR_OOM);
            sb.add(L[l], k[l], C[l], 1, kmax[l], nullptr, ls[i]);
            sp[i] = X64Spec{&ls[i], &ls[i], k[l], k[l], TcOut{H[l], k[l], 0, OUT_F64, 0}, 0};
        }
        if (sb.flush() != cudaSuccess) return tc_err(err, "x64_pchol_gram: split failed");
        int rc = gemm_x64(sp.data(), ng, flag, st, err);
        if (rc != LS_OK) return rc;
    }
    return LS_OK;
}

// out_l = op(A_l) op(B_l) (+ add_l) for k_l x k_l row-major matrices, op = identity or
// transpose (ta, tb): the small dense products of the eigen-solver and of CholeskyQR.
// The product is taken as X Y^T with X = op(A) and Y = op(B)^T in K-major rows
// (transposed copies where needed); add_l (may alias nothing, may be null) is copied to
// out_l first and the product added to it.
int x64_small(int n, const double* const A[], const int ta[], const double* const B[], const int tb[],
              const int k[], double* const out[], const double* const add[], int* flag, cudaStream_t st,
              std::string* err, const int* const skip[]) {
    for (int g0 = 0; g0 < n; g0 += kX64MaxJobs) {
        const int ng = std::min(kX64MaxJobs, n - g0);
        Arena ar(st);
        SplitBatch sb(st);
        std::vector<X64Op> xs(ng), ys(ng);
        std::vector<X64Spec> sp(ng);
        for (int i = 0; i < ng; ++i) {
            const int l = g0 + i, kk = k[l];
            const int64_t kp = pad64(kk);
            xs[i] = x64_alloc(ar, kk, kp);
            ys[i] = x64_alloc(ar, kk, kp);
            if (!xs[i].ok() || !ys[i].ok()) return tc_err(err, "x64_small: out of memory", LS_ERR_OOM);
            // X = op(A) in rows; Y = op(B)^T in rows: transposes are strided reads
            sb.add(A[l], kk, kk, ta[l] ? 1 : kk, ta[l] ? kk : 1, nullptr, xs[i]);
            sb.add(B[l], kk, kk, tb[l] ? kk : 1, tb[l] ? 1 : kk, nullptr, ys[i]);
            if (add && add[l] && add[l] != out[l] &&
                cudaMemcpyAsync(out[l], add[l], sizeof(double) * kk * kk, cudaMemcpyDeviceToDevice, st) != cudaSuccess)
                return tc_err(err, "x64_small: copy failed");
            sp[i] = X64Spec{&xs[i], &ys[i], kk, kk, TcOut{out[l], kk, 0, OUT_F64, (add && add[l]) ? 1 : 0}, 0, 0,
                            skip ? skip[l] : nullptr};
        }
        if (sb.flush() != cudaSuccess) return tc_err(err, "x64_small: split failed");
        int rc = gemm_x64(sp.data(), ng, flag, st, err);
        if (rc != LS_OK) return rc;
    }
    return LS_OK;
}

// T = S^{-1/2} by the series I - Delta/2 + 3/8 Delta^2 - 5/16 Delta^3, Delta = S - I
// (S close to I): Delta, the two powers on the tensor cores, then the combination; the
// elementwise steps take every matrix in one launch (blockIdx.y).
struct LowdinSet {
    const double* S[kX64MaxJobs];
    double* Dl[kX64MaxJobs];
    const double* D2[kX64MaxJobs];
    const double* D3[kX64MaxJobs];
    double* T[kX64MaxJobs];
    double* gate[kX64MaxJobs];   // ||S - I||_F (gated form; else null)
    int* off[kX64MaxJobs];       // gated form: 1 where the gate sends the matrix to the Cholesky pass
    int k[kX64MaxJobs];
};
// gate[j] = ||S_j - I||_F, one block per matrix (fixed reduction order)
__global__ void __launch_bounds__(1024) k_dist_identity(const __grid_constant__ LowdinSet L) {
    const int j = blockIdx.x, k = L.k[j];
    const int64_t n = (int64_t)k * k;
    double acc = 0.0;
    for (int64_t e = threadIdx.x; e < n; e += blockDim.x) {
        const double v = L.S[j][e] - ((e / k) == (e % k) ? 1.0 : 0.0);
        acc = fma(v, v, acc);
    }
    __shared__ double red[32];
    for (int o = 16; o; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
        const double g = sqrt(t);
        *L.gate[j] = g;
        *L.off[j] = !(g < kSeriesGate);   // the test k_lowdin_combine makes
    }
}
__global__ void k_minus_identity(const __grid_constant__ LowdinSet L) {
    const int j = blockIdx.y, k = L.k[j];
    const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e >= (int64_t)k * k) return;
    L.Dl[j][e] = L.S[j][e] - ((e / k) == (e % k) ? 1.0 : 0.0);
}
__global__ void k_lowdin_combine(const __grid_constant__ LowdinSet L) {
    const int j = blockIdx.y, k = L.k[j];
    const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e >= (int64_t)k * k) return;
    if (L.gate[j] && !(*L.gate[j] < kSeriesGate)) return;   // too far from I: the Cholesky pass takes it
    const double id = (e / k) == (e % k) ? 1.0 : 0.0;
    L.T[j][e] = id - 0.5 * L.Dl[j][e] + 0.375 * L.D2[j][e] - 0.3125 * L.D3[j][e];
}

int x64_lowdin(int n, const double* const S[], const int k[], double* const D2[], double* const T[], int* flag,
               cudaStream_t st, std::string* err, double* const gate[]) {
    for (int g0 = 0; g0 < n; g0 += kX64MaxJobs) {
        const int ng = std::min(kX64MaxJobs, n - g0);
        Arena ar(st);
        LowdinSet L{};
        std::vector<const double*> Dlc(ng), D2c(ng);
        std::vector<double*> D3(ng), D2m(ng);
        std::vector<int> zero(ng, 0), one(ng, 1), kk(ng);
        int64_t emax = 1;
        for (int i = 0; i < ng; ++i) {
            const int l = g0 + i;
            const int64_t e = (int64_t)k[l] * k[l];
            L.S[i] = S[l];
            L.Dl[i] = ar.get<double>(e);
            D3[i] = ar.get<double>(e);
            if (!L.Dl[i] || !D3[i]) return tc_err(err, "x64_lowdin: out of memory", LS_ERR_OOM);
            L.D2[i] = D2[l];
            L.D3[i] = D3[i];
            L.T[i] = T[l];
            L.gate[i] = gate ? gate[l] : nullptr;
            L.k[i] = kk[i] = k[l];
            Dlc[i] = L.Dl[i];
            D2c[i] = D2[l];
            D2m[i] = D2[l];
            emax = std::max(emax, e);
        }
        const dim3 grid((unsigned)((emax + 255) / 256), (unsigned)ng);
        // gated form: the powers of a matrix that the gate sends to the Cholesky pass are not
        // formed (its products read the flag that k_dist_identity writes)
        std::vector<const int*> offc(ng, nullptr);
        if (gate) {
            int* off = ar.get<int>(ng);
            if (!off) return tc_err(err, "x64_lowdin: out of memory", LS_ERR_OOM);
            for (int i = 0; i < ng; ++i) offc[i] = L.off[i] = off + i;
            k_dist_identity<<<ng, 1024, 0, st>>>(L);
            count_kernels(1);
        }
        k_minus_identity<<<grid, 256, 0, st>>>(L);
        count_kernels(1);
        // Delta is symmetric: Delta^2 = Delta Delta^T and Delta^3 = Delta^2 Delta^T need no transposes
        const int* const* skip = gate ? offc.data() : nullptr;
        int rc = x64_small(ng, Dlc.data(), zero.data(), Dlc.data(), one.data(), kk.data(), D2m.data(), nullptr, flag, st,
                           err, skip);
        if (rc == LS_OK)
            rc = x64_small(ng, D2c.data(), zero.data(), Dlc.data(), one.data(), kk.data(), D3.data(), nullptr, flag, st,
                           err, skip);
        if (rc != LS_OK) return rc;
        k_lowdin_combine<<<grid, 256, 0, st>>>(L);
        count_kernels(1);
        if (cudaGetLastError() != cudaSuccess) return tc_err(err, "x64_lowdin: launch failed");
    }
    return LS_OK;
}

// D_l = X_l Y_l^T for general strided operands (see X64Mat). Taken as D^T = Y X^T with a
// transposed store, so that the epilogue's lanes (rows of the 128-row tile) write
// consecutive entries of a row of D.
int x64_nt(int n, const X64Mat X[], const X64Mat Y[], double* const D[], const int64_t ld[], int* flag,
           cudaStream_t st, std::string* err) {
    for (int g0 = 0; g0 < n; g0 += kX64MaxJobs) {
        const int ng = std::min(kX64MaxJobs, n - g0);
        Arena ar(st);
        SplitBatch sb(st);
        std::vector<X64Op> xs(ng), ys(ng);
        std::vector<X64Spec> sp(ng);
        for (int i = 0; i < ng; ++i) {
            const int l = g0 + i;
            if (X[l].cols != Y[l].cols) return tc_err(err, "x64_nt: inner sizes differ", LS_ERR_ARG);
            const int64_t kp = pad64(std::max<int64_t>(X[l].cols, 1));
            ys[i] = x64_alloc(ar, Y[l].rows, kp);
            xs[i] = x64_alloc(ar, X[l].rows, kp);
            if (!xs[i].ok() || !ys[i].ok()) return tc_err(err, "x64_nt: out of memory", LS_ERR_OOM);
            sb.add(Y[l].p, Y[l].rows, Y[l].cols, Y[l].si, Y[l].sk, Y[l].rs, ys[i]);
            sb.add(X[l].p, X[l].rows, X[l].cols, X[l].si, X[l].sk, X[l].rs, xs[i]);
            sp[i] = X64Spec{&ys[i], &xs[i], Y[l].rows, X[l].rows, TcOut{D[l], ld[l], 0, OUT_F64, 0}, 1};
        }
        if (sb.flush() != cudaSuccess) return tc_err(err, "x64_nt: split failed");
        int rc = gemm_x64(sp.data(), ng, flag, st, err);
        if (rc != LS_OK) return rc;
    }
    return LS_OK;
}

// D = A B^T (A: M x K, B: N x K, D: M x N, row-major), then a synchronised status check
int x64_gemm_nt(const double* A, const double* B, int64_t M, int64_t N, int64_t K, double* D, cudaStream_t st,
                std::string* err) {
    Arena ar(st);
    Flag fl(ar, st);
    const int64_t kp = pad64(std::max<int64_t>(K, 1));
    X64Op as = x64_alloc(ar, M, kp), bs = x64_alloc(ar, N, kp);
    if (!fl.d || !as.ok() || !bs.ok()) return tc_err(err, "gemm_nt: out of memory", LS_ERR_OOM);
    SplitBatch sb(st);
    sb.add(A, M, K, K, 1, nullptr, as);
    sb.add(B, N, K, K, 1, nullptr, bs);
    if (sb.flush() != cudaSuccess) return tc_err(err, "gemm_nt: split failed");
    X64Spec sp{&as, &bs, M, N, TcOut{D, N, 0, OUT_F64, 0}, 0};
    int rc = gemm_x64(&sp, 1, fl.d, st, err);
    if (rc != LS_OK) return rc;
    return fl.check(err);
}

}  // namespace ls
