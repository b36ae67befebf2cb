// Mixed-precision tensor-core path for sm_103a: one TN GEMM on tcgen05.
//
//   D[z][m][n] = sum_k A[z][m][k] * B[z][n][k]        (A, B K-major, FP64 in HBM)
//
// Each operand row is scaled by a power of two 2^-e (its largest entry then
// lies in [1/2, 1)) and split into two 6-bit fixed-point digits h and m
// (multiples of 2^-6 and 2^-12) and a rest below 2^-12 carried by two BF16
// parts (to 2^-30). Products of digits are integers: h*h (units 2^-12) and
// h*m + m*h (units 2^-18) keep their K <= 1024 partial sums below 2^23 and so
// accumulate EXACTLY in two FP32 TMEM accumulators, whatever the rounding of
// the tensor core's adds. The remaining products that matter (m*m and those
// with the rest, all below 2^-12 of the result) go to a third accumulator,
// whose rounding then stays near 2^-36 of the result even if every add rounds
// the same way. The FP64 epilogue sums the three and applies 2^(e_a + e_b).
// Each contraction is good to a few 2^-30 of sum |a_k b_k|, against 2^-24
// sqrt(K) or worse for plain FP32 accumulation: the cancellation in the
// projections and in the core contraction needs the former.
//
// Tiles of 128 x 64 x 64 come into 128B-swizzled shared memory by TMA (one
// plain load per tile; no multicast), one thread issues tcgen05.mma for the
// CTA, and four epilogue warps read the accumulators back with tcgen05.ld.
// Every mbarrier wait is bounded: on timeout the kernel raises a flag, drains
// the copies it issued, frees its TMEM and returns.
//
// Uses: projection P = Z A^T (Def. 4.1 / Thm A.1(c)), the dense second step of
// the core contraction (Thm A.1(c)).
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

constexpr int TBM = 128, TBN = 64, TBK = 64, TSTAGES = 2, NPART = 4;   // parts: h, m, rest0, rest1
constexpr int TILE_A = TBM * TBK * 2;          // bytes of one bf16 A tile (16 KB)
constexpr int TILE_B = TBN * TBK * 2;          // 8 KB
constexpr int STAGE_BYTES = NPART * (TILE_A + TILE_B);
constexpr int TC_THREADS = 192;                // warp 0 TMA, warp 1 MMA + TMEM, warps 2-5 epilogue
constexpr int KCHUNK = 1024;                   // K per exact head accumulation
constexpr int TMEM_COLS = 4 * TBN;             // three FP32 accumulators (power-of-two allocation)

enum OutMode : int { OUT_F64 = 0, OUT_F32 = 1 };

struct TcOut {
    void* p;            // D
    int64_t ld;         // row stride (elements)
    int64_t zs;         // batch stride (elements)
    int mode;
    int accumulate;     // F64 only: D += result
};

__global__ void __launch_bounds__(TC_THREADS, 1)
    k_fx_gemm(const __grid_constant__ CUtensorMap mA0, const __grid_constant__ CUtensorMap mA1,
              const __grid_constant__ CUtensorMap mA2, const __grid_constant__ CUtensorMap mA3,
              const __grid_constant__ CUtensorMap mB0, const __grid_constant__ CUtensorMap mB1,
              const __grid_constant__ CUtensorMap mB2, const __grid_constant__ CUtensorMap mB3, int M, int N, int kb0,
              int nkb, int a_batched, int b_batched, const int* __restrict__ ea, int64_t ea_zs,
              const int* __restrict__ eb, int64_t eb_zs, TcOut out, int* flag) {
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    unsigned char* smem = (unsigned char*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    uint64_t* full = (uint64_t*)(smem + TSTAGES * STAGE_BYTES);
    uint64_t* empty = full + TSTAGES;
    uint64_t* accum = empty + TSTAGES;
    uint32_t* tmem_slot = (uint32_t*)(accum + 1);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int n0 = blockIdx.x * TBN, m0 = blockIdx.y * TBM, z = blockIdx.z;

    if (threadIdx.x == 0) {
        for (int s = 0; s < TSTAGES; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], 1);
        }
        mbar_init(accum, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                     "r"(TMEM_COLS));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    const uint32_t tmem = *tmem_slot;

    if (warp == 0 && lane == 0) {
        // TMA producer
        int issued = 0;
        const int za = a_batched ? z : 0, zb = b_batched ? z : 0;
        for (int kb = 0; kb < nkb; ++kb) {
            const int s = kb % TSTAGES;
            if (kb >= TSTAGES && !mbar_wait(&empty[s], ((kb / TSTAGES) + 1) & 1, flag)) break;
            unsigned char* st = smem + s * STAGE_BYTES;
            const int kx = (kb0 + kb) * TBK;
            mbar_expect_tx(&full[s], STAGE_BYTES);
            tma_load_3d(st + 0 * TILE_A, &mA0, kx, m0, za, &full[s]);
            tma_load_3d(st + 1 * TILE_A, &mA1, kx, m0, za, &full[s]);
            tma_load_3d(st + 2 * TILE_A, &mA2, kx, m0, za, &full[s]);
            tma_load_3d(st + 3 * TILE_A, &mA3, kx, m0, za, &full[s]);
            unsigned char* sb = st + NPART * TILE_A;
            tma_load_3d(sb + 0 * TILE_B, &mB0, kx, n0, zb, &full[s]);
            tma_load_3d(sb + 1 * TILE_B, &mB1, kx, n0, zb, &full[s]);
            tma_load_3d(sb + 2 * TILE_B, &mB2, kx, n0, zb, &full[s]);
            tma_load_3d(sb + 3 * TILE_B, &mB3, kx, n0, zb, &full[s]);
            issued = kb + 1;
        }
        // drain: every issued stage must have landed before the CTA may exit
        for (int kb = max(0, issued - TSTAGES); kb < issued; ++kb) {
            long long it = 0;
            while (!mbar_try_wait(&full[kb % TSTAGES], (kb / TSTAGES) & 1) && ++it < kWaitLimit) {
            }
        }
    } else if (warp == 1 && lane == 0) {
        // MMA issuer: accumulator 0 gets h*h, accumulator 1 gets h*m + m*h (both exact),
        // accumulator 2 the products below 2^-12 of the result
        const uint32_t idesc = idesc_bf16(TBM, TBN);
        const uint32_t t0 = tmem, t1 = tmem + TBN, t2 = tmem + 2 * TBN;
        for (int kb = 0; kb < nkb; ++kb) {
            const int s = kb % TSTAGES;
            if (!mbar_wait(&full[s], (kb / TSTAGES) & 1, flag)) break;
            asm volatile("tcgen05.fence::after_thread_sync;");
            const uint32_t base = smem_u32(smem + s * STAGE_BYTES);
            uint64_t a[NPART], b[NPART];
#pragma unroll
            for (int i = 0; i < NPART; ++i) {
                a[i] = smem_desc_sw128(base + i * TILE_A);
                b[i] = smem_desc_sw128(base + NPART * TILE_A + i * TILE_B);
            }
#pragma unroll
            for (int kk = 0; kk < TBK / 16; ++kk) {
                const uint64_t o = (uint64_t)((kk * 32) >> 4);   // 16 bf16 = 32 bytes along K
                const uint32_t first = (kb | kk) ? 1u : 0u;
                mma_bf16(t0, a[0] + o, b[0] + o, idesc, first);          // h h
                mma_bf16(t1, a[0] + o, b[1] + o, idesc, first);          // h m
                mma_bf16(t1, a[1] + o, b[0] + o, idesc, 1u);             // m h
                // below 2^-12: smallest first
                mma_bf16(t2, a[2] + o, b[2] + o, idesc, first);          // r0 r0
                mma_bf16(t2, a[1] + o, b[3] + o, idesc, 1u);             // m r1
                mma_bf16(t2, a[3] + o, b[1] + o, idesc, 1u);             // r1 m
                mma_bf16(t2, a[0] + o, b[3] + o, idesc, 1u);             // h r1
                mma_bf16(t2, a[3] + o, b[0] + o, idesc, 1u);             // r1 h
                mma_bf16(t2, a[1] + o, b[2] + o, idesc, 1u);             // m r0
                mma_bf16(t2, a[2] + o, b[1] + o, idesc, 1u);             // r0 m
                mma_bf16(t2, a[1] + o, b[1] + o, idesc, 1u);             // m m
                mma_bf16(t2, a[0] + o, b[2] + o, idesc, 1u);             // h r0
                mma_bf16(t2, a[2] + o, b[0] + o, idesc, 1u);             // r0 h
            }
            mma_commit(&empty[s]);
        }
        mma_commit(accum);
    } else if (warp >= 2) {
        // epilogue: warp w reads TMEM lanes 32*(w%4) .. +31
        const int q = warp & 3;
        const int row = m0 + 32 * q + lane;
        if (mbar_wait(accum, 0, flag)) {
            asm volatile("tcgen05.fence::after_thread_sync;");
            const int erow = (row < M) ? ea[(a_batched ? (int64_t)z * ea_zs : 0) + row] : 0;
            const int* ebz = eb + (b_batched ? (int64_t)z * eb_zs : 0);
            for (int c = 0; c < TBN; c += 32) {
                float v0[32], v1[32], v2[32];
                const uint32_t lanes = (uint32_t)(32 * q) << 16;
                tmem_ld32(tmem + lanes + (uint32_t)c, v0);
                tmem_ld32(tmem + lanes + (uint32_t)(TBN + c), v1);
                tmem_ld32(tmem + lanes + (uint32_t)(2 * TBN + c), v2);
                if (row >= M) continue;
                const int nb = n0 + c;
                if (out.mode == OUT_F64) {
                    double* o = (double*)out.p + (int64_t)z * out.zs + (int64_t)row * out.ld + nb;
#pragma unroll
                    for (int j = 0; j < 32; ++j)
                        if (nb + j < N) {
                            const double v =
                                ldexp((double)v0[j] + (double)v1[j] + (double)v2[j], erow + ebz[nb + j]);
                            o[j] = out.accumulate ? o[j] + v : v;
                        }
                } else {
                    float* o = (float*)out.p + (int64_t)z * out.zs + (int64_t)row * out.ld + nb;
#pragma unroll
                    for (int j = 0; j < 32; ++j)
                        if (nb + j < N)
                            o[j] = (float)ldexp((double)v0[j] + (double)v1[j] + (double)v2[j], erow + ebz[nb + j]);
                }
            }
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    if (warp == 1) {
        asm volatile("tcgen05.fence::after_thread_sync;");
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TMEM_COLS));
    }
}

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
// the tensor cores. One stage of 8 slices x (128 + 64) rows x 64 k fills
// 192 KB of shared memory; the eight accumulators fill TMEM's 512 columns.
// ---------------------------------------------------------------------------
constexpr int XSL = 8;                              // slices (digits)
constexpr int XKCHUNK = 512;                        // K per exact accumulation
constexpr int XSTAGE = XSL * (TILE_A + TILE_B);     // 192 KB
constexpr int XTMEM = XSL * TBN;                    // 512 columns

struct X64Job {
    CUtensorMap a[XSL], b[XSL];
    int M, N, nkb;        // k-blocks of 64 over all of K
    int tiles_n, b0;      // tiles along N; first block of the job
    int transposed;       // D stored at out.p[n * out.ld + m]
    const int* ea;
    const int* eb;
    TcOut out;
};
constexpr int kX64MaxJobs = 3;
struct X64Group {
    X64Job j[kX64MaxJobs];
    int n;
};

// One 128 x 64 output tile of one job per CTA, all of K: the K-chunks of 512 run in
// turn on the same eight accumulators (the MMA warp waits until the epilogue has drained
// them); the epilogue adds each chunk's recombined value into the output tile, which only
// this CTA writes.
__global__ void __launch_bounds__(TC_THREADS, 1) k_x64_gemm(const __grid_constant__ X64Group G, int* flag) {
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    unsigned char* smem = (unsigned char*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    uint64_t* full = (uint64_t*)(smem + XSTAGE);
    uint64_t* empty = full + 1;
    uint64_t* accum = empty + 1;      // accumulators of a chunk complete
    uint64_t* drained = accum + 1;    // epilogue has read them
    uint32_t* tmem_slot = (uint32_t*)(drained + 1);
    int ji = 0;
    while (ji + 1 < G.n && (int)blockIdx.x >= G.j[ji + 1].b0) ++ji;
    const X64Job& J = G.j[ji];
    const int tile = (int)blockIdx.x - J.b0;
    const int tm = tile / J.tiles_n, tn = tile - tm * J.tiles_n;
    const int n0 = tn * TBN, m0 = tm * TBM;
    const int kbc = XKCHUNK / TBK;
    const int nchunk = (J.nkb + kbc - 1) / kbc;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

    if (threadIdx.x == 0) {
        mbar_init(full, 1);
        mbar_init(empty, 1);
        mbar_init(accum, 1);
        mbar_init(drained, 4);   // one arrival per epilogue warp
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
        // TMA producer: one stage, refilled once the MMAs of the previous k-block are done
        int issued = 0;
        for (int kb = 0; kb < J.nkb; ++kb) {
            if (kb > 0 && !mbar_wait(empty, (kb - 1) & 1, flag)) break;
            const int kx = kb * TBK;
            mbar_expect_tx(full, XSTAGE);
#pragma unroll
            for (int i = 0; i < XSL; ++i) tma_load_3d(smem + i * TILE_A, &J.a[i], kx, m0, 0, full);
#pragma unroll
            for (int j = 0; j < XSL; ++j) tma_load_3d(smem + XSL * TILE_A + j * TILE_B, &J.b[j], kx, n0, 0, full);
            issued = kb + 1;
        }
        if (issued > 0) {
            long long it = 0;
            while (!mbar_try_wait(full, (issued - 1) & 1) && ++it < kWaitLimit) {
            }
        }
    } else if (warp == 1 && lane == 0) {
        // MMA issuer: pair (i, j) into the accumulator of level i + j; a chunk starts from zero
        const uint32_t idesc = idesc_bf16(TBM, TBN);
        bool ok = true;
        for (int c = 0; c < nchunk && ok; ++c) {
            if (c > 0 && !mbar_wait(drained, (c - 1) & 1, flag)) break;
            asm volatile("tcgen05.fence::after_thread_sync;");
            const int kbe = min(J.nkb, (c + 1) * kbc);
            for (int kb = c * kbc; kb < kbe; ++kb) {
                if (!mbar_wait(full, kb & 1, flag)) { ok = false; break; }
                asm volatile("tcgen05.fence::after_thread_sync;");
                const uint32_t base = smem_u32(smem);
                const bool first_kb = kb == c * kbc;
#pragma unroll
                for (int kk = 0; kk < TBK / 16; ++kk) {
                    const uint64_t o = (uint64_t)((kk * 32) >> 4);
#pragma unroll
                    for (int l = 0; l < XSL; ++l)
#pragma unroll
                        for (int i = 0; i <= l; ++i) {
                            const uint64_t a = smem_desc_sw128(base + i * TILE_A) + o;
                            const uint64_t b = smem_desc_sw128(base + XSL * TILE_A + (l - i) * TILE_B) + o;
                            mma_bf16(tmem + (uint32_t)(l * TBN), a, b, idesc, (!first_kb || kk || i) ? 1u : 0u);
                        }
                }
                mma_commit(empty);
            }
            mma_commit(accum);
        }
    } else if (warp >= 2) {
        const int q = warp & 3;
        const int row = m0 + 32 * q + lane;
        const int er = row < J.M ? J.ea[row] : 0;
        const uint32_t lanes = (uint32_t)(32 * q) << 16;
        for (int c = 0; c < nchunk; ++c) {
            if (!mbar_wait(accum, c & 1, flag)) break;
            asm volatile("tcgen05.fence::after_thread_sync;");
            const bool add = c > 0 || J.out.accumulate;
            for (int cc = 0; cc < TBN; cc += 8) {
                float S[XSL][8];
#pragma unroll
                for (int l = 0; l < XSL; ++l) tmem_ld8(tmem + lanes + (uint32_t)(l * TBN + cc), S[l]);
                if (row >= J.M) continue;
#pragma unroll
                for (int jj = 0; jj < 8; ++jj) {
                    const int col = n0 + cc + jj;
                    if (col >= J.N) continue;
                    // exact level sums (integers below 2^24), recombined by Horner steps in int64
                    long long hi = 0, lo = 0;
#pragma unroll
                    for (int l = 0; l < 4; ++l) hi = hi * 128 + (long long)__float2int_rn(S[l][jj]);
#pragma unroll
                    for (int l = 4; l < 8; ++l) lo = lo * 128 + (long long)__float2int_rn(S[l][jj]);
                    // sum_l S_l 2^(-7(l+2)) = hi 2^-35 + lo 2^-63
                    const double v = ldexp(fma((double)hi, 0x1p-35, (double)lo * 0x1p-63), er + J.eb[col]);
                    double* o = (double*)J.out.p +
                                (J.transposed ? (int64_t)col * J.out.ld + row : (int64_t)row * J.out.ld + col);
                    *o = add ? *o + v : v;
                }
            }
            asm volatile("tcgen05.fence::before_thread_sync;");
            __syncwarp();
            if (lane == 0) asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(drained)) : "memory");
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

// One CTA per row i of a K-contiguous source x(i, k) = src[i*si + k], scaled by rs[i] if
// given. E = exponent with max_k |x| in [2^(E-2), 2^(E-1)), so that x 2^-E lies in
// (-1/2, 1/2) and its digits in [-64, 64]; zero digits past cols.
__global__ void __launch_bounds__(128) k_split_x64(const double* __restrict__ src, int64_t rows, int64_t cols,
                                                   int64_t si, const double* __restrict__ rs, int64_t kpad, X64Ptrs d,
                                                   int* __restrict__ exps) {
    __shared__ unsigned long long s_mb[4];
    const int64_t i = blockIdx.x;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    unsigned long long mb = 0;
    for (int64_t k = threadIdx.x; k < cols; k += blockDim.x) mb = max(mb, abs_bits(src[i * si + k]));
    for (int o = 16; o; o >>= 1) mb = max(mb, __shfl_xor_sync(0xffffffffu, mb, o));
    if (lane == 0) s_mb[warp] = mb;
    __syncthreads();
    mb = max(max(s_mb[0], s_mb[1]), max(s_mb[2], s_mb[3]));
    const double sc = rs ? fabs(rs[i]) : 1.0;
    const double mx = sc * __longlong_as_double((long long)mb);
    const int E = mx > 0.0 ? ilogb(mx) + 2 : 0;
    if (threadIdx.x == 0) exps[i] = E;
    const double f = (rs ? rs[i] : 1.0) * ldexp(1.0, 56 - E);
    for (int64_t k = threadIdx.x; k < kpad; k += blockDim.x)
        x64_digits(k < cols ? src[i * si + k] * f : 0.0, i * kpad + k, d);
}

// ---------------------------------------------------------------------------
// operand preparation: FP64 rows -> exponent + 6-bit head + three-part rest
// ---------------------------------------------------------------------------

// One warp per row r of `batch` stacked matrices of `rows` rows:
//   x(b, i, k) = src[b*sb + i*si + k*sk] for k < cols, 0 for cols <= k < kpad;
//   e = exponent with max_k |x| in [2^(e-1), 2^e) (0 for a zero row);
//   x 2^-e = h + m + rest, h = trunc(64 x 2^-e)/64, m = trunc(4096 (x 2^-e - h))/4096,
//   rest -> two BF16 parts.
__global__ void k_split_fx(const double* __restrict__ src, int64_t rows, int64_t cols, int64_t si, int64_t sk,
                           int64_t sb, int64_t batch, int64_t kpad, __nv_bfloat16* __restrict__ ph,
                           __nv_bfloat16* __restrict__ pm, __nv_bfloat16* __restrict__ p0,
                           __nv_bfloat16* __restrict__ p1, int* __restrict__ exps) {
    const int lane = threadIdx.x & 31;
    const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    if (warp >= rows * batch) return;
    const int64_t b = warp / rows, i = warp - b * rows;
    const double* x = src + b * sb + i * si;
    double mx = 0.0;
    for (int64_t k = lane; k < cols; k += 32) mx = fmax(mx, fabs(x[k * sk]));
    for (int o = 16; o; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    const int e = mx > 0.0 ? ilogb(mx) + 1 : 0;
    if (lane == 0) exps[warp] = e;
    const int64_t off = warp * kpad;
    for (int64_t k = lane; k < kpad; k += 32) {
        const double v = k < cols ? ldexp(x[k * sk], -e) : 0.0;
        const double hd = trunc(v * 64.0) * (1.0 / 64.0);             // |v - hd| < 2^-6
        const double md = trunc((v - hd) * 4096.0) * (1.0 / 4096.0);  // |v - hd - md| < 2^-12
        const double rest = (v - hd) - md;
        ph[off + k] = __double2bfloat16(hd);   // exact: 6 significant bits
        pm[off + k] = __double2bfloat16(md);   // exact: 6 significant bits
        const __nv_bfloat16 r0 = __float2bfloat16_rn((float)rest);
        p0[off + k] = r0;
        p1[off + k] = __float2bfloat16_rn((float)(rest - (double)__bfloat162float(r0)));
    }
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
// rows x kpad bf16 matrices, `batch` of them back to back; box = box_rows x 64
bool make_map(CUtensorMap* m, const void* base, int64_t rows, int64_t kpad, int64_t batch, int box_rows) {
    auto fn = encode_fn();
    if (!fn) return false;
    cuuint64_t dims[3] = {(cuuint64_t)kpad, (cuuint64_t)rows, (cuuint64_t)batch};
    cuuint64_t strides[2] = {(cuuint64_t)(kpad * 2), (cuuint64_t)(rows * kpad * 2)};
    cuuint32_t box[3] = {(cuuint32_t)TBK, (cuuint32_t)box_rows, 1};
    cuuint32_t es[3] = {1, 1, 1};
    CUresult r = fn(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, const_cast<void*>(base), dims, strides, box, es,
                    CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                    CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS;
}

int64_t pad64(int64_t x) { return (x + 63) / 64 * 64; }

struct Fx {   // one operand in split form: head + three rest parts, and a row exponent
    __nv_bfloat16* p[NPART] = {nullptr, nullptr, nullptr, nullptr};
    int* e = nullptr;
    bool ok() const { return p[0] && p[1] && p[2] && p[3] && e; }
};

Fx fx_alloc(Arena& ar, int64_t rows_total, int64_t kpad) {
    Fx f;
    for (int i = 0; i < NPART; ++i) f.p[i] = ar.get<__nv_bfloat16>(rows_total * kpad);
    f.e = ar.get<int>(rows_total);
    return f;
}

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


cudaError_t launch_split_fx(const double* src, int64_t rows, int64_t cols, int64_t si, int64_t sk, int64_t sb,
                            int64_t batch, int64_t kpad, Fx d, cudaStream_t st) {
    const int64_t warps = rows * batch;
    k_split_fx<<<(unsigned)((warps * 32 + 255) / 256), 256, 0, st>>>(src, rows, cols, si, sk, sb, batch, kpad, d.p[0],
                                                                    d.p[1], d.p[2], d.p[3], d.e);
    count_kernels(1);
    return cudaGetLastError();
}

// D[z] (+)= A[z] B[z]^T with A: batchA x M x kpad, B: batchB x N x kpad, both in split form
int gemm_fx(const Fx& A, int64_t M, int64_t batchA, const Fx& B, int64_t N, int64_t batchB, int64_t kpad, int64_t batch,
            const TcOut& out, int* flag, cudaStream_t st, std::string* err) {
    if (M <= 0 || N <= 0 || batch <= 0) return LS_OK;
    if (kpad % TBK != 0) return tc_err(err, "tc gemm: K not padded", LS_ERR_ARG);
    CUtensorMap mA[NPART], mB[NPART];
    for (int i = 0; i < NPART; ++i)
        if (!make_map(&mA[i], A.p[i], M, kpad, batchA, TBM) || !make_map(&mB[i], B.p[i], N, kpad, batchB, TBN))
            return tc_err(err, "tc gemm: cuTensorMapEncodeTiled failed");
    const size_t smem = TSTAGES * STAGE_BYTES + 1024 + 256;
    static std::once_flag attr_once;
    static cudaError_t attr_err = cudaSuccess;
    std::call_once(attr_once, [&] {
        attr_err = cudaFuncSetAttribute(k_fx_gemm, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    });
    if (attr_err != cudaSuccess) return tc_err(err, "tc gemm: cannot reserve shared memory");
    const int nkb_all = (int)(kpad / TBK);
    const int chunk = KCHUNK / TBK;
    for (int64_t z0 = 0; z0 < batch; z0 += 65535) {
        const int64_t nz = std::min<int64_t>(65535, batch - z0);
        dim3 grid((unsigned)((N + TBN - 1) / TBN), (unsigned)((M + TBM - 1) / TBM), (unsigned)nz);
        for (int kb0 = 0; kb0 < nkb_all; kb0 += chunk) {
            TcOut o = out;
            if (kb0 > 0) o.accumulate = 1;
            const size_t esz = out.mode == OUT_F64 ? 8 : 4;
            if (z0) o.p = (char*)out.p + z0 * out.zs * esz;
            if (kb0 > 0 && out.mode != OUT_F64)
                return tc_err(err, "tc gemm: K beyond one exact chunk needs FP64 output", LS_ERR_ARG);
            // batched operands: the z offset goes through the tensor-map coordinate; the exponent
            // arrays and the output are offset here for z0 > 0
            const int* ea = A.e + (batchA > 1 ? z0 * M : 0);
            const int* eb = B.e + (batchB > 1 ? z0 * N : 0);
            if (z0 && (batchA > 1 || batchB > 1))
                return tc_err(err, "tc gemm: more than 65535 batched slabs per call", LS_ERR_ARG);
            k_fx_gemm<<<grid, TC_THREADS, smem, st>>>(mA[0], mA[1], mA[2], mA[3], mB[0], mB[1], mB[2], mB[3], (int)M,
                                                      (int)N, kb0, std::min(chunk, nkb_all - kb0), batchA > 1,
                                                      batchB > 1, ea, M, eb, N, o, flag);
            count_kernels(1);
            cudaError_t e = cudaGetLastError();
            if (e != cudaSuccess) return tc_err(err, std::string("tc gemm launch: ") + cudaGetErrorString(e));
        }
    }
    return LS_OK;
}

// rows of x(i, k) = src[i*si + k] times rs[i] (if given) into exact-slice form
cudaError_t launch_split_x64(const double* src, int64_t rows, int64_t cols, int64_t si, const double* rs,
                             const X64Op& d, cudaStream_t st) {
    if (rows <= 0) return cudaSuccess;
    k_split_x64<<<(unsigned)rows, 128, 0, st>>>(src, rows, cols, si, rs, d.kpad, d.d, d.e);
    count_kernels(1);
    return cudaGetLastError();
}

// one product of a group: D (+)= A B^T, A: M x kpad, B: N x kpad (exact-slice form)
struct X64Spec {
    const X64Op* A;
    const X64Op* B;
    int64_t M, N;
    TcOut out;
    int transposed;
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
        for (int q = 0; q < XSL; ++q)
            if (!make_map(&J.a[q], s0.A->d.p[q], s0.M, kpad, 1, TBM) || !make_map(&J.b[q], s0.B->d.p[q], s0.N, kpad, 1, TBN))
                return tc_err(err, "x64 gemm: cuTensorMapEncodeTiled failed");
        J.M = (int)s0.M;
        J.N = (int)s0.N;
        J.nkb = (int)(kpad / TBK);
        J.tiles_n = (int)((s0.N + TBN - 1) / TBN);
        J.b0 = blocks;
        J.transposed = s0.transposed;
        J.ea = s0.A->e;
        J.eb = s0.B->e;
        J.out = s0.out;
        blocks += (int)((s0.M + TBM - 1) / TBM) * J.tiles_n;
    }
    g.n = n;
    if (blocks == 0) return LS_OK;
    const size_t smem = XSTAGE + 1024 + 256;
    static std::once_flag attr_once;
    static cudaError_t attr_err = cudaSuccess;
    std::call_once(attr_once, [&] {
        attr_err = cudaFuncSetAttribute(k_x64_gemm, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    });
    if (attr_err != cudaSuccess) return tc_err(err, "x64 gemm: cannot reserve shared memory");
    k_x64_gemm<<<blocks, TC_THREADS, smem, st>>>(g, flag);
    count_kernels(1);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return tc_err(err, std::string("x64 gemm launch: ") + cudaGetErrorString(e));
    return LS_OK;
}


}  // namespace

int tc_project(const double* Z, int r, const double* a, int64_t C, int64_t N, double* P, cudaStream_t st,
               std::string* err) {
    Arena ar(st);
    Flag fl(ar, st);
    const int64_t kp = pad64(N);
    Fx zs = fx_alloc(ar, r, kp), as = fx_alloc(ar, C, kp);
    if (!fl.d || !zs.ok() || !as.ok()) return tc_err(err, "tc_project: out of memory", LS_ERR_OOM);
    if (launch_split_fx(Z, r, N, N, 1, 0, 1, kp, zs, st) != cudaSuccess ||
        launch_split_fx(a, C, N, N, 1, 0, 1, kp, as, st) != cudaSuccess)
        return tc_err(err, "tc_project: split failed");
    TcOut o{P, C, 0, OUT_F64, 0};
    int rc = gemm_fx(zs, r, 1, as, C, 1, kp, 1, o, fl.d, st, err);
    if (rc != LS_OK) return rc;
    return fl.check(err);
}

int tc_core(const double* P0, const double* P1, const double* P2, const int32_t* C, const int32_t* r,
            const int32_t* tcol, const double* xin, const int32_t* perm, const int32_t* off, int64_t T, double* B,
            int num_sms, cudaStream_t st, std::string* err) {
    (void)T;
    (void)num_sms;
    Arena ar(st);
    Flag fl(ar, st);
    const int64_t nn = (int64_t)r[1] * r[2];
    // step 1 (FP64, grouped by c0): W[c][n]; chunks of the groups bound W to ~256 MB
    const int64_t chunk = std::max<int64_t>(
        64, std::min<int64_t>(pad64(C[0]), ((int64_t)32 << 20) / std::max<int64_t>(nn, 1) / 64 * 64));
    double* P1t = ar.get<double>((int64_t)C[1] * r[1]);
    double* P2t = ar.get<double>((int64_t)C[2] * r[2]);
    double* W = ar.get<double>(chunk * nn);
    Fx w = fx_alloc(ar, nn, chunk), p0 = fx_alloc(ar, r[0], chunk);
    if (!fl.d || !P1t || !P2t || !W || !w.ok() || !p0.ok()) return tc_err(err, "tc_core: out of memory", LS_ERR_OOM);
    if (launch_transpose(P1, r[1], C[1], P1t, st) != cudaSuccess || launch_transpose(P2, r[2], C[2], P2t, st) != cudaSuccess)
        return tc_err(err, "tc_core: transpose failed");
    for (int64_t c0 = 0; c0 < C[0]; c0 += chunk) {
        const int64_t cw = std::min<int64_t>(chunk, C[0] - c0);
        const int64_t kp = pad64(cw);
        if (launch_core_group(P1t, P2t, r[1], r[2], tcol, xin, perm, off, (int)c0, (int)cw, W, st) != cudaSuccess)
            return tc_err(err, "tc_core: grouping failed");
        // step 2 on tensor cores: B_(0)[i][n] (+)= sum_c P0[i][c0 + c] W[c][n]
        if (launch_split_fx(W, nn, cw, 1, nn, 0, 1, kp, w, st) != cudaSuccess ||
            launch_split_fx(P0 + c0, r[0], cw, C[0], 1, 0, 1, kp, p0, st) != cudaSuccess)
            return tc_err(err, "tc_core: split failed");
        TcOut o{B, nn, 0, OUT_F64, c0 > 0 ? 1 : 0};
        int rc = gemm_fx(p0, r[0], 1, w, nn, 1, kp, 1, o, fl.d, st, err);
        if (rc != LS_OK) return rc;
    }
    if (cudaGetLastError() != cudaSuccess) return tc_err(err, "tc_core: launch failed");
    return fl.check(err);
}

// FP64-grade products on the tensor cores (exact slices) -------------------
// G_l = diag(w_l) A_l A_l^T diag(w_l), A_l: C_l rows of length N
int x64_gram(int n, const double* const a[], const int64_t C[], int64_t N, const double* const w[], double* const G[],
             int* flag, cudaStream_t st, std::string* err) {
    Arena ar(st);
    std::vector<X64Op> xs(n);
    std::vector<X64Spec> sp(n);
    for (int l = 0; l < n; ++l) {
        xs[l] = x64_alloc(ar, C[l], pad64(N));
        if (!xs[l].ok()) return tc_err(err, "x64_gram: out of memory", LS_ERR_OOM);
        if (launch_split_x64(a[l], C[l], N, N, w ? w[l] : nullptr, xs[l], st) != cudaSuccess)
            return tc_err(err, "x64_gram: split failed");
    }
    for (int l = 0; l < n; ++l) sp[l] = X64Spec{&xs[l], &xs[l], C[l], C[l], TcOut{G[l], C[l], 0, OUT_F64, 0}, 0};
    return gemm_x64(sp.data(), n, flag, st, err);
}

// P_l = Z_l A_l^T: Z_l r_l x N, A_l C_l x N (rows), P_l r_l x C_l
int x64_project(int n, const double* const Z[], const int r[], const double* const a[], const int64_t C[], int64_t N,
                double* const P[], int* flag, cudaStream_t st, std::string* err) {
    Arena ar(st);
    const int64_t kp = pad64(N);
    std::vector<X64Op> zs(n), as(n);
    std::vector<X64Spec> sp(n);
    for (int l = 0; l < n; ++l) {
        zs[l] = x64_alloc(ar, r[l], kp);
        as[l] = x64_alloc(ar, C[l], kp);
        if (!zs[l].ok() || !as[l].ok()) return tc_err(err, "x64_project: out of memory", LS_ERR_OOM);
        if (launch_split_x64(Z[l], r[l], N, N, nullptr, zs[l], st) != cudaSuccess ||
            launch_split_x64(a[l], C[l], N, N, nullptr, as[l], st) != cudaSuccess)
            return tc_err(err, "x64_project: split failed");
        sp[l] = X64Spec{&zs[l], &as[l], r[l], C[l], TcOut{P[l], C[l], 0, OUT_F64, 0}, 0};
    }
    return gemm_x64(sp.data(), n, flag, st, err);
}

// dst_l = T_l src_l: T_l r_l x r_l, src_l and dst_l r_l x N (rows). Computed as
// dst^T = src^T T^T (src transposed first) with a transposed store: each epilogue warp
// writes 32 consecutive entries of a row of dst.
int x64_apply(int n, const double* const T[], const int r[], const double* const src[], int64_t N,
              double* const dst[], int* flag, cudaStream_t st, std::string* err) {
    Arena ar(st);
    std::vector<X64Op> ss(n), ts(n);
    std::vector<X64Spec> sp(n);
    for (int l = 0; l < n; ++l) {
        const int64_t kp = pad64(r[l]);
        double* srcT = ar.get<double>(N * r[l]);
        ss[l] = x64_alloc(ar, N, kp);
        ts[l] = x64_alloc(ar, r[l], kp);
        if (!srcT || !ss[l].ok() || !ts[l].ok()) return tc_err(err, "x64_apply: out of memory", LS_ERR_OOM);
        if (launch_transpose(src[l], r[l], N, srcT, st) != cudaSuccess ||
            launch_split_x64(srcT, N, r[l], r[l], nullptr, ss[l], st) != cudaSuccess ||
            launch_split_x64(T[l], r[l], r[l], r[l], nullptr, ts[l], st) != cudaSuccess)
            return tc_err(err, "x64_apply: split failed");
        sp[l] = X64Spec{&ss[l], &ts[l], N, r[l], TcOut{dst[l], N, 0, OUT_F64, 0}, 1};
    }
    return gemm_x64(sp.data(), n, flag, st, err);
}

// D = A B^T (A: M x K, B: N x K, D: M x N, row-major), then a synchronised status check
int x64_gemm_nt(const double* A, const double* B, int64_t M, int64_t N, int64_t K, double* D, cudaStream_t st,
                std::string* err) {
    Arena ar(st);
    Flag fl(ar, st);
    const int64_t kp = pad64(std::max<int64_t>(K, 1));
    X64Op as = x64_alloc(ar, M, kp), bs = x64_alloc(ar, N, kp);
    if (!fl.d || !as.ok() || !bs.ok()) return tc_err(err, "gemm_nt: out of memory", LS_ERR_OOM);
    if (launch_split_x64(A, M, K, K, nullptr, as, st) != cudaSuccess ||
        launch_split_x64(B, N, K, K, nullptr, bs, st) != cudaSuccess)
        return tc_err(err, "gemm_nt: split failed");
    X64Spec sp{&as, &bs, M, N, TcOut{D, N, 0, OUT_F64, 0}, 0};
    int rc = gemm_x64(&sp, 1, fl.d, st, err);
    if (rc != LS_OK) return rc;
    return fl.check(err);
}

}  // namespace ls
