// Mixed-precision tensor-core path for sm_103a: one TN GEMM on tcgen05.
//
//   D[z][m][n] = sum_k A[z][m][k] * B[z][n][k]        (A, B K-major)
//
// Operands arrive as three BF16 parts (x = b0 + b1 + b2 holds all 24 bits of
// the FP32 value of x) and each k-step issues the six MMAs with i + j <= 2 into
// one FP32 TMEM accumulator; the dropped products are below 3 * 2^-27 |ab|, so
// each product is as good as an FP32 product. (Two parts and three MMAs lose
// 2^-18 per operand, which the cancellation in the core contraction amplifies
// past a 1e-6 target.) Tiles of 128 x 128 x 64 are brought into 128B-swizzled
// shared memory by TMA (one plain load per tile; no multicast), one thread
// issues tcgen05.mma for the CTA, and four epilogue warps read the
// accumulator back with tcgen05.ld.
// Every mbarrier wait is bounded: on timeout the kernel raises a flag, drains
// the copies it issued, frees its TMEM and returns.
//
// Uses: projection P = Z A^T (Def. 4.1 / Thm A.1(c)), the dense second step of
// the core contraction (Thm A.1(c)), and the two n-mode products of slab
// evaluation (Eq. Tucker_singePot).
#include <cuda.h>
#include <cuda_bf16.h>
#include <cudaTypedefs.h>

#include <algorithm>
#include <mutex>
#include <string>
#include <vector>

#include "lattice_sum.h"
#include "ls_common.cuh"
#include "ls_tc.cuh"

namespace ls {

namespace {

constexpr int TBM = 128, TBN = 128, TBK = 64, TSTAGES = 2, NPART = 3;
constexpr int TILE_A = TBM * TBK * 2;          // bytes of one bf16 A tile (16 KB)
constexpr int TILE_B = TBN * TBK * 2;          // 16 KB
constexpr int STAGE_BYTES = NPART * (TILE_A + TILE_B);
constexpr int TC_THREADS = 192;                // warp 0 TMA, warp 1 MMA + TMEM, warps 2-5 epilogue
constexpr long long kWaitLimit = 1LL << 22;   // try_wait polls; each may suspend briefly

enum OutMode : int { OUT_F64 = 0, OUT_F32 = 1, OUT_SPLIT = 2 };

struct TcOut {
    void* p;            // F64 / F32: D; SPLIT: part 0
    void* p2;           // SPLIT: part 1
    void* p3;           // SPLIT: part 2
    int64_t ld;         // row stride (elements)
    int64_t zs;         // batch stride (elements)
    int mode;
    int accumulate;     // F64 only: D += result
};

// x (FP32) = b0 + b1 + b2 exactly: three BF16 parts of 8 significant bits each
__device__ __forceinline__ void split3(float x, __nv_bfloat16& b0, __nv_bfloat16& b1, __nv_bfloat16& b2) {
    b0 = __float2bfloat16_rn(x);
    const float r1 = x - __bfloat162float(b0);
    b1 = __float2bfloat16_rn(r1);
    b2 = __float2bfloat16_rn(r1 - __bfloat162float(b1));
}

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, unsigned count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count));
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, unsigned bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, unsigned parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// bounded wait; returns false (and raises the flag) on timeout
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, unsigned parity, int* flag) {
    long long it = 0;
    while (!mbar_try_wait(bar, parity)) {
        if (++it > kWaitLimit) {
            atomicCAS(flag, 0, FLAG_TIMEOUT);
            return false;
        }
        if (*(volatile int*)flag != 0 && it > 1024) return false;
    }
    return true;
}

__device__ __forceinline__ void tma_load_3d(void* dst, const CUtensorMap* map, int x, int y, int z, uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], [%5];"
        ::"r"(smem_u32(dst)), "l"((uint64_t)map), "r"(x), "r"(y), "r"(z), "r"(smem_u32(bar))
        : "memory");
}

// K-major operand tile in 128B-swizzled shared memory: rows of 64 bf16 (128 B),
// 8-row swizzle atoms 1024 B apart.
__device__ __forceinline__ uint64_t smem_desc_sw128(uint32_t addr) {
    uint64_t d = 0;
    d |= (uint64_t)((addr & 0x3FFFF) >> 4);          // start address
    d |= (uint64_t)(16 >> 4) << 16;                  // leading byte offset (unused for this layout)
    d |= (uint64_t)(1024 >> 4) << 32;                // stride byte offset: next 8-row atom
    d |= (uint64_t)1 << 46;                          // descriptor version for sm_100 family
    d |= (uint64_t)2 << 61;                          // 128-byte swizzle
    return d;
}

// instruction descriptor: kind::f16, A = B = BF16, D = F32, both K-major
__host__ __device__ constexpr uint32_t idesc_bf16(int M, int N) {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void mma_bf16(uint32_t tmem, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}"
        ::"r"(tmem), "l"(a), "l"(b), "r"(idesc), "r"(acc));
}

__device__ __forceinline__ void mma_commit(uint64_t* bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
                 : "memory");
}

__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float* v) {
    uint32_t r[32];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
        "%15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
          "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
          "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}

__global__ void __launch_bounds__(TC_THREADS, 1)
    k_tc_gemm(const __grid_constant__ CUtensorMap mA0, const __grid_constant__ CUtensorMap mA1,
              const __grid_constant__ CUtensorMap mA2, const __grid_constant__ CUtensorMap mB0,
              const __grid_constant__ CUtensorMap mB1, const __grid_constant__ CUtensorMap mB2, int M, int N, int K,
              int a_batched, int b_batched, TcOut out, int* flag) {
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    unsigned char* smem = (unsigned char*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    uint64_t* full = (uint64_t*)(smem + TSTAGES * STAGE_BYTES);
    uint64_t* empty = full + TSTAGES;
    uint64_t* accum = empty + TSTAGES;
    uint32_t* tmem_slot = (uint32_t*)(accum + 1);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int n0 = blockIdx.x * TBN, m0 = blockIdx.y * TBM, z = blockIdx.z;
    const int nk = K / TBK;

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
                     "r"(TBN));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    const uint32_t tmem = *tmem_slot;

    if (warp == 0 && lane == 0) {
        // TMA producer
        int issued = 0;
        for (int kb = 0; kb < nk; ++kb) {
            const int s = kb % TSTAGES;
            if (kb >= TSTAGES && !mbar_wait(&empty[s], ((kb / TSTAGES) + 1) & 1, flag)) break;
            unsigned char* st = smem + s * STAGE_BYTES;
            mbar_expect_tx(&full[s], STAGE_BYTES);
            const int za = a_batched ? z : 0, zb = b_batched ? z : 0;
            tma_load_3d(st, &mA0, kb * TBK, m0, za, &full[s]);
            tma_load_3d(st + TILE_A, &mA1, kb * TBK, m0, za, &full[s]);
            tma_load_3d(st + 2 * TILE_A, &mA2, kb * TBK, m0, za, &full[s]);
            tma_load_3d(st + 3 * TILE_A, &mB0, kb * TBK, n0, zb, &full[s]);
            tma_load_3d(st + 3 * TILE_A + TILE_B, &mB1, kb * TBK, n0, zb, &full[s]);
            tma_load_3d(st + 3 * TILE_A + 2 * TILE_B, &mB2, kb * TBK, n0, zb, &full[s]);
            issued = kb + 1;
        }
        // drain: every issued stage must have landed before the CTA may exit
        for (int kb = max(0, issued - TSTAGES); kb < issued; ++kb) {
            long long it = 0;
            while (!mbar_try_wait(&full[kb % TSTAGES], (kb / TSTAGES) & 1) && ++it < kWaitLimit) {
            }
        }
    } else if (warp == 1 && lane == 0) {
        // MMA issuer
        const uint32_t idesc = idesc_bf16(TBM, TBN);
        bool ok = true;
        for (int kb = 0; kb < nk && ok; ++kb) {
            const int s = kb % TSTAGES;
            if (!mbar_wait(&full[s], (kb / TSTAGES) & 1, flag)) { ok = false; break; }
            asm volatile("tcgen05.fence::after_thread_sync;");
            const uint32_t base = smem_u32(smem + s * STAGE_BYTES);
            const uint64_t dA0 = smem_desc_sw128(base), dA1 = smem_desc_sw128(base + TILE_A),
                           dA2 = smem_desc_sw128(base + 2 * TILE_A);
            const uint64_t dB0 = smem_desc_sw128(base + 3 * TILE_A), dB1 = smem_desc_sw128(base + 3 * TILE_A + TILE_B),
                           dB2 = smem_desc_sw128(base + 3 * TILE_A + 2 * TILE_B);
#pragma unroll
            for (int kk = 0; kk < TBK / 16; ++kk) {
                const uint64_t off = (uint64_t)((kk * 32) >> 4);   // 16 bf16 = 32 bytes along K
                // small products first, then the leading one
                mma_bf16(tmem, dA0 + off, dB2 + off, idesc, (kb | kk) ? 1u : 0u);
                mma_bf16(tmem, dA1 + off, dB1 + off, idesc, 1u);
                mma_bf16(tmem, dA2 + off, dB0 + off, idesc, 1u);
                mma_bf16(tmem, dA0 + off, dB1 + off, idesc, 1u);
                mma_bf16(tmem, dA1 + off, dB0 + off, idesc, 1u);
                mma_bf16(tmem, dA0 + off, dB0 + off, idesc, 1u);
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
            for (int c = 0; c < TBN; c += 32) {
                float v[32];
                tmem_ld32(tmem + ((uint32_t)(32 * q) << 16) + (uint32_t)c, v);
                if (row >= M) continue;
                const int nb = n0 + c;
                if (out.mode == OUT_F64) {
                    double* o = (double*)out.p + (int64_t)z * out.zs + (int64_t)row * out.ld + nb;
#pragma unroll
                    for (int j = 0; j < 32; ++j)
                        if (nb + j < N) o[j] = out.accumulate ? o[j] + (double)v[j] : (double)v[j];
                } else if (out.mode == OUT_F32) {
                    float* o = (float*)out.p + (int64_t)z * out.zs + (int64_t)row * out.ld + nb;
#pragma unroll
                    for (int j = 0; j < 32; ++j)
                        if (nb + j < N) o[j] = v[j];
                } else {
                    const int64_t o = (int64_t)z * out.zs + (int64_t)row * out.ld + nb;
                    __nv_bfloat16* o0 = (__nv_bfloat16*)out.p + o;
                    __nv_bfloat16* o1 = (__nv_bfloat16*)out.p2 + o;
                    __nv_bfloat16* o2 = (__nv_bfloat16*)out.p3 + o;
#pragma unroll
                    for (int j = 0; j < 32; ++j)
                        if (nb + j < N) split3(v[j], o0[j], o1[j], o2[j]);
                }
            }
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    if (warp == 1) {
        asm volatile("tcgen05.fence::after_thread_sync;");
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TBN));
    }
}

// ---------------------------------------------------------------------------
// operand preparation: FP64 -> three BF16 parts with zero padding
// ---------------------------------------------------------------------------

// dst[b][i][k] for i < rows_pad, k < kpad  from  src(b, i, k) = src[b*sb + i*si + k*sk]
// (zero outside rows x cols).
__global__ void k_split(const double* __restrict__ src, int64_t rows, int64_t cols, int64_t si, int64_t sk,
                        int64_t sb, int64_t rows_pad, int64_t kpad, __nv_bfloat16* __restrict__ d0,
                        __nv_bfloat16* __restrict__ d1, __nv_bfloat16* __restrict__ d2) {
    const int64_t b = blockIdx.y;
    const int64_t n = rows_pad * kpad;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = e / kpad, k = e - i * kpad;
        const float x = (i < rows && k < cols) ? (float)src[b * sb + i * si + k * sk] : 0.f;
        split3(x, d0[b * n + e], d1[b * n + e], d2[b * n + e]);
    }
}

// Core, step 1 in FP32 (terms grouped by their mode-0 vector c0):
//   W[n][c0] = sum_{t in group(c0)} xin[t] P1[j][c1(t)] P2[l][c2(t)],  n = j*r2 + l,
// written as three BF16 parts in K-major rows of length kpad. One thread per n
// and 32 consecutive groups per CTA column.
__global__ void __launch_bounds__(128) k_core_group_split(const float* __restrict__ P1t, const float* __restrict__ P2t,
                                                          int r1, int r2, const int32_t* __restrict__ tcol,
                                                          const double* __restrict__ xin,
                                                          const int32_t* __restrict__ perm,
                                                          const int32_t* __restrict__ off, int C0, int64_t kpad,
                                                          __nv_bfloat16* __restrict__ w0, __nv_bfloat16* __restrict__ w1,
                                                          __nv_bfloat16* __restrict__ w2) {
    const int64_t nn = (int64_t)r1 * r2;
    const int64_t n = blockIdx.x * 128 + threadIdx.x;
    const int cb = blockIdx.y * 32;
    if (n >= nn) return;
    const int j = (int)(n / r2), l = (int)(n - (int64_t)j * r2);
    float acc[32];
#pragma unroll
    for (int u = 0; u < 32; ++u) {
        float a = 0.f;
        const int c = cb + u;
        if (c < C0) {
            for (int k = off[c]; k < off[c + 1]; ++k) {
                const int t = perm[k];
                a = fmaf((float)xin[t] * P1t[(int64_t)tcol[3 * t + 1] * r1 + j], P2t[(int64_t)tcol[3 * t + 2] * r2 + l], a);
            }
        }
        acc[u] = a;
    }
    __align__(16) __nv_bfloat16 h0[32], h1[32], h2[32];
#pragma unroll
    for (int u = 0; u < 32; ++u) split3(acc[u], h0[u], h1[u], h2[u]);
    uint4* o0 = (uint4*)(w0 + n * kpad + cb);
    uint4* o1 = (uint4*)(w1 + n * kpad + cb);
    uint4* o2 = (uint4*)(w2 + n * kpad + cb);
#pragma unroll
    for (int u = 0; u < 4; ++u) {
        o0[u] = ((const uint4*)h0)[u];
        o1[u] = ((const uint4*)h1)[u];
        o2[u] = ((const uint4*)h2)[u];
    }
}

__global__ void k_transpose_f32(const double* __restrict__ in, int64_t rows, int64_t cols, float* __restrict__ out) {
    __shared__ float tile[32][33];
    const int64_t c0 = blockIdx.x * 32, r0 = blockIdx.y * 32;
    for (int k = threadIdx.y; k < 32; k += blockDim.y) {
        const int64_t r = r0 + k, c = c0 + threadIdx.x;
        tile[k][threadIdx.x] = (r < rows && c < cols) ? (float)in[r * cols + c] : 0.f;
    }
    __syncthreads();
    for (int k = threadIdx.y; k < 32; k += blockDim.y) {
        const int64_t c = c0 + k, r = r0 + threadIdx.x;
        if (c < cols && r < rows) out[c * rows + r] = tile[threadIdx.x][k];
    }
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = (PFN_cuTensorMapEncodeTiled_v12000)p;
    });
    return fn;
}

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

struct Split {   // three BF16 parts of one operand
    __nv_bfloat16* p[NPART] = {nullptr, nullptr, nullptr};
    bool ok() const { return p[0] && p[1] && p[2]; }
};

// one scratch arena per call, from the stream-ordered allocator
struct Arena {
    cudaStream_t st;
    std::vector<void*> ptrs;
    explicit Arena(cudaStream_t s) : st(s) {}
    template <class T>
    T* get(int64_t n) {
        void* p = nullptr;
        if (cudaMallocAsync(&p, (size_t)std::max<int64_t>(n, 1) * sizeof(T), st) != cudaSuccess) return nullptr;
        ptrs.push_back(p);
        return (T*)p;
    }
    Split split(int64_t n) {
        Split s;
        for (int i = 0; i < NPART; ++i) s.p[i] = get<__nv_bfloat16>(n);
        return s;
    }
    ~Arena() {
        for (void* p : ptrs) cudaFreeAsync(p, st);
    }
};

int tc_err(std::string* err, const std::string& msg, int code = LS_ERR_CUDA) {
    if (err) *err = msg;
    return code;
}

cudaError_t launch_split(const double* src, int64_t rows, int64_t cols, int64_t si, int64_t sk, int64_t sb, int64_t batch,
                         int64_t rows_pad, int64_t kpad, Split d, cudaStream_t st) {
    const int64_t n = rows_pad * kpad;
    dim3 grid((unsigned)std::min<int64_t>((n + 255) / 256, 4096), (unsigned)batch);
    k_split<<<grid, 256, 0, st>>>(src, rows, cols, si, sk, sb, rows_pad, kpad, d.p[0], d.p[1], d.p[2]);
    count_kernels(1);
    return cudaGetLastError();
}

// D[z] = A[z] B[z]^T with A: batchA x M x kpad, B: batchB x N x kpad (three BF16 parts each)
int gemm_tc(Split A, int64_t M, int64_t batchA, Split B, int64_t N, int64_t batchB, int64_t kpad, int64_t batch,
            const TcOut& out, int* flag, cudaStream_t st, std::string* err) {
    if (M <= 0 || N <= 0 || batch <= 0) return LS_OK;
    if (kpad % TBK != 0) return tc_err(err, "tc gemm: K not padded", LS_ERR_ARG);
    CUtensorMap mA[NPART], mB[NPART];
    for (int i = 0; i < NPART; ++i)
        if (!make_map(&mA[i], A.p[i], M, kpad, batchA, TBM) || !make_map(&mB[i], B.p[i], N, kpad, batchB, TBN))
            return tc_err(err, "tc gemm: cuTensorMapEncodeTiled failed");
    const size_t smem = TSTAGES * STAGE_BYTES + 1024 + 256;
    static bool attr = false;
    if (!attr) {
        if (cudaFuncSetAttribute(k_tc_gemm, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
            return tc_err(err, "tc gemm: cannot reserve shared memory");
        attr = true;
    }
    for (int64_t z0 = 0; z0 < batch; z0 += 65535) {
        dim3 grid((unsigned)((N + TBN - 1) / TBN), (unsigned)((M + TBM - 1) / TBM),
                  (unsigned)std::min<int64_t>(65535, batch - z0));
        TcOut o = out;
        if (z0) {
            const size_t esz = out.mode == OUT_F64 ? 8 : out.mode == OUT_F32 ? 4 : 2;
            o.p = (char*)out.p + z0 * out.zs * esz;
            if (o.p2) o.p2 = (char*)out.p2 + z0 * out.zs * esz;
            if (o.p3) o.p3 = (char*)out.p3 + z0 * out.zs * esz;
        }
        k_tc_gemm<<<grid, TC_THREADS, smem, st>>>(mA[0], mA[1], mA[2], mB[0], mB[1], mB[2], (int)M, (int)N, (int)kpad,
                                                  batchA > 1, batchB > 1, o, flag);
        count_kernels(1);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return tc_err(err, std::string("tc gemm launch: ") + cudaGetErrorString(e));
    }
    return LS_OK;
}

// device flag shared by the tensor-core kernels of one call; checked after the call
struct Flag {
    int* d = nullptr;
    cudaStream_t st;
    Flag(Arena& a, cudaStream_t s) : st(s) {
        d = a.get<int>(1);
        if (d) cudaMemsetAsync(d, 0, sizeof(int), st);
    }
    int check(std::string* err) {
        int h = 0;
        if (cudaMemcpyAsync(&h, d, sizeof(int), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
            cudaStreamSynchronize(st) != cudaSuccess)
            return tc_err(err, "tc: status read failed");
        if (h == FLAG_TIMEOUT) return tc_err(err, "tc gemm: a bounded mbarrier wait timed out", LS_ERR_TIMEOUT);
        return LS_OK;
    }
};

}  // namespace

int tc_project(const double* Z, int r, const double* a, int64_t C, int64_t N, double* P, cudaStream_t st,
               std::string* err) {
    Arena ar(st);
    Flag fl(ar, st);
    const int64_t kp = pad64(N);
    Split zs = ar.split((int64_t)r * kp), as = ar.split(C * kp);
    if (!fl.d || !zs.ok() || !as.ok()) return tc_err(err, "tc_project: out of memory", LS_ERR_OOM);
    if (launch_split(Z, r, N, N, 1, 0, 1, r, kp, zs, st) != cudaSuccess ||
        launch_split(a, C, N, N, 1, 0, 1, C, kp, as, st) != cudaSuccess)
        return tc_err(err, "tc_project: split failed");
    TcOut o{P, nullptr, nullptr, C, 0, OUT_F64, 0};
    int rc = gemm_tc(zs, r, 1, as, C, 1, kp, 1, o, fl.d, st, err);
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
    // W rows of all groups would take nn * kpad * 4 bytes; chunk the groups to ~1 GB
    const int64_t kp_all = pad64(C[0]);
    const int64_t chunk = std::max<int64_t>(64, std::min<int64_t>(kp_all, ((int64_t)1 << 28) / std::max<int64_t>(nn, 1) / 64 * 64));
    float* P1t = ar.get<float>((int64_t)C[1] * r[1]);
    float* P2t = ar.get<float>((int64_t)C[2] * r[2]);
    Split w = ar.split(nn * chunk);
    Split p0 = ar.split((int64_t)r[0] * chunk);
    if (!fl.d || !P1t || !P2t || !w.ok() || !p0.ok()) return tc_err(err, "tc_core: out of memory", LS_ERR_OOM);
    dim3 tg1((unsigned)((C[1] + 31) / 32), (unsigned)((r[1] + 31) / 32));
    k_transpose_f32<<<tg1, dim3(32, 8), 0, st>>>(P1, r[1], C[1], P1t);
    dim3 tg2((unsigned)((C[2] + 31) / 32), (unsigned)((r[2] + 31) / 32));
    k_transpose_f32<<<tg2, dim3(32, 8), 0, st>>>(P2, r[2], C[2], P2t);
    count_kernels(2);
    for (int64_t c0 = 0; c0 < C[0]; c0 += chunk) {
        const int64_t cw = std::min<int64_t>(chunk, C[0] - c0);
        const int64_t kp = pad64(cw);
        dim3 g((unsigned)((nn + 127) / 128), (unsigned)(kp / 32));
        // groups beyond C0 inside the padded range come out as zeros
        k_core_group_split<<<g, 128, 0, st>>>(P1t, P2t, r[1], r[2], tcol, xin, perm, off + c0, (int)cw, kp, w.p[0],
                                              w.p[1], w.p[2]);
        count_kernels(1);
        if (launch_split(P0 + c0, r[0], cw, C[0], 1, 0, 1, r[0], kp, p0, st) != cudaSuccess)
            return tc_err(err, "tc_core: split failed");
        TcOut o{B, nullptr, nullptr, nn, 0, OUT_F64, c0 > 0 ? 1 : 0};
        int rc = gemm_tc(p0, r[0], 1, w, nn, 1, kp, 1, o, fl.d, st, err);
        if (rc != LS_OK) return rc;
    }
    if (cudaGetLastError() != cudaSuccess) return tc_err(err, "tc_core: launch failed");
    return fl.check(err);
}

int tc_eval(const double* const Z[3], const int32_t* r, const double* B, int64_t N, const int32_t* zidx, int nslab,
            double* work, void* out, int out_f32, int num_sms, cudaStream_t st, std::string* err) {
    (void)num_sms;
    (void)work;
    Arena ar(st);
    Flag fl(ar, st);
    const int r0 = r[0], r1 = r[1];
    const int64_t k1 = pad64(r1), k0 = pad64(r0);
    // M_s[a][b] = sum_k B[a][b][k] Z2[k][z_s]: small, FP64 CUDA cores
    double* M = ar.get<double>((int64_t)r0 * r1 * nslab);
    Split z1t = ar.split(N * k1), z0t = ar.split(N * k0), ms = ar.split((int64_t)nslab * r0 * k1);
    Split tt = ar.split((int64_t)nslab * N * k0);
    if (!fl.d || !M || !z1t.ok() || !z0t.ok() || !ms.ok() || !tt.ok()) return tc_err(err, "tc_eval: out of memory", LS_ERR_OOM);
    cudaError_t e = launch_eval_m(Z[2], r, B, N, zidx, nslab, M, st);
    if (e != cudaSuccess) return tc_err(err, std::string("tc_eval: ") + cudaGetErrorString(e));
    // operands: Z1^T [y][b], Z0^T [x][a] (K-major), M_s [a][b] per slab
    if (launch_split(Z[1], N, r1, 1, N, 0, 1, N, k1, z1t, st) != cudaSuccess ||
        launch_split(Z[0], N, r0, 1, N, 0, 1, N, k0, z0t, st) != cudaSuccess ||
        launch_split(M, r0, r1, (int64_t)r1 * nslab, nslab, 1, nslab, r0, k1, ms, st) != cudaSuccess)
        return tc_err(err, "tc_eval: split failed");
    // T_s^T[y][a] = sum_b Z1^T[y][b] M_s[a][b], written directly as three BF16 parts
    TcOut o1{tt.p[0], tt.p[1], tt.p[2], k0, N * k0, OUT_SPLIT, 0};
    if (k0 > r0) {   // the padding columns a in [r0, k0) of T^T must read as zeros
        for (int i = 0; i < NPART; ++i)
            if (cudaMemsetAsync(tt.p[i], 0, (size_t)nslab * N * k0 * 2, st) != cudaSuccess)
                return tc_err(err, "tc_eval: memset failed");
    }
    int rc = gemm_tc(z1t, N, 1, ms, r0, nslab, k1, nslab, o1, fl.d, st, err);
    if (rc != LS_OK) return rc;
    // S_s[x][y] = sum_a Z0^T[x][a] T_s^T[y][a]
    TcOut o2{out, nullptr, nullptr, N, N * N, out_f32 ? OUT_F32 : OUT_F64, 0};
    rc = gemm_tc(z0t, N, 1, tt, N, nslab, k0, nslab, o2, fl.d, st, err);
    if (rc != LS_OK) return rc;
    return fl.check(err);
}

}  // namespace ls
