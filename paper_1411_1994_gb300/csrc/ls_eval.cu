// Slab evaluation of the Tucker result on tcgen05 tensor cores (Eq.
// Tucker_singePot: the values of a Tucker tensor are n-mode products of the
// core with the three side matrices; a z-slab fixes the third index):
//
//   M_s[a][b] = sum_c B[a][b][c] Z2[c][z_s]        r0 x r1 per slab
//   T_s[y][a] = sum_b M_s[a][b] Z1[b][y]           N x r0 per slab
//   S_s[x][y] = sum_a Z0[a][x] T_s[y][a]           N x N per slab
//
// Each is one TN product D[m][n] = sum_k A[m][k] B[n][k] (A and B K-major) on
// one persistent kernel, k_dt_gemm. The output index m lies along the TMEM
// lanes and is stored contiguous, so each warp writes an output column as 32
// consecutive elements (one 128-byte line in FP32).
//
// Operand form: two exact digits and two tails. Row i of an operand is scaled
// by 2^(6 - E_i), with E_i the exponent for which max_k |x_ik| lies in
// [2^(E_i - 1), 2^E_i), and written as
//   x 2^(6-E) = d0 + d1 2^-7 + t1 + t2,
// where d0 and d1 are nearest integers in [-64, 64], t1 is the rest (below
// 2^-8) rounded to 11 significant bits, and t2 the rest after that.
// All four parts are stored as FP16 times 2^9: d0 2^9 and d1 2^2 are exact,
// and the factor keeps t2 in FP16's normal range. The form is good to 2^-30
// of a digit unit (2^-36 of 2^E). The split runs in integer arithmetic on the
// FP64 (or FP32-pair) bit pattern: a fixed-point value with 50 fraction bits,
// then the digits and the 11-bit tails. It uses no FP64 arithmetic.
//
// The products (all scaled by 2^18) accumulate in three FP32 TMEM
// accumulators:
//   acc0 = sum d0 d0: integers of magnitude at most 2^12 (before the scale),
//     exact for K <= 4096;
//   acc1 = sum (d0 d1 + d1 d0) 2^-7: multiples of 2^-7 below 2^13 K, exact
//     for K <= 2048;
//   acc2 = the products below 2^-7 of a digit unit squared, smallest first:
//     d0 t2, t2 d0, t1 t1, d1 t1, t1 d1, d1 d1, d0 t1, t1 d0 (11 MMAs a
//     k-step in all).
// The two leading levels are exact, whatever rounding the tensor core's adds
// use. That matters: they truncate, and a float accumulator holding terms at
// 2^-7 of the result drifts by about half an ulp per MMA. acc2 sits below
// 2^-14 of the result, where that drift is negligible. The dropped products
// (d1 t2, t2 d1, t1 t2, ...) are below 2^-32 of 2^(E_a + E_b) per term.
//
// The epilogue adds the three accumulators as an unevaluated FP32 pair
// (TwoSum, no FP64 arithmetic) and scales by 2^(E_a + E_b - 30). It stores one
// of three forms: FP32 (the pair rounded once), FP64, or the pair itself.
// The intermediate products M and T are kept as pairs, so with FP32 output
// the output's own rounding is the largest error left.
//
// Pipeline:
// - Persistent grid, at most one CTA per SM.
// - Warp 0: TMA producer, through a ring of shared-memory stages (k-blocks
//   of 32, 64-byte swizzle).
// - Warp 1: allocates TMEM and issues the MMAs.
// - Warps 2-9: epilogue. Two warps per TMEM lane quadrant, each taking half
//   of the tile's columns.
// With FP32 output the epilogue pulls its accumulators into registers and
// releases TMEM before it stores, so the next tile's MMAs overlap the stores.
// Tiles up to 64 wide also double-buffer TMEM.
// Every mbarrier wait is bounded. On timeout the kernel raises the flag; the
// producer drains its copies, the MMA warp waits for its MMAs, and TMEM is
// freed before exit.
#include <cuda.h>
#include <cuda_fp16.h>

#include <string.h>

#include <algorithm>
#include <mutex>
#include <string>
#include <vector>

#include "lattice_sum.h"
#include "ls_common.cuh"
#include "ls_eval.cuh"
#include "ls_tcgen05.cuh"

namespace ls {

namespace {

using namespace tc5;

constexpr int DT_BM = 128, DT_BK = 32, DT_PARTS = 4, DT_EPI_WARPS = 8;
constexpr int DT_THREADS = 64 + 32 * DT_EPI_WARPS;       // TMA warp, MMA warp, epilogue warps
constexpr int DT_TA = DT_BM * DT_BK * 2;                 // one A part tile: 8 KB
constexpr int DT_MAXK = 2048;                            // exact level-1 accumulation
constexpr int FXB = 50;                                  // fraction bits of the fixed-point split

constexpr int pow2ceil(int x) {
    int p = 32;
    while (p < x) p <<= 1;
    return p;
}

template <int BN>
struct DtCfg {
    static constexpr int TB = BN * DT_BK * 2;
    static constexpr int STAGE = DT_PARTS * (DT_TA + TB);
    static constexpr int STAGES = std::min(8, (220 * 1024) / STAGE);
    static constexpr int NBUF = 3 * BN * 2 <= 512 ? 2 : 1;
    static constexpr int TMEM_COLS = pow2ceil(3 * BN * NBUF);
    static constexpr size_t SMEM = (size_t)STAGES * STAGE + 1024 + 256;
    static_assert(3 * BN * NBUF <= 512, "three accumulators per buffer must fit TMEM");
};

struct DtJob {
    CUtensorMap a, b;          // (kpad, rows, 4 * batch) fp16, 64-byte swizzle
    int M, N, nkb;             // k-blocks of 32
    int tiles_m, tiles_n, ntiles;
    int a_batch, b_batch;      // batches held by each operand (1: shared)
    const int* ea;             // row exponents [batch][rows]
    const int* eb;
    int64_t ea_zs, eb_zs;
    void* out;                 // out[z * zs + n * ldn + m]
    int64_t ldn, zs;
    int mode;                  // DtOutMode
};

__device__ __forceinline__ float pow2f(int e) {           // e in [-126, 127]
    return __int_as_float((e + 127) << 23);
}

// v 2^e by two exact multiplications (no overflow of the factors for |e| <= 252)
__device__ __forceinline__ float scale_f32(float v, int e) {
    const int e1 = max(-126, min(127, e));
    return (v * pow2f(e1)) * pow2f(max(-126, min(127, e - e1)));
}

// a0 + a1 + a2 (a0, a1 exact, |a2| small) as an unevaluated pair hi + lo, by two
// TwoSums: hi is the sum rounded once, lo the rest to about 2^-48 of it
__device__ __forceinline__ void combine3(float a0, float a1, float a2, float& hi, float& lo) {
    const float s = a0 + a1;
    const float bb = s - a0;
    const float e = (a0 - (s - bb)) + (a1 - bb);
    const float t = e + a2;
    hi = s + t;
    const float b2 = hi - s;
    lo = (s - (hi - b2)) + (t - b2);
}

template <int BN>
__global__ void __launch_bounds__(DT_THREADS, 1) k_dt_gemm(const __grid_constant__ DtJob J, int* flag) {
    using C = DtCfg<BN>;
    constexpr int S = C::STAGES, NBUF = C::NBUF;
    constexpr int HALF = BN / 2;                  // columns per epilogue warp
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    unsigned char* smem = (unsigned char*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    uint64_t* full = (uint64_t*)(smem + S * C::STAGE);
    uint64_t* empty = full + S;
    uint64_t* tfull = empty + S;       // accumulator buffer holds a finished tile
    uint64_t* tempty = tfull + 2;      // epilogue has read it
    uint64_t* mdone = tempty + 2;      // every MMA of this CTA has completed
    uint32_t* tmem_slot = (uint32_t*)(mdone + 1);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int per_z = J.tiles_m * J.tiles_n;

    if (threadIdx.x == 0) {
        for (int s = 0; s < S; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], 1);
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(&tfull[b], 1);
            mbar_init(&tempty[b], DT_EPI_WARPS);   // one arrival per epilogue warp
        }
        mbar_init(mdone, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                     "r"(C::TMEM_COLS));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    const uint32_t tmem = *tmem_slot;

    if (warp == 0 && lane == 0) {
        // TMA producer: the four parts of A, then of B, for each k-block of each tile
        uint32_t it = 0;
        bool ok = true;
        for (int t = blockIdx.x; t < J.ntiles && ok; t += gridDim.x) {
            const int z = t / per_z, rem = t - z * per_z;
            const int tn = rem / J.tiles_m, tm = rem - tn * J.tiles_m;
            const int za = J.a_batch > 1 ? z : 0, zb = J.b_batch > 1 ? z : 0;
            for (int kb = 0; kb < J.nkb; ++kb, ++it) {
                const uint32_t s = it % S, u = it / S;
                if (u > 0 && !mbar_wait(&empty[s], (u - 1) & 1, flag)) { ok = false; break; }
                unsigned char* st = smem + s * C::STAGE;
                mbar_expect_tx(&full[s], C::STAGE);
                const int kx = kb * DT_BK;
#pragma unroll
                for (int p = 0; p < DT_PARTS; ++p)
                    tma_load_3d(st + p * DT_TA, &J.a, kx, tm * DT_BM, p * J.a_batch + za, &full[s]);
#pragma unroll
                for (int p = 0; p < DT_PARTS; ++p)
                    tma_load_3d(st + DT_PARTS * DT_TA + p * C::TB, &J.b, kx, tn * BN, p * J.b_batch + zb, &full[s]);
            }
        }
        // every issued stage must have landed before the CTA may exit
        for (uint32_t j = it > (uint32_t)S ? it - S : 0; j < it; ++j) mbar_drain(&full[j % S], (j / S) & 1);
    } else if (warp == 1 && lane == 0) {
        constexpr uint32_t idesc = idesc_f16(DT_BM, BN);
        uint32_t it = 0, lt = 0;
        bool ok = true;
        for (int t = blockIdx.x; t < J.ntiles && ok; t += gridDim.x, ++lt) {
            const uint32_t buf = lt % NBUF, u = lt / NBUF;
            if (u > 0 && !mbar_wait(&tempty[buf], (u - 1) & 1, flag)) break;
            asm volatile("tcgen05.fence::after_thread_sync;");
            const uint32_t c0 = tmem + buf * 3 * BN, c1 = c0 + BN, c2 = c0 + 2 * BN;
            for (int kb = 0; kb < J.nkb; ++kb, ++it) {
                const uint32_t s = it % S;
                if (!mbar_wait(&full[s], (it / S) & 1, flag)) { ok = false; break; }
                asm volatile("tcgen05.fence::after_thread_sync;");
                const uint32_t sa = smem_u32(smem + s * C::STAGE), sb = sa + DT_PARTS * DT_TA;
#pragma unroll
                for (int kk = 0; kk < DT_BK / 16; ++kk) {
                    const uint64_t o = (uint64_t)((kk * 32) >> 4);   // 16 bf16 = 32 bytes along K
                    const uint64_t a0 = smem_desc_sw64(sa) + o, a1 = smem_desc_sw64(sa + DT_TA) + o,
                                   a2 = smem_desc_sw64(sa + 2 * DT_TA) + o, a3 = smem_desc_sw64(sa + 3 * DT_TA) + o;
                    const uint64_t b0 = smem_desc_sw64(sb) + o, b1 = smem_desc_sw64(sb + C::TB) + o,
                                   b2 = smem_desc_sw64(sb + 2 * C::TB) + o, b3 = smem_desc_sw64(sb + 3 * C::TB) + o;
                    const uint32_t acc = (kb | kk) ? 1u : 0u;
                    mma_bf16(c0, a0, b0, idesc, acc);            // d0 d0: exact
                    mma_bf16(c1, a0, b1, idesc, acc);            // d0 d1, d1 d0: exact
                    mma_bf16(c1, a1, b0, idesc, 1u);
                    mma_bf16(c2, a0, b3, idesc, acc);            // the rest, smallest first
                    mma_bf16(c2, a3, b0, idesc, 1u);
                    mma_bf16(c2, a2, b2, idesc, 1u);
                    mma_bf16(c2, a1, b2, idesc, 1u);
                    mma_bf16(c2, a2, b1, idesc, 1u);
                    mma_bf16(c2, a1, b1, idesc, 1u);
                    mma_bf16(c2, a0, b2, idesc, 1u);
                    mma_bf16(c2, a2, b0, idesc, 1u);
                }
                mma_commit(&empty[s]);
            }
            if (!ok) break;
            mma_commit(&tfull[buf]);
        }
        // TMEM is freed only after every MMA issued here has completed
        mma_commit(mdone);
        mbar_drain(mdone, 0);
    } else if (warp >= 2) {
        // epilogue: warp w reads TMEM lanes 32 (w % 4) .. + 31, columns of its half of the tile
        const int q = warp & 3, hc = (warp - 2) >> 2;
        const uint32_t lanes = (uint32_t)(32 * q) << 16;
        uint32_t lt = 0;
        for (int t = blockIdx.x; t < J.ntiles; t += gridDim.x, ++lt) {
            const uint32_t buf = lt % NBUF;
            if (!mbar_wait(&tfull[buf], (lt / NBUF) & 1, flag)) break;
            asm volatile("tcgen05.fence::after_thread_sync;");
            const int z = t / per_z, rem = t - z * per_z;
            const int tn = rem / J.tiles_m, tm = rem - tn * J.tiles_m;
            const int m = tm * DT_BM + 32 * q + lane, n0 = tn * BN + hc * HALF;
            const bool mv = m < J.M;
            const int ea = mv ? J.ea[(J.a_batch > 1 ? z : 0) * J.ea_zs + m] - 30 : 0;
            const int* eb = J.eb + (J.b_batch > 1 ? z : 0) * J.eb_zs;
            const int nn = max(0, min(HALF, J.N - n0));
            const uint32_t col = tmem + lanes + buf * 3 * BN + hc * HALF;
            const int64_t base = (int64_t)z * J.zs + (int64_t)n0 * J.ldn + m;
            if (J.mode == DT_F32) {
                // all of this warp's values into registers, TMEM released, then the stores
                float hv[HALF];
#pragma unroll
                for (int c = 0; c < HALF; c += 16) {
                    float v0[16], v1[16], v2[16];
                    if (c < nn) {
                        tmem_ld16(col + c, v0);
                        tmem_ld16(col + BN + c, v1);
                        tmem_ld16(col + 2 * BN + c, v2);
#pragma unroll
                        for (int j = 0; j < 16; ++j) {
                            float lo;
                            combine3(v0[j], v1[j], v2[j], hv[c + j], lo);
                        }
                    }
                }
                asm volatile("tcgen05.fence::before_thread_sync;");
                __syncwarp();
                if (lane == 0) mbar_arrive(&tempty[buf]);
                if (mv) {
                    float* o = (float*)J.out + base;
#pragma unroll
                    for (int j = 0; j < HALF; ++j)
                        if (j < nn) o[j * J.ldn] = scale_f32(hv[j], ea + eb[n0 + j]);
                }
            } else {
                for (int c = 0; c < nn; c += 16) {
                    float v0[16], v1[16], v2[16];
                    tmem_ld16(col + c, v0);
                    tmem_ld16(col + BN + c, v1);
                    tmem_ld16(col + 2 * BN + c, v2);
                    if (!mv) continue;
#pragma unroll
                    for (int j = 0; j < 16; ++j) {
                        if (c + j >= nn) break;
                        float hi, lo;
                        combine3(v0[j], v1[j], v2[j], hi, lo);
                        const int e = ea + eb[n0 + c + j];
                        const int64_t at = base + (int64_t)(c + j) * J.ldn;
                        if (J.mode == DT_PAIR) {
                            reinterpret_cast<float2*>(J.out)[at] = make_float2(scale_f32(hi, e), scale_f32(lo, e));
                        } else {
                            const double v = (double)hi + (double)lo;
                            const int e1 = max(-1022, min(1023, e));
                            reinterpret_cast<double*>(J.out)[at] =
                                (v * __longlong_as_double((long long)(e1 + 1023) << 52)) *
                                __longlong_as_double((long long)(max(-1022, min(1023, e - e1)) + 1023) << 52);
                        }
                    }
                }
                asm volatile("tcgen05.fence::before_thread_sync;");
                __syncwarp();
                if (lane == 0) mbar_arrive(&tempty[buf]);
            }
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    if (warp == 1) {
        asm volatile("tcgen05.fence::after_thread_sync;");
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(C::TMEM_COLS));
    }
}

// ---------------------------------------------------------------------------
// operand split, in integer arithmetic on bit patterns
// ---------------------------------------------------------------------------

// round(m 2^k) for an unsigned significand m < 2^53, nearest-even; 0 below 2^-61
__device__ __forceinline__ unsigned long long shift_round(unsigned long long mant, int k) {
    if (k >= 0) return mant << k;
    if (k < -60) return 0;
    unsigned long long w = mant >> -k;
    const unsigned long long rem = mant & ((1ull << -k) - 1), half = 1ull << (-k - 1);
    if (rem > half || (rem == half && (w & 1))) ++w;
    return w;
}

// round(x 2^s) as an integer for finite x; the caller guarantees |x 2^s| < 2^62
__device__ __forceinline__ long long fixed_of(double x, int s) {
    const unsigned long long bits = (unsigned long long)__double_as_longlong(x);
    const int ex = (int)((bits >> 52) & 0x7ff);
    unsigned long long mant = bits & ((1ull << 52) - 1);
    if (ex == 0 && mant == 0) return 0;
    int e2 = -1074;
    if (ex) {
        mant |= 1ull << 52;
        e2 = ex - 1075;
    }
    const long long w = (long long)shift_round(mant, e2 + s);
    return (bits >> 63) ? -w : w;
}
__device__ __forceinline__ long long fixed_of(float x, int s) {
    const unsigned int bits = __float_as_uint(x);
    const int ex = (int)((bits >> 23) & 0xff);
    unsigned long long mant = bits & 0x7fffffu;
    if (ex == 0 && mant == 0) return 0;
    int e2 = -149;
    if (ex) {
        mant |= 1u << 23;
        e2 = ex - 150;
    }
    const long long w = (long long)shift_round(mant, e2 + s);
    return (bits >> 31) ? -w : w;
}

// R 2^-FXB times 2^9, rounded to FP16 (11 significant bits, nearest-even; subnormal
// below 2^-14); q = the rounded value, back in units of 2^-FXB (an integer). With
// FXB = 50 the FP16 value is R 2^-41: normal from 2^27 units up, quantum 2^17 units
// below.
__device__ __forceinline__ unsigned short f16_of_fixed(long long R, long long& q) {
    if (R == 0) {
        q = 0;
        return 0;
    }
    const unsigned neg = R < 0;
    const unsigned long long a = neg ? (unsigned long long)(-R) : (unsigned long long)R;
    const int msb = 63 - __clzll((long long)a);
    unsigned long long m;
    unsigned bits;
    if (msb >= FXB - 23) {                               // normal: keep 11 significant bits
        int sh = msb - 10;
        m = a >> sh;
        const unsigned long long rem = a & ((1ull << sh) - 1), half = 1ull << (sh - 1);
        if (rem > half || (rem == half && (m & 1))) ++m;
        if (m == 2048) {
            m = 1024;
            ++sh;
        }
        q = (long long)(m << sh);
        // value (m / 1024) 2^(sh - FXB + 19): biased exponent sh - FXB + 34
        bits = ((unsigned)(sh - FXB + 34) << 10) | (unsigned)(m & 1023);
    } else {                                             // subnormal: quantum 2^-24 = 2^(FXB - 33) units
        constexpr int sh = FXB - 33;
        m = a >> sh;
        const unsigned long long rem = a & ((1ull << sh) - 1), half = 1ull << (sh - 1);
        if (rem > half || (rem == half && (m & 1))) ++m;
        q = (long long)(m << sh);
        bits = (unsigned)m;                              // m = 1024 is the smallest normal's encoding
    }
    if (neg) q = -q;
    return (unsigned short)((neg << 15) | bits);
}

// sources: FP64 values, or FP32 pairs (hi, lo) whose sum is the value
struct SrcF64 {
    const double* p;
    __device__ unsigned long long mag(int64_t i) const {   // orders like |x|
        return (unsigned long long)__double_as_longlong(p[i]) & 0x7fffffffffffffffull;
    }
    __device__ static int exp_of(unsigned long long mb) {  // E with max|x| in [2^(E-1), 2^E)
        const int ex = (int)(mb >> 52);
        return ex ? ex - 1022 : (63 - __clzll((long long)mb)) - 1073;
    }
    __device__ long long fixed(int64_t i, int s) const { return fixed_of(p[i], s); }
};
struct SrcPair {
    const float2* p;
    __device__ unsigned long long mag(int64_t i) const { return __float_as_uint(p[i].x) & 0x7fffffffu; }
    __device__ static int exp_of(unsigned long long mb) {
        const int ex = (int)(mb >> 23);
        return ex ? ex - 126 : (63 - __clzll((long long)mb)) - 148;
    }
    __device__ long long fixed(int64_t i, int s) const {
        const float2 v = p[i];
        return fixed_of(v.x, s) + fixed_of(v.y, s);
    }
};

// One warp per row (b, i) of `batch` stacked operands:
//   x(k) = src[b*sb + row(i)*si + k*sk] for k < cols, 0 for cols <= k < kpad,
//   row(i) = ridx ? ridx[i] : i;
// written as FP16 d0 2^9, d1 2^2, t1 2^9, t2 2^9 into parts[p][b][i][k], with the row
// exponent E in exps[b*rows + i].
template <class Src>
__global__ void k_split_dt(Src src, const int32_t* __restrict__ ridx, int64_t rows, int64_t cols, int64_t si,
                           int64_t sk, int64_t sb, int64_t batch, int64_t kpad, unsigned short* __restrict__ parts,
                           int* __restrict__ exps) {
    const int lane = threadIdx.x & 31;
    const int64_t w = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    if (w >= rows * batch) return;
    const int64_t b = w / rows, i = w - b * rows;
    const int64_t x0 = b * sb + (int64_t)(ridx ? ridx[i] : i) * si;
    unsigned long long mb = 0;
    for (int64_t k = lane; k < cols; k += 32) mb = max(mb, src.mag(x0 + k * sk));
    for (int o = 16; o; o >>= 1) mb = max(mb, __shfl_xor_sync(0xffffffffu, mb, o));
    const int E = mb ? Src::exp_of(mb) : 0;
    if (lane == 0) exps[w] = E;
    const int64_t ps = batch * rows * kpad, off = w * kpad;
    for (int64_t k = lane; k < kpad; k += 32) {
        unsigned short p0 = 0, p1 = 0, p2 = 0, p3 = 0;
        if (k < cols) {
            const long long W = src.fixed(x0 + k * sk, 6 - E + FXB);   // |W| < 2^(6 + FXB)
            const long long d0 = (W + (1ll << (FXB - 1))) >> FXB;     // nearest, |d0| <= 64
            long long R = W - (d0 << FXB);                             // |R| <= 2^(FXB - 1)
            const long long d1 = (R + (1ll << (FXB - 8))) >> (FXB - 7);  // nearest, |d1| <= 64
            R -= d1 << (FXB - 7);                                      // |R| <= 2^(FXB - 8)
            long long q;
            p2 = f16_of_fixed(R, q);
            R -= q;
            p3 = f16_of_fixed(R, q);
            p0 = __half_as_ushort(__float2half_rn((float)(d0 * 512)));   // exact
            p1 = __half_as_ushort(__float2half_rn((float)(d1 * 4)));     // exact
        }
        parts[off + k] = p0;
        parts[ps + off + k] = p1;
        parts[2 * ps + off + k] = p2;
        parts[3 * ps + off + k] = p3;
    }
}

int64_t pad32(int64_t x) { return (x + 31) / 32 * 32; }

bool make_map_dt(CUtensorMap* m, const DtOp& op, int box_rows) {
    auto fn = encode_fn();
    if (!fn) return false;
    cuuint64_t dims[3] = {(cuuint64_t)op.kpad, (cuuint64_t)op.rows, (cuuint64_t)(DT_PARTS * op.batch)};
    cuuint64_t strides[2] = {(cuuint64_t)(op.kpad * 2), (cuuint64_t)(op.rows * op.kpad * 2)};
    cuuint32_t box[3] = {(cuuint32_t)DT_BK, (cuuint32_t)box_rows, 1};
    cuuint32_t es[3] = {1, 1, 1};
    CUresult r = fn(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT16, 3, op.p, dims, strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
                    CU_TENSOR_MAP_SWIZZLE_64B, CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS;
}

template <int BN>
cudaError_t launch_dt(const DtJob& J, int grid, int* flag, cudaStream_t st) {
    using C = DtCfg<BN>;
    static std::once_flag once;
    static cudaError_t attr = cudaSuccess;
    std::call_once(once, [] {
        attr = cudaFuncSetAttribute(k_dt_gemm<BN>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)C::SMEM);
    });
    if (attr != cudaSuccess) return attr;
    k_dt_gemm<BN><<<grid, DT_THREADS, C::SMEM, st>>>(J, flag);
    count_kernels(1);
    return cudaGetLastError();
}

int num_sms_now() {
    static int n = 0;
    static std::once_flag once;
    std::call_once(once, [] {
        int dev = 0;
        if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
            n = 0;
    });
    return n > 0 ? n : 1;
}

DtOp dt_alloc(Arena& ar, int64_t rows, int64_t kpad, int64_t batch) {
    DtOp o;
    o.p = ar.get<uint16_t>((int64_t)DT_PARTS * batch * rows * kpad);
    o.e = ar.get<int>(batch * rows);
    o.rows = rows;
    o.kpad = kpad;
    o.batch = batch;
    return o;
}

template <class Src>
cudaError_t dt_split(Src src, const int32_t* ridx, int64_t cols, int64_t si, int64_t sk, int64_t sb, const DtOp& d,
                     cudaStream_t st) {
    const int64_t warps = d.rows * d.batch;
    if (warps <= 0) return cudaSuccess;
    if (cols > d.kpad) return cudaErrorInvalidValue;
    k_split_dt<Src><<<(unsigned)((warps * 32 + 255) / 256), 256, 0, st>>>(src, ridx, d.rows, cols, si, sk, sb, d.batch,
                                                                          d.kpad, d.p, d.e);
    count_kernels(1);
    return cudaGetLastError();
}

int dt_gemm(const DtOp& A, const DtOp& B, int64_t M, int64_t N, int64_t batch, const DtOut& out, const DtOpts& opt,
            int* flag, cudaStream_t st, std::string* err) {
    if (M <= 0 || N <= 0 || batch <= 0) return LS_OK;
    if (A.kpad != B.kpad || A.kpad % DT_BK != 0 || A.kpad > DT_MAXK || M > A.rows || N > B.rows ||
        (A.batch != 1 && A.batch != batch) || (B.batch != 1 && B.batch != batch))
        return tc_err(err, "dt gemm: bad operands", LS_ERR_ARG);
    int bn = opt.tile_n;
    if (bn == 0) bn = N <= 32 ? 32 : N <= 64 ? 64 : 128;
    if (bn != 32 && bn != 64 && bn != 128) return tc_err(err, "dt gemm: tile_n must be 32, 64 or 128", LS_ERR_ARG);
    DtJob J;
    memset(&J, 0, sizeof J);
    if (!make_map_dt(&J.a, A, DT_BM) || !make_map_dt(&J.b, B, bn))
        return tc_err(err, "dt gemm: cuTensorMapEncodeTiled failed");
    J.M = (int)M;
    J.N = (int)N;
    J.nkb = (int)(A.kpad / DT_BK);
    J.tiles_m = (int)((M + DT_BM - 1) / DT_BM);
    J.tiles_n = (int)((N + bn - 1) / bn);
    const int64_t nt = (int64_t)J.tiles_m * J.tiles_n * batch;
    if (nt > INT32_MAX) return tc_err(err, "dt gemm: too many tiles", LS_ERR_ARG);
    J.ntiles = (int)nt;
    J.a_batch = (int)A.batch;
    J.b_batch = (int)B.batch;
    J.ea = A.e;
    J.eb = B.e;
    J.ea_zs = A.rows;
    J.eb_zs = B.rows;
    J.out = out.p;
    J.ldn = out.ldn;
    J.zs = out.zs;
    J.mode = out.mode;
    const int grid = (int)std::min<int64_t>(nt, num_sms_now());
    cudaError_t e = bn == 32 ? launch_dt<32>(J, grid, flag, st)
                    : bn == 64 ? launch_dt<64>(J, grid, flag, st)
                               : launch_dt<128>(J, grid, flag, st);
    if (e != cudaSuccess) return tc_err(err, std::string("dt gemm launch: ") + cudaGetErrorString(e));
    return LS_OK;
}

}  // namespace

// Operands of the slab evaluation that depend only on the reduced tensor, built
// on the first evaluation and kept with the context: Z0^T and Z1^T (rows y over
// the rank index) and the core (rows (a, b) over c), all in digit + tail form.
struct DtEvalCache {
    cudaStream_t st = nullptr;
    DtOp z0t, z1t, core;
    std::vector<void*> allocs;
};

void dt_eval_free(DtEvalCache* c) {
    if (!c) return;
    for (void* p : c->allocs) cudaFreeAsync(p, c->st);
    delete c;
}

int dt_eval(DtEvalCache** cache, const double* const Z[3], const int32_t* r, const double* B, int64_t N,
            const int32_t* zidx, int nslab, void* out, int out_f32, const DtOpts& opt, cudaStream_t st,
            std::string* err) {
    const int64_t r0 = r[0], r1 = r[1], r2 = r[2];
    const int64_t k0 = pad32(r0), k1 = pad32(r1), k2 = pad32(r2);
    if (k0 > DT_MAXK || k1 > DT_MAXK || k2 > DT_MAXK) return tc_err(err, "eval: rank above 2048", LS_ERR_ARG);
    if (nslab <= 0) return LS_OK;
    if (!*cache) {
        Scope sc("eval.prepare", st);
        DtEvalCache* c = new DtEvalCache();
        c->st = st;
        Arena tmp(st);
        double* zt = tmp.get<double>(N * std::max(r0, r1));
        auto keep = [&](int64_t rows, int64_t kpad) {
            DtOp o;
            void* p = nullptr;
            void* q = nullptr;
            if (cudaMallocAsync(&p, (size_t)DT_PARTS * rows * kpad * 2, st) == cudaSuccess) c->allocs.push_back(p);
            if (cudaMallocAsync(&q, (size_t)rows * sizeof(int), st) == cudaSuccess) c->allocs.push_back(q);
            o.p = (uint16_t*)p;
            o.e = (int*)q;
            o.rows = rows;
            o.kpad = kpad;
            return o;
        };
        c->z0t = keep(N, k0);
        c->z1t = keep(N, k1);
        c->core = keep(r0 * r1, k2);
        if (!zt || !c->z0t.ok() || !c->z1t.ok() || !c->core.ok()) {
            dt_eval_free(c);
            return tc_err(err, "eval: out of memory", LS_ERR_OOM);
        }
        // Z_l is r_l x N (rows are basis vectors): transpose, then split rows of length r_l
        if (launch_transpose(Z[0], r0, N, zt, st) != cudaSuccess ||
            dt_split(SrcF64{zt}, nullptr, r0, r0, 1, 0, c->z0t, st) != cudaSuccess ||
            launch_transpose(Z[1], r1, N, zt, st) != cudaSuccess ||
            dt_split(SrcF64{zt}, nullptr, r1, r1, 1, 0, c->z1t, st) != cudaSuccess ||
            dt_split(SrcF64{B}, nullptr, r2, r2, 1, 0, c->core, st) != cudaSuccess) {
            dt_eval_free(c);
            return tc_err(err, "eval: operand preparation failed");
        }
        *cache = c;
    }
    const DtEvalCache& c = **cache;
    // slabs in chunks that bound the per-call scratch to about 1 GB
    const int64_t per = r0 * r1 * 8 + DT_PARTS * r0 * k1 * 2 + r0 * 4 + N * r0 * 8 + DT_PARTS * N * k0 * 2 + N * 4 +
                        DT_PARTS * k2 * 2 + 4;
    const int chunk = (int)std::max<int64_t>(1, std::min<int64_t>(nslab, ((int64_t)1 << 30) / per));
    Arena ar(st);
    Flag fl(ar, st);
    DtOp z2s = dt_alloc(ar, chunk, k2, 1), ms = dt_alloc(ar, r0, k1, chunk), ts = dt_alloc(ar, N, k0, chunk);
    float2* Mt = ar.get<float2>((int64_t)chunk * r0 * r1);
    float2* Tt = ar.get<float2>((int64_t)chunk * N * r0);
    if (!fl.d || !z2s.ok() || !ms.ok() || !ts.ok() || !Mt || !Tt) return tc_err(err, "eval: out of memory", LS_ERR_OOM);
    const size_t esz = out_f32 ? 4 : 8;
    for (int s0 = 0; s0 < nslab; s0 += chunk) {
        const int ns = std::min(chunk, nslab - s0);
        DtOp z2 = z2s, m = ms, t = ts;
        z2.rows = ns;
        m.batch = ns;
        t.batch = ns;
        int rc;
        {
            Scope sc("eval.mt", st);
            // rows s of Z2^T: Z2[c][z_s], gathered
            if (dt_split(SrcF64{Z[2]}, zidx + s0, r2, 1, N, 0, z2, st) != cudaSuccess)
                return tc_err(err, "eval: split failed");
            // M[s][(a, b)] = sum_c core[(a, b)][c] Z2[c][z_s]
            rc = dt_gemm(c.core, z2, r0 * r1, ns, 1, DtOut{Mt, r0 * r1, 0, DT_PAIR}, opt, fl.d, st, err);
            if (rc != LS_OK) return rc;
            if (dt_split(SrcPair{Mt}, nullptr, r1, r1, 1, r0 * r1, m, st) != cudaSuccess)
                return tc_err(err, "eval: split failed");
            // T_s[y][a] = sum_b M_s[a][b] Z1^T[y][b]   (D[a][y], a on the lanes)
            rc = dt_gemm(m, c.z1t, r0, N, ns, DtOut{Tt, r0, N * r0, DT_PAIR}, opt, fl.d, st, err);
            if (rc != LS_OK) return rc;
            if (dt_split(SrcPair{Tt}, nullptr, r0, r0, 1, N * r0, t, st) != cudaSuccess)
                return tc_err(err, "eval: split failed");
        }
        {
            Scope sc("eval.slab", st);
            // S_s[x][y] = sum_a T_s[y][a] Z0^T[x][a]   (D[y][x], y on the lanes: rows of S contiguous)
            void* o = static_cast<char*>(out) + (size_t)s0 * N * N * esz;
            rc = dt_gemm(t, c.z0t, N, N, ns, DtOut{o, N, N * N, out_f32 ? DT_F32 : DT_F64}, opt, fl.d, st, err);
            if (rc != LS_OK) return rc;
        }
    }
    return fl.check(err);
}

int dt_gemm_nt(const double* A, const double* B, int64_t M, int64_t N, int64_t K, void* D, int out_f32,
               const DtOpts& opt, cudaStream_t st, std::string* err) {
    if (M <= 0 || N <= 0) return LS_OK;
    const int64_t kp = pad32(std::max<int64_t>(K, 1));
    if (kp > DT_MAXK) return tc_err(err, "gemm_nt_mixed: K above 2048", LS_ERR_ARG);
    Arena ar(st);
    Flag fl(ar, st);
    DtOp a = dt_alloc(ar, M, kp, 1), b = dt_alloc(ar, N, kp, 1);
    if (!fl.d || !a.ok() || !b.ok()) return tc_err(err, "gemm_nt_mixed: out of memory", LS_ERR_OOM);
    if (dt_split(SrcF64{A}, nullptr, K, K, 1, 0, a, st) != cudaSuccess ||
        dt_split(SrcF64{B}, nullptr, K, K, 1, 0, b, st) != cudaSuccess)
        return tc_err(err, "gemm_nt_mixed: split failed");
    // D[m][n] row-major = the kernel's D with n on the lanes: swap the operands
    int rc = dt_gemm(b, a, N, M, 1, DtOut{D, N, 0, out_f32 ? DT_F32 : DT_F64}, opt, fl.d, st, err);
    if (rc != LS_OK) return rc;
    return fl.check(err);
}

}  // namespace ls
