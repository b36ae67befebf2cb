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
// K ranges above 2048 (up to 4096) take a fourth accumulator: acc1 keeps
// d0 d1 and acc3 d1 d0, each a sum of multiples of 2^-7 below 2^12 K, exact
// for K <= 4096.
// The two leading levels are exact, whatever rounding the tensor core's adds
// use. That matters: they truncate, and a float accumulator holding terms at
// 2^-7 of the result drifts by about half an ulp per MMA. acc2 sits below
// 2^-14 of the result, where that drift stays small: on random data about
// 2^-38 K^1.5 of max|a| max|b| or less (measured: 2^-21 at K = 4096). The dropped products
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
// - Warps 2-17: epilogue. Four warps per TMEM lane quadrant, each taking a
//   quarter of the tile's columns. Each pulls its accumulators into
//   registers and releases TMEM before it stores, so the next tile's MMAs
//   overlap the stores. Tiles up to 64 wide also double-buffer TMEM.
// Every mbarrier wait is bounded. On timeout the kernel raises the flag; the
// producer drains its copies, the MMA warp waits for its MMAs, and TMEM is
// freed before exit.
#include <cuda.h>
#include <cuda_fp16.h>

#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <deque>
#include <map>
#include <mutex>
#include <string>
#include <tuple>
#include <vector>

#include "lattice_sum.h"
#include "ls_common.cuh"
#include "ls_eval.cuh"
#include "ls_tcgen05.cuh"

namespace ls {

namespace {

using namespace tc5;

constexpr int DT_BM = 128, DT_BK = 32, DT_PARTS = 4, DT_EPI_WARPS = 16;
constexpr int DT_THREADS = 64 + 32 * DT_EPI_WARPS;       // TMA warp, MMA warp, epilogue warps
constexpr int DT_TA = DT_BM * DT_BK * 2;                 // one A part tile: 8 KB
constexpr int DT_MAXK = 2048;                            // exact level-1 accumulation, three accumulators
constexpr int DT_MAXK4 = 4096;                           // the same with four
constexpr int FXB = 50;                                  // fraction bits of the fixed-point split

__host__ __device__ constexpr int pow2ceil(int x) {
    int p = 32;
    while (p < x) p <<= 1;
    return p;
}

template <int BN>
struct DtCfg {
    static constexpr int TB = BN * DT_BK * 2;
    static constexpr int STAGE = DT_PARTS * (DT_TA + TB);
    static constexpr int STAGES = std::min(8, (220 * 1024) / STAGE);
    static constexpr size_t SMEM = (size_t)STAGES * STAGE + 1024 + 256;
    static_assert(4 * BN <= 512, "four accumulators must fit TMEM");
};
// accumulator buffers (two when both fit TMEM, so that a tile's MMAs overlap the
// previous tile's epilogue) and the TMEM columns they take
__host__ __device__ constexpr int dt_nbuf(int bn, int nacc) { return nacc * bn * 2 <= 512 ? 2 : 1; }
__host__ __device__ constexpr int dt_tmem_cols(int bn, int nacc) { return pow2ceil(nacc * bn * dt_nbuf(bn, nacc)); }

struct DtJob {
    CUtensorMap a, b;          // (kpad, rows, 4 * batch) fp16, 64-byte swizzle
    int M, N, nkb;             // k-blocks of 32
    int tiles_m, tiles_n, ntiles;
    int n_fast;                // tile order: n fastest (the A operand streams once) or m fastest
    int a_batch, b_batch;      // batches held by each operand (1: shared)
    const int* ea;             // row exponents [batch][rows]
    const int* eb;
    int64_t ea_zs, eb_zs;
    void* out;                 // out[z * zs + n * ldn + m]
    int64_t ldn, zs;
    int mode;                  // DtOutMode (also the kernel's template argument)
    int nacc;                  // accumulators: 3 (K ranges <= 2048) or 4 (<= 4096)
    int accumulate;            // DT_F64 only: out += D
    const int* kb_lo;          // per-z k-block ranges [kb_lo[z], kb_lo[z + 1]) (grouped form), or
    int kb_begin, kb_end;      // one range for every z
};

// tile t -> (batch z, m-tile, n-tile)
__device__ __forceinline__ void tile_of(const DtJob& J, int t, int& z, int& tm, int& tn) {
    const int per_z = J.tiles_m * J.tiles_n;
    z = t / per_z;
    const int rem = t - z * per_z;
    if (J.n_fast) {
        tm = rem / J.tiles_n;
        tn = rem - tm * J.tiles_n;
    } else {
        tn = rem / J.tiles_m;
        tm = rem - tn * J.tiles_m;
    }
}

__device__ __forceinline__ void k_range(const DtJob& J, int z, int& k0, int& k1) {
    if (J.kb_lo) {
        k0 = J.kb_lo[z];
        k1 = J.kb_lo[z + 1];
    } else {
        k0 = J.kb_begin;
        k1 = J.kb_end;
    }
}

__device__ __forceinline__ float pow2f(int e) {           // e in [-126, 127]
    return __int_as_float((e + 127) << 23);
}

// v 2^e by two exact multiplications (no overflow of the factors for |e| <= 252)
__device__ __forceinline__ float scale_f32(float v, int e) {
    const int e1 = max(-126, min(127, e));
    return (v * pow2f(e1)) * pow2f(max(-126, min(127, e - e1)));
}

// (hi + lo) 2^e as a double without FP64 arithmetic, for a pair from combine3
// (|lo| <= ulp(hi) / 2). hi's significand goes to bit 52 of a 53-bit integer,
// lo is aligned to it and added (bits of lo below the double's last place are
// dropped: < 1 ulp), the sum renormalised by at most one place and the exponent
// biased by e. Zero, subnormal and out-of-range cases take the FP64 route.
__device__ __forceinline__ double pair_to_f64(float hi, float lo, int e) {
    const unsigned hb = __float_as_uint(hi), lb = __float_as_uint(lo);
    const int eh = (int)((hb >> 23) & 0xff), el = (int)((lb >> 23) & 0xff);
    int ed = eh - 127 + 1023 + e;
    if (eh == 0 || eh == 0xff || ed < 2 || ed > 2045) {
        const int e1 = max(-1022, min(1023, e));
        return (((double)hi + (double)lo) * __longlong_as_double((long long)(e1 + 1023) << 52)) *
               __longlong_as_double((long long)(max(-1022, min(1023, e - e1)) + 1023) << 52);
    }
    long long M = (long long)((hb & 0x7fffffu) | 0x800000u) << 29;        // units 2^(eh - 127 - 52)
    if (el != 0) {
        const long long ml = (long long)((lb & 0x7fffffu) | 0x800000u);
        const int k = el - eh + 29;                                        // lo = ml 2^k units, k <= 5
        const long long lv = k >= 0 ? ml << k : (k > -40 ? ml >> -k : 0);
        M += ((hb ^ lb) >> 31) ? -lv : lv;
    }
    if (M >= (1ll << 53)) {
        M >>= 1;
        ++ed;
    } else if (M < (1ll << 52)) {
        M <<= 1;
        --ed;
    }
    const unsigned long long bits =
        ((unsigned long long)(hb >> 31) << 63) | ((unsigned long long)ed << 52) | ((unsigned long long)M & ((1ull << 52) - 1));
    return __longlong_as_double((long long)bits);
}

__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
    s = a + b;
    const float bb = s - a;
    e = (a - (s - bb)) + (b - bb);
}

// a0 + a1 + a2 (a0, a1 exact, |a2| small) as an unevaluated pair hi + lo, by two
// TwoSums: hi is the sum rounded once, lo the rest to about 2^-48 of it
__device__ __forceinline__ void combine3(float a0, float a1, float a2, float& hi, float& lo) {
    float s, e;
    two_sum(a0, a1, s, e);
    const float t = e + a2;
    hi = s + t;
    const float b2 = hi - s;
    lo = (s - (hi - b2)) + (t - b2);
}
template <int BN, int MODE>
__global__ void __launch_bounds__(DT_THREADS, 1) k_dt_gemm(const __grid_constant__ DtJob J, int* flag) {
    using C = DtCfg<BN>;
    constexpr int S = C::STAGES;
    const int nacc = J.nacc, NBUF = dt_nbuf(BN, nacc), tcols = dt_tmem_cols(BN, nacc);
    constexpr int QC = BN / 4;                    // columns per epilogue warp
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    unsigned char* smem = (unsigned char*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    uint64_t* full = (uint64_t*)(smem + S * C::STAGE);
    uint64_t* empty = full + S;
    uint64_t* tfull = empty + S;       // accumulator buffer holds a finished tile
    uint64_t* tempty = tfull + 2;      // epilogue has read it
    uint64_t* mdone = tempty + 2;      // every MMA of this CTA has completed
    uint32_t* tmem_slot = (uint32_t*)(mdone + 1);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

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
                     "r"(tcols));
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
            int z, tm, tn;
            tile_of(J, t, z, tm, tn);
            const int za = J.a_batch > 1 ? z : 0, zb = J.b_batch > 1 ? z : 0;
            int k0, k1;
            k_range(J, z, k0, k1);
            for (int kb = k0; kb < k1; ++kb, ++it) {
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
            const uint32_t c0 = tmem + buf * nacc * BN, c1 = c0 + BN, c2 = c0 + 2 * BN,
                           c3 = nacc == 4 ? c0 + 3 * BN : c1;
            int k0, k1;
            k_range(J, t / (J.tiles_m * J.tiles_n), k0, k1);
            for (int kb = k0; kb < k1; ++kb, ++it) {
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
                    const uint32_t acc = (kb != k0 || kk) ? 1u : 0u;
                    mma_bf16(c0, a0, b0, idesc, acc);            // d0 d0: exact
                    mma_bf16(c1, a0, b1, idesc, acc);            // d0 d1, d1 d0: exact
                    mma_bf16(c3, a1, b0, idesc, nacc == 4 ? acc : 1u);
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
        // epilogue: warp w reads TMEM lanes 32 (w % 4) .. + 31 and a quarter of the tile's
        // columns; it takes all of its values into registers, releases the accumulators to
        // the next tile's MMAs, then scales and stores
        const int q = warp & 3, hc = (warp - 2) >> 2;
        const uint32_t lanes = (uint32_t)(32 * q) << 16;
        uint32_t lt = 0;
        for (int t = blockIdx.x; t < J.ntiles; t += gridDim.x, ++lt) {
            const uint32_t buf = lt % NBUF;
            if (!mbar_wait(&tfull[buf], (lt / NBUF) & 1, flag)) break;
            asm volatile("tcgen05.fence::after_thread_sync;");
            int z, tm, tn;
            tile_of(J, t, z, tm, tn);
            const int m = tm * DT_BM + 32 * q + lane, n0 = tn * BN + hc * QC;
            const int nn = max(0, min(QC, J.N - n0));
            const uint32_t col = tmem + lanes + buf * nacc * BN + hc * QC;
            int k0, k1;
            k_range(J, z, k0, k1);
            const bool live = k1 > k0;   // an empty K range leaves the accumulators unwritten: zeros
            float hv[QC], lv[QC];
#pragma unroll
            for (int c = 0; c < QC; c += 8) {
                if (c < nn) {
                    float v0[8], v1[8], v2[8];
                    if (nacc == 4) {
                        // the two level-1 sums by TwoSum; its rounding error joins acc2
                        float v3[8];
                        tmem_ld8(col + BN + c, v1);
                        tmem_ld8(col + 3 * BN + c, v3);
#pragma unroll
                        for (int j = 0; j < 8; ++j) two_sum(v1[j], v3[j], v1[j], v3[j]);
                        tmem_ld8(col + 2 * BN + c, v2);
#pragma unroll
                        for (int j = 0; j < 8; ++j) v2[j] += v3[j];
                    } else {
                        tmem_ld8(col + BN + c, v1);
                        tmem_ld8(col + 2 * BN + c, v2);
                    }
                    tmem_ld8(col + c, v0);
#pragma unroll
                    for (int j = 0; j < 8; ++j)
                        combine3(live ? v0[j] : 0.f, live ? v1[j] : 0.f, live ? v2[j] : 0.f, hv[c + j], lv[c + j]);
                }
            }
            asm volatile("tcgen05.fence::before_thread_sync;");
            __syncwarp();
            if (lane == 0) mbar_arrive(&tempty[buf]);
            if (m >= J.M) continue;
            const int ea = J.ea[(J.a_batch > 1 ? z : 0) * J.ea_zs + m] - 30;
            const int* eb = J.eb + (J.b_batch > 1 ? z : 0) * J.eb_zs + n0;
            const int64_t base = (int64_t)z * J.zs + (int64_t)n0 * J.ldn + m;
#pragma unroll
            for (int j = 0; j < QC; ++j) {
                if (j >= nn) break;
                const int e = ea + eb[j];
                const int64_t at = base + (int64_t)j * J.ldn;
                if (MODE == DT_F32) {
                    reinterpret_cast<float*>(J.out)[at] = scale_f32(hv[j], e);
                } else if (MODE == DT_PAIR) {
                    reinterpret_cast<float2*>(J.out)[at] = make_float2(scale_f32(hv[j], e), scale_f32(lv[j], e));
                } else {
                    const double sv = pair_to_f64(hv[j], lv[j], e);
                    double* o = reinterpret_cast<double*>(J.out) + at;
                    *o = J.accumulate ? *o + sv : sv;
                }
            }
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    if (warp == 1) {
        asm volatile("tcgen05.fence::after_thread_sync;");
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(tcols));
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

// Split sources: element (b, i, k) of `batch` stacked operands (row i, column k).
//   SrcF64:    p[b*sb + row(i)*si + k*sk], row(i) = ridx ? ridx[i] : i
//   SrcPair:   the same over FP32 pairs (hi, lo) whose sum is the value
//   SrcIdx:    w[k] P[i*ld + idx[k]] (0 where idx[k] < 0): the columns of a projected
//              side matrix that the canonical terms use, in the order of a term list
//              (one batch; idx and w resolved from the term map once, k_term_index)
// mag() orders like |x|; exp_of() gives E with max|x| in [2^(E-1), 2^E) from it.
struct SrcF64 {
    static constexpr bool pair = false;
    const double* p;
    int64_t si, sk, sb;
    const int32_t* ridx;
    __device__ double at(int64_t b, int64_t i, int64_t k) const { return p[b * sb + (ridx ? ridx[i] : i) * si + k * sk]; }
    __device__ unsigned long long mag(int64_t b, int64_t i, int64_t k) const {
        return (unsigned long long)__double_as_longlong(at(b, i, k)) & 0x7fffffffffffffffull;
    }
    __device__ static int exp_of(unsigned long long mb) {
        const int ex = (int)(mb >> 52);
        return ex ? ex - 1022 : (63 - __clzll((long long)mb)) - 1073;
    }
    __device__ long long fixed(int64_t b, int64_t i, int64_t k, int s) const { return fixed_of(at(b, i, k), s); }
};
struct SrcPair {
    static constexpr bool pair = true;
    const float2* p;
    int64_t si, sk, sb;
    __device__ float2 at(int64_t b, int64_t i, int64_t k) const { return p[b * sb + i * si + k * sk]; }
    __device__ unsigned long long mag(int64_t b, int64_t i, int64_t k) const {
        return __float_as_uint(at(b, i, k).x) & 0x7fffffffu;
    }
    __device__ static int exp_of(unsigned long long mb) {
        const int ex = (int)(mb >> 23);
        return ex ? ex - 126 : (63 - __clzll((long long)mb)) - 148;
    }
    __device__ long long fixed(int64_t b, int64_t i, int64_t k, int s) const {
        const float2 v = at(b, i, k);
        return fixed_of(v.x, s) + fixed_of(v.y, s);
    }
};

// A gathered operand whose column map is already resolved: x(i, k) = w[k] P[i*ld + idx[k]]
// (w may be NULL), 0 where idx[k] < 0: with idx[k] = tcol[3 tmap[k] + mode] and
// w[k] = w[tmap[k]] resolved beforehand, an entry is two independent reads and one
// dependent one.
struct SrcIdx {
    static constexpr bool pair = false;
    const double* P;
    int64_t ld;
    const int32_t* idx;
    const double* w;
    __device__ double at(int64_t, int64_t i, int64_t k) const {
        const int c = idx[k];
        if (c < 0) return 0.0;
        const double v = P[i * ld + c];
        return w ? w[k] * v : v;
    }
    __device__ unsigned long long mag(int64_t b, int64_t i, int64_t k) const {
        return (unsigned long long)__double_as_longlong(at(b, i, k)) & 0x7fffffffffffffffull;
    }
    __device__ static int exp_of(unsigned long long mb) { return SrcF64::exp_of(mb); }
    __device__ long long fixed(int64_t b, int64_t i, int64_t k, int s) const { return fixed_of(at(b, i, k), s); }
};
// the core's column maps of modes 1 and 2 and the term weights over the padded term list
__global__ void k_term_index(const int32_t* __restrict__ tmap, const int32_t* __restrict__ tcol,
                             const double* __restrict__ xin, int64_t tpad, int32_t* __restrict__ idx1,
                             int32_t* __restrict__ idx2, double* __restrict__ w1) {
    const int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (k >= tpad) return;
    const int t = tmap[k];
    idx1[k] = t < 0 ? -1 : tcol[3 * (int64_t)t + 1];
    idx2[k] = t < 0 ? -1 : tcol[3 * (int64_t)t + 2];
    w1[k] = t < 0 ? 0.0 : xin[t];
}

// The same four parts from an FP32 pair (hi, lo) in FP32 arithmetic: the scaled
// value as a pair, nearest-integer digits (the differences are exact), the rest
// carried by TwoSum, the tails by the hardware FP16 conversion. Agrees with the
// integer route to the form's accuracy.
__device__ __forceinline__ void split_pair(float2 v, int E, unsigned short& p0, unsigned short& p1, unsigned short& p2,
                                           unsigned short& p3) {
    const float hs = scale_f32(v.x, 6 - E), ls = scale_f32(v.y, 6 - E);
    const float d0 = rintf(hs);
    float rh, rl;
    two_sum(hs - d0, ls, rh, rl);                    // the rest after d0, |.| <= 1/2
    const float d1 = rintf(rh * 128.f);
    float vh, vl;
    two_sum((rh * 128.f - d1) * 4.f, rl * 512.f, vh, vl);   // the rest after d1, times 2^9
    const __half t1 = __float2half_rn(vh);
    const __half t2 = __float2half_rn((vh - __half2float(t1)) + vl);
    p0 = __half_as_ushort(__float2half_rn(d0 * 512.f));
    p1 = __half_as_ushort(__float2half_rn(d1 * 4.f));
    p2 = __half_as_ushort(t1);
    p3 = __half_as_ushort(t2);
}

// the four parts of one entry, given its row exponent E
template <class Src>
__device__ __forceinline__ void split_entry(const Src& src, int64_t b, int64_t i, int64_t k, int E, unsigned short& p0,
                                            unsigned short& p1, unsigned short& p2, unsigned short& p3) {
    if constexpr (Src::pair) {
        split_pair(src.at(b, i, k), E, p0, p1, p2, p3);
        return;
    }
    const long long W = src.fixed(b, i, k, 6 - E + FXB);        // |W| < 2^(6 + FXB)
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

// One warp per row (b, i) of `batch` stacked operands: x(k) = src(b, i, k) for k < cols,
// 0 for cols <= k < kpad; written as FP16 d0 2^9, d1 2^2, t1 2^9, t2 2^9 into
// parts[p][b][i][k], with the row exponent E in exps[b*rows + i].
template <class Src>
__global__ void k_split_dt(Src src, int64_t rows, int64_t cols, int64_t batch, int64_t kpad,
                           unsigned short* __restrict__ parts, int* __restrict__ exps) {
    const int lane = threadIdx.x & 31;
    const int64_t w = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    if (w >= rows * batch) return;
    const int64_t b = w / rows, i = w - b * rows;
    unsigned long long mb = 0;
    for (int64_t k = lane; k < cols; k += 32) mb = max(mb, src.mag(b, i, k));
    for (int o = 16; o; o >>= 1) mb = max(mb, __shfl_xor_sync(0xffffffffu, mb, o));
    const int E = mb ? Src::exp_of(mb) : 0;
    if (lane == 0) exps[w] = E;
    const int64_t ps = batch * rows * kpad, off = w * kpad;
    for (int64_t k = lane; k < kpad; k += 32) {
        unsigned short p0 = 0, p1 = 0, p2 = 0, p3 = 0;
        if (k < cols) split_entry(src, b, i, k, E, p0, p1, p2, p3);
        parts[off + k] = p0;
        parts[ps + off + k] = p1;
        parts[2 * ps + off + k] = p2;
        parts[3 * ps + off + k] = p3;
    }
}

// Long rows, in two passes with the whole grid busy. Pass 1: mb[row] = max |x| bits
// (blocks of 256 threads over 1024-entry segments of one row; mb zeroed before).
template <class Src>
__global__ void k_rowmax(Src src, int64_t rows, int64_t cols, unsigned long long* __restrict__ mb) {
    const int64_t row = blockIdx.y, b = row / rows, i = row - b * rows;
    unsigned long long m = 0;
    for (int64_t k = blockIdx.x * 1024 + threadIdx.x; k < min(cols, (int64_t)(blockIdx.x + 1) * 1024); k += 256)
        m = max(m, src.mag(b, i, k));
    for (int o = 16; o; o >>= 1) m = max(m, __shfl_xor_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0 && m) atomicMax(mb + row, m);
}
// Pass 2: four consecutive entries (row, k .. k + 3) a thread (kpad is a multiple of 32),
// each part's four values stored as one 8-byte word.
template <class Src>
__global__ void k_split_rows(Src src, int64_t rows, int64_t cols, int64_t batch, int64_t kpad,
                             const unsigned long long* __restrict__ mb, unsigned short* __restrict__ parts,
                             int* __restrict__ exps) {
    const int64_t row = blockIdx.y, b = row / rows, i = row - b * rows;
    const int64_t k = 4 * (blockIdx.x * (int64_t)blockDim.x + threadIdx.x);
    if (k >= kpad) return;
    const int E = mb[row] ? Src::exp_of(mb[row]) : 0;
    if (k == 0) exps[row] = E;
    unsigned short q[4][4];   // [part][entry]
#pragma unroll
    for (int u = 0; u < 4; ++u) {
        q[0][u] = q[1][u] = q[2][u] = q[3][u] = 0;
        if (k + u < cols) split_entry(src, b, i, k + u, E, q[0][u], q[1][u], q[2][u], q[3][u]);
    }
    const int64_t ps = batch * rows * kpad, off = row * kpad + k;
#pragma unroll
    for (int p = 0; p < 4; ++p)
        *reinterpret_cast<uint2*>(parts + p * ps + off) =
            make_uint2((unsigned)q[p][0] | ((unsigned)q[p][1] << 16), (unsigned)q[p][2] | ((unsigned)q[p][3] << 16));
}

// Operand rows n of a pair matrix stored transposed, x(n, k) = W[k * ld + n] (k < cols):
// pass 1 has a thread per row walk k (reads coalesced across rows); pass 2 splits
// 64 x 64 tiles through shared memory so that both the reads (along n) and the
// writes (along k: 128 bytes of a row and part, a whole line) are contiguous.
__global__ void k_rowmax_tr(const float2* __restrict__ W, int64_t ld, int64_t rows, int64_t cols,
                            unsigned long long* __restrict__ mb) {
    const int64_t n = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (n >= rows) return;
    unsigned int m = 0;
    for (int64_t k = 0; k < cols; ++k) m = max(m, __float_as_uint(W[k * ld + n].x) & 0x7fffffffu);
    mb[n] = m;
}
constexpr int kTrRows = 64, kTrK = 64;
__global__ void __launch_bounds__(256) k_split_tr(const float2* __restrict__ W, int64_t ld, int64_t rows, int64_t cols,
                                                  int64_t kpad, const unsigned long long* __restrict__ mb,
                                                  unsigned short* __restrict__ parts, int* __restrict__ exps) {
    __shared__ unsigned int tile[4][kTrRows][kTrK / 2 + 1];   // [part][row][k pairs of u16], padded
    const int64_t n0 = blockIdx.x * (int64_t)kTrRows, k0 = blockIdx.y * (int64_t)kTrK;
    const int tx = threadIdx.x & 63, ty = threadIdx.x >> 6;   // 64 rows x 4 k-lanes
    const int64_t n = n0 + tx;
    const SrcPair src{W, 1, ld, 0};
    const int E = (n < rows && mb[n]) ? SrcPair::exp_of(mb[n]) : 0;
    if (blockIdx.y == 0 && ty == 0 && n < rows) exps[n] = E;
    // the thread's sixteen entries loaded first (sixteen reads in flight), then split
    constexpr int NV = kTrK / 4;
    float2 v[NV];
#pragma unroll
    for (int q = 0; q < NV; ++q) {
        const int kk = ty * 2 + 8 * (q >> 1) + (q & 1);
        v[q] = (n < rows && k0 + kk < cols) ? src.at(0, n, k0 + kk) : make_float2(0.f, 0.f);
    }
#pragma unroll
    for (int q = 0; q < NV; q += 2) {
        const int kk = ty * 2 + 8 * (q >> 1);
        unsigned short a[4] = {0, 0, 0, 0}, c[4] = {0, 0, 0, 0};
        if (n < rows && k0 + kk < cols) split_pair(v[q], E, a[0], a[1], a[2], a[3]);
        if (n < rows && k0 + kk + 1 < cols) split_pair(v[q + 1], E, c[0], c[1], c[2], c[3]);
#pragma unroll
        for (int p = 0; p < 4; ++p) tile[p][tx][kk >> 1] = (unsigned)a[p] | ((unsigned)c[p] << 16);
    }
    __syncthreads();
    // write: each row n of the tile is 64 u16 = 32 words per part, a warp per row and part
    const int64_t ps = rows * kpad;
    for (int e = threadIdx.x; e < 4 * kTrRows * (kTrK / 2); e += 256) {
        const int p = e / (kTrRows * (kTrK / 2)), rr = (e / (kTrK / 2)) % kTrRows, w = e % (kTrK / 2);
        const int64_t nn = n0 + rr, kk = k0 + 2 * w;
        if (nn < rows && kk < kpad)
            reinterpret_cast<unsigned int*>(parts + p * ps + nn * kpad + kk)[0] = tile[p][rr][w];
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

template <int BN, int MODE>
cudaError_t launch_dt(const DtJob& J, int grid, int* flag, cudaStream_t st) {
    using C = DtCfg<BN>;
    static std::once_flag once;
    static cudaError_t attr = cudaSuccess;
    std::call_once(once, [] {
        attr = cudaFuncSetAttribute(k_dt_gemm<BN, MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)C::SMEM);
    });
    if (attr != cudaSuccess) return attr;
    k_dt_gemm<BN, MODE><<<grid, DT_THREADS, C::SMEM, st>>>(J, flag);
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
cudaError_t dt_split(Src src, int64_t cols, const DtOp& d, cudaStream_t st) {
    const int64_t nrows = d.rows * d.batch;
    if (nrows <= 0) return cudaSuccess;
    if (cols > d.kpad) return cudaErrorInvalidValue;
    if (cols <= 1024 || nrows > 65535) {
        // a warp per row, one pass (short rows, or enough rows to fill the GPU)
        k_split_dt<Src><<<(unsigned)((nrows * 32 + 255) / 256), 256, 0, st>>>(src, d.rows, cols, d.batch, d.kpad, d.p,
                                                                               d.e);
        count_kernels(1);
        return cudaGetLastError();
    }
    if (nrows > 65535) return cudaErrorInvalidValue;
    Arena ar(st);
    unsigned long long* mb = ar.get<unsigned long long>(nrows);
    if (!mb) return cudaErrorMemoryAllocation;
    cudaError_t e = cudaMemsetAsync(mb, 0, nrows * sizeof(unsigned long long), st);
    if (e != cudaSuccess) return e;
    k_rowmax<Src><<<dim3((unsigned)((cols + 1023) / 1024), (unsigned)nrows), 256, 0, st>>>(src, d.rows, cols, mb);
    k_split_rows<Src><<<dim3((unsigned)((d.kpad / 4 + 255) / 256), (unsigned)nrows), 256, 0, st>>>(
        src, d.rows, cols, d.batch, d.kpad, mb, d.p, d.e);
    count_kernels(2);
    return cudaGetLastError();
}

// rows n < d.rows of x(n, k) = W[k * ld + n], k < cols (W: FP32 pairs), into d (one batch)
cudaError_t dt_split_tr(const float2* W, int64_t ld, int64_t cols, const DtOp& d, cudaStream_t st) {
    if (d.rows <= 0) return cudaSuccess;
    if (cols > d.kpad || d.batch != 1 || d.kpad % 32) return cudaErrorInvalidValue;
    Arena ar(st);
    unsigned long long* mb = ar.get<unsigned long long>(d.rows);
    if (!mb) return cudaErrorMemoryAllocation;
    k_rowmax_tr<<<(unsigned)((d.rows + 255) / 256), 256, 0, st>>>(W, ld, d.rows, cols, mb);
    k_split_tr<<<dim3((unsigned)((d.rows + kTrRows - 1) / kTrRows), (unsigned)((d.kpad + kTrK - 1) / kTrK)), 256, 0, st>>>(
        W, ld, d.rows, cols, d.kpad, mb, d.p, d.e);
    count_kernels(2);
    return cudaGetLastError();
}

// K ranges of a product, in k-blocks of 32: kb_lo (device, batch + 1 entries) gives
// batch z the range [kb_lo[z], kb_lo[z + 1]) (the caller guarantees at most 2048
// entries each); otherwise every batch takes [kb_begin, kb_end) (kb_end < 0: all of
// kpad), at most 4096 entries.
struct DtK {
    const int* kb_lo = nullptr;
    int kb_begin = 0, kb_end = -1;
};

// Tile widths chosen by measurement: product shape (output mode, M, N, K span in
// k-blocks or -1 for per-batch ranges, batch) -> tile_n. Filled by dt_gemm_tuned, read
// by dt_gemm when no width is asked for; shapes never tuned take the width by N.
using TuneKey = std::tuple<int, int64_t, int64_t, int64_t, int64_t>;
struct TuneTable {
    std::mutex mu;
    std::map<TuneKey, int> best;
};
TuneTable& tune_table() {
    static TuneTable* t = new TuneTable();
    return *t;
}
TuneKey tune_key(int mode, int64_t M, int64_t N, int64_t batch, const DtK& kr, int nkb) {
    const int64_t span = kr.kb_lo ? -1 : (int64_t)((kr.kb_end < 0 ? nkb : kr.kb_end) - kr.kb_begin);
    return TuneKey{mode, M, N, span, batch};
}

int dt_gemm(const DtOp& A, const DtOp& B, int64_t M, int64_t N, int64_t batch, const DtOut& out, const DtOpts& opt,
            int* flag, cudaStream_t st, std::string* err, DtK kr = DtK{}) {
    if (M <= 0 || N <= 0 || batch <= 0) return LS_OK;
    const int nkb = (int)(A.kpad / DT_BK);
    if (kr.kb_end < 0) kr.kb_end = nkb;
    if (A.kpad != B.kpad || A.kpad % DT_BK != 0 || M > A.rows || N > B.rows ||
        (A.batch != 1 && A.batch != batch) || (B.batch != 1 && B.batch != batch) ||
        (!kr.kb_lo && (kr.kb_begin < 0 || kr.kb_end > nkb || kr.kb_end - kr.kb_begin > DT_MAXK4 / DT_BK)) ||
        (out.accumulate && out.mode != DT_F64))
        return tc_err(err, "dt gemm: bad operands", LS_ERR_ARG);
    int bn = opt.tile_n;
    if (bn == 0) {
        TuneTable& tt = tune_table();
        std::lock_guard<std::mutex> g(tt.mu);
        const auto it = tt.best.find(tune_key(out.mode, M, N, batch, kr, nkb));
        if (it != tt.best.end()) bn = it->second;
    }
    if (bn == 0) bn = N <= 32 ? 32 : N <= 64 ? 64 : 128;
    if (bn != 32 && bn != 64 && bn != 128) return tc_err(err, "dt gemm: tile_n must be 32, 64 or 128", LS_ERR_ARG);
    DtJob J;
    memset(&J, 0, sizeof J);
    if (!make_map_dt(&J.a, A, DT_BM) || !make_map_dt(&J.b, B, bn))
        return tc_err(err, "dt gemm: cuTensorMapEncodeTiled failed");
    J.M = (int)M;
    J.N = (int)N;
    J.nkb = nkb;
    J.tiles_m = (int)((M + DT_BM - 1) / DT_BM);
    J.tiles_n = (int)((N + bn - 1) / bn);
    const int64_t nt = (int64_t)J.tiles_m * J.tiles_n * batch;
    if (nt > INT32_MAX) return tc_err(err, "dt gemm: too many tiles", LS_ERR_ARG);
    J.ntiles = (int)nt;
    // the smaller operand stays resident in L2 while the larger one streams once
    J.n_fast = M * A.batch > N * B.batch;
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
    J.nacc = (!kr.kb_lo && kr.kb_end - kr.kb_begin > DT_MAXK / DT_BK) ? 4 : 3;
    J.accumulate = out.accumulate;
    J.kb_lo = kr.kb_lo;
    J.kb_begin = kr.kb_begin;
    J.kb_end = kr.kb_end;
    const int grid = (int)std::min<int64_t>(nt, num_sms_now());
    cudaError_t e;
    switch ((bn << 2) | out.mode) {
        case (32 << 2) | DT_F32: e = launch_dt<32, DT_F32>(J, grid, flag, st); break;
        case (32 << 2) | DT_F64: e = launch_dt<32, DT_F64>(J, grid, flag, st); break;
        case (32 << 2) | DT_PAIR: e = launch_dt<32, DT_PAIR>(J, grid, flag, st); break;
        case (64 << 2) | DT_F32: e = launch_dt<64, DT_F32>(J, grid, flag, st); break;
        case (64 << 2) | DT_F64: e = launch_dt<64, DT_F64>(J, grid, flag, st); break;
        case (64 << 2) | DT_PAIR: e = launch_dt<64, DT_PAIR>(J, grid, flag, st); break;
        case (128 << 2) | DT_F32: e = launch_dt<128, DT_F32>(J, grid, flag, st); break;
        case (128 << 2) | DT_F64: e = launch_dt<128, DT_F64>(J, grid, flag, st); break;
        default: e = launch_dt<128, DT_PAIR>(J, grid, flag, st); break;
    }
    if (e != cudaSuccess) return tc_err(err, std::string("dt gemm launch: ") + cudaGetErrorString(e));
    return LS_OK;
}

// The product with each tile width in turn, timed by CUDA events on the stream (one run
// to warm up, then two timed; the stream is synchronised), the fastest recorded for
// its shape. Every width gives the same result bit for bit, so the product is left
// computed; the output must not accumulate. Appends "name": {times, best} to report.
int dt_gemm_tuned(const DtOp& A, const DtOp& B, int64_t M, int64_t N, int64_t batch, const DtOut& out, int* flag,
                  cudaStream_t st, std::string* err, const char* name, std::string* report) {
    if (M <= 0 || N <= 0 || batch <= 0) return LS_OK;
    if (out.accumulate) return tc_err(err, "dt tune: accumulating products cannot be rerun", LS_ERR_ARG);
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
        if (e0) cudaEventDestroy(e0);
        return tc_err(err, "dt tune: event creation failed");
    }
    const int widths[3] = {32, 64, 128};
    float ms[3] = {0.f, 0.f, 0.f};
    int rc = LS_OK;
    for (int w = 0; w < 3 && rc == LS_OK; ++w) {
        DtOpts o;
        o.tile_n = widths[w];
        rc = dt_gemm(A, B, M, N, batch, out, o, flag, st, err);
        if (rc == LS_OK && cudaEventRecord(e0, st) != cudaSuccess) rc = tc_err(err, "dt tune: event record failed");
        for (int rep = 0; rep < 2 && rc == LS_OK; ++rep) rc = dt_gemm(A, B, M, N, batch, out, o, flag, st, err);
        if (rc == LS_OK && (cudaEventRecord(e1, st) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
                            cudaEventElapsedTime(&ms[w], e0, e1) != cudaSuccess))
            rc = tc_err(err, "dt tune: timing failed");
        ms[w] *= 0.5f;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (rc != LS_OK) return rc;
    int best = 0;
    for (int w = 1; w < 3; ++w)
        if (ms[w] < ms[best]) best = w;
    {
        const int nkb = (int)(A.kpad / DT_BK);
        TuneTable& tt = tune_table();
        std::lock_guard<std::mutex> g(tt.mu);
        tt.best[tune_key(out.mode, M, N, batch, DtK{}, nkb)] = widths[best];
    }
    if (report) {
        char buf[256];
        snprintf(buf, sizeof buf, "%s\"%s\": {\"M\": %lld, \"N\": %lld, \"batch\": %lld, \"ms\": [%.4f, %.4f, %.4f], \"tile_n\": %d}",
                 report->empty() ? "" : ", ", name, (long long)M, (long long)N, (long long)batch, ms[0], ms[1], ms[2],
                 widths[best]);
        *report += buf;
    }
    return LS_OK;
}


// Scratch for a chunked product: the free device memory / div, clamped to [lo, hi]; a
// need of at most lo is granted without asking the driver.
int64_t scratch_budget(int64_t need, int div, int64_t lo, int64_t hi) {
    if (need <= lo) return lo;
    size_t fr = 0, tot = 0;
    if (cudaMemGetInfo(&fr, &tot) != cudaSuccess) fr = 0;
    return std::max(lo, std::min(hi, (int64_t)(fr / div)));
}

}  // namespace

// Host-to-device uploads through a process-wide ring of pinned host memory: the
// caller's bytes are copied into the ring at once (the caller may reuse its buffer
// on return) and the copy runs asynchronously on the stream. A pageable upload
// would make the host wait for the stream to drain first, and the GPU would idle
// while the host enqueued the next kernels. A region of the ring is reused only
// after the event recorded behind its copy has completed.
namespace {
struct PinnedRing {
    std::mutex mu;
    char* buf = nullptr;
    size_t cap = 0, head = 0;
    std::deque<std::tuple<size_t, size_t, cudaEvent_t>> inflight;   // [begin, end) in copy order
    std::vector<cudaEvent_t> spare;
};
PinnedRing& pinned_ring() {
    static PinnedRing* r = new PinnedRing();
    return *r;
}
cudaError_t ring_retire_front(PinnedRing& R) {
    cudaEvent_t e = std::get<2>(R.inflight.front());
    const cudaError_t rc = cudaEventSynchronize(e);
    R.spare.push_back(e);
    R.inflight.pop_front();
    return rc;
}
}  // namespace

namespace {
struct LaunchCache {
    std::mutex mu;
    std::map<const void*, size_t> smem;
    std::map<std::tuple<const void*, int, size_t>, int> occ;
};
LaunchCache& launch_cache() {
    static LaunchCache* c = new LaunchCache();
    return *c;
}
}  // namespace

cudaError_t grow_smem(const void* kernel, size_t bytes) {
    LaunchCache& L = launch_cache();
    std::lock_guard<std::mutex> g(L.mu);
    size_t& done = L.smem[kernel];
    if (bytes <= done) return cudaSuccess;
    const cudaError_t e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    if (e == cudaSuccess) done = bytes;
    return e;
}

cudaError_t blocks_per_sm(const void* kernel, int threads, size_t smem, int* out) {
    LaunchCache& L = launch_cache();
    std::lock_guard<std::mutex> g(L.mu);
    const auto key = std::make_tuple(kernel, threads, smem);
    const auto it = L.occ.find(key);
    if (it != L.occ.end()) {
        *out = it->second;
        return cudaSuccess;
    }
    const cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(out, kernel, threads, smem);
    if (e == cudaSuccess) L.occ[key] = *out;
    return e;
}

cudaError_t upload_h2d(void* dst, const void* src, size_t bytes, cudaStream_t st) {
    if (bytes == 0) return cudaSuccess;
    PinnedRing& R = pinned_ring();
    std::lock_guard<std::mutex> g(R.mu);
    cudaError_t e;
    const size_t need = (bytes + 255) & ~(size_t)255;
    // copies already done free their regions
    while (!R.inflight.empty() && cudaEventQuery(std::get<2>(R.inflight.front())) == cudaSuccess)
        if ((e = ring_retire_front(R)) != cudaSuccess) return e;
    if (need > R.cap) {
        while (!R.inflight.empty())
            if ((e = ring_retire_front(R)) != cudaSuccess) return e;
        const size_t old = R.cap;
        if (R.buf) cudaFreeHost(R.buf);
        R.buf = nullptr;
        R.cap = R.head = 0;
        const size_t cap = std::max<size_t>({need, (size_t)8 << 20, 2 * old});
        if ((e = cudaMallocHost(&R.buf, cap)) != cudaSuccess) return e;
        R.cap = cap;
    }
    if (R.head + need > R.cap) R.head = 0;
    // wait for the copies that still read the region about to be written (oldest first)
    while (!R.inflight.empty()) {
        bool overlap = false;
        for (auto& f : R.inflight)
            if (std::get<0>(f) < R.head + need && R.head < std::get<1>(f)) overlap = true;
        if (!overlap) break;
        if ((e = ring_retire_front(R)) != cudaSuccess) return e;
    }
    memcpy(R.buf + R.head, src, bytes);
    if ((e = cudaMemcpyAsync(dst, R.buf + R.head, bytes, cudaMemcpyHostToDevice, st)) != cudaSuccess) return e;
    cudaEvent_t ev;
    if (!R.spare.empty()) {
        ev = R.spare.back();
        R.spare.pop_back();
    } else if ((e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming)) != cudaSuccess) {
        return e;
    }
    if ((e = cudaEventRecord(ev, st)) != cudaSuccess) return e;
    R.inflight.emplace_back(R.head, R.head + need, ev);
    R.head += need;
    return cudaSuccess;
}

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
            std::string* err, std::string* tune_report) {
    const int64_t r0 = r[0], r1 = r[1], r2 = r[2];
    const int64_t k0 = pad32(r0), k1 = pad32(r1), k2 = pad32(r2);
    if (k0 > DT_MAXK4 || k1 > DT_MAXK4 || k2 > DT_MAXK4) return tc_err(err, "eval: rank above 4096", LS_ERR_ARG);
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
            dt_split(SrcF64{zt, r0, 1, 0, nullptr}, r0, c->z0t, st) != cudaSuccess ||
            launch_transpose(Z[1], r1, N, zt, st) != cudaSuccess ||
            dt_split(SrcF64{zt, r1, 1, 0, nullptr}, r1, c->z1t, st) != cudaSuccess ||
            dt_split(SrcF64{B, r2, 1, 0, nullptr}, r2, c->core, st) != cudaSuccess) {
            dt_eval_free(c);
            return tc_err(err, "eval: operand preparation failed");
        }
        *cache = c;
    }
    const DtEvalCache& c = **cache;
    // Slabs in two levels of chunks. An outer chunk takes M for its slabs in one pass
    // over the core (M as pairs, r0 r1 a slab); an inner chunk then splits its M, and
    // forms T and S. Scratch: about a quarter of the free memory, 1 to 16 GB.
    const int64_t per_m = r0 * r1 * 8 + DT_PARTS * k2 * 2 + 4;
    const int64_t per_t = DT_PARTS * r0 * k1 * 2 + r0 * 4 + N * r0 * 8 + DT_PARTS * N * k0 * 2 + N * 4;
    const int64_t budget = scratch_budget((int64_t)nslab * (per_m + per_t) * 2, 4, (int64_t)1 << 30, (int64_t)16 << 30);
    const int mchunk = (int)std::max<int64_t>(1, std::min<int64_t>(nslab, budget / 2 / per_m));
    const int tchunk = (int)std::max<int64_t>(1, std::min<int64_t>(mchunk, budget / 2 / per_t));
    Arena ar(st);
    Flag fl(ar, st);
    DtOp z2s = dt_alloc(ar, mchunk, k2, 1), ms = dt_alloc(ar, r0, k1, tchunk), ts = dt_alloc(ar, N, k0, tchunk);
    float2* Mt = ar.get<float2>((int64_t)mchunk * r0 * r1);
    float2* Tt = ar.get<float2>((int64_t)tchunk * N * r0);
    if (!fl.d || !z2s.ok() || !ms.ok() || !ts.ok() || !Mt || !Tt) return tc_err(err, "eval: out of memory", LS_ERR_OOM);
    const size_t esz = out_f32 ? 4 : 8;
    for (int s0 = 0; s0 < nslab; s0 += mchunk) {
        const int nm = std::min(mchunk, nslab - s0);
        int rc;
        {
            Scope sc("eval.mt", st);
            DtOp z2 = z2s;
            z2.rows = nm;
            // rows s of Z2^T: Z2[c][z_s], gathered
            if (dt_split(SrcF64{Z[2], 1, N, 0, zidx + s0}, r2, z2, st) != cudaSuccess)
                return tc_err(err, "eval: split failed");
            // M[s][(a, b)] = sum_c core[(a, b)][c] Z2[c][z_s]
            const DtOut mo{Mt, r0 * r1, 0, DT_PAIR};
            rc = tune_report && s0 == 0 ? dt_gemm_tuned(c.core, z2, r0 * r1, nm, 1, mo, fl.d, st, err, "M", tune_report)
                                        : dt_gemm(c.core, z2, r0 * r1, nm, 1, mo, opt, fl.d, st, err);
            if (rc != LS_OK) return rc;
        }
        for (int s1 = 0; s1 < nm; s1 += tchunk) {
            const int ns = std::min(tchunk, nm - s1);
            DtOp m = ms, t = ts;
            m.batch = ns;
            t.batch = ns;
            {
                Scope sc("eval.mt", st);
                if (dt_split(SrcPair{Mt + (int64_t)s1 * r0 * r1, r1, 1, r0 * r1}, r1, m, st) != cudaSuccess)
                    return tc_err(err, "eval: split failed");
                // T_s[y][a] = sum_b M_s[a][b] Z1^T[y][b]   (D[a][y], a on the lanes)
                const DtOut to{Tt, r0, N * r0, DT_PAIR};
                rc = tune_report && s0 == 0 && s1 == 0
                         ? dt_gemm_tuned(m, c.z1t, r0, N, ns, to, fl.d, st, err, "T", tune_report)
                         : dt_gemm(m, c.z1t, r0, N, ns, to, opt, fl.d, st, err);
                if (rc != LS_OK) return rc;
                if (dt_split(SrcPair{Tt, r0, 1, N * r0}, r0, t, st) != cudaSuccess)
                    return tc_err(err, "eval: split failed");
            }
            {
                Scope sc("eval.slab", st);
                // S_s[x][y] = sum_a T_s[y][a] Z0^T[x][a]   (D[y][x], y on the lanes: rows of S contiguous)
                void* o = static_cast<char*>(out) + (size_t)(s0 + s1) * N * N * esz;
                const DtOut so{o, N, N * N, out_f32 ? DT_F32 : DT_F64};
                rc = tune_report && s0 == 0 && s1 == 0
                         ? dt_gemm_tuned(t, c.z0t, N, N, ns, so, fl.d, st, err, "S", tune_report)
                         : dt_gemm(t, c.z0t, N, N, ns, so, opt, fl.d, st, err);
                if (rc != LS_OK) return rc;
            }
        }
    }
    return fl.check(err);
}

int dt_gemm_nt(const double* A, const double* B, int64_t M, int64_t N, int64_t K, void* D, int out_f32,
               const DtOpts& opt, cudaStream_t st, std::string* err) {
    if (M <= 0 || N <= 0) return LS_OK;
    const int64_t kp = pad32(std::max<int64_t>(K, 1));
    if (kp > DT_MAXK4 && out_f32) return tc_err(err, "gemm_nt_mixed: K above 4096 needs FP64 output", LS_ERR_ARG);
    Arena ar(st);
    Flag fl(ar, st);
    DtOp a = dt_alloc(ar, M, kp, 1), b = dt_alloc(ar, N, kp, 1);
    if (!fl.d || !a.ok() || !b.ok()) return tc_err(err, "gemm_nt_mixed: out of memory", LS_ERR_OOM);
    if (dt_split(SrcF64{A, K, 1, 0, nullptr}, K, a, st) != cudaSuccess ||
        dt_split(SrcF64{B, K, 1, 0, nullptr}, K, b, st) != cudaSuccess)
        return tc_err(err, "gemm_nt_mixed: split failed");
    // D[m][n] row-major = the kernel's D with n on the lanes: swap the operands; K in
    // chunks of 4096 (each exact in its leading levels), added in FP64
    const int nkb = (int)(kp / DT_BK), ckb = DT_MAXK4 / DT_BK;
    for (int k0 = 0; k0 < nkb; k0 += ckb) {
        DtOut o{D, N, 0, out_f32 ? DT_F32 : DT_F64};
        o.accumulate = k0 > 0;
        DtK kr;
        kr.kb_begin = k0;
        kr.kb_end = std::min(nkb, k0 + ckb);
        int rc = dt_gemm(b, a, N, M, 1, o, opt, fl.d, st, err, kr);
        if (rc != LS_OK) return rc;
    }
    return fl.check(err);
}

int dt_core(const double* P0, const double* P1, const double* P2, const int32_t* C, const int32_t* r,
            const int32_t* tcol, const double* xin, const int32_t* perm, const int32_t* off, int64_t T, double* Bc,
            int* flag, cudaStream_t st, std::string* err) {
    const int64_t C0 = C[0], r0 = r[0], r1 = r[1], r2 = r[2], nn = r1 * r2;
    if (C0 <= 0 || T <= 0) return LS_OK;
    // groups of terms by mode-0 column, each padded to whole k-blocks
    std::vector<int> kb_lo(C0 + 1, 0);
    for (int64_t g = 0; g < C0; ++g) {
        const int n = off[g + 1] - off[g];
        if (n > DT_MAXK) return tc_err(err, "core: more than 2048 terms share one mode-0 column", LS_ERR_ARG);
        kb_lo[g + 1] = kb_lo[g] + (n + DT_BK - 1) / DT_BK;
    }
    const int64_t tpad = (int64_t)kb_lo[C0] * DT_BK;
    // one upload: the group k-block offsets, then the padded term list
    std::vector<int32_t> up((C0 + 1) + tpad, -1);
    std::copy(kb_lo.begin(), kb_lo.end(), up.begin());
    int32_t* tmap = up.data() + (C0 + 1);
    for (int64_t g = 0; g < C0; ++g)
        for (int u = 0; u < off[g + 1] - off[g]; ++u) tmap[(int64_t)kb_lo[g] * DT_BK + u] = perm[off[g] + u];
    Arena ar(st);
    int* d_kb = ar.get<int>((C0 + 1) + tpad);
    int32_t* d_tmap = d_kb + (C0 + 1);
    int32_t* d_idx1 = ar.get<int32_t>(2 * tpad);
    int32_t* d_idx2 = d_idx1 ? d_idx1 + tpad : nullptr;
    double* d_w1 = ar.get<double>(tpad);
    // Output columns (j, k) in ranges of jc values of j, groups in chunks of gc (each
    // one exact K range of step 2, up to 4096): W (pairs) and its split form take
    // 16 bytes a (group, j, k), within about a third of the free memory (1 to 32 GB).
    const int64_t budget = scratch_budget(16 * std::min<int64_t>(C0, DT_MAXK4) * nn, 3, (int64_t)1 << 30, (int64_t)32 << 30);
    int64_t gc = std::min<int64_t>(C0, DT_MAXK4);
    if (16 * gc * r2 > budget) gc = std::max<int64_t>(DT_BK, budget / (16 * r2) / DT_BK * DT_BK);
    const int64_t jc = std::max<int64_t>(1, std::min<int64_t>(r1, budget / (16 * gc * r2)));
    DtOp a = dt_alloc(ar, r2, tpad, 1), b = dt_alloc(ar, jc, tpad, 1);
    float2* W = ar.get<float2>(gc * jc * r2);
    DtOp ws = dt_alloc(ar, jc * r2, pad32(gc), 1), p0s = dt_alloc(ar, r0, pad32(gc), 1);
    if (!d_kb || !d_idx1 || !d_w1 || !a.ok() || !b.ok() || !W || !ws.ok() || !p0s.ok())
        return tc_err(err, "core: out of memory", LS_ERR_OOM);
    {
        Scope sc("core.operands", st);
        if (upload_h2d(d_kb, up.data(), up.size() * sizeof(int32_t), st) != cudaSuccess)
            return tc_err(err, "core: upload failed");
        count_h2d((int64_t)(up.size() * sizeof(int32_t)));
        // the column maps and weights over the padded term list, once
        k_term_index<<<(unsigned)((tpad + 255) / 256), 256, 0, st>>>(d_tmap, tcol, xin, tpad, d_idx1, d_idx2, d_w1);
        count_kernels(1);
        // step 1's A operand over the padded term list: A[k][t] = P2[k][c2(t)]
        if (dt_split(SrcIdx{P2, (int64_t)C[2], d_idx2, nullptr}, tpad, a, st) != cudaSuccess)
            return tc_err(err, "core: split failed");
    }
    const DtOpts opt;
    for (int64_t j0 = 0; j0 < r1; j0 += jc) {
        const int64_t nj = std::min(jc, r1 - j0);
        DtOp bj = b;
        bj.rows = nj;
        {
            Scope sc("core.operands", st);
            // step 1's B operand: B[j][t] = xin[t] P1[j][c1(t)], rows j0 .. j0 + nj
            if (dt_split(SrcIdx{P1 + j0 * C[1], (int64_t)C[1], d_idx1, d_w1}, tpad, bj, st) != cudaSuccess)
                return tc_err(err, "core: split failed");
        }
        for (int64_t g0 = 0; g0 < C0; g0 += gc) {
            const int64_t ng = std::min(gc, C0 - g0);
            int rc;
            {
                Scope sc("core.step1", st);
                // step 1: W[g][j][k] = sum_{t in group g} xin[t] P1[j][c1(t)] P2[k][c2(t)]  (k on the lanes)
                DtK k1;
                k1.kb_lo = d_kb + g0;
                rc = dt_gemm(a, bj, r2, nj, ng, DtOut{W, r2, nj * r2, DT_PAIR}, opt, flag, st, err, k1);
                if (rc != LS_OK) return rc;
            }
            DtOp w = ws, p = p0s;
            w.rows = nj * r2;
            {
                Scope sc("core.wsplit", st);
                if (dt_split_tr(W, nj * r2, ng, w, st) != cudaSuccess ||
                    dt_split(SrcF64{P0 + g0, C0, 1, 0, nullptr}, ng, p, st) != cudaSuccess)
                    return tc_err(err, "core: split failed");
            }
            {
                Scope sc("core.step2", st);
                // step 2: B[i][(j, k)] (+)= sum_g W[g][(j, k)] P0[i][g]  ((j, k) on the lanes)
                DtOut o{Bc + j0 * r2, nn, 0, DT_F64};
                o.accumulate = g0 > 0;
                DtK k2;
                k2.kb_end = (int)(pad32(ng) / DT_BK);
                rc = dt_gemm(w, p, nj * r2, r0, 1, o, opt, flag, st, err, k2);
                if (rc != LS_OK) return rc;
            }
        }
    }
    return LS_OK;
}

}  // namespace ls
