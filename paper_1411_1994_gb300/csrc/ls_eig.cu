// Symmetric eigen-solver of the truncation step (Thm 2.1 / Algorithm 1 take
// the SVD of each side matrix; here the eigen-decomposition of its k x k
// Gram matrix H = L^T L after the pivoted Cholesky compression): cyclic
// two-sided block Jacobi.
//
// Representation: the diagonal D of the rotated matrix as an unevaluated
// hi + lo FP32 pair, the off-diagonal part E in FP32 (full symmetric
// storage), and the accumulated rotation as I + F with F in FP32. Every
// stored entry carries its own relative rounding, so the iteration keeps the
// relative accuracy that Jacobi has on graded positive definite matrices.
// Run a second time on the nearly diagonal U^T H U (U from the first run,
// orthonormalised and re-projected in FP64-grade arithmetic), the angles are
// small, E and F are small, and the FP32 rounding of E and F is small in
// absolute terms: the second run reaches off-diagonal ratios of 1e-10 without
// any FP64 sweep.
//
// Two forms of the same rounds: one thread-block cluster per matrix with the
// matrix in shared memory (k_jacobi_blk), and one cooperative grid for
// every matrix of a launch with the matrices in global memory (k_jacobi_gblk,
// any k). The file also holds the FP32 Cholesky + inverse of CholeskyQR's
// first pass (k_chol32_multi).
#include <cooperative_groups.h>

#include <algorithm>

#include "ls_common.cuh"
#include "ls_grid.cuh"

namespace cg = cooperative_groups;

namespace ls {

namespace {

constexpr int kEigThreads = 1024;

struct DfMode {
    const double* H; double* outD; double* outF; DevStatus* st;
    int64_t ldd; int k; int add_identity; double abs_floor; double tau; double tol;
};

// v mod n for 0 <= v < 2 n (one compare: the round-robin indices below stay in that range, and
// a division by a runtime n is a long dependent chain on the critical path of a round)
__device__ __forceinline__ int mod_lt2n(int v, int n) { return v >= n ? v - n : v; }

// pair-block i (0 <= i < Cp / 2) of round t (0 <= t < Cp - 1) of the round-robin over Cp blocks
__device__ __forceinline__ void rr_pair_e(int t, int i, int Cp, int& p, int& q) {
    const int n1 = Cp - 1;
    int a, b;
    if (i == 0) { a = n1; b = t; }
    else { a = mod_lt2n(t + i, n1); b = mod_lt2n(t - i + n1, n1); }
    p = min(a, b);
    q = max(a, b);
}

// The diagonal is kept as an unevaluated sum hi + lo of two FP32 numbers
// (about 48 significant bits) and updated with error-free FP32 additions
// (Knuth's TwoSum, then a renormalising Fast2Sum): no FP64 instruction in
// the iteration itself, whose few FP64 lanes per SM would serialise it.
struct DF {
    float hi, lo;
};
__device__ __forceinline__ DF df_from(double d) {
    const float h = (float)d;
    return DF{h, (float)(d - (double)h)};
}
__device__ __forceinline__ double df_to(DF x) { return (double)x.hi + (double)x.lo; }
__device__ __forceinline__ DF df_add(DF x, float y) {
    const float s = __fadd_rn(x.hi, y);
    const float bb = __fsub_rn(s, x.hi);
    const float e = __fadd_rn(__fsub_rn(x.hi, __fsub_rn(s, bb)), __fsub_rn(y, bb));
    const float lo = __fadd_rn(x.lo, e);
    const float h2 = __fadd_rn(s, lo);
    return DF{h2, __fsub_rn(lo, __fsub_rn(h2, s))};
}
// a - b rounded to FP32
__device__ __forceinline__ float df_diff(DF a, DF b) { return __fadd_rn(__fsub_rn(a.hi, b.hi), __fsub_rn(a.lo, b.lo)); }

// The rotation of a pair from (d_p, d_q, e_pq): the tangent t only steers
// (an inexact t leaves a residue of that relative size in e_pq, as FP32
// rounding does), so it is taken with the hardware approximations; c is then
// made consistent with t, c = (1 + t^2)^(-1/2) with one Newton step on the
// approximate rsqrt, and s = t c, so that c^2 + s^2 = 1 to an ulp or two.
// c - 1 = -t^2 c / (1 + 1/c) is kept apart for the accumulated rotations.
__device__ __forceinline__ float rcp_a(float x) {
    float y;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
__device__ __forceinline__ float sqrt_a(float x) {
    float y;
    asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
__device__ __forceinline__ float rsqrt_a(float x) {
    float y;
    asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
struct RotCS {
    float t, c, s, cm1;
};
__device__ __forceinline__ RotCS jacobi_rot(float dq_minus_dp, float epq) {
    const float theta = dq_minus_dp * rcp_a(2.f * epq);
    const float t = copysignf(rcp_a(fabsf(theta) + sqrt_a(fmaf(theta, theta, 1.f))), theta);
    const float x = fmaf(t, t, 1.f);
    float c = rsqrt_a(x);
    c = c * fmaf(-0.5f * x, c * c, 1.5f);
    return RotCS{t, c, t * c, -(t * t) * c * rcp_a(fmaf(x, c, 1.f))};
}

// rotation criterion (a decision only, so taken in FP32; the sweep-start scan
// and the angle phase use this one function and therefore agree)
struct Crit {
    float floor, tau, tol2;
    __device__ __forceinline__ bool operator()(DF app, DF aqq, float apq) const {
        const float a = app.hi, b = aqq.hi;
        return fabsf(apq) > floor && fmaxf(a, b) >= tau && apq * apq > tol2 * fabsf(a * b);
    }
};

// the device's SM count (queried once)
int sm_count() {
    static const int n = [] {
        int dev = 0, v = 0;
        if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
            return 1;
        return std::max(1, v);
    }();
    return n;
}
// dynamic shared memory available to the kernel (its static variables take a few bytes)
int smem_optin() {
    int dev = 0, v = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return 0;
    if (cudaDeviceGetAttribute(&v, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess) return 0;
    return std::max(0, v - 1024);
}

// ---------------------------------------------------------------------------
// Block form of the same iteration: indices in blocks of BJ = 8, a round-robin
// over the m blocks pairs them into m/2 pair-blocks of 16 indices per round
// (m - 1 rounds a sweep). Each pair-block's 16 x 16 subproblem receives one
// inner cyclic sweep (a warp, in registers; the diagonal as hi/lo pairs), whose
// rotations accumulate into Q = I + F_Q; then every off-diagonal tile of
// pair-blocks is rotated as E_AB <- Q_A^T E_AB Q_B (a warp per tile, dense
// FP32), and F <- F + F_Q + F F_Q on the F rows. In the first round of a
// sweep the inner sweeps rotate every index pair of each pair-block (so every
// pair within a block); in the other rounds only the pairs across the two
// blocks (8 inner rounds). A sweep thus rotates every pair at least once, and
// a round is dense arithmetic instead of one synchronisation per rotation.
// E is held in full (symmetric) storage; K = m * BJ <= jacobi_blk_max_k().
// ---------------------------------------------------------------------------
constexpr int BJ = 8, BJ2 = 16, BJ2SQ = 256;
// threads of the block kernel: 128 registers a thread, so the tile products stay in registers
constexpr int kBlkThreads = 512;
// padded strides: E rows K + 4 (16-byte aligned rows, column walks over 8 banks), 16 x 16
// scratch rows 17 (row-wise walks conflict-free)
constexpr int SP = BJ2 + 1, SPSQ = BJ2 * SP;
// rows of F a half-warp updates at a time
constexpr int kFR = 4;

struct BjArgs {
    const DfMode* m; int max_sweeps; int cs; int rows_per;
};

// block (of size BJ) of position u (0..15) in pair-block (I, J)
__device__ __forceinline__ int bj_index(int I, int J, int u) { return u < BJ ? I * BJ + u : J * BJ + (u - BJ); }

// shared-memory layout: offsets in bytes
struct BjLayout {
    int K, ldE, nb;
    size_t ctl, D, E, Q, pb, act, tiles, ndep, lists, qrem, F;   // CTA 0: ctl .. lists; others: ctl qrem F
    size_t e_bytes, f_bytes;
    __host__ __device__ BjLayout(int k, int rows_per) {
        int m = (k + BJ - 1) / BJ;
        m += m & 1;
        K = m * BJ;
        ldE = K + 4;
        nb = m / 2;
        ctl = 0;
        D = 16;
        E = D + 8 * (size_t)K;
        Q = E + 4 * (size_t)K * ldE;
        pb = Q + 4 * (size_t)2 * nb * BJ2SQ;                 // Q, pb, act and F_Q: two rounds' worth
        act = pb + 4 * (size_t)2 * nb;
        tiles = act + 4 * (size_t)2 * nb;
        ndep = tiles + 4 * (size_t)nb * nb;
        lists = ndep + 4 * (size_t)m;
        e_bytes = lists + (((size_t)m * nb * (nb - 1) / 2 + 15) & ~(size_t)15);
        qrem = 16;
        F = qrem + 4 * (size_t)2 * nb * SPSQ;
        f_bytes = F + 4 * (size_t)rows_per * K;
    }
};

// ---------------------------------------------------------------------------
// The inner sweep of one pair-block by one warp, in registers (both forms run it).
// Lanes 0..15 hold the columns of the 16 x 16 subproblem E_s (zero diagonal) and the
// diagonal entry d of position i = lane; lanes 16..31 hold the columns of F_Q
// (Q = I + F_Q, zero at the start), position i = lane - 16. Inner round `it`
// rotates 8 disjoint position pairs (u, v), u < v: in the full form (the first round
// of a sweep) the round-robin pairs of all 16 positions, otherwise u = l and
// v = 8 + ((l + it) mod 8). Lane u takes the rotation from (d_u, d_v, e_uv) when
// both indices are below k and the pair qualifies; then E_s <- J^T E_s J (rows in
// each lane, then columns with the partner lane's column), F_Q <- F_Q J + (J - I)
// with c - 1 taken directly, d_u -= t e_uv, d_v += t e_uv, and the pair's 2 x 2 block
// of E_s is set to zero. Returns the rotations taken by this lane.
//
// The rows of a column sit in registers in an order that turns with the inner
// rounds, so that every round pairs the same registers: (l, 8 + l) in the cross
// form, where register 8 + j holds row 8 + ((j + it) mod 8); (15, 0) and
// (l, 15 - l) in the full form, where register s < 15 holds row (s + it) mod 15.
// The round loop then needs no unrolling and the code stays small.
// ---------------------------------------------------------------------------
// (indices mod 15 by conditional steps: the arguments stay within one period of 0..14)
__device__ __forceinline__ int mod15(int v) {
    v = v < 0 ? v + (BJ2 - 1) : v;
    return v >= BJ2 - 1 ? v - (BJ2 - 1) : v;
}
template <bool FULL>
__device__ __forceinline__ int in_partner(int it, int i) {
    if (FULL) return i == BJ2 - 1 ? it : (i == it ? BJ2 - 1 : mod15(2 * it - i));
    return i < BJ ? BJ + ((i + it) & (BJ - 1)) : ((i - BJ - it) & (BJ - 1));
}
// register of row `row` in inner round it
template <bool FULL>
__device__ __forceinline__ int in_reg(int it, int row) {
    if (FULL) return row == BJ2 - 1 ? row : mod15(row - it);
    return row < BJ ? row : BJ + ((row - BJ - it) & (BJ - 1));
}
// row held by register r in inner round it
template <bool FULL>
__device__ __forceinline__ int in_row(int it, int r) {
    if (FULL) return r == BJ2 - 1 ? r : mod15(r + it);
    return r < BJ ? r : BJ + ((r - BJ + it) & (BJ - 1));
}
// v[p] for a runtime p, by a tree of selects on the bits of p
__device__ __forceinline__ float pick16(const float (&v)[BJ2], int p) {
    float a[8], b[4];
#pragma unroll
    for (int i = 0; i < 8; ++i) a[i] = (p & 1) ? v[2 * i + 1] : v[2 * i];
#pragma unroll
    for (int i = 0; i < 4; ++i) b[i] = (p & 2) ? a[2 * i + 1] : a[2 * i];
    const float c0 = (p & 4) ? b[1] : b[0], c1 = (p & 4) ? b[3] : b[2];
    return (p & 8) ? c1 : c0;
}

template <bool FULL>
__device__ __forceinline__ unsigned int inner_sweep(float (&x)[BJ2], DF& d, int I, int Jb, int k, const Crit& qualifies) {
    const int lane = threadIdx.x & 31, pos = lane & (BJ2 - 1);
    const bool is_e = lane < BJ2;
    const bool in_k = bj_index(I, Jb, pos) < k;
    constexpr int NIT = FULL ? BJ2 - 1 : BJ;
    unsigned int nrot = 0;
#pragma unroll 1
    for (int it = 0; it < NIT; ++it) {
        const int pt = in_partner<FULL>(it, pos);
        const bool owner = pos < pt;
        const int rpos = in_reg<FULL>(it, pos), rpt = in_reg<FULL>(it, pt);
        // the pair's rotation, taken by its lane u
        const float dph = __shfl_sync(0xffffffffu, d.hi, pt), dpl = __shfl_sync(0xffffffffu, d.lo, pt);
        const int pk = __shfl_sync(0xffffffffu, (int)in_k, pt);
        const float epq = pick16(x, rpt);
        float c = 1.f, sn = 0.f, cm1 = 0.f, te = 0.f;
        int act = 0;
        if (is_e && owner && in_k && pk) {
            const DF dq{dph, dpl};
            if (qualifies(d, dq, epq)) {
                const RotCS g = jacobi_rot(df_diff(dq, d), epq);
                c = g.c;
                sn = g.s;
                cm1 = g.cm1;
                te = g.t * epq;
                act = 1;
                ++nrot;
            }
        }
        // rows of E_s: the fixed register pairs, each with its pair's rotation from lane u
        if (is_e) {
#pragma unroll
            for (int l = 0; l < BJ; ++l) {
                const int p = FULL ? (l == 0 ? BJ2 - 1 : l) : l;
                const int q = FULL ? (l == 0 ? 0 : BJ2 - 1 - l) : BJ + l;
                const int rowp = in_row<FULL>(it, p), rowq = in_row<FULL>(it, q);
                const int u = rowp < rowq ? rowp : rowq;
                const float cl = __shfl_sync(0x0000ffffu, c, u);
                const float s0 = __shfl_sync(0x0000ffffu, sn, u);
                const float sl = rowp < rowq ? s0 : -s0;
                const float xp = x[p], xq = x[q];
                x[p] = cl * xp - sl * xq;
                x[q] = sl * xp + cl * xq;
            }
        }
        // columns: this lane's pair rotation and the partner lane's column
        const int own = owner ? pos : pt;
        c = __shfl_sync(0xffffffffu, c, own);
        sn = __shfl_sync(0xffffffffu, sn, own);
        cm1 = __shfl_sync(0xffffffffu, cm1, own);
        te = __shfl_sync(0xffffffffu, te, own);
        act = __shfl_sync(0xffffffffu, act, own);
        float o[BJ2];
        const int plane = (lane & BJ2) | pt;
#pragma unroll
        for (int r = 0; r < BJ2; ++r) o[r] = __shfl_sync(0xffffffffu, x[r], plane);
        // both halves: u's column c x_u - s x_v, v's column s x_u + c x_v; then E_s's pair
        // block is zeroed and F_Q takes J - I (c - 1 on the diagonal, -s and s off it)
#pragma unroll
        for (int r = 0; r < BJ2; ++r) x[r] = owner ? c * x[r] - sn * o[r] : sn * o[r] + c * x[r];
        if (act) {
            const float add_pos = is_e ? 0.f : cm1, add_pt = is_e ? 0.f : (owner ? -sn : sn);
#pragma unroll
            for (int r = 0; r < BJ2; ++r) {
                if (r == rpos) x[r] = is_e ? 0.f : x[r] + add_pos;
                if (r == rpt) x[r] = is_e ? 0.f : x[r] + add_pt;
            }
            if (is_e) d = df_add(d, owner ? -te : te);
        }
        // turn the register order to the next round's
        if (FULL) {
            const float x0 = x[0];
#pragma unroll
            for (int r = 0; r < BJ2 - 2; ++r) x[r] = x[r + 1];
            x[BJ2 - 2] = x0;
        } else {
            const float x8 = x[BJ];
#pragma unroll
            for (int r = BJ; r < BJ2 - 1; ++r) x[r] = x[r + 1];
            x[BJ2 - 1] = x8;
        }
    }
    return nrot;
}

// Round pipeline of the cluster form. CTA 0 holds D, E, Q and the tables; CTAs 1..cs-1
// hold rows of F and run the inner sweeps. A round t splits CTA 0's tiles in two: the
// "dependency" tiles, each holding an 8 x 8 block that round t + 1 pairs (one per pair-block
// of round t + 1), and the rest. After the dependency tiles a cluster barrier lets CTAs 1..
// run round t + 1's inner sweeps (and F's update of round t) while CTA 0 finishes the other
// tiles of round t: those touch no block that round t + 1's inner sweeps read or write. Q,
// the pair-block table, the rotation flags and F_Q are kept for two rounds (by parity). The
// last round of a sweep is not overlapped: CTA 0 then scans for a qualifying pair.
__global__ void __launch_bounds__(kBlkThreads) k_jacobi_blk(BjArgs A) {
    cg::cluster_group cl = cg::this_cluster();
    const int rank = (int)cl.block_rank(), cs = A.cs;
    const int job = blockIdx.x / cs;
    const DfMode J = A.m[job];
    const int k = J.k;
    const BjLayout Ly(k, A.rows_per);
    const int K = Ly.K, ldE = Ly.ldE, nb = Ly.nb, m = 2 * nb;
    extern __shared__ __align__(16) unsigned char smem[];
    unsigned char* s0 = rank == 0 ? smem : cl.map_shared_rank(smem, 0);
    int* ctl = reinterpret_cast<int*>(smem + Ly.ctl);       // this CTA's copy of the stop decision
    DF* D = reinterpret_cast<DF*>(s0 + Ly.D);
    float* E = reinterpret_cast<float*>(s0 + Ly.E);
    float* Qr = reinterpret_cast<float*>(s0 + Ly.Q);         // [2][nb][16][16], Q = I + F_Q
    int* pbr = reinterpret_cast<int*>(s0 + Ly.pb);           // [2][nb]: I | J << 16
    int* actr = reinterpret_cast<int*>(s0 + Ly.act);         // [2][nb]: pair-block rotated
    float* El = reinterpret_cast<float*>(smem + Ly.E);       // CTA 0's own views
    const float* Ql = reinterpret_cast<const float*>(smem + Ly.Q);
    const int* pbl = reinterpret_cast<const int*>(smem + Ly.pb);
    const int* actl = reinterpret_cast<const int*>(smem + Ly.act);
    int* tiles = reinterpret_cast<int*>(smem + Ly.tiles);    // tiles a | b << 8, a < b
    int* ndep = reinterpret_cast<int*>(smem + Ly.ndep);      // per round: its dependency tiles
    unsigned char* lists = smem + Ly.lists;                   // per round: dependency tiles, then the rest
    float* qrem = reinterpret_cast<float*>(smem + Ly.qrem);  // CTAs >= 1: [2][nb] F_Q of own pair-blocks
    float* F = reinterpret_cast<float*>(smem + Ly.F);        // CTAs >= 1: rows j0 .. j1 of F
    __shared__ unsigned int s_active;                         // CTA 0: rotations of this sweep
    unsigned int* active = rank == 0 ? &s_active : cl.map_shared_rank(&s_active, 0);
    const int tid = threadIdx.x, nthr = blockDim.x;
    const int warp = tid >> 5, lane = tid & 31, nw = nthr >> 5;
    const Crit qualifies{(float)J.abs_floor, (float)J.tau, (float)(J.tol * J.tol)};
    const int j0 = rank >= 1 ? min(K, (rank - 1) * A.rows_per) : 0;
    const int j1 = rank >= 1 ? min(K, j0 + A.rows_per) : 0;
    const int ntile = nb * (nb - 1) / 2;
    const int nF = cs - 1;                                    // CTAs of F rows and inner sweeps
    const int iw = (nb + nF - 1) / nF;                        // their warps 0 .. iw-1: inner sweeps

    int base = 0;
    if (rank == 0) {
        for (int a = tid; a < K; a += nthr) D[a] = df_from(a < k ? J.H[(int64_t)a * k + a] : 0.0);
        for (int a = warp; a < K; a += nw)
            for (int c = lane; c < K; c += 32)
                E[a * ldE + c] = (a < k && c < k && a != c) ? (float)J.H[(int64_t)a * k + c] : 0.f;
        if (tid == 0) {
            s_active = 0;
            int n = 0;
            for (int a = 0; a < nb; ++a)
                for (int b = a + 1; b < nb; ++b) tiles[n++] = a | (b << 8);
        }
        __syncthreads();
        // the tile order of each round t: first the tiles holding a block that round t + 1
        // pairs (ndep[t] of them), then the others; in the last round of a sweep all tiles in
        // order (ndep = 0). Round t pairs block X with (2 t - X) mod (m - 1), and m - 1 with t.
        for (int t = warp; t < m - 1; t += nw) {
            const bool next = t + 1 < m - 1;
            const int n1 = m - 1, tt = t + 1;
            auto partner = [&](int X) { return X == n1 ? tt : X == tt ? n1 : ((2 * tt - X) % n1 + n1) % n1; };
            auto is_dep = [&](int i) {
                const int ab = tiles[i];
                int Ia, Ja, Ib, Jbb;
                rr_pair_e(t, ab & 255, m, Ia, Ja);
                rr_pair_e(t, ab >> 8, m, Ib, Jbb);
                const int pI = partner(Ia), pJ = partner(Ja);
                return pI == Ib || pI == Jbb || pJ == Ib || pJ == Jbb;
            };
            unsigned char* lt = lists + t * ntile;
            int nd = 0;
            for (int c0 = 0; c0 < ntile; c0 += 32) {
                const int i = c0 + lane;
                const bool dep = next && i < ntile && is_dep(i);
                const unsigned bal = __ballot_sync(0xffffffffu, dep);
                if (dep) lt[nd + __popc(bal & ((1u << lane) - 1))] = (unsigned char)i;
                nd += __popc(bal);
            }
            int nr = nd;
            for (int c0 = 0; c0 < ntile; c0 += 32) {
                const int i = c0 + lane;
                const bool rest = i < ntile && !(next && is_dep(i));
                const unsigned bal = __ballot_sync(0xffffffffu, rest);
                if (rest) lt[nr + __popc(bal & ((1u << lane) - 1))] = (unsigned char)i;
                nr += __popc(bal);
            }
            if (lane == 0) ndep[t] = nd;
        }
        base = J.st->sweeps;
    } else {
        for (int e = tid; e < (j1 - j0) * K; e += nthr) F[e] = 0.f;
    }
    cl.sync();

    // inner sweep of pair-block sub in round t (CTAs >= 1, warps 0 .. iw-1)
    auto inner = [&](int t, int sub) {
        const int par = t & 1;
        int I, Jb;
        rr_pair_e(t, sub, m, I, Jb);
        const int pos = lane & (BJ2 - 1), gi = bj_index(I, Jb, pos);
        float x[BJ2];
        DF d{0.f, 0.f};
        if (lane < BJ2) {
#pragma unroll
            for (int r = 0; r < BJ2; ++r) x[r] = E[bj_index(I, Jb, r) * ldE + gi];
            d = D[gi];
        } else {
#pragma unroll
            for (int r = 0; r < BJ2; ++r) x[r] = 0.f;
        }
        unsigned int nrot = t == 0 ? inner_sweep<true>(x, d, I, Jb, k, qualifies)
                                   : inner_sweep<false>(x, d, I, Jb, k, qualifies);
        for (int o = 16; o; o >>= 1) nrot += __shfl_xor_sync(0xffffffffu, nrot, o);
        if (lane < BJ2) {
#pragma unroll
            for (int r = 0; r < BJ2; ++r) E[bj_index(I, Jb, r) * ldE + gi] = x[r];
            D[gi] = d;
        } else {
            // F_Q here (the F updates of the other CTAs read it through the cluster window),
            // Q = I + F_Q to CTA 0
            float* qr = qrem + (size_t)par * nb * SPSQ + sub * SPSQ + pos;
#pragma unroll
            for (int r = 0; r < BJ2; ++r) qr[r * SP] = x[r];
            float* Qs = Qr + (size_t)par * nb * BJ2SQ + sub * BJ2SQ;
#pragma unroll
            for (int r = 0; r < BJ2; ++r) Qs[r * BJ2 + pos] = x[r] + (r == pos ? 1.f : 0.f);
        }
        if (lane == 0) {
            pbr[par * nb + sub] = I | (Jb << 16);
            actr[par * nb + sub] = nrot > 0;
            if (nrot) atomicAdd(active, nrot);
        }
    };
    // the inner sweeps of round t on CTAs >= 1
    auto inner_round = [&](int t) {
        if (rank >= 1 && warp < iw)
            for (int sub = (rank - 1) + nF * warp; sub < nb; sub += nF * iw) inner(t, sub);
    };

    // the same tile rotation with a whole warp per tile (lanes 16..31 take the tile's rows 8..15),
    // for the few tiles that the next round waits for: half the latency, the same arithmetic
    auto tile_wide = [&](int t, int l0, int l1) {
        const int par = t & 1;
        const float* Q = Ql + (size_t)par * nb * BJ2SQ;
        const int* pb = pbl + par * nb;
        const int* act = actl + par * nb;
        float* E = El;
        const int l16 = lane & 15;
        const int rr = (l16 >> 1) + BJ * (lane >> 4), c0 = (l16 & 1) * BJ;
        for (int task = l0 + warp; task < l1; task += nw) {
            const int ab = tiles[lists[t * ntile + task]];
            const int a = ab & 255, b = ab >> 8;
            if (!act[a] && !act[b]) continue;
            const int pa = pb[a], pbb = pb[b];
            const int Ia = pa & 0xffff, Ja = pa >> 16, Ib = pbb & 0xffff, Jb2 = pbb >> 16;
            const float* Qa = Q + a * BJ2SQ;
            const float* Qb = Q + b * BJ2SQ;
            const int colb = c0 ? Jb2 * BJ : Ib * BJ;
            float t0[BJ];
#pragma unroll
            for (int c = 0; c < BJ; ++c) t0[c] = 0.f;
#pragma unroll
            for (int j = 0; j < BJ2; ++j) {
                const float qa = Qa[j * BJ2 + rr];
                const float* xr = E + bj_index(Ia, Ja, j) * ldE + colb;
                const float4 x0 = *reinterpret_cast<const float4*>(xr);
                const float4 x1 = *reinterpret_cast<const float4*>(xr + 4);
                const float xv[BJ] = {x0.x, x0.y, x0.z, x0.w, x1.x, x1.y, x1.z, x1.w};
#pragma unroll
                for (int c = 0; c < BJ; ++c) t0[c] = fmaf(qa, xv[c], t0[c]);
            }
            const int cp = c0 ^ BJ;
            float z[BJ];
#pragma unroll
            for (int c = 0; c < BJ; ++c) z[c] = 0.f;
#pragma unroll
            for (int jj = 0; jj < BJ; ++jj) {
                const float tv = t0[jj];
                const float ov = __shfl_xor_sync(0xffffffffu, tv, 1);
                const float4 qs0 = *reinterpret_cast<const float4*>(Qb + (c0 + jj) * BJ2 + c0);
                const float4 qs1 = *reinterpret_cast<const float4*>(Qb + (c0 + jj) * BJ2 + c0 + 4);
                const float4 qo0 = *reinterpret_cast<const float4*>(Qb + (cp + jj) * BJ2 + c0);
                const float4 qo1 = *reinterpret_cast<const float4*>(Qb + (cp + jj) * BJ2 + c0 + 4);
                z[0] = fmaf(tv, qs0.x, fmaf(ov, qo0.x, z[0]));
                z[1] = fmaf(tv, qs0.y, fmaf(ov, qo0.y, z[1]));
                z[2] = fmaf(tv, qs0.z, fmaf(ov, qo0.z, z[2]));
                z[3] = fmaf(tv, qs0.w, fmaf(ov, qo0.w, z[3]));
                z[4] = fmaf(tv, qs1.x, fmaf(ov, qo1.x, z[4]));
                z[5] = fmaf(tv, qs1.y, fmaf(ov, qo1.y, z[5]));
                z[6] = fmaf(tv, qs1.z, fmaf(ov, qo1.z, z[6]));
                z[7] = fmaf(tv, qs1.w, fmaf(ov, qo1.w, z[7]));
            }
            // every lane has read this tile's E rows before any store
            __syncwarp();
            const int row = bj_index(Ia, Ja, rr);
            float* w = E + row * ldE + colb;
            *reinterpret_cast<float4*>(w) = make_float4(z[0], z[1], z[2], z[3]);
            *reinterpret_cast<float4*>(w + 4) = make_float4(z[4], z[5], z[6], z[7]);
#pragma unroll
            for (int c = 0; c < BJ; ++c) E[(colb + c) * ldE + row] = z[c];
            __syncwarp();
        }
    };
    // off-diagonal tiles of round t on CTA 0, tiles lists[l0 .. l1): E_ab <- Q_a^T E_ab Q_b,
    // two tiles per warp (a half-warp each); lane: rows r0, r0 + 8 of the tile, columns
    // c0..c0+7 (one block of the column pair-block); the product with Q_b takes the partner
    // lane's half of the intermediate rows by shuffle
    auto tile_range = [&](int t, int l0, int l1) {
        const int par = t & 1;
        const float* Q = Ql + (size_t)par * nb * BJ2SQ;
        const int* pb = pbl + par * nb;
        const int* act = actl + par * nb;
        float* E = El;
        const int h = lane >> 4, l16 = lane & 15;
        const int r0 = l16 >> 1, c0 = (l16 & 1) * BJ;
        for (int task0 = l0 + 2 * warp; task0 < l1; task0 += 2 * nw) {
            const int task = task0 + h;
            const bool live = task < l1;
            const int ab = tiles[lists[t * ntile + (live ? task : task0)]];
            const int a = ab & 255, b = ab >> 8;
            if (__all_sync(0xffffffffu, !live || (!act[a] && !act[b]))) continue;
            const int pa = pb[a], pbb = pb[b];
            const int Ia = pa & 0xffff, Ja = pa >> 16, Ib = pbb & 0xffff, Jb2 = pbb >> 16;
            const float* Qa = Q + a * BJ2SQ;
            const float* Qb = Q + b * BJ2SQ;
            const int colb = c0 ? Jb2 * BJ : Ib * BJ;
            float t0[BJ], t1[BJ];
#pragma unroll
            for (int c = 0; c < BJ; ++c) { t0[c] = 0.f; t1[c] = 0.f; }
#pragma unroll
            for (int j = 0; j < BJ2; ++j) {
                const float qa0 = Qa[j * BJ2 + r0], qa1 = Qa[j * BJ2 + r0 + BJ];
                const float* xr = E + bj_index(Ia, Ja, j) * ldE + colb;
                const float4 x0 = *reinterpret_cast<const float4*>(xr);
                const float4 x1 = *reinterpret_cast<const float4*>(xr + 4);
                const float xv[BJ] = {x0.x, x0.y, x0.z, x0.w, x1.x, x1.y, x1.z, x1.w};
#pragma unroll
                for (int c = 0; c < BJ; ++c) {
                    t0[c] = fmaf(qa0, xv[c], t0[c]);
                    t1[c] = fmaf(qa1, xv[c], t1[c]);
                }
            }
            const int cp = c0 ^ BJ;
            const int row0 = bj_index(Ia, Ja, r0), row1 = bj_index(Ia, Ja, r0 + BJ);
#pragma unroll
            for (int half_row = 0; half_row < 2; ++half_row) {
                float z[BJ];
#pragma unroll
                for (int c = 0; c < BJ; ++c) z[c] = 0.f;
#pragma unroll
                for (int jj = 0; jj < BJ; ++jj) {
                    const float tv = half_row ? t1[jj] : t0[jj];
                    const float ov = __shfl_xor_sync(0xffffffffu, tv, 1);
                    const float4 qs0 = *reinterpret_cast<const float4*>(Qb + (c0 + jj) * BJ2 + c0);
                    const float4 qs1 = *reinterpret_cast<const float4*>(Qb + (c0 + jj) * BJ2 + c0 + 4);
                    const float4 qo0 = *reinterpret_cast<const float4*>(Qb + (cp + jj) * BJ2 + c0);
                    const float4 qo1 = *reinterpret_cast<const float4*>(Qb + (cp + jj) * BJ2 + c0 + 4);
                    z[0] = fmaf(tv, qs0.x, fmaf(ov, qo0.x, z[0]));
                    z[1] = fmaf(tv, qs0.y, fmaf(ov, qo0.y, z[1]));
                    z[2] = fmaf(tv, qs0.z, fmaf(ov, qo0.z, z[2]));
                    z[3] = fmaf(tv, qs0.w, fmaf(ov, qo0.w, z[3]));
                    z[4] = fmaf(tv, qs1.x, fmaf(ov, qo1.x, z[4]));
                    z[5] = fmaf(tv, qs1.y, fmaf(ov, qo1.y, z[5]));
                    z[6] = fmaf(tv, qs1.z, fmaf(ov, qo1.z, z[6]));
                    z[7] = fmaf(tv, qs1.w, fmaf(ov, qo1.w, z[7]));
                }
                // every lane has read this tile's E rows (first product) before any store
                __syncwarp();
                if (live) {
                    const int row = half_row ? row1 : row0;
                    float* w = E + row * ldE + colb;
                    *reinterpret_cast<float4*>(w) = make_float4(z[0], z[1], z[2], z[3]);
                    *reinterpret_cast<float4*>(w + 4) = make_float4(z[4], z[5], z[6], z[7]);
#pragma unroll
                    for (int c = 0; c < BJ; ++c) E[(colb + c) * ldE + row] = z[c];
                }
            }
            __syncwarp();
        }
    };
    // F <- F + F_Q + F F_Q for round t on this CTA's rows (CTAs >= 1), by half-warps: a
    // half-warp per pair-block and a group of rows; lane x of the half holds column x of F_Q in
    // registers. Beside the inner sweeps (overlap) only the warps on the other SMSPs of the SM
    // take part (warp w runs on SMSP w mod 4), so the inner sweeps' latency-bound chains keep
    // their issue slots; otherwise every warp does.
    auto f_update = [&](int t, bool overlap) {
        if (rank < 1) return;
        const int par = t & 1;
        const bool split = overlap && iw < 4;
        if (split && (warp & 3) < iw) return;
        if (overlap && !split && warp < iw) return;
        const int nwp = split ? (nw >> 2) * (4 - iw) : overlap ? nw - iw : nw;
        const int wi = split ? (warp >> 2) * (4 - iw) + (warp & 3) - iw : overlap ? warp - iw : warp;
        const int hw = 2 * wi + (lane >> 4), x = lane & 15, nhw = 2 * nwp;
        const unsigned int half = 0xffffu << (lane & 16);
        const int nr = j1 - j0;
        const int groups = max(1, nhw / nb);
        for (int task = hw; task < groups * nb; task += nhw) {
            const int a = task % nb, g = task / nb;
            int Ia, Ja;
            rr_pair_e(t, a, m, Ia, Ja);
            // F_Q of pair-block a, from the CTA that ran its inner sweep
            const float* fq = cl.map_shared_rank(qrem, 1 + a % nF) + (size_t)par * nb * SPSQ + a * SPSQ;
            float fcol[BJ2];
            bool nz = false;
#pragma unroll
            for (int y = 0; y < BJ2; ++y) {
                fcol[y] = fq[y * SP + x];
                nz |= fcol[y] != 0.f;
            }
            // F_Q = 0 (no rotation in this pair-block): F is unchanged
            const bool any = __any_sync(half, nz);
            // kFR rows at a time (independent chains; each element's sum keeps its order)
            for (int jl0 = g * kFR; jl0 < nr && any; jl0 += groups * kFR) {
                float acc[kFR];
#pragma unroll
                for (int q = 0; q < kFR; ++q) {
                    const int jl = jl0 + q;
                    if (jl >= nr) break;
                    const int j = j0 + jl;
                    const float* row = F + (size_t)jl * K;
                    const float4 f0 = *reinterpret_cast<const float4*>(row + Ia * BJ);
                    const float4 f1 = *reinterpret_cast<const float4*>(row + Ia * BJ + 4);
                    const float4 f2 = *reinterpret_cast<const float4*>(row + Ja * BJ);
                    const float4 f3 = *reinterpret_cast<const float4*>(row + Ja * BJ + 4);
                    const float fv[BJ2] = {f0.x, f0.y, f0.z, f0.w, f1.x, f1.y, f1.z, f1.w,
                                           f2.x, f2.y, f2.z, f2.w, f3.x, f3.y, f3.z, f3.w};
                    float v = row[bj_index(Ia, Ja, x)];
#pragma unroll
                    for (int y = 0; y < BJ2; ++y) v = fmaf(fv[y], fcol[y], v);
                    // row j of F_Q (embedded) when j is one of the pair-block's indices
                    const int bj = j / BJ;
                    if (bj == Ia) v += pick16(fcol, j - Ia * BJ);
                    else if (bj == Ja) v += pick16(fcol, BJ + j - Ja * BJ);
                    acc[q] = v;
                }
                // every lane has read these rows before any store
                __syncwarp(half);
#pragma unroll
                for (int q = 0; q < kFR; ++q)
                    if (jl0 + q < nr) F[(size_t)(jl0 + q) * K + bj_index(Ia, Ja, x)] = acc[q];
            }
        }
    };

    int sweep = 0;
    for (; sweep <= A.max_sweeps; ++sweep) {
        // sweep start: CTA 0 records the finished sweep's rotations and looks for a pair that
        // qualifies; every CTA reads the decision after the barrier
        if (rank == 0) {
            int need = 0;
            for (int a = warp; a < k && !need; a += nw)
                for (int c = a + 1 + lane; c < k; c += 32)
                    if (qualifies(D[a], D[c], El[a * ldE + c])) { need = 1; break; }
            need = __syncthreads_or(need);
            if (tid == 0) {
                int stop = 0;
                if (!need) stop = 1;
                else if (sweep == A.max_sweeps) {
                    stop = 1;
                    atomicCAS(&J.st->flag, FLAG_OK, FLAG_NOCONVERGE);
                }
                if (sweep > 0) J.st->sweep_active[(base + sweep - 1) & 63] = s_active;
                s_active = 0;
                for (int c = 0; c < cs; ++c) cl.map_shared_rank(ctl, c)[0] = stop;
            }
        }
        cl.sync();
        if (ctl[0]) break;
        inner_round(0);
        cl.sync();
        for (int t = 0; t < m - 1; ++t) {
            const bool next = t + 1 < m - 1;   // round t + 1 is in this sweep: overlap it
            const int nd = rank == 0 ? ndep[t] : 0;
            if (rank == 0) tile_wide(t, 0, nd);
            if (next) {
                cl.sync();
                // CTA 0: the other tiles of round t; CTAs >= 1: round t + 1's inner sweeps and
                // round t's F update on their other warps
                if (rank == 0) tile_range(t, nd, ntile);
                inner_round(t + 1);
                f_update(t, true);
            } else {
                if (rank == 0) tile_range(t, nd, ntile);
                f_update(t, false);
            }
            cl.sync();
        }
    }
    if (rank == 0) {
        for (int a = tid; a < k; a += nthr) J.outD[(int64_t)a * J.ldd] = df_to(D[a]);
        if (tid == 0) J.st->sweeps = base + sweep;
    } else {
        for (int e = tid; e < (j1 - j0) * K; e += nthr) {
            const int jl = e / K, n = e - jl * K;
            const int j = j0 + jl;
            if (j < k && n < k) J.outF[(int64_t)j * k + n] = (double)F[e] + ((J.add_identity && j == n) ? 1.0 : 0.0);
        }
    }
    cl.sync();
}

// ---------------------------------------------------------------------------
// Cholesky and triangular inverse in FP32, one CTA per matrix, held in shared
// memory: the first, conditioning pass of CholeskyQR (its result need only
// make the rows well conditioned; the second pass restores FP64 accuracy).
// Right-looking unblocked factorisation (a warp per trailing row, lanes over
// its columns), then the in-place inverse column by column from the last:
// column j of L^{-1} = -(1/l_jj) L^{-1}_{trailing} l_{j+1:, j}.
// ---------------------------------------------------------------------------
__device__ __forceinline__ float warp_sum(float v) {
    for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

__global__ void __launch_bounds__(kEigThreads) k_chol32_multi(const CholJob* jobs) {
    const CholJob J = jobs[blockIdx.x];
    if (J.gate && *J.gate < kSeriesGate) return;   // the series pass took this matrix
    const int r = J.r;
    extern __shared__ __align__(16) float A[];   // r x r, row-major (lower part)
    float* tmp = A + (size_t)r * r;               // r
    __shared__ int s_bad;
    const int tid = threadIdx.x, nthr = blockDim.x;
    const int warp = tid >> 5, lane = tid & 31, nw = nthr >> 5;
    for (int i = warp; i < r; i += nw)
        for (int l = lane; l <= i; l += 32) A[i * r + l] = (float)J.A[(int64_t)i * r + l];
    if (tid == 0) s_bad = 0;
    __syncthreads();
    for (int j = 0; j < r; ++j) {
        if (tid == 0) {
            float d = A[j * r + j];
            if (!(d > 0.f)) { s_bad = 1; d = 1.f; }
            A[j * r + j] = sqrtf(d);
        }
        __syncthreads();
        const float inv = 1.f / A[j * r + j];
        for (int i = j + 1 + tid; i < r; i += nthr) A[i * r + j] *= inv;
        __syncthreads();
        for (int i = j + 1 + warp; i < r; i += nw) {
            const float aij = A[i * r + j];
            for (int l = j + 1 + lane; l <= i; l += 32) A[i * r + l] = fmaf(-aij, A[l * r + j], A[i * r + l]);
        }
        __syncthreads();
    }
    for (int j = r - 1; j >= 0; --j) {
        for (int i = j + 1 + tid; i < r; i += nthr) tmp[i] = A[i * r + j];
        __syncthreads();
        const float djj = 1.f / A[j * r + j];
        for (int i = j + 1 + warp; i < r; i += nw) {
            float acc = 0.f;
            for (int l = j + 1 + lane; l <= i; l += 32) acc = fmaf(A[i * r + l], tmp[l], acc);
            acc = warp_sum(acc);
            if (lane == 0) A[i * r + j] = -djj * acc;
        }
        __syncthreads();
        if (tid == 0) A[j * r + j] = djj;
        __syncthreads();
    }
    for (int i = warp; i < r; i += nw)
        for (int l = lane; l < r; l += 32) J.Li[(int64_t)i * r + l] = l <= i ? (double)A[i * r + l] : 0.0;
    if (tid == 0 && s_bad) atomicCAS(&J.st->flag, FLAG_OK, FLAG_NOT_SPD);
}


// ---------------------------------------------------------------------------
// The same block Jacobi for matrices beyond one CTA's shared memory: one
// cooperative grid for every matrix of the launch, D (hi/lo FP32), E (FP32,
// full symmetric storage, three buffers by round), the rotation accumulator F
// and the pair-block rotations Q (two buffers by round) in global memory
// (L2-resident: a few MB a matrix at k = 512). One phase a round, between
// bounded counting barriers:
//   - a warp per pair-block of round g (warp 0 of different SMs) forms its
//     16 x 16 diagonal block of the state after round g - 1: the two diagonal
//     8 x 8 blocks as round g - 1's inner sweeps left them (buffer g mod 3),
//     the cross block from round g - 1's tile of the two pair-blocks that held
//     them (buffer g - 1 mod 3) and that round's rotations, by the tile
//     product's own arithmetic; it runs the inner sweep exactly as the cluster
//     kernel does (the same function) and writes the block to buffer g + 1
//     mod 3, D and F_Q;
//   - meanwhile the other warps rotate round g - 1's tiles (E_ab <- Q_a^T E_ab
//     Q_b, both triangles; a half-warp each, operands staged in shared memory)
//     from buffer g - 1 mod 3 into buffer g mod 3, copying those of pair-blocks
//     that did not rotate, and apply round
//     g - 1's rotations to F (F <- F + F_Q + F F_Q, a half-warp per pair-block
//     and group of 16 rows, a lane per row).
// So a round costs one barrier and its inner sweeps, with the tiles off the
// critical path. Matrices of different sizes keep their own round and sweep
// counters. A matrix stops after a sweep in which no pair qualified, or at the
// sweep limit. The decision is read by every CTA from the same counter after
// the same barrier, so control flow stays uniform. The outputs and the sweep
// report are those of the cluster kernel. For the same input it gives the same
// result, with one more sweep reported: that sweep is the empty one that
// confirms convergence, where the cluster kernel scans instead.
// ---------------------------------------------------------------------------
constexpr int kGbThreads = 512;
constexpr int kGbMaxModes = 128;

struct GbMode {
    const double* H; double* outD; double* outF; DevStatus* st;
    int64_t ldd; int k; int add_identity;
    float floor, tau, tol2;
    int K, ldE, nb, m;
    // E [3][K][ldE]: round mod 3; Q [2][nb][16 x 16] and act [2][nb]: round parity; cnt[3]:
    // rotations a sweep (sweep mod 3)
    DF* D; float* E; float* F; float* Q; int* act; unsigned int* cnt;
};
struct GbArgs {
    const GbMode* m; int nm; int max_sweeps; DevStatus* bar;
};
static_assert(sizeof(GbMode) % sizeof(int) == 0 && alignof(GbMode) <= 16, "descriptors are copied as words");

// F <- F + F_Q + F F_Q on the 16 columns of pair-block a of round `round` for
// the rows 16 g .. 16 g + 15: a half-warp, lane x owns row 16 g + x; the
// half-warp stages F_Q in sq. The same products in the same order as the
// cluster kernel's F update.
__device__ __forceinline__ void gb_f_rows(const GbMode& J, int round, const float* Qp, int a, int g, int x,
                                          unsigned int half, float* sq) {
    int Ia, Ja;
    rr_pair_e(round, a, J.m, Ia, Ja);
    const float4* fq4 = reinterpret_cast<const float4*>(Qp + (int64_t)a * BJ2SQ);
#pragma unroll
    for (int q = 0; q < 4; ++q) reinterpret_cast<float4*>(sq)[x * 4 + q] = fq4[x * 4 + q];
    const int row = g * BJ2 + x;
    float* fr = J.F + (int64_t)row * J.K;
    const float4 f0 = *reinterpret_cast<const float4*>(fr + Ia * BJ);
    const float4 f1 = *reinterpret_cast<const float4*>(fr + Ia * BJ + 4);
    const float4 f2 = *reinterpret_cast<const float4*>(fr + Ja * BJ);
    const float4 f3 = *reinterpret_cast<const float4*>(fr + Ja * BJ + 4);
    const float f[BJ2] = {f0.x, f0.y, f0.z, f0.w, f1.x, f1.y, f1.z, f1.w,
                          f2.x, f2.y, f2.z, f2.w, f3.x, f3.y, f3.z, f3.w};
    __syncwarp(half);
    float o[BJ2];
#pragma unroll
    for (int c = 0; c < BJ2; ++c) o[c] = f[c];
    // F_Q rows as float4 broadcasts: a quarter of the shared-memory reads of scalar ones
    const float4* sq4 = reinterpret_cast<const float4*>(sq);
#pragma unroll
    for (int y = 0; y < BJ2; ++y)
#pragma unroll
        for (int c4 = 0; c4 < BJ2 / 4; ++c4) {
            const float4 q = sq4[y * (BJ2 / 4) + c4];
            o[4 * c4] = fmaf(f[y], q.x, o[4 * c4]);
            o[4 * c4 + 1] = fmaf(f[y], q.y, o[4 * c4 + 1]);
            o[4 * c4 + 2] = fmaf(f[y], q.z, o[4 * c4 + 2]);
            o[4 * c4 + 3] = fmaf(f[y], q.w, o[4 * c4 + 3]);
        }
    // the F_Q term: rows of F inside the pair-block (F holds I + F)
    const int bj = row / BJ;
    const int lr = bj == Ia ? row - Ia * BJ : (bj == Ja ? BJ + row - Ja * BJ : -1);
    if (lr >= 0) {
#pragma unroll
        for (int c4 = 0; c4 < BJ2 / 4; ++c4) {
            const float4 q = sq4[lr * (BJ2 / 4) + c4];
            o[4 * c4] += q.x;
            o[4 * c4 + 1] += q.y;
            o[4 * c4 + 2] += q.z;
            o[4 * c4 + 3] += q.w;
        }
    }
    *reinterpret_cast<float4*>(fr + Ia * BJ) = make_float4(o[0], o[1], o[2], o[3]);
    *reinterpret_cast<float4*>(fr + Ia * BJ + 4) = make_float4(o[4], o[5], o[6], o[7]);
    *reinterpret_cast<float4*>(fr + Ja * BJ) = make_float4(o[8], o[9], o[10], o[11]);
    *reinterpret_cast<float4*>(fr + Ja * BJ + 4) = make_float4(o[12], o[13], o[14], o[15]);
    __syncwarp(half);   // every lane has read sq before the next item stages its F_Q
}

// pair-block of round t holding block X (blocks of BJ indices, m of them) and whether X is its
// second half (the larger block index): the inverse of rr_pair_e
__device__ __forceinline__ void rr_block_of(int t, int X, int m, int& i, int& second) {
    const int n1 = m - 1, nb = m / 2;
    if (X == n1) { i = 0; second = 1; return; }
    if (X == t) { i = 0; second = 0; return; }
    const int dd = mod_lt2n(X - t + n1, n1);
    int a, b;
    if (dd <= nb - 1) { i = dd; a = X; b = mod_lt2n(t - dd + n1, n1); }
    else { i = n1 - dd; a = mod_lt2n(t + i, n1); b = X; }
    second = X == max(a, b) ? 1 : 0;
}

__global__ void __launch_bounds__(kGbThreads, 1) k_jacobi_gblk(GbArgs A) {
    __shared__ int s_sweep[kGbMaxModes], s_round[kGbMaxModes], s_done[kGbMaxModes], s_base[kGbMaxModes];
    __shared__ int s_gr[kGbMaxModes];   // global index of the matrix's next round (its A phase)
    __shared__ int s_ran[kGbMaxModes];  // this phase runs the matrix's next round
    __shared__ int s_pr[kGbMaxModes];   // round (within its sweep) whose tiles and F update are pending, -1: none
    __shared__ int s_pg[kGbMaxModes];   // its global index
    __shared__ int s_pa[kGbMaxModes + 1], s_pt[kGbMaxModes + 1], s_pf[kGbMaxModes + 1];
    __shared__ int s_live;
    // per half-warp: F_Q of an F item, E_ab, Q_a, Q_b of a tile, or (the inner sweeps' warps) the
    // previous round's tile, its rotations and the cross block they give
    extern __shared__ __align__(16) float gb_smem[];
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int nwarp_cta = kGbThreads / 32;
    const int slot = warp * gridDim.x + blockIdx.x, nwarps = gridDim.x * nwarp_cta;
    // the warps in the order 1, 2, 3, 5, ..., 15, then 4, 8, 12, 0 (warp 0 takes the inner sweeps)
    const int frank = (warp & 3) == 0 ? (warp == 0 ? nwarp_cta - 1 : nwarp_cta - nwarp_cta / 4 + (warp >> 2) - 1)
                                      : warp - 1 - (warp >> 2);
    const int fslot = frank * gridDim.x + blockIdx.x;
    const int h = lane >> 4, l16 = lane & 15;
    const unsigned int half = 0xffffu << (lane & 16);
    float* sq = gb_smem + (size_t)(warp * 2 + h) * 3 * BJ2SQ;
    float* sw = gb_smem + (size_t)(warp * 2) * 3 * BJ2SQ;   // the whole warp's staging (6 x 256 floats)
    const int nm = A.nm;
    // the job descriptors in shared memory (read in every phase; global reads would miss L1
    // after each barrier's fence)
    GbMode* Ms = reinterpret_cast<GbMode*>(gb_smem + (size_t)(kGbThreads / 16) * 3 * BJ2SQ);
    {
        const int words = nm * (int)(sizeof(GbMode) / sizeof(int));
        const int* src = reinterpret_cast<const int*>(A.m);
        int* dst = reinterpret_cast<int*>(Ms);
        for (int i = tid; i < words; i += kGbThreads) dst[i] = src[i];
        __syncthreads();
    }
    unsigned int epoch = 0;
    auto barrier = [&]() { return count_barrier(A.bar, ++epoch * gridDim.x); };
    auto ebuf = [&](const GbMode& J, int g) { return J.E + (int64_t)(g % 3) * J.K * J.ldE; };
    // half-item fh of the pending F updates (decoded over the matrices with one pending)
    auto f_item = [&](int fh) {
        int j = 0;
        while (j < nm - 1 && (s_pf[j + 1] <= fh || s_pr[j] < 0)) ++j;
        const GbMode& J = Ms[j];
        const int rest = fh - s_pf[j], groups = J.K / BJ2;
        const int a = rest / groups, g = rest - a * groups, par = s_pg[j] & 1;
        if (!J.act[par * J.nb + a]) return;   // uniform over the half-warp
        gb_f_rows(J, s_pr[j], J.Q + (int64_t)par * J.nb * BJ2SQ, a, g, l16, half, sq);
    };

    // initial state (buffer 0 = the state before round 0): D from diag(H), E from the
    // off-diagonal of H, F = 0, counters 0
    for (int j = 0; j < nm; ++j) {
        const GbMode& J = Ms[j];
        const int64_t ne = (int64_t)J.K * J.ldE;
        for (int64_t e = blockIdx.x * (int64_t)kGbThreads + tid; e < ne; e += (int64_t)gridDim.x * kGbThreads) {
            const int r = (int)(e / J.ldE), c = (int)(e - (int64_t)r * J.ldE);
            J.E[e] = (r < J.k && c < J.k && r != c) ? (float)J.H[(int64_t)r * J.k + c] : 0.f;
            if (c == 0) J.D[r] = df_from(r < J.k ? J.H[(int64_t)r * J.k + r] : 0.0);
        }
        const int64_t nf = (int64_t)J.K * J.K;
        for (int64_t e = blockIdx.x * (int64_t)kGbThreads + tid; e < nf; e += (int64_t)gridDim.x * kGbThreads) J.F[e] = 0.f;
        if (blockIdx.x == 0 && tid < 3) J.cnt[tid] = 0;
    }
    if (tid < nm) {
        s_sweep[tid] = 0;
        s_round[tid] = 0;
        s_done[tid] = 0;
        s_base[tid] = Ms[tid].st->sweeps;
        s_gr[tid] = 0;
        s_pr[tid] = -1;
        s_pg[tid] = 0;
    }
    bool ok = barrier();

    // One phase a round: the inner sweeps of every live matrix's next round g (warp 0 of
    // different SMs; they read the state after round g - 1: the diagonal blocks from buffer
    // g % 3, and their cross block from round g - 1's tile in buffer (g - 1) % 3 with that
    // round's rotations, by the tile product's own arithmetic) beside the tiles and the F
    // update of round g - 1 (the other warps: buffer (g - 1) % 3 into buffer g % 3, which the
    // inner sweeps of round g - 1 have already filled with their diagonal blocks). One
    // barrier a phase.
    while (ok) {
        if (tid == 0) {
            int pa = 0, pt = 0, pf = 0, live = 0;
            for (int j = 0; j < nm; ++j) {
                s_pa[j] = pa;
                s_pt[j] = pt;
                s_pf[j] = pf;
                const GbMode& J = Ms[j];
                s_ran[j] = !s_done[j];
                if (s_ran[j]) pa += J.nb;
                if (s_pr[j] >= 0) {
                    pt += J.nb * (J.nb - 1) / 2;
                    pf += J.nb * (J.K / BJ2);
                }
                live |= s_ran[j] || s_pr[j] >= 0;
            }
            s_pa[nm] = pa;
            s_pt[nm] = pt;
            s_pf[nm] = pf;
            s_live = live;
        }
        __syncthreads();
        if (!s_live) break;

        // ---- inner sweeps of round g, a warp per pair-block
        const int nA = s_pa[nm];
        for (int item = slot; item < nA; item += nwarps) {
            int j = 0;
            while (j < nm - 1 && (s_pa[j + 1] <= item || !s_ran[j])) ++j;
            const GbMode& J = Ms[j];
            const int a = item - s_pa[j], t = s_round[j], g = s_gr[j], par = g & 1;
            const Crit qualifies{J.floor, J.tau, J.tol2};
            int I, Jb;
            rr_pair_e(t, a, J.m, I, Jb);
            const int pos = lane & (BJ2 - 1);
            const int64_t gi = bj_index(I, Jb, pos);
            const float* Ec = ebuf(J, g);   // the state after round g - 1
            float x[BJ2];
            DF d{0.f, 0.f};
            if (g == 0) {
                if (lane < BJ2) {
#pragma unroll
                    for (int r = 0; r < BJ2; ++r) x[r] = Ec[(int64_t)bj_index(I, Jb, r) * J.ldE + gi];
                    d = J.D[gi];
                } else {
#pragma unroll
                    for (int r = 0; r < BJ2; ++r) x[r] = 0.f;
                }
            } else {
                // the cross block [I, Jb] after round g - 1: round g - 1 paired I and Jb into
                // different pair-blocks; their tile (rows: the smaller pair-block index) rotated
                const int tp = t == 0 ? J.m - 2 : t - 1, pp = (g - 1) & 1;
                int ia, ha, ib, hb;
                rr_block_of(tp, I, J.m, ia, ha);
                rr_block_of(tp, Jb, J.m, ib, hb);
                const bool swap = ia > ib;   // the tile's rows hold Jb: the block is [Jb, I]
                const int ra = swap ? ib : ia, rb = swap ? ia : ib;
                const int hr = swap ? hb : ha, hc = swap ? ha : hb;
                int Ira, Jra, Irb, Jrb;
                rr_pair_e(tp, ra, J.m, Ira, Jra);
                rr_pair_e(tp, rb, J.m, Irb, Jrb);
                float* sE = sw;
                float* sQa = sw + BJ2SQ;
                float* sQb = sw + 2 * BJ2SQ;
                float* sT = sw + 3 * BJ2SQ;   // [8][16]: the tile rows hr*8 .. +7 of Q_a^T E
                float* sR = sT + 8 * BJ2;     // [8][8]: the block
                // the two diagonal blocks (buffer g % 3) and d, loaded beside the tile and its
                // rotations below: one trip to L2 instead of two; the cross entries come later
                if (lane < BJ2) {
#pragma unroll
                    for (int r = 0; r < BJ2; ++r)
                        if ((r < BJ) == (pos < BJ)) x[r] = Ec[(int64_t)bj_index(I, Jb, r) * J.ldE + gi];
                    d = J.D[gi];
                } else {
#pragma unroll
                    for (int r = 0; r < BJ2; ++r) x[r] = 0.f;
                }
                {
                    const float* Ep = ebuf(J, g - 1);
                    const float4* qa4 = reinterpret_cast<const float4*>(J.Q + ((int64_t)pp * J.nb + ra) * BJ2SQ);
                    const float4* qb4 = reinterpret_cast<const float4*>(J.Q + ((int64_t)pp * J.nb + rb) * BJ2SQ);
                    // lane: tile row lane / 2, its half (lane & 1) of the 16 columns; Q: float4s lane, lane + 32
                    const int tr = lane >> 1, th = lane & 1;
                    const float* er = Ep + (int64_t)bj_index(Ira, Jra, tr) * J.ldE + (th ? Jrb : Irb) * BJ;
                    const float4 e0 = *reinterpret_cast<const float4*>(er);
                    const float4 e1 = *reinterpret_cast<const float4*>(er + 4);
                    const float4 a0 = qa4[lane], a1 = qa4[lane + 32], b0 = qb4[lane], b1 = qb4[lane + 32];
                    __syncwarp();   // the previous item's readers of the staging area are done
                    reinterpret_cast<float4*>(sE)[tr * 4 + th * 2] = e0;
                    reinterpret_cast<float4*>(sE)[tr * 4 + th * 2 + 1] = e1;
                    reinterpret_cast<float4*>(sQa)[lane] = a0;
                    reinterpret_cast<float4*>(sQa)[lane + 32] = a1;
                    reinterpret_cast<float4*>(sQb)[lane] = b0;
                    reinterpret_cast<float4*>(sQb)[lane + 32] = b1;
                    __syncwarp();
                }
                // T[row][col] = sum_jj (Q_a[jj][row] + [jj == row]) E[jj][col], rows hr*8 .. +7, in the
                // tile product's order; a lane takes column lane & 15 of four consecutive rows (one
                // float4 of Q_a and one entry of E a step)
                {
                    const int col = lane & 15, rq = (lane >> 4) * 4, row0 = hr * BJ + rq;
                    float acc[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
                    for (int jj = 0; jj < BJ2; ++jj) {
                        const float4 q = *reinterpret_cast<const float4*>(sQa + jj * BJ2 + row0);
                        const float e = sE[jj * BJ2 + col];
                        acc[0] = fmaf(q.x + (jj == row0 ? 1.f : 0.f), e, acc[0]);
                        acc[1] = fmaf(q.y + (jj == row0 + 1 ? 1.f : 0.f), e, acc[1]);
                        acc[2] = fmaf(q.z + (jj == row0 + 2 ? 1.f : 0.f), e, acc[2]);
                        acc[3] = fmaf(q.w + (jj == row0 + 3 ? 1.f : 0.f), e, acc[3]);
                    }
#pragma unroll
                    for (int u = 0; u < 4; ++u) sT[(rq + u) * BJ2 + col] = acc[u];
                }
                __syncwarp();
                // the block: columns hc*8 .. +7 of T Q_b, the tile product's pairing of column halves;
                // a lane takes column cc of rows rr and rr + 4 (the same Q_b entries for both)
                {
                    const int rr = lane >> 3, cc = lane & 7;
                    const int c0 = hc * BJ, cp = c0 ^ BJ, tc = c0 + cc;
                    float qs[BJ], qo[BJ];
#pragma unroll
                    for (int jj = 0; jj < BJ; ++jj) {
                        qs[jj] = sQb[(c0 + jj) * BJ2 + tc] + ((c0 + jj) == tc ? 1.f : 0.f);
                        qo[jj] = sQb[(cp + jj) * BJ2 + tc] + ((cp + jj) == tc ? 1.f : 0.f);
                    }
#pragma unroll
                    for (int h2 = 0; h2 < 2; ++h2) {
                        const float* trow = sT + (rr + 4 * h2) * BJ2;
                        const float4 t0 = *reinterpret_cast<const float4*>(trow + c0);
                        const float4 t1 = *reinterpret_cast<const float4*>(trow + c0 + 4);
                        const float4 o0 = *reinterpret_cast<const float4*>(trow + cp);
                        const float4 o1 = *reinterpret_cast<const float4*>(trow + cp + 4);
                        const float tv[BJ] = {t0.x, t0.y, t0.z, t0.w, t1.x, t1.y, t1.z, t1.w};
                        const float ov[BJ] = {o0.x, o0.y, o0.z, o0.w, o1.x, o1.y, o1.z, o1.w};
                        float z = 0.f;
#pragma unroll
                        for (int jj = 0; jj < BJ; ++jj) z = fmaf(tv[jj], qs[jj], fmaf(ov[jj], qo[jj], z));
                        sR[(rr + 4 * h2) * BJ + cc] = z;
                    }
                }
                __syncwarp();
                // the 16 x 16 block's cross entries from sR (sR = [I, Jb], or [Jb, I] when
                // swapped; the other cross block is its transpose)
                if (lane < BJ2) {
#pragma unroll
                    for (int r = 0; r < BJ2; ++r) {
                        const bool rI = r < BJ, cI = pos < BJ;
                        if (rI != cI) {
                            // [I, Jb][u][v] with u the row in block I, v the column in block Jb
                            const int u = rI ? r : pos, v = rI ? pos - BJ : r - BJ;
                            x[r] = swap ? sR[v * BJ + u] : sR[u * BJ + v];
                        }
                    }
                }
            }
            unsigned int nrot = t == 0 ? inner_sweep<true>(x, d, I, Jb, J.k, qualifies)
                                       : inner_sweep<false>(x, d, I, Jb, J.k, qualifies);
            for (int o = 16; o; o >>= 1) nrot += __shfl_xor_sync(0xffffffffu, nrot, o);
            float* En = ebuf(J, g + 1);   // the state after round g: its diagonal blocks
            float* Qa = J.Q + ((int64_t)par * J.nb + a) * BJ2SQ;
            if (lane < BJ2) {
#pragma unroll
                for (int r = 0; r < BJ2; ++r) En[(int64_t)bj_index(I, Jb, r) * J.ldE + gi] = x[r];
                J.D[gi] = d;
            } else {
#pragma unroll
                for (int r = 0; r < BJ2; ++r) Qa[r * BJ2 + pos] = x[r];   // F_Q; Q = I + F_Q
            }
            if (lane == 0) {
                J.act[par * J.nb + a] = nrot > 0;
                if (nrot) atomicAdd(&J.cnt[s_sweep[j] % 3], nrot);
            }
            __syncwarp();
        }

        // ---- round g - 1's tiles (buffer (g - 1) % 3 rotated into buffer g % 3; a tile of two
        // pair-blocks that did not rotate is copied) and its F update, on the warps of the other
        // SMSPs first (warp 0's SMSP runs the inner sweep alone: sharing it slows the sweep more
        // than the extra warps speed up the tiles)
        {
            const int r0 = l16 >> 1, c0 = (l16 & 1) * BJ;
            const int ntile = s_pt[nm];
            for (int task0 = 2 * fslot; task0 < ntile; task0 += 2 * nwarps) {
                const int task = task0 + h;
                const bool live = task < ntile;
                const int tt = live ? task : task0;
                int j = 0;
                while (j < nm - 1 && (s_pt[j + 1] <= tt || s_pr[j] < 0)) ++j;
                const GbMode& J = Ms[j];
                const int pg = s_pg[j], par = pg & 1;
                // tile index -> (a, b), a < b: row a has nb - 1 - a tiles
                int rem = tt - s_pt[j], a = 0;
                while (a < J.nb - 1 && rem >= J.nb - 1 - a) { rem -= J.nb - 1 - a; ++a; }
                const int b = a + 1 + rem;
                const int t = s_pr[j];
                int Ia, Ja, Ib, Jb2;
                rr_pair_e(t, a, J.m, Ia, Ja);
                rr_pair_e(t, b, J.m, Ib, Jb2);
                const float* Es = ebuf(J, pg);
                float* Ed = ebuf(J, pg + 1);
                // a tile of two pair-blocks that did not rotate is copied (both triangles); the
                // product runs where either half-warp's tile needs it (the other half's Q are then
                // identities, so it copies exactly by the same arithmetic)
                const int* act = J.act + par * J.nb;
                if (!__any_sync(0xffffffffu, live && (act[a] | act[b]))) {
                    if (live) {
                        const int ra = bj_index(Ia, Ja, l16), rb = bj_index(Ib, Jb2, l16);
                        const float* sa = Es + (int64_t)ra * J.ldE;
                        const float* sb = Es + (int64_t)rb * J.ldE;
                        float* da = Ed + (int64_t)ra * J.ldE;
                        float* db = Ed + (int64_t)rb * J.ldE;
                        const float4 u0 = *reinterpret_cast<const float4*>(sa + Ib * BJ);
                        const float4 u1 = *reinterpret_cast<const float4*>(sa + Ib * BJ + 4);
                        const float4 u2 = *reinterpret_cast<const float4*>(sa + Jb2 * BJ);
                        const float4 u3 = *reinterpret_cast<const float4*>(sa + Jb2 * BJ + 4);
                        const float4 w0 = *reinterpret_cast<const float4*>(sb + Ia * BJ);
                        const float4 w1 = *reinterpret_cast<const float4*>(sb + Ia * BJ + 4);
                        const float4 w2 = *reinterpret_cast<const float4*>(sb + Ja * BJ);
                        const float4 w3 = *reinterpret_cast<const float4*>(sb + Ja * BJ + 4);
                        *reinterpret_cast<float4*>(da + Ib * BJ) = u0;
                        *reinterpret_cast<float4*>(da + Ib * BJ + 4) = u1;
                        *reinterpret_cast<float4*>(da + Jb2 * BJ) = u2;
                        *reinterpret_cast<float4*>(da + Jb2 * BJ + 4) = u3;
                        *reinterpret_cast<float4*>(db + Ia * BJ) = w0;
                        *reinterpret_cast<float4*>(db + Ia * BJ + 4) = w1;
                        *reinterpret_cast<float4*>(db + Ja * BJ) = w2;
                        *reinterpret_cast<float4*>(db + Ja * BJ + 4) = w3;
                    }
                    continue;
                }
                float* sE = sq;
                float* sQa = sq + BJ2SQ;
                float* sQb = sq + 2 * BJ2SQ;
                {
                    const float4* qa4 = reinterpret_cast<const float4*>(J.Q + ((int64_t)par * J.nb + a) * BJ2SQ);
                    const float4* qb4 = reinterpret_cast<const float4*>(J.Q + ((int64_t)par * J.nb + b) * BJ2SQ);
                    const float* er = Es + (int64_t)bj_index(Ia, Ja, l16) * J.ldE;
                    float4 v[12];
#pragma unroll
                    for (int q = 0; q < 4; ++q) {
                        v[q] = qa4[l16 * 4 + q];
                        v[4 + q] = qb4[l16 * 4 + q];
                    }
                    v[8] = *reinterpret_cast<const float4*>(er + Ib * BJ);
                    v[9] = *reinterpret_cast<const float4*>(er + Ib * BJ + 4);
                    v[10] = *reinterpret_cast<const float4*>(er + Jb2 * BJ);
                    v[11] = *reinterpret_cast<const float4*>(er + Jb2 * BJ + 4);
                    __syncwarp();   // the previous item's readers of this staging area are done
#pragma unroll
                    for (int q = 0; q < 4; ++q) {
                        reinterpret_cast<float4*>(sQa)[l16 * 4 + q] = v[q];
                        reinterpret_cast<float4*>(sQb)[l16 * 4 + q] = v[4 + q];
                        reinterpret_cast<float4*>(sE)[l16 * 4 + q] = v[8 + q];
                    }
                    __syncwarp();
                }
                const float* Qa = sQa;
                const float* Qb = sQb;
                const int colb = c0 ? Jb2 * BJ : Ib * BJ;
                float t0[BJ], t1[BJ];
#pragma unroll
                for (int c = 0; c < BJ; ++c) { t0[c] = 0.f; t1[c] = 0.f; }
#pragma unroll
                for (int jj = 0; jj < BJ2; ++jj) {
                    const float qa0 = Qa[jj * BJ2 + r0] + (jj == r0 ? 1.f : 0.f);
                    const float qa1 = Qa[jj * BJ2 + r0 + BJ] + (jj == r0 + BJ ? 1.f : 0.f);
                    const float* xr = sE + jj * BJ2 + c0;
                    const float4 x0 = *reinterpret_cast<const float4*>(xr);
                    const float4 x1 = *reinterpret_cast<const float4*>(xr + 4);
                    const float xv[BJ] = {x0.x, x0.y, x0.z, x0.w, x1.x, x1.y, x1.z, x1.w};
#pragma unroll
                    for (int c = 0; c < BJ; ++c) {
                        t0[c] = fmaf(qa0, xv[c], t0[c]);
                        t1[c] = fmaf(qa1, xv[c], t1[c]);
                    }
                }
                const int ldE = J.ldE;
                const int cp = c0 ^ BJ;
                const int row0 = bj_index(Ia, Ja, r0), row1 = bj_index(Ia, Ja, r0 + BJ);
#pragma unroll
                for (int half_row = 0; half_row < 2; ++half_row) {
                    float z[BJ];
#pragma unroll
                    for (int c = 0; c < BJ; ++c) z[c] = 0.f;
#pragma unroll
                    for (int jj = 0; jj < BJ; ++jj) {
                        const float tv = half_row ? t1[jj] : t0[jj];
                        const float ov = __shfl_xor_sync(0xffffffffu, tv, 1);
                        const float4* qs4 = reinterpret_cast<const float4*>(Qb + (c0 + jj) * BJ2 + c0);
                        const float4* qo4 = reinterpret_cast<const float4*>(Qb + (cp + jj) * BJ2 + c0);
                        const float4 s0 = qs4[0], s1 = qs4[1], o0 = qo4[0], o1 = qo4[1];
                        const float qsv[BJ] = {s0.x, s0.y, s0.z, s0.w, s1.x, s1.y, s1.z, s1.w};
                        const float qov[BJ] = {o0.x, o0.y, o0.z, o0.w, o1.x, o1.y, o1.z, o1.w};
#pragma unroll
                        for (int c = 0; c < BJ; ++c) {
                            const float qs = qsv[c] + ((c0 + jj) == (c0 + c) ? 1.f : 0.f);
                            const float qo = qov[c] + ((cp + jj) == (c0 + c) ? 1.f : 0.f);
                            z[c] = fmaf(tv, qs, fmaf(ov, qo, z[c]));
                        }
                    }
                    if (live) {
                        const int row = half_row ? row1 : row0;
                        float* w = Ed + (int64_t)row * ldE + colb;
                        *reinterpret_cast<float4*>(w) = make_float4(z[0], z[1], z[2], z[3]);
                        *reinterpret_cast<float4*>(w + 4) = make_float4(z[4], z[5], z[6], z[7]);
#pragma unroll
                        for (int c = 0; c < BJ; ++c) Ed[(int64_t)(colb + c) * ldE + row] = z[c];
                    }
                }
                __syncwarp();
            }
            const int nF = s_pf[nm];
            for (int fw = fslot; 2 * fw < nF; fw += nwarps) {
                const int fh = 2 * fw + h;
                if (fh < nF) f_item(fh);
            }
        }
        __syncthreads();
        if (!(ok = barrier())) break;
        // the round just run is pending (tiles, F); the next one, or the end of the sweep
        if (tid < nm) {
            const int j = tid;
            const GbMode& J = Ms[j];
            if (s_ran[j]) {
                s_pr[j] = s_round[j];
                s_pg[j] = s_gr[j];
                ++s_gr[j];
                if (s_round[j] == J.m - 2) {
                    const int sw = s_sweep[j];
                    const unsigned int c = *(volatile unsigned int*)&J.cnt[sw % 3];
                    if (blockIdx.x == 0) {
                        J.st->sweep_active[(s_base[j] + sw) & 63] = c;
                        J.cnt[(sw + 2) % 3] = 0;   // read two sweeps ago; added to next sweep but one
                    }
                    if (c == 0) {
                        s_done[j] = 1;   // converged: this sweep confirmed it
                    } else if (sw + 1 >= A.max_sweeps) {
                        s_done[j] = 1;   // sweep limit
                        if (blockIdx.x == 0) atomicCAS(&J.st->flag, FLAG_OK, FLAG_NOCONVERGE);
                    } else {
                        s_round[j] = 0;
                        ++s_sweep[j];
                    }
                } else {
                    ++s_round[j];
                }
            } else {
                s_pr[j] = -1;
            }
        }
        __syncthreads();
    }
    // results (also after a failed barrier, so the host sees the flag and the partial state)
    const bool timed_out = !ok;
    for (int j = 0; j < nm; ++j) {
        const GbMode& J = Ms[j];
        for (int64_t e = blockIdx.x * (int64_t)kGbThreads + tid; e < (int64_t)J.k * J.k; e += (int64_t)gridDim.x * kGbThreads) {
            const int r = (int)(e / J.k), c = (int)(e - (int64_t)r * J.k);
            J.outF[e] = (double)J.F[(int64_t)r * J.K + c] + ((J.add_identity && r == c) ? 1.0 : 0.0);
        }
        for (int r = blockIdx.x * kGbThreads + tid; r < J.k; r += gridDim.x * kGbThreads) J.outD[(int64_t)r * J.ldd] = df_to(J.D[r]);
        if (blockIdx.x == 0 && tid == 0) {
            J.st->sweeps = s_base[j] + s_sweep[j] + 1;
            if (timed_out) atomicCAS(&J.st->flag, FLAG_OK, FLAG_TIMEOUT);
        }
    }
}

}  // namespace

int chol32_max_r() {
    const int cap = smem_optin();
    int r = 1;
    while (4 * ((size_t)(r + 1) * (r + 1) + (r + 1)) <= (size_t)cap) ++r;
    return r;
}

cudaError_t launch_chol32_multi(const CholJob* jobs, int njobs, cudaStream_t st) {
    if (njobs < 1) return cudaSuccess;
    int rmax = 1;
    for (int m = 0; m < njobs; ++m) rmax = std::max(rmax, jobs[m].r);
    if (rmax > chol32_max_r()) return cudaErrorInvalidValue;
    const size_t smem = 4 * ((size_t)rmax * rmax + rmax);
    cudaError_t e = grow_smem((const void*)k_chol32_multi, smem);
    if (e != cudaSuccess) return e;
    CholJob* dj = nullptr;
    e = cudaMallocAsync(&dj, sizeof(CholJob) * njobs, st);
    if (e != cudaSuccess) return e;
    e = upload_h2d(dj, jobs, sizeof(CholJob) * njobs, st);
    if (e == cudaSuccess) {
        k_chol32_multi<<<njobs, kEigThreads, smem, st>>>(dj);
        count_kernels(1);
        e = cudaGetLastError();
    }
    cudaFreeAsync(dj, st);
    return e;
}

int jacobi_blk_max_k() {
    const int cap = smem_optin();
    int k = BJ2;
    while (k < 4096 && BjLayout(k + BJ2, 1).e_bytes <= (size_t)cap) k += BJ2;
    return k;
}

cudaError_t launch_jacobi_blk(const DfJob* jobs, int njobs, int max_sweeps, cudaStream_t st) {
    if (njobs < 1) return cudaSuccess;
    const int cap = smem_optin();
    int kmax = 1;
    for (int m = 0; m < njobs; ++m) kmax = std::max(kmax, jobs[m].k);
    const BjLayout L0(kmax, 1);
    // one thread per rotation of an inner round
    if (L0.e_bytes > (size_t)cap || L0.nb * (BJ2 / 2) > kBlkThreads) return cudaErrorInvalidValue;
    // F rows and inner sweeps over nF CTAs: seven (an 8-CTA cluster, two inner sweeps a CTA on
    // their own SMSPs) while every cluster of the launch fits on the GPU at once; else three, so
    // that twice as many matrices run side by side
    int nF = njobs * 8 <= sm_count() ? 7 : 3;
    int rows_per = (L0.K + nF - 1) / nF;
    while (BjLayout(kmax, rows_per).f_bytes > (size_t)cap && nF < 7) rows_per = (L0.K + ++nF - 1) / nF;
    const BjLayout L1(kmax, rows_per);
    if (L1.f_bytes > (size_t)cap) return cudaErrorInvalidValue;
    const size_t smem = std::max(L1.e_bytes, L1.f_bytes);
    cudaError_t e = grow_smem((const void*)k_jacobi_blk, smem);
    if (e != cudaSuccess) return e;
    std::vector<DfMode> hm(njobs);
    for (int m = 0; m < njobs; ++m) {
        const DfJob& J = jobs[m];
        hm[m] = DfMode{J.H, J.outD, J.outF, J.st, J.ldd, J.k, J.add_identity, J.abs_floor, J.tau, J.tol};
    }
    DfMode* dm = nullptr;
    e = cudaMallocAsync(&dm, sizeof(DfMode) * njobs, st);
    if (e != cudaSuccess) return e;
    e = upload_h2d(dm, hm.data(), sizeof(DfMode) * njobs, st);
    if (e == cudaSuccess) {
        const int cs = 1 + nF;
        BjArgs a{dm, max_sweeps > 63 ? 63 : max_sweeps, cs, rows_per};
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3((unsigned)(njobs * cs));
        cfg.blockDim = dim3(kBlkThreads);
        cfg.dynamicSmemBytes = smem;
        cfg.stream = st;
        cudaLaunchAttribute attr[1];
        attr[0].id = cudaLaunchAttributeClusterDimension;
        attr[0].val.clusterDim.x = (unsigned)cs;
        attr[0].val.clusterDim.y = 1;
        attr[0].val.clusterDim.z = 1;
        cfg.attrs = attr;
        cfg.numAttrs = 1;
        count_kernels(1);
        e = cudaLaunchKernelEx(&cfg, k_jacobi_blk, a);
    }
    cudaFreeAsync(dm, st);
    return e;
}

// The grid block form: every job of the launch in one cooperative grid, the
// matrices in global memory (any k). Jobs beyond kGbMaxModes run in further launches.
cudaError_t launch_jacobi_gblk(const DfJob* jobs, int njobs, int max_sweeps, int num_sms, cudaStream_t st) {
    for (int j0 = 0; j0 < njobs; j0 += kGbMaxModes) {
        const int nm = std::min(kGbMaxModes, njobs - j0);
        std::vector<GbMode> hm(nm);
        std::vector<size_t> off(nm);
        const size_t st_bytes = (sizeof(DevStatus) + 255) / 256 * 256;
        size_t total = st_bytes;   // barrier status first
        auto carve = [&](size_t bytes) {
            const size_t o = total;
            total += (bytes + 255) / 256 * 256;
            return o;
        };
        struct Offs { size_t D, E, F, Q, act, cnt; };
        std::vector<Offs> of(nm);
        for (int i = 0; i < nm; ++i) {
            const DfJob& J = jobs[j0 + i];
            int m = (J.k + BJ - 1) / BJ;
            m += m & 1;
            if (m < 2) m = 2;
            const int K = m * BJ, ldE = K + 4, nb = m / 2;
            of[i] = Offs{carve(sizeof(DF) * (size_t)K), carve(3 * 4 * (size_t)K * ldE), carve(4 * (size_t)K * K),
                         carve(2 * 4 * (size_t)nb * BJ2SQ), carve(2 * 4 * (size_t)nb), carve(16)};
            hm[i] = GbMode{J.H, J.outD, J.outF, J.st, J.ldd, J.k, J.add_identity,
                           (float)J.abs_floor, (float)J.tau, (float)(J.tol * J.tol), K, ldE, nb, m,
                           nullptr, nullptr, nullptr, nullptr, nullptr, nullptr};
        }
        const size_t modes_at = carve(sizeof(GbMode) * nm);
        unsigned char* ws = nullptr;
        cudaError_t e = cudaMallocAsync(&ws, total, st);
        if (e != cudaSuccess) return e;
        for (int i = 0; i < nm; ++i) {
            hm[i].D = reinterpret_cast<DF*>(ws + of[i].D);
            hm[i].E = reinterpret_cast<float*>(ws + of[i].E);
            hm[i].F = reinterpret_cast<float*>(ws + of[i].F);
            hm[i].Q = reinterpret_cast<float*>(ws + of[i].Q);
            hm[i].act = reinterpret_cast<int*>(ws + of[i].act);
            hm[i].cnt = reinterpret_cast<unsigned int*>(ws + of[i].cnt);
        }
        e = cudaMemsetAsync(ws, 0, st_bytes, st);
        if (e == cudaSuccess)
            e = upload_h2d(ws + modes_at, hm.data(), sizeof(GbMode) * nm, st);
        // 96 KB of staging, then the job descriptors
        const size_t smem = (size_t)(kGbThreads / 16) * 3 * BJ2SQ * sizeof(float) + sizeof(GbMode) * nm;
        int per_sm = 0;
        if (e == cudaSuccess) e = grow_smem((const void*)k_jacobi_gblk, smem);
        if (e == cudaSuccess) e = blocks_per_sm((const void*)k_jacobi_gblk, kGbThreads, smem, &per_sm);
        if (e == cudaSuccess && per_sm < 1) e = cudaErrorInvalidConfiguration;
        if (e == cudaSuccess) {
            GbArgs a{reinterpret_cast<const GbMode*>(ws + modes_at), nm, max_sweeps > 63 ? 63 : max_sweeps,
                     reinterpret_cast<DevStatus*>(ws)};
            void* args[] = {&a};
            count_kernels(1);
            e = cudaLaunchCooperativeKernel((void*)k_jacobi_gblk, dim3((unsigned)std::max(1, num_sms)),
                                            dim3(kGbThreads), args, smem, st);
        }
        cudaFreeAsync(ws, st);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

}  // namespace ls
