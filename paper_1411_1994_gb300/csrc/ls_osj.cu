// One-sided (Hestenes) Jacobi in FP64 and the elementwise steps of the
// reduction's non-squaring singular-value route.
//
// Def. 4.1 truncates each side matrix by its singular values. The Gram route
// (eigenvalues of A^T A) squares them, so values below about sqrt(u) sigma_1
// drown in the Gram matrix's rounding. The FP64 path therefore takes the
// singular values and the final rotation from B = Q^T A_w, with Q an
// orthonormal basis of the side matrix's range found by two deflated Gram
// passes, by one-sided Jacobi on the rows of B: plane rotations of pairs of
// rows, applied to B and accumulated in M, until every pair of rows is
// orthogonal to within tol. The rotations never form B B^T, so each singular
// value keeps the relative accuracy of its row (Demmel & Veselic, SIAM J.
// Matrix Anal. Appl. 13 (1992)); B starts close to row-orthogonal (Q comes
// from the Gram eigenvectors), so two or three sweeps suffice.
//
// Parallel ordering: the round-robin tournament (pairs (m'-1, t) and
// ((t+i) mod (m'-1), (t-i) mod (m'-1))), m'/2 disjoint pairs a round, m'-1
// rounds a sweep, m' = m rounded up to even (the extra index is idle). One
// warp per pair; one cooperative grid for up to three matrices, CTAs split
// between them, with a bounded group barrier after every round.
#include <algorithm>
#include <vector>

#include "ls_common.cuh"
#include "ls_grid.cuh"

namespace ls {
namespace {

constexpr int kOsjThreads = 256;
constexpr int kOsjWarps = kOsjThreads / 32;
constexpr int kOsjMaxJobs = 3;
constexpr float kCosDone = 1e-9f;

struct OsjMode {
    double* B; int64_t ldb; int C; double* M; int m; double* sig2; DevStatus* st; double tol; unsigned* cmax;
    int cta0, ncta;
};
struct OsjArgs {
    OsjMode j[kOsjMaxJobs];
    int n;
    int max_sweeps;
};

__device__ __forceinline__ void tour_pair(int t, int i, int mp, int& p, int& q) {
    const int n1 = mp - 1;
    int a, b;
    if (i == 0) { a = n1; b = t; }
    else { a = (t + i) % n1; b = (t - i + n1) % n1; }
    p = min(a, b);
    q = max(a, b);
}

__device__ __forceinline__ double warp_sum(double v) {
    for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

__global__ void __launch_bounds__(kOsjThreads) k_osj(const __grid_constant__ OsjArgs A) {
    int ji = 0;
    while (ji + 1 < A.n && (int)blockIdx.x >= A.j[ji + 1].cta0) ++ji;
    const OsjMode& J = A.j[ji];
    const int cb = (int)blockIdx.x - J.cta0;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int gw = cb * kOsjWarps + warp, nw = J.ncta * kOsjWarps;
    const int m = J.m, C = J.C, mp = m + (m & 1);
    const unsigned nb = (unsigned)J.ncta;
    __shared__ int s_rot;
    __shared__ unsigned s_cmax;
    // M = I
    for (int64_t e = (int64_t)cb * kOsjThreads + threadIdx.x; e < (int64_t)m * m; e += (int64_t)nb * kOsjThreads)
        __stcg(J.M + e, (e / m == e % m) ? 1.0 : 0.0);
    if (!group_barrier(J.st, nb)) return;
    int sweeps = 0;
    bool converged = m < 2;
    for (int s = 0; s < A.max_sweeps && !converged; ++s) {
        if (threadIdx.x == 0) { s_rot = 0; s_cmax = 0u; }
        __syncthreads();
        for (int t = 0; t < mp - 1; ++t) {
            for (int i = gw; i < mp / 2; i += nw) {
                int p, q;
                tour_pair(t, i, mp, p, q);
                if (q >= m) continue;   // the idle index of an odd m
                // rows written by other CTAs in earlier rounds: loads and stores go through L2
                // (__ldcg / __stcg), never a stale L1 line
                double* bp = J.B + (int64_t)p * J.ldb;
                double* bq = J.B + (int64_t)q * J.ldb;
                double a = 0.0, b = 0.0, g = 0.0;
#pragma unroll 8
                for (int k = lane; k < C; k += 32) {
                    const double x = __ldcg(bp + k), y = __ldcg(bq + k);
                    a = fma(x, x, a);
                    b = fma(y, y, b);
                    g = fma(x, y, g);
                }
                a = warp_sum(a);
                b = warp_sum(b);
                g = warp_sum(g);
                if (g == 0.0 || !(fabs(g) > J.tol * sqrt(a * b))) continue;
                // the largest |cos| of the sweep, as the bits of a positive float (they order alike)
                if (lane == 0) atomicMax(&s_cmax, __float_as_uint((float)(fabs(g) / sqrt(a * b))));
                // tan of the angle that makes rows p and q orthogonal (the smaller root)
                const double zeta = (b - a) / (2.0 * g);
                const double t_ = fabs(zeta) > 1e100 ? 0.5 / zeta
                                                     : copysign(1.0, zeta) / (fabs(zeta) + sqrt(1.0 + zeta * zeta));
                const double c = 1.0 / sqrt(1.0 + t_ * t_), sn = c * t_;
#pragma unroll 8
                for (int k = lane; k < C; k += 32) {
                    const double x = __ldcg(bp + k), y = __ldcg(bq + k);
                    __stcg(bp + k, fma(c, x, -sn * y));
                    __stcg(bq + k, fma(sn, x, c * y));
                }
                double* mpp = J.M + (int64_t)p * m;
                double* mq = J.M + (int64_t)q * m;
#pragma unroll 8
                for (int k = lane; k < m; k += 32) {
                    const double x = __ldcg(mpp + k), y = __ldcg(mq + k);
                    __stcg(mpp + k, fma(c, x, -sn * y));
                    __stcg(mq + k, fma(sn, x, c * y));
                }
                if (lane == 0) atomicAdd(&s_rot, 1);
            }
            if (t == mp - 2) {
                // this CTA's rotations of the sweep, before the sweep's last barrier
                __syncthreads();
                if (threadIdx.x == 0 && s_rot > 0) {
                    atomicAdd(&J.st->sweep_active[s < 64 ? s : 63], (unsigned)s_rot);
                    atomicMax(&J.cmax[s < 64 ? s : 63], s_cmax);
                }
            }
            if (!group_barrier(J.st, nb)) return;
        }
        sweeps = s + 1;
        // done after a sweep without rotations, or one whose largest |cos| was below kCosDone:
        // Jacobi converges quadratically, so the next sweep would find cosines of about
        // kCosDone^2, below the rounding of the dot products
        const unsigned cm = *(volatile unsigned*)&J.cmax[s < 64 ? s : 63];
        converged = *(volatile unsigned*)&J.st->sweep_active[s < 64 ? s : 63] == 0u ||
                    __uint_as_float(cm) < kCosDone;
    }
    // squared row norms: the squared singular values
    for (int i = gw; i < m; i += nw) {
        const double* bi = J.B + (int64_t)i * J.ldb;
        double a = 0.0;
        for (int k = lane; k < C; k += 32) {
            const double x = __ldcg(bi + k);
            a = fma(x, x, a);
        }
        a = warp_sum(a);
        if (lane == 0) J.sig2[i] = a;
    }
    if (cb == 0 && threadIdx.x == 0) {
        J.st->sweeps = sweeps;
        if (!converged) atomicCAS(&J.st->flag, FLAG_OK, FLAG_NOCONVERGE);
    }
}

__global__ void k_resid_rows(const double* __restrict__ A, const double* __restrict__ w, const double* __restrict__ D,
                             int64_t rows, int64_t N, double* __restrict__ E) {
    const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e >= rows * N) return;
    const int64_t c = e / N;
    E[e] = (w ? w[c] : 1.0) * A[e] - D[e];
}

__global__ void k_sub(double* __restrict__ Y, const double* __restrict__ D, int64_t n) {
    const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e < n) Y[e] -= D[e];
}

__global__ void k_gather_rows(const double* __restrict__ M, int64_t len, const int32_t* __restrict__ perm, int r,
                              const double* __restrict__ scale, double* __restrict__ out) {
    const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e >= (int64_t)r * len) return;
    const int j = (int)(e / len);
    const int64_t k = e - (int64_t)j * len;
    const double v = M[(int64_t)perm[j] * len + k];
    out[e] = scale ? v * scale[j] : v;
}

// Frobenius scaling of the Tucker side blocks: block j = rows [j w, (j + 1) w) of A (row
// length N); nrm[j] = its Frobenius norm, out = sqrt(mult[j]) / nrm[j] times the block
// (zero for a zero block). One CTA per block, fixed reduction order.
__global__ void __launch_bounds__(256) k_block_frob(const double* __restrict__ A, int w, int64_t N,
                                                    const double* __restrict__ mult, double* __restrict__ nrm,
                                                    double* __restrict__ out) {
    const int j = blockIdx.x;
    const double* a = A + (int64_t)j * w * N;
    const int64_t n = (int64_t)w * N;
    double acc = 0.0;
    for (int64_t e = threadIdx.x; e < n; e += blockDim.x) acc = fma(a[e], a[e], acc);
    __shared__ double red[8];
    acc = warp_sum(acc);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
    __syncthreads();
    __shared__ double s_f;
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int k = 0; k < 8; ++k) t += red[k];
        const double f = sqrt(t);
        nrm[j] = f;
        s_f = f > 0.0 ? sqrt(mult[j]) / f : 0.0;
    }
    __syncthreads();
    double* o = out + (int64_t)j * w * N;
    for (int64_t e = threadIdx.x; e < n; e += blockDim.x) o[e] = a[e] * s_f;
}

// out = sum_e x[e]^p, p = 2 or 3 (one CTA, fixed order)
__global__ void __launch_bounds__(256) k_sum_powers(const double* __restrict__ x, int64_t n, int p,
                                                    double* __restrict__ out) {
    double acc = 0.0;
    for (int64_t e = threadIdx.x; e < n; e += blockDim.x) acc = fma(p == 3 ? x[e] * x[e] : x[e], x[e], acc);
    __shared__ double red[8];
    acc = warp_sum(acc);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int k = 0; k < 8; ++k) t += red[k];
        *out = t;
    }
}

unsigned blocks_for(int64_t n) { return (unsigned)((n + 255) / 256); }

// The bounded group barrier on its own: a two-CTA cooperative grid in which CTA 1 arrives
// (absent = 0) or returns without arriving (absent = 1); CTA 0 waits with `limit` polls, so
// with an absent partner the wait runs out and raises FLAG_TIMEOUT instead of hanging.
__global__ void k_wait_probe(DevStatus* st, int absent, long long limit) {
    if (blockIdx.x == 1 && absent) return;
    group_barrier_n(st, 2u, limit);
}

}  // namespace

cudaError_t launch_osj(const OsjJob* jobs, int njobs, int max_sweeps, int num_sms, cudaStream_t st) {
    if (njobs < 1) return cudaSuccess;
    int per_sm = 0;
    if (blocks_per_sm((const void*)k_osj, kOsjThreads, 0, &per_sm) != cudaSuccess || per_sm < 1) per_sm = 1;
    const int resident = per_sm * num_sms;
    for (int j0 = 0; j0 < njobs; j0 += kOsjMaxJobs) {
        const int nj = std::min(kOsjMaxJobs, njobs - j0);
        // a warp per pair of a round, the CTAs of the launch within one wave
        std::vector<int> want(nj);
        int total = 0;
        for (int i = 0; i < nj; ++i) {
            const int m = jobs[j0 + i].m;
            want[i] = std::max(1, ((m + 1) / 2 + kOsjWarps - 1) / kOsjWarps);
            total += want[i];
        }
        // at most one CTA per SM in all (cheaper group barriers), split in proportion to the
        // pairs, at least one each: sum = nj + (cap - nj) at most
        const int cap = std::max(nj, std::min(resident, num_sms));
        OsjArgs a{};
        a.n = nj;
        a.max_sweeps = max_sweeps;
        int cta = 0;
        for (int i = 0; i < nj; ++i) {
            const OsjJob& J = jobs[j0 + i];
            int nc = want[i];
            if (total > cap)
                nc = 1 + (int)((int64_t)(want[i] - 1) * (cap - nj) / std::max(1, total - nj));
            a.j[i] = OsjMode{J.B, J.ldb, J.C, J.M, J.m, J.sig2, J.st, J.tol, J.cmax, cta, nc};
            cta += nc;
        }
        void* args[] = {&a};
        count_kernels(1);
        cudaError_t e = cudaLaunchCooperativeKernel((void*)k_osj, dim3(cta), dim3(kOsjThreads), args, 0, st);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

cudaError_t launch_wait_probe(DevStatus* st, int absent, long long limit, cudaStream_t stream) {
    void* args[] = {&st, &absent, &limit};
    count_kernels(1);
    return cudaLaunchCooperativeKernel((void*)k_wait_probe, dim3(2), dim3(32), args, 0, stream);
}

cudaError_t launch_resid_rows(const double* A, const double* w, const double* D, int64_t rows, int64_t N, double* E,
                              cudaStream_t st) {
    if (rows * N == 0) return cudaSuccess;
    k_resid_rows<<<blocks_for(rows * N), 256, 0, st>>>(A, w, D, rows, N, E);
    count_kernels(1);
    return cudaGetLastError();
}

cudaError_t launch_sub(double* Y, const double* D, int64_t n, cudaStream_t st) {
    if (n == 0) return cudaSuccess;
    k_sub<<<blocks_for(n), 256, 0, st>>>(Y, D, n);
    count_kernels(1);
    return cudaGetLastError();
}

cudaError_t launch_gather_rows(const double* M, int64_t len, const int32_t* perm, int r, const double* scale,
                               double* out, cudaStream_t st) {
    if ((int64_t)r * len == 0) return cudaSuccess;
    k_gather_rows<<<blocks_for((int64_t)r * len), 256, 0, st>>>(M, len, perm, r, scale, out);
    count_kernels(1);
    return cudaGetLastError();
}

cudaError_t launch_block_frob(const double* A, int w, int64_t N, int nblocks, const double* mult, double* nrm,
                              double* out, cudaStream_t st) {
    if (nblocks < 1) return cudaSuccess;
    k_block_frob<<<nblocks, 256, 0, st>>>(A, w, N, mult, nrm, out);
    count_kernels(1);
    return cudaGetLastError();
}

cudaError_t launch_sum_cubes(const double* x, int64_t n, double* out, cudaStream_t st) {
    k_sum_powers<<<1, 256, 0, st>>>(x, n, 3, out);
    count_kernels(1);
    return cudaGetLastError();
}

cudaError_t launch_sum_squares(const double* x, int64_t n, double* out, cudaStream_t st) {
    k_sum_powers<<<1, 256, 0, st>>>(x, n, 2, out);
    count_kernels(1);
    return cudaGetLastError();
}

}  // namespace ls
