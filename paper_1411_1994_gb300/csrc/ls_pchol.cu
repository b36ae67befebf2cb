// Pivoted Cholesky of the weighted Gram matrix (the compression that precedes
// the eigen-solver of the truncation step, Thm 2.1 / Algorithm 1), held in
// shared memory by one thread-block cluster per matrix: CTA r owns rows
// [r0, r1) of G and of L and their residual diagonal d. Per step every CTA
// reduces the published (max d, argmax, sum d) candidates of all CTAs in the
// same order, reads row p of L from its owner's shared memory, computes its
// rows of the new column l_j = (G_jp - L_j . L_p) / sqrt(d_p) (FP64; each
// dot product in four quarters, one per warp, so that the four SMSPs' FP64
// units share the work, added in a fixed order), updates d and publishes its
// next candidate into every CTA's shared
// memory (double-buffered by step parity): one cluster barrier per step and no
// global-memory traffic inside the loop. Greedy diagonal pivoting with ties to
// the smaller index; the iteration stops when the remaining trace is <= delta
// or after kmax columns, as the grid form in ls_f64.cu does.
#include <cooperative_groups.h>

#include <algorithm>
#include <map>
#include <mutex>

#include "ls_common.cuh"

namespace cg = cooperative_groups;

namespace ls {

namespace {

constexpr int kPcThreads = 128;   // four warps: the quarters of each dot product

static_assert(kPcThreads == 128, "the row dot products are split over exactly four warps");
// rows a thread of the panel kernel finishes (its rows' column of S waits in registers): the
// launcher takes at most kCpRowsPerThread * kPcThreads rows a CTA
constexpr int kCpRowsPerThread = 4;

struct PcMode {
    const double* G; double* L; double* resid; int* piv; DevStatus* st; int C; int kmax; double delta;
};
struct PcArgs {
    const PcMode* m; int cs; int rows_per;
};
struct Cand {
    double sum, mx;   // sum of d, max d (exact)
    long long key;    // order of (max d, -index): see cand_key
    long long pad;
};

// (max d, smallest index among near-equal maxima) as one integer: FP64 on this
// part has few lanes, so the arg-max runs on the integer pipe (d >= 0 orders
// like its bits); the low 24 mantissa bits give way to the index, so maxima
// within 2^-28 relative go to the smaller index. The pivot's exact value
// travels with the key.
__device__ __forceinline__ unsigned long long cand_key(double v, int ix) {
    const unsigned long long b = (unsigned long long)__double_as_longlong(v);
    return (b & ~0xffffffull) | (unsigned long long)(0xffffff - ix);   // low 24 bits: index, smaller wins
}

__global__ void __launch_bounds__(kPcThreads) k_pchol_cluster(PcArgs A) {
    cg::cluster_group cl = cg::this_cluster();
    const int rank = (int)cl.block_rank();
    const PcMode J = A.m[blockIdx.x / A.cs];
    const int C = J.C, kmax = J.kmax, rp = A.rows_per;
    // odd row strides: the threads of a step read one column across their rows
    const int ldG = C | 1, ldL = kmax | 1;
    const int r0 = min(C, rank * rp), r1 = min(C, r0 + rp), nr = r1 - r0;
    extern __shared__ __align__(16) unsigned char smem[];
    double* Gs = reinterpret_cast<double*>(smem);                 // [rp][ldG]
    double* Ls = Gs + (size_t)rp * ldG;                           // [rp][ldL]
    double* d = Ls + (size_t)rp * ldL;                            // [rp]
    double* lrow = d + rp;                                        // [kmax]
    double* part = lrow + kmax;                                   // [4][rp] quarter sums
    Cand* cand = reinterpret_cast<Cand*>(part + 4 * (size_t)rp);  // [2][cs]
    __shared__ double s_dmax, s_sum, s_inv;
    __shared__ int s_p;
    const int tid = threadIdx.x, nthr = blockDim.x;
    const int warp = tid >> 5, lane = tid & 31;

    for (int e = tid; e < nr * C; e += nthr) {
        const int jl = e / C, c = e - jl * C;
        Gs[(size_t)jl * ldG + c] = J.G[(int64_t)r0 * C + e];
    }
    __syncthreads();
    for (int jl = tid; jl < nr; jl += nthr) d[jl] = Gs[(size_t)jl * ldG + r0 + jl];
    __syncthreads();
    // this CTA's candidate (warp 0): the arg-max by integer keys, the sum by a butterfly
    auto publish = [&](int parity) {
        if (warp != 0) return;
        unsigned long long key = 0;
        double sm = 0.0, mx = 0.0;
        for (int jl = lane; jl < nr; jl += 32) {
            const double v = d[jl];
            sm += v;
            const unsigned long long kk = cand_key(v, r0 + jl);
            if (kk > key) { key = kk; mx = v; }
        }
        for (int o = 16; o; o >>= 1) {
            const unsigned long long k2 = __shfl_xor_sync(0xffffffffu, key, o);
            const double m2 = __shfl_xor_sync(0xffffffffu, mx, o);
            if (k2 > key) { key = k2; mx = m2; }
            sm += __shfl_xor_sync(0xffffffffu, sm, o);
        }
        if (lane < A.cs) cl.map_shared_rank(cand, lane)[parity * A.cs + rank] = Cand{sm, mx, (long long)key, 0};
    };
    publish(0);
    cl.sync();
    int k = 0;
    double sum = 0.0;
    for (;; ++k) {
        const int par = k & 1;
        // every CTA reduces the candidates of all CTAs in rank order
        if (warp == 0) {
            unsigned long long key = 0;
            double sm = 0.0, mx = 0.0;
            if (lane < A.cs) {
                const Cand c = cand[par * A.cs + lane];
                key = (unsigned long long)c.key;
                sm = c.sum;
                mx = c.mx;
            }
            for (int o = 16; o; o >>= 1) {
                const unsigned long long k2 = __shfl_xor_sync(0xffffffffu, key, o);
                const double m2 = __shfl_xor_sync(0xffffffffu, mx, o);
                if (k2 > key) { key = k2; mx = m2; }
                sm += __shfl_xor_sync(0xffffffffu, sm, o);
            }
            if (lane == 0) {
                s_p = key == 0 ? -1 : 0xffffff - (int)(key & 0xffffffull);
                s_dmax = key == 0 ? 0.0 : mx;
                s_sum = sm;
                s_inv = mx > 0.0 ? 1.0 / sqrt(mx) : 0.0;   // once, not in every thread
            }
        }
        __syncthreads();
        const double dmax = s_dmax;
        const int p = s_p;
        sum = s_sum;
        if (k >= kmax || !(sum > J.delta) || p < 0 || !(dmax > 0.0)) break;
        // row p of L (columns 0..k-1) from its owner
        {
            const int owner = p / rp;
            const double* src = cl.map_shared_rank(Ls, owner) + (size_t)(p - owner * rp) * ldL;
            for (int t = tid; t < k; t += nthr) lrow[t] = src[t];
        }
        __syncthreads();
        const double inv = s_inv;
        // L_j . L_p in quarters of the k range, warp w the w-th quarter of every row (a thread
        // per row), two partial sums a thread
        {
            const int qlen = (k + 3) >> 2, t0 = min(k, warp * qlen), t1 = min(k, t0 + qlen);
            for (int jl = lane; jl < nr; jl += 32) {
                const double* lj = Ls + (size_t)jl * ldL;
                double a0 = 0.0, a1 = 0.0;
                int t = t0;
                for (; t + 1 < t1; t += 2) {
                    a0 = fma(lj[t], lrow[t], a0);
                    a1 = fma(lj[t + 1], lrow[t + 1], a1);
                }
                if (t < t1) a0 = fma(lj[t], lrow[t], a0);
                part[warp * rp + jl] = a0 + a1;
            }
        }
        __syncthreads();
        // l_j = (G_jp - L_j . L_p) / sqrt(d_p), the quarters added in order
        for (int jl = tid; jl < nr; jl += nthr) {
            const double dot = ((part[jl] + part[rp + jl]) + part[2 * rp + jl]) + part[3 * rp + jl];
            const double l = (Gs[(size_t)jl * ldG + p] - dot) * inv;
            Ls[(size_t)jl * ldL + k] = l;
            d[jl] = (r0 + jl == p) ? 0.0 : fmax(d[jl] - l * l, 0.0);
        }
        if (rank == 0 && tid == 0) J.piv[k] = p;
        __syncthreads();
        publish(par ^ 1);
        cl.sync();
    }
    // L rows to global memory (C x kmax, row-major; columns k.. are not used)
    for (int e = tid; e < nr * k; e += nthr) {
        const int jl = e / k, t = e - jl * k;
        J.L[(int64_t)(r0 + jl) * kmax + t] = Ls[(size_t)jl * ldL + t];
    }
    if (rank == 0 && tid == 0) {
        J.st->sweeps = k;
        *J.resid = sum;
    }
    cl.sync();
}

// ---------------------------------------------------------------------------
// The panel form for matrices whose rows of G do not fit a cluster: one
// cluster per matrix continues the factorisation at column k0 = st->sweeps,
// with S = G - L[:, :k0] L[:, :k0]^T in global memory (the Schur complement the
// caller's tensor-core product formed after the previous panel), and takes up
// to pw pivots. CTA r keeps its rows' residual diagonal and their entries of
// the panel's columns in shared memory; column p of S comes from global memory
// (one round trip a step), row p of the panel from its owner's shared memory.
// The panel's columns also go to Lp (C x pw, zero past the last pivot taken,
// zero throughout once the factorisation has ended), so that the caller can
// queue the Schur update S -= Lp Lp^T without a read-back. The same steps,
// candidate keys and quarter sums as the whole-matrix kernel above.
// ---------------------------------------------------------------------------
struct CpMode {
    const double* S; double* L; double* Lp; double* d; double* resid; int* piv; DevStatus* st; int C; int kmax;
    double delta;
};
struct CpArgs {
    const CpMode* m; int cs; int rows_per; int pw;
};

__global__ void __launch_bounds__(kPcThreads) k_pchol_cpanel(CpArgs A) {
    cg::cluster_group cl = cg::this_cluster();
    const int rank = (int)cl.block_rank();
    const CpMode J = A.m[blockIdx.x / A.cs];
    const int C = J.C, kmax = J.kmax, rp = A.rows_per, pw = A.pw;
    const int ldL = pw | 1;
    const int r0 = min(C, rank * rp), r1 = min(C, r0 + rp), nr = r1 - r0;
    const int tid = threadIdx.x, nthr = blockDim.x;
    const int warp = tid >> 5, lane = tid & 31;
    // where the previous panel left the factorisation (every CTA reads the same words)
    const int k0 = *(volatile int*)&J.st->sweeps;
    if (*(volatile int*)&J.st->done || k0 >= kmax) {
        for (int64_t e = tid; e < (int64_t)nr * pw; e += nthr) J.Lp[(int64_t)r0 * pw + e] = 0.0;
        if (rank == 0 && tid == 0) J.st->done = 1;
        return;   // every CTA of the cluster leaves here: no cluster barrier is pending
    }
    const int kend = min(kmax, k0 + pw);
    extern __shared__ __align__(16) unsigned char smem[];
    double* Ls = reinterpret_cast<double*>(smem);                 // [rp][ldL] the panel's columns
    double* d = Ls + (size_t)rp * ldL;                            // [rp]
    double* lrow = d + rp;                                        // [pw]
    double* part = lrow + pw;                                     // [4][rp] quarter sums
    Cand* cand = reinterpret_cast<Cand*>(part + 4 * (size_t)rp);  // [2][cs]
    __shared__ double s_dmax, s_sum, s_inv;
    __shared__ int s_p;

    for (int jl = tid; jl < nr; jl += nthr)
        d[jl] = k0 == 0 ? J.S[(int64_t)(r0 + jl) * C + r0 + jl] : J.d[r0 + jl];
    __syncthreads();
    auto publish = [&](int parity) {
        if (warp != 0) return;
        unsigned long long key = 0;
        double sm = 0.0, mx = 0.0;
        for (int jl = lane; jl < nr; jl += 32) {
            const double v = d[jl];
            sm += v;
            const unsigned long long kk = cand_key(v, r0 + jl);
            if (kk > key) { key = kk; mx = v; }
        }
        for (int o = 16; o; o >>= 1) {
            const unsigned long long k2 = __shfl_xor_sync(0xffffffffu, key, o);
            const double m2 = __shfl_xor_sync(0xffffffffu, mx, o);
            if (k2 > key) { key = k2; mx = m2; }
            sm += __shfl_xor_sync(0xffffffffu, sm, o);
        }
        if (lane < A.cs) cl.map_shared_rank(cand, lane)[parity * A.cs + rank] = Cand{sm, mx, (long long)key, 0};
    };
    publish(0);
    cl.sync();
    int k = k0;
    bool done = false;
    double sum = 0.0;
    for (;; ++k) {
        const int par = (k - k0) & 1;
        if (warp == 0) {
            unsigned long long key = 0;
            double sm = 0.0, mx = 0.0;
            if (lane < A.cs) {
                const Cand c = cand[par * A.cs + lane];
                key = (unsigned long long)c.key;
                sm = c.sum;
                mx = c.mx;
            }
            for (int o = 16; o; o >>= 1) {
                const unsigned long long k2 = __shfl_xor_sync(0xffffffffu, key, o);
                const double m2 = __shfl_xor_sync(0xffffffffu, mx, o);
                if (k2 > key) { key = k2; mx = m2; }
                sm += __shfl_xor_sync(0xffffffffu, sm, o);
            }
            if (lane == 0) {
                s_p = key == 0 ? -1 : 0xffffff - (int)(key & 0xffffffull);
                s_dmax = key == 0 ? 0.0 : mx;
                s_sum = sm;
                s_inv = mx > 0.0 ? 1.0 / sqrt(mx) : 0.0;
            }
        }
        __syncthreads();
        const double dmax = s_dmax;
        const int p = s_p;
        sum = s_sum;
        if (k >= kmax || !(sum > J.delta) || p < 0 || !(dmax > 0.0)) {
            done = true;
            break;
        }
        if (k >= kend) break;
        const int kk = k - k0;
        // column p of S for the own rows, into registers: S[j][p] from S's upper triangle (the
        // Schur updates leave the lower one behind); its trip to L2 runs beside the dot products,
        // and the thread that loads row jl is the one that finishes it below
        double gc[kCpRowsPerThread];
#pragma unroll
        for (int u = 0; u < kCpRowsPerThread; ++u) {
            const int jl = tid + u * kPcThreads, j = r0 + jl;
            gc[u] = jl < nr ? __ldcg(J.S + (j < p ? (int64_t)j * C + p : (int64_t)p * C + j)) : 0.0;
        }
        // the panel part of row p from its owner
        {
            const int owner = p / rp;
            const double* src = cl.map_shared_rank(Ls, owner) + (size_t)(p - owner * rp) * ldL;
            for (int t = tid; t < kk; t += nthr) lrow[t] = src[t];
        }
        __syncthreads();
        const double inv = s_inv;
        {
            const int qlen = (kk + 3) >> 2, t0 = min(kk, warp * qlen), t1 = min(kk, t0 + qlen);
            for (int jl = lane; jl < nr; jl += 32) {
                const double* lj = Ls + (size_t)jl * ldL;
                double a0 = 0.0, a1 = 0.0;
                int t = t0;
                for (; t + 1 < t1; t += 2) {
                    a0 = fma(lj[t], lrow[t], a0);
                    a1 = fma(lj[t + 1], lrow[t + 1], a1);
                }
                if (t < t1) a0 = fma(lj[t], lrow[t], a0);
                part[warp * rp + jl] = a0 + a1;
            }
        }
        __syncthreads();
#pragma unroll
        for (int u = 0; u < kCpRowsPerThread; ++u) {
            const int jl = tid + u * kPcThreads;
            if (jl >= nr) break;
            const double dot = ((part[jl] + part[rp + jl]) + part[2 * rp + jl]) + part[3 * rp + jl];
            const double l = (gc[u] - dot) * inv;
            Ls[(size_t)jl * ldL + kk] = l;
            __stcg(J.L + (int64_t)(r0 + jl) * kmax + k, l);
            __stcg(J.Lp + (int64_t)(r0 + jl) * pw + kk, l);
            d[jl] = (r0 + jl == p) ? 0.0 : fmax(d[jl] - l * l, 0.0);
        }
        if (rank == 0 && tid == 0) J.piv[k] = p;
        __syncthreads();
        publish(par ^ 1);
        cl.sync();
    }
    for (int jl = tid; jl < nr; jl += nthr) J.d[r0 + jl] = d[jl];
    // the panel's columns past the last pivot taken are zero
    const int taken = k - k0;
    for (int64_t e = tid; e < (int64_t)nr * (pw - taken); e += nthr) {
        const int64_t jl = e / (pw - taken), t = taken + e % (pw - taken);
        J.Lp[(r0 + jl) * pw + t] = 0.0;
    }
    if (rank == 0 && tid == 0) {
        J.st->sweeps = k;
        J.st->done = done ? 1 : 0;
        *J.resid = sum;
    }
    cl.sync();
}

size_t cp_smem(int cs, int rp, int pw) {
    return 8 * ((size_t)rp * (pw | 1) + rp + pw + 4 * (size_t)rp) + sizeof(Cand) * 2 * (size_t)cs;
}

size_t pc_smem(int C, int kmax, int cs, int rp) {
    return 8 * ((size_t)rp * (C | 1) + (size_t)rp * (kmax | 1) + rp + kmax + 4 * (size_t)rp) + sizeof(Cand) * 2 * (size_t)cs;
}

int sm_count_pc() {
    static const int n = [] {
        int dev = 0, v = 0;
        if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
            return 1;
        return std::max(1, v);
    }();
    return n;
}

int smem_cap() {
    int dev = 0, v = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return 0;
    if (cudaDeviceGetAttribute(&v, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess) return 0;
    return std::max(0, v - 1024);
}

// The kernel's attributes are set once, and its dynamic shared memory only when a launch
// needs more than before; whether a 16-CTA cluster fits one GPC is asked once per shared-
// memory size. (These driver calls cost tens of microseconds of host time each, inside
// every reduction otherwise.)
std::mutex g_pc_mu;
cudaError_t allow_cluster16() {
    static cudaError_t e = cudaFuncSetAttribute(k_pchol_cluster, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    return e;
}
cudaError_t reserve_smem(size_t bytes) {
    static size_t done = 0;
    std::lock_guard<std::mutex> g(g_pc_mu);
    if (bytes <= done) return cudaSuccess;
    const cudaError_t e = cudaFuncSetAttribute(k_pchol_cluster, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    if (e == cudaSuccess) done = bytes;
    return e;
}
bool cluster16_fits(cudaLaunchConfig_t cfg) {
    static std::map<size_t, bool> known;
    std::lock_guard<std::mutex> g(g_pc_mu);
    const auto it = known.find(cfg.dynamicSmemBytes);
    if (it != known.end()) return it->second;
    int nclusters = 0;
    cfg.gridDim = dim3(16);
    const bool ok = cudaOccupancyMaxActiveClusters(&nclusters, k_pchol_cluster, &cfg) == cudaSuccess && nclusters >= 1;
    if (!ok) cudaGetLastError();
    known[cfg.dynamicSmemBytes] = ok;
    return ok;
}


// the panel kernel's attributes, as for the whole-matrix kernel
cudaError_t cp_allow_cluster16() {
    static cudaError_t e = cudaFuncSetAttribute(k_pchol_cpanel, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    return e;
}
cudaError_t cp_reserve_smem(size_t bytes) {
    static size_t done = 0;
    std::lock_guard<std::mutex> g(g_pc_mu);
    if (bytes <= done) return cudaSuccess;
    const cudaError_t e = cudaFuncSetAttribute(k_pchol_cpanel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    if (e == cudaSuccess) done = bytes;
    return e;
}
bool cp_cluster16_fits(cudaLaunchConfig_t cfg) {
    static std::map<size_t, bool> known;
    std::lock_guard<std::mutex> g(g_pc_mu);
    const auto it = known.find(cfg.dynamicSmemBytes);
    if (it != known.end()) return it->second;
    int nclusters = 0;
    cfg.gridDim = dim3(16);
    const bool ok = cudaOccupancyMaxActiveClusters(&nclusters, k_pchol_cpanel, &cfg) == cudaSuccess && nclusters >= 1;
    if (!ok) cudaGetLastError();
    known[cfg.dynamicSmemBytes] = ok;
    return ok;
}
// (columns so far, done) of every job of a panel launch, for the caller's one read-back
__global__ void k_cpanel_report(const CpMode* m, int n, int* out) {
    for (int j = threadIdx.x; j < n; j += blockDim.x) {
        out[2 * j] = m[j].st->sweeps;
        out[2 * j + 1] = m[j].st->done;
    }
}

}  // namespace

// largest cluster (16, else 8) whose CTAs can hold rows of G and L for C, kmax
int pchol_cluster_size(int C, int kmax) {
    const size_t cap = (size_t)smem_cap();
    for (int cs : {16, 8}) {
        const int rp = (C + cs - 1) / cs;
        if (pc_smem(C, kmax, cs, rp) <= cap) return cs;
    }
    return 0;
}

cudaError_t launch_pchol_cluster(const PcholJob* jobs, int njobs, cudaStream_t st) {
    if (njobs < 1) return cudaSuccess;
    int Cmax = 1, kmaxm = 1;
    for (int m = 0; m < njobs; ++m) {
        Cmax = std::max<int>(Cmax, (int)jobs[m].C);
        kmaxm = std::max(kmaxm, jobs[m].kmax);
    }
    int cs = pchol_cluster_size(Cmax, kmaxm);
    if (cs == 0) return cudaErrorInvalidValue;
    cudaError_t e;
    if (cs > 8 && (e = allow_cluster16()) != cudaSuccess) return e;
    size_t smem = pc_smem(Cmax, kmaxm, cs, (Cmax + cs - 1) / cs);
    if ((e = reserve_smem(smem)) != cudaSuccess) return e;
    cudaLaunchConfig_t cfg = {};
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = (unsigned)cs;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.blockDim = dim3(kPcThreads);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    // a 16-CTA cluster must fit one GPC: fall back to 8 where it does not
    if (cs > 8 && !cluster16_fits(cfg)) {
        cs = 8;
        smem = pc_smem(Cmax, kmaxm, cs, (Cmax + cs - 1) / cs);
        if (smem > (size_t)smem_cap()) return cudaErrorInvalidValue;
        if ((e = reserve_smem(smem)) != cudaSuccess) return e;
        attr[0].val.clusterDim.x = 8;
    }
    const int rp2 = (Cmax + cs - 1) / cs;
    cfg.dynamicSmemBytes = pc_smem(Cmax, kmaxm, cs, rp2);
    std::vector<PcMode> hm(njobs);
    for (int m = 0; m < njobs; ++m) {
        const PcholJob& J = jobs[m];
        hm[m] = PcMode{J.G, J.L, J.cand + kPcholCand - 1, J.piv, J.st, (int)J.C, J.kmax, J.delta};
    }
    PcMode* dm = nullptr;
    e = cudaMallocAsync(&dm, sizeof(PcMode) * njobs, st);
    if (e != cudaSuccess) return e;
    e = upload_h2d(dm, hm.data(), sizeof(PcMode) * njobs, st);
    if (e == cudaSuccess) {
        PcArgs a{dm, cs, rp2};
        cfg.gridDim = dim3((unsigned)(njobs * cs));
        count_kernels(1);
        e = cudaLaunchKernelEx(&cfg, k_pchol_cluster, a);
    }
    cudaFreeAsync(dm, st);
    return e;
}

// whether the panel form's clusters (16 CTAs, else 8) hold every job's rows for this panel width
bool pchol_cpanel_fits(int64_t Cmax, int panel) {
    const size_t cap = (size_t)smem_cap();
    return cp_smem(8, (int)((Cmax + 7) / 8), panel) <= cap && (Cmax + 7) / 8 <= kCpRowsPerThread * kPcThreads;
}

cudaError_t launch_pchol_cpanel(const PcholJob* jobs, int panel, int njobs, int* d_report, cudaStream_t st) {
    if (njobs < 1) return cudaSuccess;
    int64_t Cmax = 1;
    for (int m = 0; m < njobs; ++m) {
        Cmax = std::max<int64_t>(Cmax, jobs[m].C);
        if (!jobs[m].Lp) return cudaErrorInvalidValue;
    }
    const size_t cap = (size_t)smem_cap();
    // 16 CTAs a matrix while the clusters of the launch fit the GPU side by side, else 8
    int cs = (njobs * 16 <= sm_count_pc() && cp_smem(16, (int)((Cmax + 15) / 16), panel) <= cap) ? 16 : 8;
    if (cp_smem(cs, (int)((Cmax + cs - 1) / cs), panel) > cap) return cudaErrorInvalidValue;
    cudaError_t e;
    if (cs > 8 && (e = cp_allow_cluster16()) != cudaSuccess) return e;
    cudaLaunchConfig_t cfg = {};
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = (unsigned)cs;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.blockDim = dim3(kPcThreads);
    cfg.dynamicSmemBytes = cp_smem(cs, (int)((Cmax + cs - 1) / cs), panel);
    cfg.stream = st;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    if ((e = cp_reserve_smem(cfg.dynamicSmemBytes)) != cudaSuccess) return e;
    // a 16-CTA cluster must fit one GPC: fall back to 8 where it does not
    if (cs > 8 && !cp_cluster16_fits(cfg)) {
        cs = 8;
        attr[0].val.clusterDim.x = 8;
        cfg.dynamicSmemBytes = cp_smem(cs, (int)((Cmax + cs - 1) / cs), panel);
        if ((e = cp_reserve_smem(cfg.dynamicSmemBytes)) != cudaSuccess) return e;
    }
    const int rp = (int)((Cmax + cs - 1) / cs);
    if (rp > kCpRowsPerThread * kPcThreads) return cudaErrorInvalidValue;
    std::vector<CpMode> hm(njobs);
    for (int m = 0; m < njobs; ++m) {
        const PcholJob& J = jobs[m];
        hm[m] = CpMode{J.G, J.L, J.Lp, J.d, J.cand + kPcholCand - 1, J.piv, J.st, (int)J.C, J.kmax, J.delta};
    }
    CpMode* dm = nullptr;
    e = cudaMallocAsync(&dm, sizeof(CpMode) * njobs, st);
    if (e != cudaSuccess) return e;
    e = upload_h2d(dm, hm.data(), sizeof(CpMode) * njobs, st);
    if (e == cudaSuccess) {
        CpArgs a{dm, cs, rp, panel};
        cfg.gridDim = dim3((unsigned)(njobs * cs));
        count_kernels(1);
        e = cudaLaunchKernelEx(&cfg, k_pchol_cpanel, a);
    }
    if (e == cudaSuccess && d_report) {
        k_cpanel_report<<<1, 128, 0, st>>>(dm, njobs, d_report);
        count_kernels(1);
        e = cudaGetLastError();
    }
    cudaFreeAsync(dm, st);
    return e;
}

}  // namespace ls
