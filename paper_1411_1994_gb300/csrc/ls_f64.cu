// FP64 kernels of the lattice-sum path (sm_103a).
//
// GB300 runs FP64 on CUDA cores at about 2 DFMA/clock/SM (~1.25 TFLOP/s for
// the whole GPU), ~58x below its FP32 rate. Every FP64 step here is written
// to spread over all SMs: the contractions use one register-blocked DFMA
// GEMM (64x64 tiles, 4x4 outputs per thread) with operand gathers done in
// the tile loaders, and the two inherently sequential algorithms (Jacobi
// eigen-solver, blocked Cholesky) run as cooperative grids with a bounded
// software grid barrier instead of one launch per step.
#include <math.h>

#include <algorithm>
#include <vector>

#include "ls_common.cuh"
#include "ls_grid.cuh"

namespace ls {

namespace {

// ---------------------------------------------------------------------------
// G0 / G1 / G2 and small elementwise kernels
// ---------------------------------------------------------------------------
// Gauss-Legendre rule on [-1, 1] for the Galerkin cell averages
constexpr int kGl = 24;
struct GlRule {
    double x[kGl], w[kGl];
};

__global__ void k_genvec(double* g, int R, int64_t N, double h, double sinc_step, double t_scale, int kernel,
                         double kappa, int galerkin, GlRule gl) {
    // the Newton kernel's nodes are q = 0..R-1; every other kernel's density vanishes at t = 0,
    // so its nodes are q = 1..R
    const bool newton = kernel == LS_KERNEL_YUKAWA && kappa == 0.0;
    const int row = blockIdx.y, q = row + (newton ? 0 : 1);
    const double u = q * sinc_step;
    const double t = sinh(u) / t_scale;
    const double spi = 1.7724538509055160273;   // sqrt(pi)
    double w;
    if (kernel == LS_KERNEL_SLATER) {
        // exp(-kappa r) = (kappa/sqrt(pi)) int t^-2 exp(-kappa^2/(4 t^2)) exp(-r^2 t^2) dt (Eq. LalpSlater)
        w = sinc_step * cosh(u) / t_scale * (kappa / spi) / (t * t) * exp(-kappa * kappa / (4.0 * t * t));
    } else if (kernel == LS_KERNEL_DIPOLE) {
        // 1/r^3 = (4/sqrt(pi)) int t^2 exp(-r^2 t^2) dt (Eq. LalpPoly at n = 3/2)
        w = sinc_step * cosh(u) / t_scale * (4.0 / spi) * t * t;
    } else {
        w = (q == 0) ? sinc_step / (t_scale * spi) : 2.0 * sinc_step * cosh(u) / (t_scale * spi);
        // Yukawa exp(-kappa r)/r = (2/sqrt(pi)) int exp(-kappa^2/(4 t^2)) exp(-r^2 t^2) dt (Eq. LalpYukawa)
        if (kappa > 0.0) w *= exp(-kappa * kappa / (4.0 * t * t));
    }
    const double a = cbrt(w);
    const double t2 = t * t;
    for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < 2 * N;
         j += (int64_t)gridDim.x * blockDim.x) {
        const double x = ((double)(j - N) + 0.5) * h;
        double v;
        if (!galerkin) {
            v = exp(-t2 * (x * x));
        } else if (t == 0.0) {
            v = 1.0;
        } else if (t * h <= 10.0) {
            // average over the cell [x - h/2, x + h/2]: the Gaussian is smooth on the cell's scale
            double acc = 0.0;
#pragma unroll 4
            for (int i = 0; i < kGl; ++i) {
                const double y = t * (x + 0.5 * h * gl.x[i]);
                acc += gl.w[i] * exp(-y * y);
            }
            v = 0.5 * acc;
        } else {
            // a narrow Gaussian: the cell lies on one side of 0, and erfc of its near end dominates
            const double c0 = x - 0.5 * h, c1 = x + 0.5 * h;
            const double d = c0 >= 0.0 ? erfc(t * c0) - erfc(t * c1) : erfc(-t * c1) - erfc(-t * c0);
            v = 0.88622692545275801365 / (t * h) * d;   // sqrt(pi)/2
        }
        g[row * 2 * N + j] = a * v;
    }
}

// nodes and weights of the n-point Gauss-Legendre rule: the roots of P_n by Newton's method
// from the Chebyshev-like start cos(pi (i + 3/4) / (n + 1/2)), P_n and P_n' by the three-term
// recurrence; w_i = 2 / ((1 - x_i^2) P_n'(x_i)^2)
GlRule gauss_legendre() {
    GlRule r{};
    const int n = kGl;
    for (int i = 0; i < (n + 1) / 2; ++i) {
        double x = cos(3.14159265358979323846 * (i + 0.75) / (n + 0.5)), dp = 1.0;
        for (int it = 0; it < 100; ++it) {
            double p0 = 1.0, p1 = x;
            for (int k = 2; k <= n; ++k) {
                const double p2 = ((2.0 * k - 1.0) * x * p1 - (k - 1.0) * p0) / k;
                p0 = p1;
                p1 = p2;
            }
            dp = n * (x * p1 - p0) / (x * x - 1.0);
            const double dx = p1 / dp;
            x -= dx;
            if (fabs(dx) < 1e-16) break;
        }
        {
            double p0 = 1.0, p1 = x;
            for (int k = 2; k <= n; ++k) {
                const double p2 = ((2.0 * k - 1.0) * x * p1 - (k - 1.0) * p0) / k;
                p0 = p1;
                p1 = p2;
            }
            dp = n * (x * p1 - p0) / (x * x - 1.0);
        }
        const double wi = 2.0 / ((1.0 - x * x) * dp * dp);
        r.x[i] = -x;
        r.w[i] = wi;
        r.x[n - 1 - i] = x;
        r.w[n - 1 - i] = wi;
    }
    return r;
}

// columns c0 .. c0 + ncols - 1, element (c, i) at out[c * N + i]: blocks walk the
// (column, run of kAsmPer * blockDim.x elements) pairs in a grid-stride loop, so that a
// launch of a few blocks per SM covers any number of columns; each thread keeps kAsmPer
// independent sums (its elements blockDim.x apart) in flight
constexpr int kAsmPer = 4;
__global__ void k_assemble(const double* __restrict__ g, int64_t N, const int32_t* __restrict__ colq,
                           const int32_t* __restrict__ woff, const int32_t* __restrict__ wcnt,
                           const int32_t* __restrict__ win, int64_t c0, int64_t ncols, double* __restrict__ out) {
    const int64_t run = (int64_t)kAsmPer * blockDim.x;
    const int64_t runs = (N + run - 1) / run, items = ncols * runs;
    for (int64_t w = blockIdx.x; w < items; w += gridDim.x) {
        const int64_t cl = w / runs, i0 = (w - cl * runs) * run + threadIdx.x, c = c0 + cl;
        const double* gq = g + (int64_t)__ldg(colq + c) * 2 * N + N;
        const int o = __ldg(woff + c), n = __ldg(wcnt + c);
        double acc[kAsmPer];
#pragma unroll
        for (int u = 0; u < kAsmPer; ++u) acc[u] = 0.0;
        for (int k = 0; k < n; ++k) {
            const double* gk = gq - __ldg(win + o + k);
#pragma unroll
            for (int u = 0; u < kAsmPer; ++u) {
                const int64_t i = i0 + (int64_t)u * blockDim.x;
                if (i < N) acc[u] += gk[i];
            }
        }
#pragma unroll
        for (int u = 0; u < kAsmPer; ++u) {
            const int64_t i = i0 + (int64_t)u * blockDim.x;
            if (i < N) out[c * N + i] = acc[u];
        }
    }
}

__global__ void k_norm_columns(double* a, int64_t N, double* norms) {
    const int64_t c = blockIdx.x;
    double* row = a + c * N;
    double s = 0.0;
    for (int64_t i = threadIdx.x; i < N; i += blockDim.x) s += row[i] * row[i];
    __shared__ double red[32];
    for (int o = 16; o; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x < 32) {
        s = (threadIdx.x < (blockDim.x >> 5)) ? red[threadIdx.x] : 0.0;
        for (int o = 16; o; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        if (threadIdx.x == 0) red[0] = s;
    }
    __syncthreads();
    const double nrm = sqrt(red[0]);
    if (threadIdx.x == 0) norms[c] = nrm;
    const double inv = nrm > 0.0 ? 1.0 / nrm : 0.0;
    for (int64_t i = threadIdx.x; i < N; i += blockDim.x) row[i] *= inv;
}

__global__ void k_identity(double* V, int64_t C) {
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < C * C;
         e += (int64_t)gridDim.x * blockDim.x)
        V[e] = (e / C == e % C) ? 1.0 : 0.0;
}

__global__ void k_fold_norms(const double* xi, const int32_t* tcol, int64_t T, const double* n0,
                             const double* n1, const double* n2, double* xin) {
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < T;
         t += (int64_t)gridDim.x * blockDim.x)
        xin[t] = xi[t] * n0[tcol[3 * t]] * n1[tcol[3 * t + 1]] * n2[tcol[3 * t + 2]];
}

// ---------------------------------------------------------------------------
// register-blocked DFMA GEMM with functor operands
//   C(z, m, n) = sum_k A(z, m, k) * B(z, k, n)
// A::kfast / B::kfast say which index is contiguous in memory, so that the
// tile loaders walk memory in order.
// ---------------------------------------------------------------------------
constexpr int GBM = 64, GBN = 64, GBK = 16;

// acc += A(z, m0:m0+64, kb:ke) * B(z, kb:ke, n0:n0+64) for this thread's 4 x 4 outputs
// (rows ty + 16 i, columns tx + 16 j of the tile)
template <class AOp, class BOp>
__device__ __forceinline__ void gemm_tile(const AOp& A, const BOp& B, int z, int M, int N, int kb, int ke, int m0,
                                          int n0, double (&As)[GBK][GBM], double (&Bs)[GBK][GBN],
                                          double (&acc)[4][4]) {
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = 0.0;
    for (int k0 = kb; k0 < ke; k0 += GBK) {
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int e = threadIdx.x + 256 * u;
            int mm, kk;
            if (AOp::kfast) { kk = e % GBK; mm = e / GBK; } else { mm = e % GBM; kk = e / GBM; }
            const int gm = m0 + mm, gk = k0 + kk;
            As[kk][mm] = (gm < M && gk < ke) ? A(z, gm, gk) : 0.0;
            int nn;
            if (BOp::kfast) { kk = e % GBK; nn = e / GBK; } else { nn = e % GBN; kk = e / GBN; }
            const int gn = n0 + nn, gk2 = k0 + kk;
            Bs[kk][nn] = (gn < N && gk2 < ke) ? B(z, gk2, gn) : 0.0;
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < GBK; ++kk) {
            double a[4], b[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) a[i] = As[kk][ty + 16 * i];
#pragma unroll
            for (int j = 0; j < 4; ++j) b[j] = Bs[kk][tx + 16 * j];
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) acc[i][j] = fma(a[i], b[j], acc[i][j]);
        }
        __syncthreads();
    }
}

template <class AOp, class BOp, class COp>
__global__ void __launch_bounds__(256) k_gemm_f64(int M, int N, int K, AOp A, BOp B, COp Cst) {
    __shared__ double As[GBK][GBM];
    __shared__ double Bs[GBK][GBN];
    const int z = blockIdx.z;
    const int m0 = blockIdx.y * GBM, n0 = blockIdx.x * GBN;
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    double acc[4][4];
    gemm_tile(A, B, z, M, N, 0, K, m0, n0, As, Bs, acc);
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const int m = m0 + ty + 16 * i;
        if (m >= M) continue;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int n = n0 + tx + 16 * j;
            if (n < N) Cst(z, m, n, acc[i][j]);
        }
    }
}

template <class AOp, class BOp, class COp>
cudaError_t gemm_f64(int M, int N, int K, int batch, AOp A, BOp B, COp Cst, cudaStream_t st) {
    if (M <= 0 || N <= 0 || batch <= 0) return cudaSuccess;
    dim3 grid((N + GBN - 1) / GBN, (M + GBM - 1) / GBM, batch);
    k_gemm_f64<<<grid, 256, 0, st>>>(M, N, K, A, B, Cst);
    count_kernels(1);
    return cudaGetLastError();
}

// operand functors ----------------------------------------------------------
struct RowK {            // X(m, k) = p[m * ld + k]        (k contiguous)
    static constexpr bool kfast = true;
    const double* p; int64_t ld;
    __device__ double operator()(int, int m, int k) const { return p[m * ld + k]; }
};
struct KRowN {           // X(k, n) = p[k * ld + n]        (n contiguous)
    static constexpr bool kfast = false;
    const double* p; int64_t ld;
    __device__ double operator()(int, int k, int n) const { return p[k * ld + n]; }
};
struct StoreRow {        // C[z*zs + m*ld + n] = v
    double* p; int64_t ld; int64_t zs;
    __device__ void operator()(int z, int m, int n, double v) const { p[z * zs + m * ld + n] = v; }
};

// eval step 1: A(m=(a,b), k) = B[m*r2 + k], B(k, n=s) = Z2[k*N + zidx[s]]
struct EvalZ3 {
    static constexpr bool kfast = true;
    const double* Z; int64_t N; const int32_t* zidx;
    __device__ double operator()(int, int k, int n) const { return Z[k * N + zidx[n]]; }
};
// eval step 2: A(z=s; m=a, k=b) = M[(a*r1 + b)*ns + s]
struct EvalM {
    static constexpr bool kfast = false;
    const double* M; int r1; int ns;
    __device__ double operator()(int z, int m, int k) const { return M[((int64_t)m * r1 + k) * ns + z]; }
};
// eval step 3: A(z; m=x, k=a) = Z0[a*N + x] ; B(z; k=a, n=y) = T[z*r0*N + a*N + y]
struct ColK {           // X(m, k) = p[k * ld + m]   (m contiguous)
    static constexpr bool kfast = false;
    const double* p; int64_t ld;
    __device__ double operator()(int, int m, int k) const { return p[k * ld + m]; }
};
struct KRowNBatched {
    static constexpr bool kfast = false;
    const double* p; int64_t ld; int64_t zs;
    __device__ double operator()(int z, int k, int n) const { return p[z * zs + k * ld + n]; }
};
struct StoreOut {
    void* p; int64_t N; int f32;
    __device__ void operator()(int z, int m, int n, double v) const {
        const int64_t o = ((int64_t)z * N + m) * N + n;
        if (f32) static_cast<float*>(p)[o] = (float)v;
        else static_cast<double*>(p)[o] = v;
    }
};

// ---------------------------------------------------------------------------
// parallel cyclic Jacobi (round-robin pairing), cooperative grid
// ---------------------------------------------------------------------------
__device__ __forceinline__ void rr_pair(int t, int i, int Cp, int& p, int& q) {
    const int n1 = Cp - 1;
    int a, b;
    if (i == 0) { a = n1; b = t; }
    else { a = (t + i) % n1; b = (t - i + n1) % n1; }
    p = min(a, b);
    q = max(a, b);
}
// partner of index a in round t, and the index of its pair
__device__ __forceinline__ int rr_partner(int t, int a, int n1) {
    if (a == n1) return t;
    if (a == t) return n1;
    return ((2 * t - a) % n1 + n1) % n1;
}
__device__ __forceinline__ int rr_index(int t, int a, int n1) {
    if (a == n1 || a == t) return 0;
    const int d = ((a - t) % n1 + n1) % n1;
    return min(d, n1 - d);
}

// Parallel cyclic Jacobi for several symmetric matrices at once: CTAs
// [cta0, cta0 + ncta) of the grid work on job m with their own bounded group
// barrier. Only the upper triangle of G is read and written. One barrier per
// round: the three pivot entries of every pair of the next round are copied to
// a double-buffered snapshot by the threads that write them, so the rotations
// of a round never read entries that the same round overwrites. A rotation is
// skipped when |a_pq| is below the absolute floor (the rounding noise of the
// FP64 Gram matrix), below tol * sqrt(|a_pp a_qq|), or when both diagonal
// entries are below tau: such directions lie far below the truncation
// threshold, are discarded together, and mixing them changes neither the
// retained subspace nor the trace of the discarded block. A sweep without
// rotations ends the iteration.
struct JacobiMode {
    double* G; double* V; double* snap; DevStatus* st; int C; int cta0; int ncta; double abs_floor; double tau;
};
struct JacobiArgs {
    const JacobiMode* m; int nmodes; int max_sweeps; double tol;
};

// the job whose CTA range [cta0, cta0 + ncta) holds blockIdx.x (jobs sorted by cta0)
template <class Job>
__device__ __forceinline__ int find_job(const Job* m, int n) {
    int lo = 0, hi = n - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if ((int)blockIdx.x >= m[mid].cta0) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

__device__ __forceinline__ double& gsym(double* G, int C, int a, int b) {
    return a <= b ? G[(int64_t)a * C + b] : G[(int64_t)b * C + a];
}

__global__ void __launch_bounds__(256) k_jacobi_multi(JacobiArgs A) {
    const JacobiMode J = A.m[find_job(A.m, A.nmodes)];
    const int lb = blockIdx.x - J.cta0, nb = J.ncta;
    const int C = J.C, Cp = C + (C & 1), P = Cp / 2, n1 = Cp - 1;
    // shared: c[P], s[P] (double), p[P], q[P], next partner[Cp], next pair index[Cp] (int)
    extern __shared__ double sm[];
    double* sc = sm;
    double* ss = sm + P;
    int* sp = (int*)(ss + P);
    int* sq = sp + P;
    int* npart = sq + P;
    int* nidx = npart + Cp;
    __shared__ unsigned int s_active;
    double* G = J.G;
    double* V = J.V;
    const int64_t nthr = (int64_t)nb * blockDim.x;
    const int64_t gtid = (int64_t)lb * blockDim.x + threadIdx.x;
    const int64_t items_g = (int64_t)P * P;
    const int64_t items = items_g + (int64_t)C * P;
    for (int64_t i = gtid; i < P; i += nthr) {
        int p, q;
        rr_pair(0, (int)i, Cp, p, q);
        J.snap[3 * i + 0] = G[(int64_t)p * C + p];
        J.snap[3 * i + 1] = q < C ? G[(int64_t)q * C + q] : 0.0;
        J.snap[3 * i + 2] = q < C ? G[(int64_t)p * C + q] : 0.0;
    }
    if (!group_barrier(J.st, nb)) return;
    int cur = 0;
    for (int sweep = 0; sweep < A.max_sweeps; ++sweep) {
        if (threadIdx.x == 0) s_active = 0;
        __syncthreads();
        for (int t = 0; t < n1; ++t) {
            const int tn = (t + 1 == n1) ? 0 : t + 1;
            const double* D = J.snap + (int64_t)cur * 3 * P;
            double* Dn = J.snap + (int64_t)(cur ^ 1) * 3 * P;
            for (int i = threadIdx.x; i < P; i += blockDim.x) {
                int p, q;
                rr_pair(t, i, Cp, p, q);
                sp[i] = p;
                sq[i] = q;
                double c = 1.0, s = 0.0;
                if (q < C) {
                    const double app = __ldcg(D + 3 * i), aqq = __ldcg(D + 3 * i + 1), apq = __ldcg(D + 3 * i + 2);
                    if (fabs(apq) > J.abs_floor && fmax(app, aqq) >= J.tau &&
                        fabs(apq) * fabs(apq) > A.tol * A.tol * fabs(app * aqq)) {
                        // The angle only steers convergence, so it is taken in FP32; the rotation
                        // itself is orthogonal to FP64 rounding: c = (1 + t^2)^(-1/2) by two FP64
                        // Newton steps from the FP32 estimate, s = t c.
                        const float theta = (float)((aqq - app) / (2.0 * apq));
                        const float tf = copysignf(1.f, theta) / (fabsf(theta) + sqrtf(fmaf(theta, theta, 1.f)));
                        const double tt = (double)tf;
                        const double x = fma(tt, tt, 1.0);
                        double cc = (double)rsqrtf((float)x);
                        cc = cc * fma(-0.5 * x, cc * cc, 1.5);
                        cc = cc * fma(-0.5 * x, cc * cc, 1.5);
                        c = cc;
                        s = tt * cc;
                        if (lb == 0) atomicAdd(&s_active, 1u);
                    }
                }
                sc[i] = c;
                ss[i] = s;
            }
            for (int a = threadIdx.x; a < Cp; a += blockDim.x) {
                npart[a] = rr_partner(tn, a, n1);
                nidx[a] = rr_index(tn, a, n1);
            }
            __syncthreads();
            if (t == n1 - 1 && lb == 0 && threadIdx.x == 0) J.st->sweep_active[sweep & 63] = s_active;
            for (int64_t it = gtid; it < items; it += nthr) {
                if (it < items_g) {
                    const int i = (int)(it / P), i2 = (int)(it - (int64_t)i * P);
                    if (i2 < i) continue;                       // upper block triangle only
                    const double c1 = sc[i], s1 = ss[i], c2 = sc[i2], s2 = ss[i2];
                    const int p = sp[i], q = sq[i], p2 = sp[i2], q2 = sq[i2];
                    const bool vq = q < C, vq2 = q2 < C;        // p, p2 < C always
                    const int rows[2] = {p, q}, cols[2] = {p2, q2};
                    int piv = 0;
#pragma unroll
                    for (int u = 0; u < 2; ++u)
#pragma unroll
                        for (int v = 0; v < 2; ++v) {
                            const int a = rows[u], b = cols[v];
                            if (a >= C || b >= C) continue;
                            if (i == i2 && u > v) continue;      // (q,p) of a diagonal block = (p,q)
                            if (a == b || npart[a] == b) piv |= 1 << (2 * u + v);
                        }
                    const bool active = (s1 != 0.0 || s2 != 0.0);
                    if (!active && !piv) continue;
                    double x[4];
                    x[0] = __ldcg(&gsym(G, C, p, p2));
                    x[1] = vq2 ? __ldcg(&gsym(G, C, p, q2)) : 0.0;
                    x[2] = vq ? __ldcg(&gsym(G, C, q, p2)) : 0.0;
                    x[3] = (vq && vq2) ? __ldcg(&gsym(G, C, q, q2)) : 0.0;
                    double z[4] = {x[0], x[1], x[2], x[3]};
                    if (active) {
                        const double ypp = c1 * x[0] - s1 * x[2], ypq = c1 * x[1] - s1 * x[3];
                        const double yqp = s1 * x[0] + c1 * x[2], yqq = s1 * x[1] + c1 * x[3];
                        z[0] = c2 * ypp - s2 * ypq;
                        z[1] = s2 * ypp + c2 * ypq;
                        z[2] = c2 * yqp - s2 * yqq;
                        z[3] = s2 * yqp + c2 * yqq;
                        __stcg(&gsym(G, C, p, p2), z[0]);
                        if (vq2) __stcg(&gsym(G, C, p, q2), z[1]);
                        if (vq && i != i2) __stcg(&gsym(G, C, q, p2), z[2]);
                        if (vq && vq2) __stcg(&gsym(G, C, q, q2), z[3]);
                    }
                    if (piv) {
#pragma unroll
                        for (int u = 0; u < 2; ++u)
#pragma unroll
                            for (int v = 0; v < 2; ++v) {
                                if (!(piv & (1 << (2 * u + v)))) continue;
                                const int a = min(rows[u], cols[v]), b = max(rows[u], cols[v]);
                                const int k = nidx[a];
                                const int slot = (a == b) ? (a < npart[a] ? 0 : 1) : 2;
                                __stcg(Dn + 3 * k + slot, z[2 * u + v]);
                            }
                    }
                } else {
                    const int64_t r = it - items_g;
                    const int j = (int)(r / P), i2 = (int)(r - (int64_t)j * P);
                    const double c2 = sc[i2], s2 = ss[i2];
                    if (s2 == 0.0) continue;
                    const int p2 = sp[i2], q2 = sq[i2];
                    const double vp = __ldcg(V + (int64_t)j * C + p2);
                    const double vv = __ldcg(V + (int64_t)j * C + q2);
                    __stcg(V + (int64_t)j * C + p2, c2 * vp - s2 * vv);
                    __stcg(V + (int64_t)j * C + q2, s2 * vp + c2 * vv);
                }
            }
            if (!group_barrier(J.st, nb)) return;
            cur ^= 1;
        }
        const unsigned int act = __ldcg(&J.st->sweep_active[sweep & 63]);
        if (act == 0) {
            if (gtid == 0) J.st->sweeps = sweep + 1;
            return;
        }
    }
    if (gtid == 0) {
        J.st->sweeps = -A.max_sweeps;
        atomicCAS(&J.st->flag, FLAG_OK, FLAG_NOCONVERGE);
    }
}

// doubles order like these integer keys (sign-adjusted bit patterns)
__device__ __forceinline__ unsigned long long order_key(double v) {
    const unsigned long long b = (unsigned long long)__double_as_longlong(v);
    return (b >> 63) ? ~b : (b | 0x8000000000000000ull);
}
// the double whose key this is
__device__ __forceinline__ double key_value(unsigned long long k) {
    return __longlong_as_double((long long)((k >> 63) ? (k & 0x7fffffffffffffffull) : ~k));
}

// ---------------------------------------------------------------------------
// Pivoted Cholesky of up to three PSD matrices at once, one panel of pivots a
// launch (cooperative grid, CTAs split between the jobs): G P = L L^T with
// greedy diagonal pivoting, stopped when the trace of the Schur complement
// drops below delta. The launch continues the factorisation at column
// k0 = st->sweeps of L with S = G - L[:, :k0] L[:, :k0]^T, the Schur complement
// that the caller's tensor-core product formed after the previous panel, and
// takes up to pw pivots, or fewer where the stopping rule ends it; it also
// writes the panel's columns to Lp (C x pw, zero past the last pivot taken:
// zero throughout once the factorisation has ended), so that the caller can
// queue the next Schur update S -= Lp Lp^T without reading anything back. Each CTA owns a
// contiguous range of rows and keeps, in shared memory, their residual
// diagonal and their entries of L in the panel's first kc columns (the global
// copy of L is written as well: other CTAs read row p from it, and it is the
// output). One step:
//   1. warp 0 reduces the per-CTA (max, argmax, sum) candidates of the
//      residual diagonal (the maximum compared as integer keys, ties to the
//      smaller index; the sum in a fixed order, so every CTA decides alike);
//   2. all threads load the panel part of row p of L and column p of S into
//      shared memory;
//   3. the other warps form the in-panel dot products of the new column, four
//      rows a warp, while warp 0 takes 1 / sqrt(d_p);
//   4. a thread per row scales its entry, updates the residual diagonal, and
//      warp 0 publishes the CTA's candidate (double-buffered by step parity);
//   5. the job's CTAs meet at a counting barrier.
// FP64 arithmetic runs at a small fraction of the FP32 rate on this GPU: the
// panel form leaves the bulk of it (the products with the earlier columns) to
// the tensor cores, and keeps every scalar FP64 operation (reductions, the
// square root, comparisons) on one warp instead of repeating it in each.
// st->sweeps receives the columns of L so far, st->done 1 once the stopping
// rule ended the factorisation, cand[kPcholCand - 1] the residual trace.
// ---------------------------------------------------------------------------
struct PcholMode {
    const double* S; double* L; double* Lp; double* d; double* cand; int* piv; DevStatus* st; int C; int kmax;
    int cta0; int ncta; int kc; int pw; double delta;
};
struct PcholArgs {
    const PcholMode* m; int nmodes;
};

// (key, index) maximum over a warp, ties to the smaller index (>= 0); every
// lane receives the result
__device__ __forceinline__ void warp_argmax(unsigned long long& key, int& ix) {
    for (int o = 16; o; o >>= 1) {
        const unsigned long long k2 = __shfl_xor_sync(0xffffffffu, key, o);
        const int i2 = __shfl_xor_sync(0xffffffffu, ix, o);
        if (k2 > key || (k2 == key && i2 >= 0 && (ix < 0 || i2 < ix))) { key = k2; ix = i2; }
    }
}

constexpr int kPcRows = 4;   // rows of the new column a warp forms at once

// rows of column p of S a thread of k_pchol_multi holds in registers (the rest in shared memory)
constexpr int kPmRowsPerThread = 2;

__global__ void __launch_bounds__(256) k_pchol_multi(PcholArgs A) {
    const PcholMode J = A.m[find_job(A.m, A.nmodes)];
    const int lb = blockIdx.x - J.cta0, nb = J.ncta;
    const int C = J.C, kc = J.kc;
    // rows of this CTA: [r0, r1)
    const int per = (C + nb - 1) / nb;
    const int r0 = min(C, lb * per), r1 = min(C, r0 + per), nr = r1 - r0;
    const int pw = J.pw;
    // where the previous panel left the factorisation (every CTA reads the same words)
    const int k0 = *(volatile int*)&J.st->sweeps;
    if (*(volatile int*)&J.st->done || k0 >= J.kmax) {
        // ended: a zero panel, so that the queued Schur update changes nothing
        for (int64_t e = threadIdx.x; e < (int64_t)nr * pw; e += blockDim.x) J.Lp[(int64_t)r0 * pw + e] = 0.0;
        if (lb == 0 && threadIdx.x == 0) J.st->done = 1;
        return;
    }
    const int kend = min(J.kmax, k0 + pw);
    extern __shared__ double smd[];
    double* lrow = smd;                 // [pw] the panel part of row p of L
    double* ds = lrow + pw;             // [per] residual diagonal of the own rows
    double* gp = ds + per;              // [per] S[own rows, p]
    double* sacc = gp + per;            // [per] dot products of the step
    double* Ls = sacc + per;            // [per][kc] own rows of L, the panel's first kc columns
    __shared__ double s_dmax, s_sum, s_inv;
    __shared__ int s_p;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31, nw = blockDim.x >> 5;
    // warp 0: this CTA's (max, argmax, sum) of the residual diagonal, published by step parity
    auto publish = [&](int parity) {
        unsigned long long key = order_key(-1.0);
        int ix = -1;
        double sm = 0.0;
        for (int jl = lane; jl < nr; jl += 32) {
            const double v = ds[jl];
            const unsigned long long kv = order_key(v);
            sm += v;
            if (kv > key) { key = kv; ix = r0 + jl; }
        }
        warp_argmax(key, ix);
        for (int o = 16; o; o >>= 1) sm += __shfl_xor_sync(0xffffffffu, sm, o);
        if (lane == 0) {
            double* c = J.cand + ((int64_t)parity * nb + lb) * 3;
            __stcg(c, key_value(key));
            __stcg(c + 1, (double)ix);
            __stcg(c + 2, sm);
        }
    };
    // the residual diagonal: diag(G) at the start, else as the previous panel left it
    for (int jl = tid; jl < nr; jl += blockDim.x)
        ds[jl] = k0 == 0 ? __ldcg(J.S + (int64_t)(r0 + jl) * C + r0 + jl) : __ldcg(J.d + r0 + jl);
    __syncthreads();
    if (warp == 0) publish(0);
    unsigned int epoch = 1;
    if (!count_barrier(J.st, epoch * nb)) return;
    int k = k0;
    bool done = false;
    for (;; ++k) {
        const int par = k & 1;
        // 1. warp 0 reduces the candidates of all CTAs of the job
        if (warp == 0) {
            unsigned long long key = order_key(-1.0);
            int p = -1;
            double sum = 0.0;
            for (int c = lane; c < nb; c += 32) {
                const double* cc = J.cand + ((int64_t)par * nb + c) * 3;
                const unsigned long long k2 = order_key(__ldcg(cc));
                const int i2 = (int)__ldcg(cc + 1);
                if (k2 > key || (k2 == key && i2 >= 0 && (p < 0 || i2 < p))) { key = k2; p = i2; }
                sum += __ldcg(cc + 2);
            }
            warp_argmax(key, p);
            for (int o = 16; o; o >>= 1) sum += __shfl_xor_sync(0xffffffffu, sum, o);
            if (lane == 0) {
                s_p = p;
                s_dmax = key_value(key);
                s_sum = sum;
            }
        }
        __syncthreads();
        const int p = s_p;
        const double dmax = s_dmax;
        // stop when the residual trace is small enough, or at kmax columns; the panel ends at kend
        if (k >= J.kmax || !(s_sum > J.delta) || p < 0 || !(dmax > 0.0)) {
            done = true;
            break;
        }
        if (k >= kend) break;
        // 2. column p of S and the panel part of row p of L (written by its owner in earlier
        // steps). S[j][p] comes from S's upper triangle (the Schur updates leave the lower one
        // behind); a thread's first kPmRowsPerThread rows wait in registers, so that their trip
        // to L2 runs beside the dot products (the thread finishes those rows in step 4)
        double gc[kPmRowsPerThread];
#pragma unroll
        for (int u = 0; u < kPmRowsPerThread; ++u) {
            const int jl = tid + u * (int)blockDim.x, j = r0 + jl;
            gc[u] = jl < nr ? __ldcg(J.S + (j < p ? (int64_t)j * C + p : (int64_t)p * C + j)) : 0.0;
        }
        for (int jl = tid + kPmRowsPerThread * (int)blockDim.x; jl < nr; jl += blockDim.x) {
            const int j = r0 + jl;
            gp[jl] = __ldcg(J.S + (j < p ? (int64_t)j * C + p : (int64_t)p * C + j));
        }
        for (int t = k0 + tid; t < k; t += blockDim.x) lrow[t - k0] = __ldcg(J.L + (int64_t)p * J.kmax + t);
        __syncthreads();
        // 3. dot products, kPcRows rows a warp (warp 0 last), and 1 / sqrt(d_p) on warp 0
        if (tid == 0) s_inv = 1.0 / sqrt(dmax);
        const int ngroups = (nr + kPcRows - 1) / kPcRows;
        const int kk = k - k0, ks = min(kk, kc);   // in-panel columns before k; those in shared memory
        for (int gi = (warp + nw - 1) % nw; gi < ngroups; gi += nw) {
            int rl[kPcRows];
#pragma unroll
            for (int q = 0; q < kPcRows; ++q) rl[q] = min(gi * kPcRows + q, nr - 1);
            double acc[kPcRows];
#pragma unroll
            for (int q = 0; q < kPcRows; ++q) acc[q] = 0.0;
            int t = lane;
            for (; t < ks; t += 32) {
                const double lv = lrow[t];
#pragma unroll
                for (int q = 0; q < kPcRows; ++q) acc[q] = fma(Ls[(size_t)rl[q] * kc + t], lv, acc[q]);
            }
            for (; t < kk; t += 32) {
                const double lv = lrow[t];
#pragma unroll
                for (int q = 0; q < kPcRows; ++q)
                    acc[q] = fma(__ldcg(J.Lp + (int64_t)(r0 + rl[q]) * pw + t), lv, acc[q]);
            }
            // transposed butterfly: 6 additions for the four sums (lane 8 q holds row q)
            const bool hi = lane & 16;
            double v0 = (hi ? acc[2] : acc[0]) + __shfl_xor_sync(0xffffffffu, hi ? acc[0] : acc[2], 16);
            double v1 = (hi ? acc[3] : acc[1]) + __shfl_xor_sync(0xffffffffu, hi ? acc[1] : acc[3], 16);
            const bool b3 = lane & 8;
            double w = (b3 ? v1 : v0) + __shfl_xor_sync(0xffffffffu, b3 ? v0 : v1, 8);
            for (int o = 4; o; o >>= 1) w += __shfl_xor_sync(0xffffffffu, w, o);
            const int q = lane >> 3;
            if ((lane & 7) == 0 && gi * kPcRows + q < nr) sacc[gi * kPcRows + q] = w;
        }
        __syncthreads();
        // 4. the new column of L and the residual diagonal
        const double inv = s_inv;
        auto finish = [&](int jl, double g) {
            const int j = r0 + jl;
            const double l = (g - sacc[jl]) * inv;
            if (kk < kc) Ls[(size_t)jl * kc + kk] = l;
            __stcg(J.L + (int64_t)j * J.kmax + k, l);
            __stcg(J.Lp + (int64_t)j * pw + kk, l);
            ds[jl] = (j == p) ? 0.0 : fmax(ds[jl] - l * l, 0.0);
        };
#pragma unroll
        for (int u = 0; u < kPmRowsPerThread; ++u) {
            const int jl = tid + u * (int)blockDim.x;
            if (jl < nr) finish(jl, gc[u]);
        }
        for (int jl = tid + kPmRowsPerThread * (int)blockDim.x; jl < nr; jl += blockDim.x) finish(jl, gp[jl]);
        if (lb == 0 && tid == 0) J.piv[k] = p;
        __syncthreads();
        if (warp == 0) publish(par ^ 1);
        // 5. the job's CTAs meet
        if (!count_barrier(J.st, ++epoch * nb)) return;
    }
    for (int jl = tid; jl < nr; jl += blockDim.x) J.d[r0 + jl] = ds[jl];
    // the panel's columns past the last pivot taken are zero
    for (int64_t e = tid; e < (int64_t)nr * (pw - (k - k0)); e += blockDim.x) {
        const int64_t jl = e / (pw - (k - k0)), t = (k - k0) + e % (pw - (k - k0));
        J.Lp[(r0 + jl) * pw + t] = 0.0;
    }
    if (lb == 0 && tid == 0) {
        J.st->sweeps = k;                          // columns of L
        J.st->done = done ? 1 : 0;
        J.cand[kPcholCand - 1] = s_sum;            // residual trace: energy outside span(L)
    }
}

// ---------------------------------------------------------------------------
// eigenvalue sort + eps-rank selection, one CTA per matrix. The ranking compares
// integer keys (doubles order like their sign-adjusted bit patterns), and the
// tail sums are suffix sums taken by one warp (contiguous chunks a lane, then a
// shuffle scan), so that neither the O(C^2) comparisons nor the C additions queue
// on one SMSP's FP64 unit.
// ---------------------------------------------------------------------------
struct SelJob {
    const double* G; int C; int forced; const double* extra; int32_t* perm; double* lam; double* isl; double* out;
    int64_t dstride; double resolution;
};
constexpr int kSelMax = 16;
struct SelArgs {
    SelJob j[kSelMax];
    double eps, resolution;
};
__global__ void __launch_bounds__(1024) k_sort_select(const __grid_constant__ SelArgs A) {
    const SelJob& J = A.j[blockIdx.x];
    const int C = J.C;
    const double* G = J.G;
    const int64_t ds = J.dstride;
    extern __shared__ double s_lam[];                     // [C] sorted, then the suffix sums [C + 1]
    double* suf = s_lam + C;
    for (int k = threadIdx.x; k < C; k += blockDim.x) {
        const double lk = G[(int64_t)k * ds];
        const unsigned long long kk = order_key(lk);
        int rank = 0;
        for (int j = 0; j < C; ++j) {
            const unsigned long long kj = order_key(G[(int64_t)j * ds]);
            rank += (kj > kk) || (kj == kk && j < k);
        }
        J.perm[rank] = k;
        s_lam[rank] = lk;
    }
    __syncthreads();
    // suffix sums of max(lambda, 0): suf[k] = sum_{j >= k}, suf[C] = 0 (warp 0)
    if (threadIdx.x < 32) {
        const int lane = threadIdx.x, per = (C + 31) / 32, b = lane * per, e = min(C, b + per);
        double run = 0.0;
        for (int j = e - 1; j >= b; --j) run += fmax(s_lam[j], 0.0);   // this chunk's total
        // exclusive scan from the right: the totals of the chunks after this one
        double after = 0.0, x = run;
        for (int o = 1; o < 32; o <<= 1) {
            const double y = __shfl_down_sync(0xffffffffu, x, o);
            if (lane + o < 32) x += y;
        }
        after = __shfl_down_sync(0xffffffffu, x, 1);
        if (lane == 31) after = 0.0;
        double acc = after;
        for (int j = e - 1; j >= b; --j) {
            acc += fmax(s_lam[j], 0.0);
            suf[j] = acc;
        }
        if (lane == 0) suf[C] = 0.0;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        // energy outside the compressed problem belongs to the discarded tail
        const double ex = J.extra ? fmax(*J.extra, 0.0) : 0.0;
        const double total = ex + suf[0];
        int r;
        double tail_at_r;
        if (J.forced > 0) {
            // a forced rank is clipped to the eigenvalues the FP64 Gram matrix resolves
            const double res = J.resolution >= 0.0 ? J.resolution : A.resolution;
            int nres = 0;
            while (nres < C && s_lam[nres] > res) ++nres;
            r = max(1, min(min(J.forced, C), nres));
            tail_at_r = ex + suf[r];
        } else {
            // smallest r >= 1 whose tail qualifies (the suffix sums only fall with r)
            const double lim = A.eps * A.eps * total;
            int lo = 1, hi = C;   // suf[C] = 0 qualifies
            while (lo < hi) {
                const int mid = (lo + hi) >> 1;
                if (ex + suf[mid] <= lim) hi = mid;
                else lo = mid + 1;
            }
            r = lo;
            tail_at_r = ex + suf[r];
        }
        J.out[0] = (double)r;
        J.out[1] = tail_at_r;
        J.out[2] = total;
    }
    // lam[] becomes the singular values sigma_k = sqrt(max(lambda_k, 0))
    for (int k = threadIdx.x; k < C; k += blockDim.x) {
        const double lk = s_lam[k];
        J.isl[k] = lk > 0.0 ? rsqrt(lk) : 0.0;
        J.lam[k] = sqrt(fmax(lk, 0.0));
    }
}

// ---------------------------------------------------------------------------
// blocked Cholesky (lower, in place on A r x r) as one cooperative grid, and
// the forward substitution Z = L^{-1} Y (rows of Y independent per column)
// ---------------------------------------------------------------------------
constexpr int CHB = 32;

// Blocked right-looking Cholesky A = L L^T (lower, in place) followed by the
// triangular inverse Li = L^{-1} (lower, zeros above) of several matrices in
// one cooperative grid, CTAs split between the jobs: a counting barrier after
// each panel step and after each block row of Li.
struct CholMode {
    double* A; double* Li; DevStatus* st; int r; int cta0; int ncta; const double* gate;
};
struct CholArgs {
    const CholMode* m; int nmodes;
};
__global__ void __launch_bounds__(256) k_chol_inv_multi(CholArgs Ar) {
    __shared__ double D[CHB][CHB + 1];
    const CholMode J = Ar.m[find_job(Ar.m, Ar.nmodes)];
    // the series pass took this matrix: every CTA of the job leaves together
    if (J.gate && *J.gate < kSeriesGate) return;
    const int lb = blockIdx.x - J.cta0, nb = J.ncta;
    double* A = J.A;
    double* Li = J.Li;
    const int r = J.r;
    DevStatus* st = J.st;
    const int64_t nthr = (int64_t)nb * blockDim.x;
    const int64_t gtid = (int64_t)lb * blockDim.x + threadIdx.x;
    const int nbk = (r + CHB - 1) / CHB;
    unsigned int epoch = 0;   // counting barriers of the job's CTAs (st->arrive zeroed by the launcher)
    __shared__ double s_rcp[CHB];   // 1 / L_kk of the panel
    __shared__ double colk[CHB];    // the column being eliminated, scaled
    // entry e of a lower triangle, row by row: (tri_r[e], tri_c[e]), tri_c <= tri_r
    __shared__ unsigned char tri_r[CHB * (CHB + 1) / 2], tri_c[CHB * (CHB + 1) / 2];
    for (int t = threadIdx.x; t < CHB; t += blockDim.x)
        for (int c = 0; c <= t; ++c) {
            tri_r[t * (t + 1) / 2 + c] = (unsigned char)t;
            tri_c[t * (t + 1) / 2 + c] = (unsigned char)c;
        }
    __syncthreads();
    __shared__ double sI[CHB][CHB + 1], sK[CHB][CHB + 1];   // panel rows of a trailing tile
    for (int j0 = 0; j0 < r; j0 += CHB) {
        const int b = min(CHB, r - j0);
        if (lb == 0) {
            for (int e = threadIdx.x; e < b * b; e += blockDim.x) {
                const int i = e / b, k = e % b;
                D[i][k] = __ldcg(A + (int64_t)(j0 + i) * r + j0 + k);
            }
            __syncthreads();
            for (int k = 0; k < b; ++k) {
                // warp 0: the pivot d = D[k][k], y ~ d^(-1/2) (the FP32 seed and one Newton step
                // in FP64, good to about 2^-46: this first factorisation only has to bring Y
                // within reach of the second pass), then column k scaled into colk and D
                if (threadIdx.x < 32) {
                    const int i = threadIdx.x;
                    const double d = D[k][k];
                    double y = 1.0;
                    if (d > 0.0) {
                        y = (double)rsqrtf((float)d);
                        y = y * fma(-0.5 * d, y * y, 1.5);
                    } else if (i == 0) {
                        atomicCAS(&st->flag, FLAG_OK, FLAG_NOT_SPD);
                    }
                    if (i == k) {
                        D[k][k] = d > 0.0 ? d * y : 1.0;
                        s_rcp[k] = y;
                    } else if (i > k && i < b) {
                        const double l = D[i][k] * y;
                        D[i][k] = l;
                        colk[i] = l;
                    }
                }
                __syncthreads();
                // the rank-one update of the trailing triangle (rows and columns k + 1 .. b - 1),
                // one entry a thread through the triangle table: as few warps as entries need
                {
                    const int n = b - 1 - k;
                    for (int e = threadIdx.x; e < n * (n + 1) / 2; e += blockDim.x) {
                        const int i = k + 1 + tri_r[e], l = k + 1 + tri_c[e];
                        D[i][l] -= colk[i] * colk[l];
                    }
                }
                __syncthreads();
            }
            for (int e = threadIdx.x; e < b * b; e += blockDim.x) {
                const int i = e / b, k = e % b;
                __stcg(A + (int64_t)(j0 + i) * r + j0 + k, k <= i ? D[i][k] : 0.0);
            }
        }
        if (!count_barrier(st, ++epoch * nb)) return;
        // every CTA stages L11 (and the reciprocals of its diagonal) in shared memory for the panel solve
        for (int e = threadIdx.x; e < b * b; e += blockDim.x) {
            const int i = e / b, k = e % b;
            D[i][k] = __ldcg(A + (int64_t)(j0 + i) * r + j0 + k);
        }
        __syncthreads();
        if (threadIdx.x < b) s_rcp[threadIdx.x] = 1.0 / D[threadIdx.x][threadIdx.x];
        __syncthreads();
        // the panel solve x L11^T = a for every row below the block: a warp per row, lane k
        // holding x_k; step k lane k finishes x_k and every later lane takes its product (one
        // FP64 instruction a step for the warp instead of one a row); rows over all CTAs
        {
            const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nwc = blockDim.x >> 5;
            const double lkk_rcp = lane < b ? s_rcp[lane] : 1.0;
            for (int64_t i = j0 + b + lb + (int64_t)nb * wid; i < r; i += (int64_t)nb * nwc) {
                double acc = lane < b ? __ldcg(A + i * r + j0 + lane) : 0.0;
                double xk = 0.0;
                for (int k = 0; k < b; ++k) {
                    const double xkk = __shfl_sync(0xffffffffu, acc * lkk_rcp, k);   // x_k (lane k's value)
                    if (lane == k) xk = xkk;
                    if (lane > k && lane < b) acc = fma(-xkk, D[lane][k], acc);
                }
                if (lane < b) __stcg(A + i * r + j0 + lane, xk);
            }
        }
        if (!count_barrier(st, ++epoch * nb)) return;
        // the trailing update A22 -= L21 L21^T on its lower 32 x 32 tiles, a CTA per tile: both
        // tiles' panel rows staged in shared memory (coalesced), thread (ty, tx) four rows
        {
            const int n2 = r - j0 - b;
            const int nt = (n2 + CHB - 1) / CHB;
            const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
            for (int item = lb; item < nt * (nt + 1) / 2; item += nb) {
                int ti = 0, rem = item;
                while (rem > ti) { rem -= ti + 1; ++ti; }
                const int tk = rem;   // tk <= ti
                __syncthreads();   // the previous tile's readers of sI, sK are done
                for (int e = threadIdx.x; e < CHB * CHB; e += blockDim.x) {
                    const int rr = e >> 5, c = e & 31;
                    const int ri = ti * CHB + rr, rk = tk * CHB + rr;
                    sI[rr][c] = (ri < n2 && c < b) ? __ldcg(A + (int64_t)(j0 + b + ri) * r + j0 + c) : 0.0;
                    sK[rr][c] = (rk < n2 && c < b) ? __ldcg(A + (int64_t)(j0 + b + rk) * r + j0 + c) : 0.0;
                }
                __syncthreads();
                const int k = tk * CHB + tx;
                if (k < n2) {
                    for (int rr = ty; rr < CHB; rr += blockDim.x >> 5) {
                        const int i = ti * CHB + rr;
                        if (i >= n2 || k > i) continue;
                        double acc = 0.0;
#pragma unroll 8
                        for (int l = 0; l < CHB; ++l) acc = fma(sI[rr][l], sK[tx][l], acc);
                        double* o = A + (int64_t)(j0 + b + i) * r + j0 + b + k;
                        __stcg(o, __ldcg(o) - acc);
                    }
                }
            }
        }
        if (!count_barrier(st, ++epoch * nb)) return;
    }
    // Li: zero the strict upper part, invert the diagonal blocks (one CTA each)
    for (int64_t e = gtid; e < (int64_t)r * r; e += nthr) {
        const int64_t i = e / r, k = e % r;
        if (k / CHB > i / CHB) __stcg(Li + e, 0.0);
    }
    __shared__ double Lb[CHB][CHB + 1];
    for (int I = lb; I < nbk; I += nb) {
        const int i0 = I * CHB, b = min(CHB, r - i0);
        for (int e = threadIdx.x; e < b * b; e += blockDim.x) {
            const int i = e / b, k = e % b;
            Lb[i][k] = __ldcg(A + (int64_t)(i0 + i) * r + i0 + k);
        }
        __syncthreads();
        // column k of inv(L_II): forward substitution, one thread per column
        for (int k = threadIdx.x; k < b; k += blockDim.x) {
            for (int i = 0; i < b; ++i) {
                double s = (i == k) ? 1.0 : 0.0;
                for (int l = k; l < i; ++l) s -= Lb[i][l] * D[l][k];
                D[i][k] = (i < k) ? 0.0 : s / Lb[i][i];
            }
        }
        __syncthreads();
        for (int e = threadIdx.x; e < b * b; e += blockDim.x) {
            const int i = e / b, k = e % b;
            __stcg(Li + (int64_t)(i0 + i) * r + i0 + k, D[i][k]);
        }
        __syncthreads();
    }
    if (!count_barrier(st, ++epoch * nb)) return;
    // block rows I = 1..: Li[I][J] = -inv(L_II) sum_{K=J}^{I-1} L[I][K] Li[K][J]
    for (int I = 1; I < nbk; ++I) {
        const int i0 = I * CHB, bi = min(CHB, r - i0);
        // all (J, element) pairs of this block row in parallel: S first, kept in Li; each dot
        // product over eight lanes (strided k), added by a butterfly
        const int q8 = threadIdx.x & 7;
        for (int64_t e8 = gtid; e8 < (int64_t)8 * bi * i0; e8 += nthr) {
            const int64_t e = e8 >> 3;   // the eight lanes of an element take the same trip count
            const int ii = (int)(e / i0), jj = (int)(e % i0);   // row i0+ii, column jj < i0
            const int J = jj / CHB;
            const double* ar = A + (int64_t)(i0 + ii) * r;
            double s0 = 0.0, s1 = 0.0;
            int kk = J * CHB + q8;
            for (; kk + 8 < i0; kk += 16) {
                s0 = fma(__ldcg(ar + kk), __ldcg(Li + (int64_t)kk * r + jj), s0);
                s1 = fma(__ldcg(ar + kk + 8), __ldcg(Li + (int64_t)(kk + 8) * r + jj), s1);
            }
            if (kk < i0) s0 = fma(__ldcg(ar + kk), __ldcg(Li + (int64_t)kk * r + jj), s0);
            double sum = s0 + s1;
            for (int o = 4; o; o >>= 1) sum += __shfl_xor_sync(0xffffffffu, sum, o);
            if (q8 == 0) __stcg(Li + (int64_t)(i0 + ii) * r + jj, sum);
        }
        if (!count_barrier(st, ++epoch * nb)) return;
        for (int64_t e = gtid; e < (int64_t)bi * i0; e += nthr) {
            const int ii = (int)(e / i0), jj = (int)(e % i0);
            double s = 0.0;
            for (int kk = 0; kk <= ii; ++kk)
                s -= __ldcg(Li + (int64_t)(i0 + ii) * r + i0 + kk) * __ldcg(Li + (int64_t)(i0 + kk) * r + jj);
            // result for (ii, jj) reads column jj of S rows <= ii: write to a staging slot
            __stcg(A + (int64_t)(i0 + ii) * r + jj, s);   // the strict lower block part of A is no longer needed
        }
        if (!count_barrier(st, ++epoch * nb)) return;
        for (int64_t e = gtid; e < (int64_t)bi * i0; e += nthr) {
            const int ii = (int)(e / i0), jj = (int)(e % i0);
            __stcg(Li + (int64_t)(i0 + ii) * r + jj, __ldcg(A + (int64_t)(i0 + ii) * r + jj));
        }
        if (!count_barrier(st, ++epoch * nb)) return;
    }
}

// out[c][j] = in[j][c]   (in: rows x cols)
__global__ void k_transpose(const double* __restrict__ in, int64_t rows, int64_t cols, double* __restrict__ out) {
    __shared__ double tile[32][33];
    const int64_t c0 = blockIdx.x * 32, r0 = blockIdx.y * 32;
    for (int k = threadIdx.y; k < 32; k += blockDim.y) {
        const int64_t r = r0 + k, c = c0 + threadIdx.x;
        tile[k][threadIdx.x] = (r < rows && c < cols) ? in[r * cols + c] : 0.0;
    }
    __syncthreads();
    for (int k = threadIdx.y; k < 32; k += blockDim.y) {
        const int64_t c = c0 + k, r = r0 + threadIdx.x;
        if (c < cols && r < rows) out[c * rows + r] = tile[threadIdx.x][k];
    }
}

// Core, step 1 (terms grouped by their mode-0 vector c0):
//   W[c0 - cbeg][j*r2 + l] = sum_{t : c0(t) = c0} xin[t] P1[j][c1(t)] P2[l][c2(t)]
// with P1t = P1^T (C1 x r1) and P2t = P2^T (C2 x r2) so that l runs along
// contiguous memory. One CTA per (1024 outputs, c0); a thread takes four
// consecutive outputs, so one product xin P1 serves four FMAs (FP64 issue is
// the limit here), and the group's term data is staged in shared memory.
constexpr int kCoreOut = 4;
constexpr int kCoreStage = 256;
__global__ void __launch_bounds__(256) k_core_group_f64(const double* __restrict__ P1t, const double* __restrict__ P2t,
                                                        int r1, int r2, const int32_t* __restrict__ tcol,
                                                        const double* __restrict__ xin, const int32_t* __restrict__ perm,
                                                        const int32_t* __restrict__ off, int cbeg, double* __restrict__ W) {
    __shared__ double s_x[kCoreStage];
    __shared__ int s_c1[kCoreStage], s_c2[kCoreStage];
    const int64_t nn = (int64_t)r1 * r2;
    const int c0 = cbeg + blockIdx.y;
    const int64_t n0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) * kCoreOut;
    int jj[kCoreOut], ll[kCoreOut];
#pragma unroll
    for (int u = 0; u < kCoreOut; ++u) {
        const int64_t n = n0 + u < nn ? n0 + u : nn - 1;
        jj[u] = (int)(n / r2);
        ll[u] = (int)(n - (int64_t)jj[u] * r2);
    }
    const bool one_row = jj[0] == jj[kCoreOut - 1];
    double acc[kCoreOut] = {0.0, 0.0, 0.0, 0.0};
    const int kb = off[c0], ke = off[c0 + 1];
    for (int k0 = kb; k0 < ke; k0 += kCoreStage) {
        const int nk = min(kCoreStage, ke - k0);
        __syncthreads();
        for (int i = threadIdx.x; i < nk; i += blockDim.x) {
            const int t = perm[k0 + i];
            s_x[i] = xin[t];
            s_c1[i] = tcol[3 * t + 1];
            s_c2[i] = tcol[3 * t + 2];
        }
        __syncthreads();
        if (n0 >= nn) continue;
        for (int i = 0; i < nk; ++i) {
            const double* p1 = P1t + (int64_t)s_c1[i] * r1;
            const double* p2 = P2t + (int64_t)s_c2[i] * r2;
            if (one_row) {
                const double a = s_x[i] * p1[jj[0]];
#pragma unroll
                for (int u = 0; u < kCoreOut; ++u) acc[u] = fma(a, p2[ll[u]], acc[u]);
            } else {
#pragma unroll
                for (int u = 0; u < kCoreOut; ++u) acc[u] = fma(s_x[i] * p1[jj[u]], p2[ll[u]], acc[u]);
            }
        }
    }
#pragma unroll
    for (int u = 0; u < kCoreOut; ++u)
        if (n0 + u < nn) W[(int64_t)blockIdx.y * nn + n0 + u] = acc[u];
}

struct StoreRowAcc {     // C[m*ld + n] (+)= v
    double* p; int64_t ld; int accumulate;
    __device__ void operator()(int, int m, int n, double v) const {
        double* q = p + m * ld + n;
        *q = accumulate ? *q + v : v;
    }
};

template <class K>
int coop_blocks(K kernel, int threads, size_t smem, int num_sms, int64_t want) {
    int per_sm = 0;
    if (blocks_per_sm((const void*)kernel, threads, smem, &per_sm) != cudaSuccess || per_sm < 1)
        per_sm = 1;
    int64_t cap = (int64_t)per_sm * num_sms;
    int64_t n = want < cap ? want : cap;
    return (int)(n < 1 ? 1 : n);
}

}  // namespace

// ---------------------------------------------------------------------------
// launchers
// ---------------------------------------------------------------------------
cudaError_t launch_genvec(double* g, int R, int64_t N, double h, double sinc_step, double t_scale,
                          int kernel, double kappa, bool galerkin, cudaStream_t st) {
    static const GlRule gl = gauss_legendre();
    dim3 grid((unsigned)((2 * N + 255) / 256 < 1024 ? (2 * N + 255) / 256 : 1024), R);
    k_genvec<<<grid, 256, 0, st>>>(g, R, N, h, sinc_step, t_scale, kernel, kappa, galerkin ? 1 : 0, gl);
    count_kernels(1);
    return cudaGetLastError();
}

cudaError_t launch_assemble(const double* g, int64_t N, const int32_t* colq, const int32_t* woff,
                            const int32_t* wcnt, const int32_t* win, int64_t c0, int64_t ncols,
                            double* out, cudaStream_t st) {
    if (ncols <= 0) return cudaSuccess;
    static int nsm = 0;
    if (nsm == 0) {
        int dev = 0;
        if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
            nsm = 1;
    }
    const int64_t blocks = std::min<int64_t>(ncols * ((N + 256 * kAsmPer - 1) / (256 * kAsmPer)), (int64_t)nsm * 8);
    k_assemble<<<(unsigned)blocks, 256, 0, st>>>(g, N, colq, woff, wcnt, win, c0, ncols, out);
    count_kernels(1);
    return cudaGetLastError();
}

cudaError_t launch_norm_columns(double* a, int64_t C, int64_t N, double* norms, cudaStream_t st) {
    if (C <= 0) return cudaSuccess;
    k_norm_columns<<<(unsigned)C, 256, 0, st>>>(a, N, norms);
    count_kernels(1);
    return cudaGetLastError();
}

cudaError_t launch_identity(double* V, int64_t C, cudaStream_t st) {
    k_identity<<<(unsigned)((C * C + 255) / 256 < 4096 ? (C * C + 255) / 256 : 4096), 256, 0, st>>>(V, C);
    count_kernels(1);
    return cudaGetLastError();
}

// Split `cap` co-resident CTAs between jobs in proportion to `want`, at least
// one each; jobs beyond `cap` go to later launches. Returns the CTA counts.
static std::vector<int> split_ctas(const std::vector<int64_t>& want, int64_t cap) {
    const int n = (int)want.size();
    int64_t total = 0;
    for (int64_t w : want) total += w;
    std::vector<int> out(n, 1);
    if (total <= cap) {
        for (int i = 0; i < n; ++i) out[i] = (int)std::max<int64_t>(1, want[i]);
        return out;
    }
    const int64_t spare = std::max<int64_t>(0, cap - n);
    const int64_t extra_total = std::max<int64_t>(1, total - n);
    for (int i = 0; i < n; ++i) out[i] = 1 + (int)((std::max<int64_t>(1, want[i]) - 1) * spare / extra_total);
    return out;
}

cudaError_t launch_jacobi_multi(const JacobiJob* jobs, int njobs, int max_sweeps, double tol, int num_sms,
                                cudaStream_t st) {
    if (njobs < 1) return cudaSuccess;
    size_t smem = 0;
    std::vector<int64_t> want(njobs);
    for (int m = 0; m < njobs; ++m) {
        const int64_t C = jobs[m].C;
        const int64_t P = (C + (C & 1)) / 2;
        smem = std::max(smem, (size_t)(2 * sizeof(double) * P + sizeof(int) * (2 * P + 2 * (C + (C & 1)))));
        const int64_t items = P * P + C * P;
        want[m] = items <= 2048 ? 1 : (items + 1023) / 1024;
    }
    if (smem > 48 * 1024) {
        cudaError_t e = grow_smem((const void*)k_jacobi_multi, smem);
        if (e != cudaSuccess) return e;
    }
    int per_sm = 0;
    if (blocks_per_sm((const void*)k_jacobi_multi, 256, smem, &per_sm) != cudaSuccess || per_sm < 1)
        per_sm = 1;
    const int64_t resident = (int64_t)per_sm * num_sms;
    // a few large jobs: about two CTAs per SM in total (cheaper group barriers); many jobs:
    // every co-resident CTA
    const int64_t cap = njobs <= 3 ? std::min<int64_t>(resident, 2 * (int64_t)num_sms) : resident;
    // waves of at most `resident` jobs (one CTA each at least)
    for (int j0 = 0; j0 < njobs; j0 += (int)resident) {
        const int nj = (int)std::min<int64_t>(resident, njobs - j0);
        std::vector<int64_t> w(want.begin() + j0, want.begin() + j0 + nj);
        std::vector<int> nc = split_ctas(w, std::min(cap, resident));
        std::vector<JacobiMode> hm(nj);
        int cta = 0;
        for (int m = 0; m < nj; ++m) {
            const JacobiJob& J = jobs[j0 + m];
            hm[m] = JacobiMode{J.G, J.V, J.snap, J.st, (int)J.C, cta, nc[m], J.abs_floor, J.tau};
            cta += nc[m];
        }
        JacobiMode* dm = nullptr;
        cudaError_t e = cudaMallocAsync(&dm, sizeof(JacobiMode) * nj, st);
        if (e != cudaSuccess) return e;
        e = upload_h2d(dm, hm.data(), sizeof(JacobiMode) * nj, st);
        if (e == cudaSuccess) {
            JacobiArgs a{dm, nj, max_sweeps > 64 ? 64 : max_sweeps, tol};
            void* args[] = {&a};
            count_kernels(1);
            e = cudaLaunchCooperativeKernel((void*)k_jacobi_multi, dim3(cta), dim3(256), args, smem, st);
        }
        cudaFreeAsync(dm, st);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

cudaError_t launch_sort_select(int n, const SortSelectJob* jobs, double eps, double resolution, cudaStream_t st) {
    for (int j0 = 0; j0 < n; j0 += kSelMax) {
        const int nj = std::min(kSelMax, n - j0);
        SelArgs a{};
        a.eps = eps;
        a.resolution = resolution;
        int cmax = 1;
        for (int i = 0; i < nj; ++i) {
            const SortSelectJob& J = jobs[j0 + i];
            a.j[i] = SelJob{J.G, (int)J.C, J.forced, J.extra, J.perm, J.lam, J.inv_sqrt_lam, J.out,
                            J.dstride > 0 ? J.dstride : J.C + 1, J.resolution};
            cmax = std::max(cmax, (int)J.C);
        }
        const size_t smem = sizeof(double) * (2 * (size_t)cmax + 1);
        if (smem > 48 * 1024) {
            cudaError_t e = grow_smem((const void*)k_sort_select, smem);
            if (e != cudaSuccess) return e;
        }
        k_sort_select<<<nj, 1024, smem, st>>>(a);
        count_kernels(1);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

// (columns of L so far, done) of every job of a panel launch, for the caller's one read-back
__global__ void k_pchol_report(const PcholMode* m, int n, int* out) {
    for (int j = threadIdx.x; j < n; j += blockDim.x) {
        out[2 * j] = m[j].st->sweeps;
        out[2 * j + 1] = m[j].st->done;
    }
}

cudaError_t launch_pchol_panel(const PcholJob* jobs, int panel, int njobs, int num_sms, int* d_report, cudaStream_t st) {
    if (njobs < 1) return cudaSuccess;
    int dev = 0, optin = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess)
        optin = 48 * 1024;
    const int64_t budget = std::max<int64_t>(0, optin - 1024);   // the kernel's static variables take a few bytes
    std::vector<int64_t> want(njobs);
    // a warp per four rows and step; the candidate scratch holds 1024 CTAs per job
    for (int m = 0; m < njobs; ++m) want[m] = std::min<int64_t>(1024, std::max<int64_t>(1, (jobs[m].C + 7) / 8));
    // one CTA per SM (the own rows of L fill its shared memory): at most num_sms jobs a launch
    for (int j0 = 0, nj = 0; j0 < njobs; j0 += nj) {
        nj = std::min(num_sms, njobs - j0);
        std::vector<int64_t> w(want.begin() + j0, want.begin() + j0 + nj);
        std::vector<int> nc = split_ctas(w, num_sms);
        std::vector<PcholMode> hm(nj);
        size_t smem = 0;
        int cta = 0;
        for (int m = 0; m < nj; ++m) {
            const PcholJob& J = jobs[j0 + m];
            if (!J.Lp || panel < 1) return cudaErrorInvalidValue;
            const int64_t per = (J.C + nc[m] - 1) / nc[m];
            const int64_t fixed = 8 * ((int64_t)panel + 3 * per);   // row p of L, d, S[., p], the dots
            // panel columns of the own rows of L held in shared memory (the rest is read from L2)
            const int64_t kc = std::min<int64_t>(panel, std::max<int64_t>(0, (budget - fixed) / (8 * per)));
            smem = std::max(smem, (size_t)(fixed + 8 * per * kc));
            hm[m] = PcholMode{J.G, J.L, J.Lp, J.d, J.cand, J.piv, J.st, (int)J.C, J.kmax, cta, nc[m], (int)kc, panel,
                              J.delta};
            cta += nc[m];
            cudaError_t e = cudaMemsetAsync(&J.st->arrive, 0, sizeof(unsigned int), st);
            if (e != cudaSuccess) return e;
        }
        if ((int64_t)smem > budget) return cudaErrorInvalidValue;
        if (smem > 48 * 1024) {
            cudaError_t e = grow_smem((const void*)k_pchol_multi, smem);
            if (e != cudaSuccess) return e;
        }
        int per_sm = 0;
        if (blocks_per_sm((const void*)k_pchol_multi, 256, smem, &per_sm) != cudaSuccess || per_sm < 1 ||
            (int64_t)per_sm * num_sms < cta)
            return cudaErrorCooperativeLaunchTooLarge;
        PcholMode* dm = nullptr;
        cudaError_t e = cudaMallocAsync(&dm, sizeof(PcholMode) * nj, st);
        if (e != cudaSuccess) return e;
        e = upload_h2d(dm, hm.data(), sizeof(PcholMode) * nj, st);
        if (e == cudaSuccess) {
            PcholArgs a{dm, nj};
            void* args[] = {&a};
            count_kernels(1);
            e = cudaLaunchCooperativeKernel((void*)k_pchol_multi, dim3(cta), dim3(256), args, smem, st);
        }
        if (e == cudaSuccess && d_report) {
            k_pchol_report<<<1, 128, 0, st>>>(dm, nj, d_report + 2 * j0);
            count_kernels(1);
            e = cudaGetLastError();
        }
        cudaFreeAsync(dm, st);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

cudaError_t launch_chol_inv_multi(const CholJob* jobs, int njobs, int num_sms, cudaStream_t st) {
    if (njobs < 1) return cudaSuccess;
    std::vector<int64_t> want(njobs);
    for (int m = 0; m < njobs; ++m) want[m] = std::max<int64_t>(1, ((int64_t)jobs[m].r * jobs[m].r + 1023) / 1024);
    int per_sm = 0;
    if (blocks_per_sm((const void*)k_chol_inv_multi, 256, 0, &per_sm) != cudaSuccess || per_sm < 1)
        per_sm = 1;
    const int64_t resident = (int64_t)per_sm * num_sms;
    const int64_t cap = std::min<int64_t>(resident, std::max<int64_t>(num_sms, njobs));
    for (int j0 = 0; j0 < njobs; j0 += (int)resident) {
        const int nj = (int)std::min<int64_t>(resident, njobs - j0);
        std::vector<int64_t> w(want.begin() + j0, want.begin() + j0 + nj);
        std::vector<int> nc = split_ctas(w, cap);
        std::vector<CholMode> hm(nj);
        int cta = 0;
        for (int m = 0; m < nj; ++m) {
            const CholJob& J = jobs[j0 + m];
            hm[m] = CholMode{J.A, J.Li, J.st, J.r, cta, nc[m], J.gate};
            cudaError_t e0 = cudaMemsetAsync(&J.st->arrive, 0, sizeof(unsigned int), st);
            if (e0 != cudaSuccess) return e0;
            cta += nc[m];
        }
        CholMode* dm = nullptr;
        cudaError_t e = cudaMallocAsync(&dm, sizeof(CholMode) * nj, st);
        if (e != cudaSuccess) return e;
        e = upload_h2d(dm, hm.data(), sizeof(CholMode) * nj, st);
        if (e == cudaSuccess) {
            CholArgs a{dm, nj};
            void* args[] = {&a};
            count_kernels(1);
            e = cudaLaunchCooperativeKernel((void*)k_chol_inv_multi, dim3(cta), dim3(256), args, 0, st);
        }
        cudaFreeAsync(dm, st);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

cudaError_t launch_fold_norms(const double* xi, const int32_t* tcol, int64_t T, const double* n0,
                              const double* n1, const double* n2, double* xin, cudaStream_t st) {
    if (T <= 0) return cudaSuccess;
    k_fold_norms<<<(unsigned)((T + 255) / 256 < 4096 ? (T + 255) / 256 : 4096), 256, 0, st>>>(xi, tcol, T, n0, n1,
                                                                                             n2, xin);
    count_kernels(1);
    return cudaGetLastError();
}

cudaError_t launch_transpose(const double* in, int64_t rows, int64_t cols, double* out, cudaStream_t st) {
    dim3 grid((unsigned)((cols + 31) / 32), (unsigned)((rows + 31) / 32));
    k_transpose<<<grid, dim3(32, 8), 0, st>>>(in, rows, cols, out);
    count_kernels(1);
    return cudaGetLastError();
}

cudaError_t launch_core_f64(const double* P0, const double* P1t, const double* P2t, const int32_t* C, const int32_t* r,
                            const int32_t* tcol, const double* xin, const int32_t* perm, const int32_t* off,
                            double* W, int64_t w_cols, double* B, cudaStream_t st) {
    const int64_t nn = (int64_t)r[1] * r[2];
    for (int64_t c0 = 0; c0 < C[0]; c0 += w_cols) {
        const int cw = (int)std::min<int64_t>(w_cols, C[0] - c0);
        dim3 grid((unsigned)((nn + 256 * kCoreOut - 1) / (256 * kCoreOut)), (unsigned)cw);
        k_core_group_f64<<<grid, 256, 0, st>>>(P1t, P2t, r[1], r[2], tcol, xin, perm, off, (int)c0, W);
        count_kernels(1);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
        // B[i][n] (+)= sum_{c in chunk} P0[i][c0 + c] W[c][n]
        e = gemm_f64(r[0], (int)nn, cw, 1, RowK{P0 + c0, C[0]}, KRowN{W, nn},
                     StoreRowAcc{B, nn, c0 > 0 ? 1 : 0}, st);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

cudaError_t launch_core_step1_f64(const double* P1t, const double* P2t, int r1, int r2, const int32_t* tcol,
                                  const double* xin, const int32_t* perm, const int32_t* off, int cbeg, int ncols,
                                  double* W, cudaStream_t st) {
    const int64_t nn = (int64_t)r1 * r2;
    if (ncols < 1 || nn < 1) return cudaSuccess;
    dim3 grid((unsigned)((nn + 256 * kCoreOut - 1) / (256 * kCoreOut)), (unsigned)ncols);
    k_core_group_f64<<<grid, 256, 0, st>>>(P1t, P2t, r1, r2, tcol, xin, perm, off, cbeg, W);
    count_kernels(1);
    return cudaGetLastError();
}

cudaError_t launch_eval_f64(const double* const Z[3], const int32_t* r, const double* B, int64_t N,
                            const int32_t* zidx, int nslab, double* work, void* out, int out_f32,
                            cudaStream_t st) {
    const int r0 = r[0], r1 = r[1], r2 = r[2];
    double* M = work;                                  // [(a*r1+b)][s]
    double* T = work + (int64_t)r0 * r1 * nslab;       // [s][a][y]
    cudaError_t e = gemm_f64(r0 * r1, nslab, r2, 1, RowK{B, r2}, EvalZ3{Z[2], N, zidx},
                             StoreRow{M, nslab, 0}, st);
    if (e != cudaSuccess) return e;
    // T_s[a][y] = sum_b M_s[a][b] Z1[b][y]
    e = gemm_f64(r0, (int)N, r1, nslab, EvalM{M, r1, nslab}, KRowN{Z[1], N},
                 StoreRow{T, N, (int64_t)r0 * N}, st);
    if (e != cudaSuccess) return e;
    // S_s[x][y] = sum_a Z0[a][x] T_s[a][y]
    return gemm_f64((int)N, (int)N, r0, nslab, ColK{Z[0], N}, KRowNBatched{T, N, (int64_t)r0 * N},
                    StoreOut{out, N, out_f32}, st);
}

}  // namespace ls
