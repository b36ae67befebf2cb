// Galerkin matrix of the Tucker potential in a rank-one basis, Eq. (nuc_pot):
// v_km = <G_k (.) G_m, T> = sum_abc B_abc M0[km][a] M1[km][b] M2[km][c] with
// M_l[km][a] = sum_i g_k^l(i) g_m^l(i) Z_l[a][i] (1D Hadamard and scalar
// products). The elementwise and contraction steps live here; the products
// M_l = H_l Z_l^T and Y = M2 B^T run on the FP64-grade tensor-core product.
#include "ls_common.cuh"

namespace ls {
namespace {

// H[p][i] = g[k_p][i] * g[m_p][i] for the pairs p < np (rows of length N)
__global__ void k_hadamard_pairs(const double* __restrict__ g, int64_t N, const int2* __restrict__ pairs, int np,
                                 double* __restrict__ H) {
    const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e >= (int64_t)np * N) return;
    const int p = (int)(e / N);
    const int64_t i = e - (int64_t)p * N;
    const int2 km = pairs[p];
    H[e] = g[(int64_t)km.x * N + i] * g[(int64_t)km.y * N + i];
}

// v_p = sum_a M0[p][a] sum_b Y[p][a r1 + b] M1[p][b]; written to V[k][m] and V[m][k].
// One CTA per pair, fixed reduction order.
__global__ void __launch_bounds__(256) k_galerkin_contract(const double* __restrict__ Y, const double* __restrict__ M0,
                                                           const double* __restrict__ M1, int r0, int r1,
                                                           const int2* __restrict__ pairs, int nb,
                                                           double* __restrict__ V) {
    const int p = blockIdx.x;
    const double* y = Y + (int64_t)p * r0 * r1;
    const double* m0 = M0 + (int64_t)p * r0;
    const double* m1 = M1 + (int64_t)p * r1;
    double acc = 0.0;
    for (int a = threadIdx.x; a < r0; a += blockDim.x) {
        double z = 0.0;
        const double* ya = y + (int64_t)a * r1;
        for (int b = 0; b < r1; ++b) z = fma(ya[b], m1[b], z);
        acc = fma(m0[a], z, acc);
    }
    __shared__ double red[8];
    for (int o = 16; o; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
        const int2 km = pairs[p];
        V[(int64_t)km.x * nb + km.y] = t;
        V[(int64_t)km.y * nb + km.x] = t;
    }
}

}  // namespace

cudaError_t launch_hadamard_pairs(const double* g, int64_t N, const int2* pairs, int np, double* H, cudaStream_t st) {
    if ((int64_t)np * N == 0) return cudaSuccess;
    k_hadamard_pairs<<<(unsigned)(((int64_t)np * N + 255) / 256), 256, 0, st>>>(g, N, pairs, np, H);
    count_kernels(1);
    return cudaGetLastError();
}

cudaError_t launch_galerkin_contract(const double* Y, const double* M0, const double* M1, int r0, int r1,
                                     const int2* pairs, int np, int nb, double* V, cudaStream_t st) {
    if (np == 0) return cudaSuccess;
    k_galerkin_contract<<<np, 256, 0, st>>>(Y, M0, M1, r0, r1, pairs, nb, V);
    count_kernels(1);
    return cudaGetLastError();
}

}  // namespace ls
