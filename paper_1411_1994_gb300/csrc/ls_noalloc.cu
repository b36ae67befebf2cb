// Slab evaluation that allocates no device memory.
//
// lattice_sum_eval_slab needs scratch space for the two intermediate products
// of every slab (M = B x3 Z3[:, i3] and T = M Z2) and takes it from the
// stream-ordered allocator. Some callers cannot allocate device memory at the
// point where they want values: a host application that reserved all of its
// device memory in one arena at start-up and forbids further allocations, or a
// latency-critical loop that must not wait on the driver's allocator. For them
// lattice_sum_eval_slab_noalloc runs the same FP64 kernels with their scratch
// in the file-scope array below, which every GPU that loads this library holds
// for the life of the process.
#include <cuda.h>   // CUcontext and the driver prototypes (reached through the runtime, no -lcuda)

#include <algorithm>
#include <mutex>
#include <string>

#include "ls_common.cuh"

namespace {

// 32 MiB of scratch: slab indices first, then the per-slab products.
constexpr int64_t kScratchBytes = 32ll << 20;
constexpr int64_t kIndexBytes = 64ll << 10;          // up to 16384 int32 slab indices per chunk
constexpr int64_t kWorkDoubles = (kScratchBytes - kIndexBytes) / 8;

static __device__ __align__(256) unsigned char g_eval_scratch[kScratchBytes];

// Slab indices travel to the device as a kernel argument (copied at launch), so
// no host buffer has to outlive the call and no host-to-device copy is made.
constexpr int kIdxPerLaunch = 960;   // 3840 bytes of indices, within the 4 KB argument limit
struct IdxPack {
    int32_t n;
    int32_t z[kIdxPerLaunch];
};

__global__ void k_put_indices(int32_t* dst, IdxPack p) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < p.n) dst[i] = p.z[i];
}

// The array's device address, looked up once per device and context. A context
// that was torn down and created again (cudaDeviceReset) gets a new id, and the
// address is looked up again for it.
struct ScratchAddr {
    unsigned long long ctx_id = 0;
    void* ptr = nullptr;
};
std::mutex g_mu;
ScratchAddr g_scratch[64];

typedef CUresult (*CtxGetCurrentFn)(CUcontext*);
typedef CUresult (*CtxGetIdFn)(CUcontext, unsigned long long*);

// id of the calling thread's current context, or 0 when the driver cannot say
unsigned long long current_ctx_id() {
    static CtxGetCurrentFn get_cur = nullptr;
    static CtxGetIdFn get_id = nullptr;
    static bool tried = false;
    if (!tried) {
        tried = true;
        void* f = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            get_cur = reinterpret_cast<CtxGetCurrentFn>(f);
        f = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            get_id = reinterpret_cast<CtxGetIdFn>(f);
    }
    if (!get_cur || !get_id) return 0;
    CUcontext c = nullptr;
    unsigned long long id = 0;
    if (get_cur(&c) != CUDA_SUCCESS || !c || get_id(c, &id) != CUDA_SUCCESS) return 0;
    return id;
}

int fail(int code, const std::string& msg) {
    ls::set_global_error(msg.c_str());
    return code;
}

}  // namespace

extern "C" int lattice_sum_eval_slab_noalloc(const double* Z0, const double* Z1, const double* Z2, const double* core,
                                             const int32_t* ranks, int64_t N, const int64_t* z_index, int32_t nslab,
                                             void* out_dev, int32_t out_dtype, void* stream) {
    if (!Z0 || !Z1 || !Z2 || !core || !ranks || (nslab > 0 && (!z_index || !out_dev)) || nslab < 0)
        return fail(LS_ERR_ARG, "eval_slab_noalloc: NULL argument");
    if (out_dtype != LS_OUT_F64 && out_dtype != LS_OUT_F32) return fail(LS_ERR_ARG, "eval_slab_noalloc: bad out_dtype");
    if (N < 1 || N > (1 << 20)) return fail(LS_ERR_ARG, "eval_slab_noalloc: N out of range");
    const int32_t r[3] = {ranks[0], ranks[1], ranks[2]};
    if (r[0] < 1 || r[1] < 1 || r[2] < 1) return fail(LS_ERR_ARG, "eval_slab_noalloc: ranks must be >= 1");
    for (int32_t s = 0; s < nslab; ++s)
        if (z_index[s] < 0 || z_index[s] >= N) return fail(LS_ERR_ARG, "eval_slab_noalloc: z index out of range");
    if (nslab == 0) return LS_OK;
    // scratch per slab: M (r0 r1) + T (r0 N) doubles
    const int64_t per = (int64_t)r[0] * r[1] + (int64_t)r[0] * N;
    if (per > kWorkDoubles)
        return fail(LS_ERR_ARG, "eval_slab_noalloc: one slab needs " + std::to_string(per * 8) +
                                    " bytes of scratch; the static maximum is " + std::to_string(kWorkDoubles * 8));
    const int64_t chunk = std::min<int64_t>({(int64_t)nslab, kWorkDoubles / per, kIndexBytes / 4});

    // once per device (and context), with that device current: the device address of the array
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64)
        return fail(LS_ERR_CUDA, "eval_slab_noalloc: no usable CUDA device");
    void* base = nullptr;
    {
        std::lock_guard<std::mutex> g(g_mu);
        const unsigned long long id = current_ctx_id();
        ScratchAddr& sa = g_scratch[dev];
        if (!sa.ptr || id == 0 || id != sa.ctx_id) {
            void* p = nullptr;
            cudaError_t e = cudaGetSymbolAddress(&p, g_eval_scratch);
            if (e != cudaSuccess)
                return fail(LS_ERR_CUDA, std::string("eval_slab_noalloc: cudaGetSymbolAddress: ") + cudaGetErrorString(e));
            sa.ptr = p;
            sa.ctx_id = id;
        }
        base = sa.ptr;
    }
    int32_t* d_z = static_cast<int32_t*>(base);
    double* work = reinterpret_cast<double*>(static_cast<unsigned char*>(base) + kIndexBytes);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const double* Z[3] = {Z0, Z1, Z2};
    const size_t esz = out_dtype == LS_OUT_F32 ? 4 : 8;
    for (int64_t s0 = 0; s0 < nslab; s0 += chunk) {
        const int64_t ns = std::min<int64_t>(chunk, nslab - s0);
        // this chunk's indices into the array's index area (kernel arguments, ordered after
        // the previous chunk's kernels on this stream)
        cudaError_t e = cudaSuccess;
        for (int64_t b0 = 0; b0 < ns && e == cudaSuccess; b0 += kIdxPerLaunch) {
            IdxPack pk;
            pk.n = (int32_t)std::min<int64_t>(kIdxPerLaunch, ns - b0);
            for (int32_t s = 0; s < pk.n; ++s) pk.z[s] = (int32_t)z_index[s0 + b0 + s];
            k_put_indices<<<(pk.n + 255) / 256, 256, 0, st>>>(d_z + b0, pk);
            ls::count_kernels(1);
            e = cudaGetLastError();
        }
        if (e == cudaSuccess) {
            char* o = static_cast<char*>(out_dev) + (size_t)s0 * N * N * esz;
            e = ls::launch_eval_f64(Z, r, core, N, d_z, (int)ns, work, o, out_dtype == LS_OUT_F32, st);
        }
        if (e != cudaSuccess)
            return fail(LS_ERR_CUDA, std::string("eval_slab_noalloc: ") + cudaGetErrorString(e));
    }
    return LS_OK;
}
