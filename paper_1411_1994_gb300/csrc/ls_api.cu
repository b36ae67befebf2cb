// Host implementation of the C ABI declared in include/lattice_sum.h.
//
// The host side only validates arguments, snaps site positions to grid
// vertices, deduplicates defect windows and keeps the term -> column maps;
// every arithmetic step of the path runs in the kernels of ls_f64.cu and
// ls_tc.cu. Device buffers come from the stream-ordered allocator
// (cudaMallocAsync), so building and dropping contexts in a loop does not
// pay for cudaMalloc after the first round.
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <deque>
#include <atomic>
#include <mutex>
#include <map>
#include <string>
#include <unordered_map>
#include <vector>

#include "ls_common.cuh"
#include "ls_eval.cuh"
#include "ls_tc.cuh"

using namespace ls;

namespace ls {
void count_kernels(int n);
}

namespace {

thread_local std::string g_create_error;

// ---------------------------------------------------------------------------
// tracing: CUDA-event pairs per step, kernel-launch and copy-byte counters
// ---------------------------------------------------------------------------
struct TraceRec {
    const char* name;
    cudaEvent_t a, b;
    int kernels;
};
struct Tracer {
    std::mutex mu;
    bool on = false;
    std::vector<TraceRec> recs;
    std::vector<cudaEvent_t> pool;
    std::atomic<long long> kernels{0}, h2d{0}, d2h{0};
    cudaEvent_t get() {
        if (!pool.empty()) {
            cudaEvent_t e = pool.back();
            pool.pop_back();
            return e;
        }
        cudaEvent_t e = nullptr;
        cudaEventCreate(&e);
        return e;
    }
};
Tracer& tracer() {
    static Tracer* t = new Tracer();
    return *t;
}

struct HostBlock {
    ls_block b;
    std::vector<int32_t> m[3];   // vertex index of each site, per mode
};

// Defect window lists of one mode -> key index (the order of first appearance), looked up by a
// 64-bit hash of the list and compared on a hit: no allocation per lookup (a context with
// thousands of defects looks one up per defect and mode).
struct KeyIndex {
    std::unordered_multimap<uint64_t, int32_t> by_hash;   // lists of two or more windows
    std::vector<int32_t> single;       // one-window lists (point defects, single sites): by vertex
    std::vector<int32_t> flat;         // key k: flat[off[k] .. off[k + 1])
    std::vector<int64_t> off{0};
    static uint64_t hash(const int32_t* w, int n) {
        uint64_t h = 1469598103934665603ull ^ (uint64_t)n;   // FNV-1a over the words
        for (int i = 0; i < n; ++i) {
            h ^= (uint32_t)w[i];
            h *= 1099511628211ull;
        }
        return h;
    }
    int32_t size() const { return (int32_t)(off.size() - 1); }
    int32_t find(const int32_t* w, int n, uint64_t h) const {
        if (n == 1 && w[0] >= 0) return w[0] < (int32_t)single.size() ? single[w[0]] : -1;
        const auto rng = by_hash.equal_range(h);
        for (auto it = rng.first; it != rng.second; ++it) {
            const int32_t k = it->second;
            if (off[k + 1] - off[k] == n && std::equal(w, w + n, flat.begin() + off[k])) return k;
        }
        return -1;
    }
    int32_t add(const int32_t* w, int n, uint64_t h) {
        const int32_t k = size();
        flat.insert(flat.end(), w, w + n);
        off.push_back((int64_t)flat.size());
        if (n == 1 && w[0] >= 0) {
            if (w[0] >= (int32_t)single.size()) single.resize((size_t)w[0] + 1, -1);
            single[w[0]] = k;
        } else {
            by_hash.emplace(h, k);
        }
        return k;
    }
};

struct ModeCols {
    int64_t C = 0, cap = 0;
    double* d_cols = nullptr;                    // [cap][N]
    std::vector<int32_t> colq, woff, wcnt, win;  // host descriptors
    int32_t* d_desc = nullptr;                   // colq | woff | wcnt (3 * cap) on device
    int32_t* d_win = nullptr;
    int64_t wincap = 0;
    KeyIndex keys;                               // defect window set -> key index
    std::vector<int32_t> count;                  // terms per column
};

// capacity for `more` elements, growing geometrically (repeated calls stay linear)
template <class V>
void reserve_more(V& v, size_t more) {
    if (v.size() + more > v.capacity()) v.reserve(std::max(v.size() + more, 2 * v.capacity()));
}

}  // namespace

struct ls_ctx {
    ls_params p{};
    cudaStream_t st = nullptr;
    int num_sms = 0;
    double h = 0.0;
    std::string err;
    std::vector<HostBlock> blocks;
    double* d_g = nullptr;
    ModeCols mode[3];
    std::vector<int32_t> tcol;   // [T][3]
    std::vector<double> xi;      // [T]
    bool reduced = false;
    // reduction outputs
    int32_t r[3] = {0, 0, 0};
    double* d_norms[3] = {nullptr, nullptr, nullptr};
    double* d_sigma[3] = {nullptr, nullptr, nullptr};
    double* d_Z[3] = {nullptr, nullptr, nullptr};
    double* d_P[3] = {nullptr, nullptr, nullptr};
    double* d_B = nullptr;
    double* d_Q[3] = {nullptr, nullptr, nullptr};   // non-squaring route: orthonormal basis of each side matrix's range
    int32_t mq[3] = {0, 0, 0};                      // its dimension
    ls_tucker_info last_info{};                     // what the reduction reported
    int32_t* d_tcol = nullptr;
    double* d_xi = nullptr;
    double* d_xin = nullptr;
    DtEvalCache* eval_cache = nullptr;   // tensor-core operands of the slab evaluation
    std::vector<void*> allocs;
    // Tucker-reference variant (LS_FLAG_TUCKER_REF; Thm 3.1(B), Sec. 4.1, Thm 4.3)
    bool tucker = false;
    int r_ref = 0;
    double* d_t = nullptr;       // [r_ref][2N] reference Tucker vectors
    double* d_gp = nullptr;      // [R][2N] projected reference vectors g'_q = t^T t g_q
    double bnorm2 = 0.0;         // ||b||^2 of the reference core
    ModeCols tmode[3];           // side matrices: the r_ref windowed Tucker vectors of each key
    std::vector<int32_t> tkey;   // [S][3] key of each Tucker term in each mode
    std::vector<double> txi;     // [S] charge (change) of each Tucker term
    const double* gsrc() const { return tucker ? d_gp : d_g; }
};

namespace {

int fail(ls_ctx* ctx, int code, const char* fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    if (ctx) ctx->err = buf;
    else g_create_error = buf;
    return code;
}

#define CU(call)                                                                                  \
    do {                                                                                          \
        cudaError_t e_ = (call);                                                                  \
        if (e_ != cudaSuccess)                                                                    \
            return fail(ctx, e_ == cudaErrorMemoryAllocation ? LS_ERR_OOM : LS_ERR_CUDA, "%s: %s (%s:%d)", \
                        #call, cudaGetErrorString(e_), __FILE__, __LINE__);                       \
    } while (0)

// failure injection for tests: the n-th context allocation from now fails (-1: none)
std::atomic<long long> g_fail_after{-1};

template <class T>
cudaError_t dalloc(ls_ctx* ctx, T** p, int64_t count) {
    *p = nullptr;
    if (count <= 0) count = 1;
    long long n = g_fail_after.load();
    while (n >= 0 && !g_fail_after.compare_exchange_weak(n, n - 1)) {}
    if (n == 0) return cudaErrorMemoryAllocation;
    void* q = nullptr;
    cudaError_t e = cudaMallocAsync(&q, (size_t)count * sizeof(T), ctx->st);
    if (e != cudaSuccess) return e;
    ctx->allocs.push_back(q);
    *p = static_cast<T*>(q);
    return cudaSuccess;
}

void dfree(ls_ctx* ctx, void* p) {
    if (!p) return;
    auto it = std::find(ctx->allocs.begin(), ctx->allocs.end(), p);
    if (it != ctx->allocs.end()) ctx->allocs.erase(it);
    cudaFreeAsync(p, ctx->st);
}

bool snap_vertex(const ls_ctx* ctx, double pos, int32_t* m) {
    const double x = floor((pos - ctx->p.box_lo) / ctx->h + 0.5);
    if (!(x >= 0.0 && x <= (double)ctx->p.N)) return false;
    *m = (int32_t)x;
    return true;
}

void keep_pool(int dev) {
    static bool done[64] = {false};
    if (dev < 0 || dev >= 64 || done[dev]) return;
    cudaMemPool_t pool;
    if (cudaDeviceGetDefaultMemPool(&pool, dev) == cudaSuccess) {
        uint64_t thr = UINT64_MAX;
        cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr);
    }
    done[dev] = true;
}

// make room for `add` more columns in mode l and append their descriptors;
// then assemble them on the device
int append_columns_to(ls_ctx* ctx, ModeCols& mc, const double* gsrc, const std::vector<int32_t>& q,
                      const std::vector<std::vector<int32_t>>& wins);
int append_columns(ls_ctx* ctx, int l, const std::vector<int32_t>& q, const std::vector<std::vector<int32_t>>& wins) {
    return append_columns_to(ctx, ctx->mode[l], ctx->gsrc(), q, wins);
}
// the Tucker side columns of new keys: r_ref windowed (or assembled) reference Tucker vectors each
int append_side(ls_ctx* ctx, int l, const std::vector<std::vector<int32_t>>& key_wins) {
    std::vector<int32_t> q;
    std::vector<std::vector<int32_t>> wins;
    for (const auto& w : key_wins)
        for (int k = 0; k < ctx->r_ref; ++k) {
            q.push_back(k);
            wins.push_back(w);
        }
    return append_columns_to(ctx, ctx->tmode[l], ctx->d_t, q, wins);
}
int append_columns_to(ls_ctx* ctx, ModeCols& mc, const double* gsrc, const std::vector<int32_t>& q,
                      const std::vector<std::vector<int32_t>>& wins) {
    const int64_t add = (int64_t)q.size();
    if (add == 0) return LS_OK;
    const int64_t N = ctx->p.N;
    const int64_t c0 = mc.C;
    if (mc.C + add > mc.cap) {
        int64_t ncap = std::max<int64_t>(mc.C + add, 2 * mc.cap);
        double* nc = nullptr;
        int32_t* nd = nullptr;
        CU(dalloc(ctx, &nc, ncap * N));
        CU(dalloc(ctx, &nd, 3 * ncap));
        if (mc.C > 0) CU(cudaMemcpyAsync(nc, mc.d_cols, (size_t)mc.C * N * sizeof(double), cudaMemcpyDeviceToDevice, ctx->st));
        dfree(ctx, mc.d_cols);
        dfree(ctx, mc.d_desc);
        mc.d_cols = nc;
        mc.d_desc = nd;
        mc.cap = ncap;
    }
    for (int64_t i = 0; i < add; ++i) {
        mc.colq.push_back(q[i]);
        mc.woff.push_back((int32_t)mc.win.size());
        mc.wcnt.push_back((int32_t)wins[i].size());
        for (int32_t m : wins[i]) mc.win.push_back(m);
        mc.count.push_back(0);
    }
    mc.C += add;
    if ((int64_t)mc.win.size() > mc.wincap) {
        int64_t nw = std::max<int64_t>((int64_t)mc.win.size(), 2 * mc.wincap);
        int32_t* d = nullptr;
        CU(dalloc(ctx, &d, nw));
        dfree(ctx, mc.d_win);
        mc.d_win = d;
        mc.wincap = nw;
    }
    // descriptors live at d_desc: colq [0,cap), woff [cap,2cap), wcnt [2cap,3cap)
    CU(upload_h2d(mc.d_desc, mc.colq.data(), mc.C * sizeof(int32_t), ctx->st));
    count_h2d((int64_t)(mc.C * sizeof(int32_t)));
    CU(upload_h2d(mc.d_desc + mc.cap, mc.woff.data(), mc.C * sizeof(int32_t), ctx->st));
    count_h2d((int64_t)(mc.C * sizeof(int32_t)));
    CU(upload_h2d(mc.d_desc + 2 * mc.cap, mc.wcnt.data(), mc.C * sizeof(int32_t), ctx->st));
    count_h2d((int64_t)(mc.C * sizeof(int32_t)));
    CU(upload_h2d(mc.d_win, mc.win.data(), mc.win.size() * sizeof(int32_t), ctx->st));
    count_h2d((int64_t)(mc.win.size() * sizeof(int32_t)));
    Scope sc_asm("assemble", ctx->st);
    CU(launch_assemble(gsrc, N, mc.d_desc, mc.d_desc + mc.cap, mc.d_desc + 2 * mc.cap, mc.d_win, c0, add,
                       mc.d_cols, ctx->st));
    // (the uploads went through pinned staging: the host vectors may change at once)
    return LS_OK;
}

// The reference Tucker tensor of the Tucker-reference variant (Eq. TuckRef_sum, Thm 3.1(B)):
// the RHOSVD of the reference canonical tensor sum_q g_q (x) g_q (x) g_q on the doubled grid.
// Its side matrix has the unit vectors g_q/|g_q| as columns; one-sided Jacobi on those R rows
// (M G = rotated rows of norms sigma_k) gives the leading left singular vectors of the side
// matrix as the rotated rows over sigma_k; r_ref by the eps rule at ref_eps. Then the
// projected vectors g'_q = t^T (t g_q) (the reference tensor written as a canonical sum,
// b = sum_q h_q^(x3), h_q = t g_q) and ||b||^2 = sum_{q,q'} (h_q . h_q')^3.
int make_reference_tucker(ls_ctx* ctx) {
    cudaStream_t st = ctx->st;
    const int R = ctx->p.R;
    const int64_t N2 = 2 * ctx->p.N;
    const double u = 1.1102230246251565e-16;
    double *gn = nullptr, *nrm = nullptr, *M = nullptr, *sig2 = nullptr, *lam = nullptr, *isl = nullptr,
           *sel = nullptr, *H = nullptr, *HH = nullptr, *b2 = nullptr;
    int32_t* perm = nullptr;
    DevStatus* ds = nullptr;
    unsigned* cmax = nullptr;
    CU(dalloc(ctx, &gn, R * N2));
    CU(dalloc(ctx, &nrm, R));
    CU(dalloc(ctx, &M, (int64_t)R * R));
    CU(dalloc(ctx, &sig2, R));
    CU(dalloc(ctx, &lam, R));
    CU(dalloc(ctx, &isl, R));
    CU(dalloc(ctx, &sel, 3));
    CU(dalloc(ctx, &perm, R));
    CU(dalloc(ctx, &ds, 2));
    CU(dalloc(ctx, &cmax, 64));
    CU(cudaMemsetAsync(ds, 0, 2 * sizeof(DevStatus), st));
    CU(cudaMemsetAsync(cmax, 0, 64 * sizeof(unsigned), st));
    CU(cudaMemcpyAsync(gn, ctx->d_g, sizeof(double) * R * N2, cudaMemcpyDeviceToDevice, st));
    CU(launch_norm_columns(gn, R, N2, nrm, st));
    const OsjJob J{gn, N2, (int)N2, M, R, sig2, ds, 8.0 * u * sqrt((double)N2), cmax};
    CU(launch_osj(&J, 1, 40, ctx->num_sms, st));
    SortSelectJob sj{sig2, R, 0, nullptr, perm, lam, isl, sel};
    sj.dstride = 1;
    sj.resolution = 0.0;
    CU(launch_sort_select(1, &sj, ctx->p.ref_eps, 0.0, st));
    double hsel[3];
    DevStatus hds;
    CU(cudaMemcpyAsync(hsel, sel, sizeof hsel, cudaMemcpyDeviceToHost, st));
    CU(cudaMemcpyAsync(&hds, ds, sizeof hds, cudaMemcpyDeviceToHost, st));
    CU(cudaStreamSynchronize(st));
    if (hds.flag == FLAG_TIMEOUT) return fail(ctx, LS_ERR_TIMEOUT, "create: reference Tucker: a bounded wait timed out");
    if (hds.flag == FLAG_NOCONVERGE) return fail(ctx, LS_ERR_NOCONVERGE, "create: reference Tucker: no convergence");
    const int r = ctx->r_ref = std::max(1, (int)hsel[0]);
    CU(dalloc(ctx, &ctx->d_t, (int64_t)r * N2));
    CU(dalloc(ctx, &ctx->d_gp, R * N2));
    CU(dalloc(ctx, &H, (int64_t)r * R));
    CU(dalloc(ctx, &HH, (int64_t)R * R));
    CU(dalloc(ctx, &b2, 1));
    // t_k = (rotated row perm[k]) / sigma_k
    CU(launch_gather_rows(gn, N2, perm, r, isl, ctx->d_t, st));
    {
        std::string err;
        X64Mat xs[1], ys[1];
        int64_t ld[1];
        double* D[1];
        xs[0] = X64Mat{ctx->d_t, r, N2, N2, 1, nullptr};   // t (r x 2N)
        ys[0] = X64Mat{ctx->d_g, R, N2, N2, 1, nullptr};   // g (R x 2N)
        ld[0] = R;
        D[0] = H;
        int rc = x64_nt(1, xs, ys, D, ld, &ds[1].flag, st, &err);   // H = t g^T (r x R)
        xs[0] = X64Mat{H, R, r, 1, R, nullptr};               // H^T (R x r)
        ys[0] = X64Mat{ctx->d_t, N2, r, 1, N2, nullptr};      // t^T (2N x r)
        ld[0] = N2;
        D[0] = ctx->d_gp;
        if (rc == LS_OK) rc = x64_nt(1, xs, ys, D, ld, &ds[1].flag, st, &err);   // g' = H^T t
        ys[0] = X64Mat{H, R, r, 1, R, nullptr};
        ld[0] = R;
        D[0] = HH;
        if (rc == LS_OK) rc = x64_nt(1, xs, ys, D, ld, &ds[1].flag, st, &err);   // H^T H (R x R)
        if (rc != LS_OK) return fail(ctx, rc, "create: reference Tucker: %s", err.c_str());
    }
    CU(launch_sum_cubes(HH, (int64_t)R * R, b2, st));
    DevStatus hd1;
    CU(cudaMemcpyAsync(&ctx->bnorm2, b2, sizeof(double), cudaMemcpyDeviceToHost, st));
    CU(cudaMemcpyAsync(&hd1, ds + 1, sizeof hd1, cudaMemcpyDeviceToHost, st));
    CU(cudaStreamSynchronize(st));
    if (hd1.flag == FLAG_TIMEOUT) return fail(ctx, LS_ERR_TIMEOUT, "create: reference Tucker: a bounded wait timed out");
    for (void* q : {(void*)gn, (void*)nrm, (void*)M, (void*)sig2, (void*)lam, (void*)isl, (void*)sel, (void*)perm,
                    (void*)ds, (void*)cmax, (void*)H, (void*)HH, (void*)b2})
        dfree(ctx, q);
    return LS_OK;
}

// max over r of |sum_q w_q exp(-t_q^2 r^2) - p(r)| / m(r) for the kernel family (see
// LS_KERNEL_*): p = exp(-kappa r)/r, m = 1/r (the Newton kernel at kappa = 0: the relative
// error); p = exp(-kappa r), m = 1 (Slater); p = 1/r^3, m = 1/r^3 (dipole). Weights
// w = h a(t) cosh(u)/s with the Laplace-Gauss densities a(t) of Sec. 2.3 (halved at u = 0).
double quad_max_err(int R, double hs, double s, int kernel, double kappa, const std::vector<double>& r) {
    std::vector<double> t(R), w(R);
    const double spi = 1.7724538509055160273;
    const int q0 = (kernel == LS_KERNEL_YUKAWA && kappa == 0.0) ? 0 : 1;
    for (int i = 0; i < R; ++i) {
        const int q = i + q0;
        t[i] = sinh(q * hs) / s;
        if (kernel == LS_KERNEL_SLATER) {
            w[i] = hs * cosh(q * hs) / s * (kappa / spi) / (t[i] * t[i]) * exp(-kappa * kappa / (4.0 * t[i] * t[i]));
        } else if (kernel == LS_KERNEL_DIPOLE) {
            w[i] = hs * cosh(q * hs) / s * (4.0 / spi) * t[i] * t[i];
        } else {
            w[i] = (q == 0) ? hs / (s * spi) : 2.0 * hs * cosh(q * hs) / (s * spi);
            if (kappa > 0.0) w[i] *= exp(-kappa * kappa / (4.0 * t[i] * t[i]));
        }
    }
    double e = 0.0;
    for (double x : r) {
        double acc = 0.0;
        for (int i = 0; i < R; ++i) acc += w[i] * exp(-t[i] * t[i] * x * x);
        double d;
        if (kernel == LS_KERNEL_SLATER) d = fabs(acc - exp(-kappa * x));
        else if (kernel == LS_KERNEL_DIPOLE) d = fabs(x * x * x * acc - 1.0);
        else d = fabs(x * acc - exp(-kappa * x));
        e = std::max(e, d);
    }
    return e;
}

// the kernel family and its parameter: LS_OK or a message
const char* kernel_args_bad(int kernel, double kappa) {
    if (kernel != LS_KERNEL_YUKAWA && kernel != LS_KERNEL_SLATER && kernel != LS_KERNEL_DIPOLE) return "unknown kernel";
    if (!(kappa >= 0.0) || !std::isfinite(kappa)) return "kappa must be finite and >= 0";
    if (kernel == LS_KERNEL_SLATER && !(kappa > 0.0)) return "the Slater kernel needs kappa > 0";
    if (kernel == LS_KERNEL_DIPOLE && kappa != 0.0) return "the dipole kernel takes kappa = 0";
    return nullptr;
}

}  // namespace

namespace ls {
void count_kernels(int n) { tracer().kernels += n; }
void count_h2d(int64_t n) { tracer().h2d += n; }
void count_d2h(int64_t n) { tracer().d2h += n; }
void set_global_error(const char* msg) { g_create_error = msg; }

// The reference-vector cache (LS_FLAG_CACHE_GENVEC): the inputs of k_genvec, bit for bit,
// and the vectors it wrote, in device memory owned by the cache (cudaMalloc: the entries
// outlive every context and stream). FIFO of at most kGenvecCacheMax entries.
struct GenvecKey {
    int dev; int64_t N; double h; int R; double sinc_step, t_scale; int kernel; double kappa; int galerkin;
    bool operator==(const GenvecKey& o) const {
        return dev == o.dev && N == o.N && memcmp(&h, &o.h, 8) == 0 && R == o.R &&
               memcmp(&sinc_step, &o.sinc_step, 8) == 0 && memcmp(&t_scale, &o.t_scale, 8) == 0 &&
               kernel == o.kernel && memcmp(&kappa, &o.kappa, 8) == 0 && galerkin == o.galerkin;
    }
};
struct GenvecEntry {
    GenvecKey key;
    double* d;
};
constexpr size_t kGenvecCacheMax = 8;
std::mutex g_genvec_mu;
std::deque<GenvecEntry>& genvec_cache() {
    static std::deque<GenvecEntry>* c = new std::deque<GenvecEntry>();
    return *c;
}

Scope::Scope(const char* n, cudaStream_t s) : name(n), st(s) {
    nvtxRangePushA(n);
    Tracer& t = tracer();
    if (!t.on) return;
    std::lock_guard<std::mutex> g(t.mu);
    a = t.get();
    k0 = t.kernels.load();
    cudaEventRecord(a, st);
}

Scope::~Scope() {
    nvtxRangePop();
    if (!a) return;
    Tracer& t = tracer();
    std::lock_guard<std::mutex> g(t.mu);
    cudaEvent_t b = t.get();
    cudaEventRecord(b, st);
    t.recs.push_back({name, a, b, (int)(t.kernels.load() - k0)});
}
}  // namespace ls

extern "C" {

int lattice_sum_fit_t_scale(int32_t R, double sinc_step, double r_min, double r_max, double* t_scale_out,
                            double* max_rel_err_out) {
    return lattice_sum_fit_t_scale_kernel(R, sinc_step, LS_KERNEL_YUKAWA, 0.0, r_min, r_max, t_scale_out,
                                          max_rel_err_out);
}

int lattice_sum_fit_t_scale_kernel(int32_t R, double sinc_step, int32_t kernel, double kappa, double r_min,
                                   double r_max, double* t_scale_out, double* max_rel_err_out) {
    ls_ctx* ctx = nullptr;
    if (R < 1 || R > 256 || !(sinc_step > 0) || !(r_min > 0) || !(r_max > r_min) || !t_scale_out ||
        kernel_args_bad(kernel, kappa))
        return fail(ctx, LS_ERR_ARG, "fit_t_scale: bad arguments");
    std::vector<double> r(600);
    for (int i = 0; i < 600; ++i) r[i] = r_min * pow(r_max / r_min, i / 599.0);
    double best = 1e300, bx = 0.0;
    const double lo = log(1e-2);
    double hi = log(1e5);
    // for kappa > 0 keep the first node's screening factor representable: kappa^2/(4 t_1^2) <= 600
    if (kappa > 0.0) hi = std::min(hi, log(sinh(sinc_step) * sqrt(2400.0) / kappa));
    if (!(hi > lo)) return fail(ctx, LS_ERR_ARG, "fit_t_scale: kappa=%g too large for sinc_step=%g", kappa, sinc_step);
    const int ns = 241;
    std::vector<double> xs(ns), es(ns);
    for (int i = 0; i < ns; ++i) {
        xs[i] = lo + (hi - lo) * i / (ns - 1);
        es[i] = quad_max_err(R, sinc_step, exp(xs[i]), kernel, kappa, r);
        if (es[i] < best) { best = es[i]; bx = i; }
    }
    int bi = (int)bx;
    double a = xs[std::max(bi - 1, 0)], b = xs[std::min(bi + 1, ns - 1)];
    const double gr = (sqrt(5.0) - 1.0) / 2.0;
    double c = b - gr * (b - a), d = a + gr * (b - a);
    double fc = quad_max_err(R, sinc_step, exp(c), kernel, kappa, r), fd = quad_max_err(R, sinc_step, exp(d), kernel, kappa, r);
    for (int it = 0; it < 60; ++it) {
        if (fc < fd) { b = d; d = c; fd = fc; c = b - gr * (b - a); fc = quad_max_err(R, sinc_step, exp(c), kernel, kappa, r); }
        else { a = c; c = d; fc = fd; d = a + gr * (b - a); fd = quad_max_err(R, sinc_step, exp(d), kernel, kappa, r); }
    }
    const double x = 0.5 * (a + b);
    *t_scale_out = exp(x);
    if (max_rel_err_out) *max_rel_err_out = quad_max_err(R, sinc_step, exp(x), kernel, kappa, r);
    return LS_OK;
}

int lattice_sum_create(ls_ctx** out, const ls_params* params, const ls_block* blocks, int32_t nblocks,
                       void* stream) {
    ls::NvtxRange nvtx_("lattice_sum_create");
    ls_ctx* ctx = nullptr;
    if (!out || !params || !blocks || nblocks < 1) return fail(ctx, LS_ERR_ARG, "create: NULL argument or no block");
    *out = nullptr;
    const ls_params& p = *params;
    if (p.N < 2 || p.N > (1 << 20)) return fail(ctx, LS_ERR_ARG, "create: N=%lld out of range", (long long)p.N);
    if (!(p.box_hi > p.box_lo)) return fail(ctx, LS_ERR_ARG, "create: empty box");
    if (p.R < 1 || p.R > 64) return fail(ctx, LS_ERR_ARG, "create: R=%d out of range [1,64]", p.R);
    if (!(p.sinc_step > 0) || !(p.t_scale > 0)) return fail(ctx, LS_ERR_ARG, "create: sinc_step and t_scale must be > 0");
    if (p.precision != LS_FP64 && p.precision != LS_MIXED) return fail(ctx, LS_ERR_ARG, "create: unknown precision %d", p.precision);
    if ((p.flags & ~(LS_FLAG_GALERKIN | LS_FLAG_SVD_GRAM | LS_FLAG_SVD_ONESIDED | LS_FLAG_TUCKER_REF |
                     LS_FLAG_CACHE_GENVEC)) != 0)
        return fail(ctx, LS_ERR_ARG, "create: unknown flags 0x%x", p.flags);
    if ((p.flags & LS_FLAG_TUCKER_REF) && !(p.ref_eps > 0.0 && p.ref_eps < 1.0))
        return fail(ctx, LS_ERR_ARG, "create: LS_FLAG_TUCKER_REF needs 0 < ref_eps < 1");
    if ((p.flags & LS_FLAG_TUCKER_REF) && (p.flags & LS_FLAG_SVD_GRAM))
        return fail(ctx, LS_ERR_ARG, "create: the Tucker-reference variant takes the non-squaring route");
    if ((p.flags & LS_FLAG_SVD_GRAM) && (p.flags & LS_FLAG_SVD_ONESIDED))
        return fail(ctx, LS_ERR_ARG, "create: LS_FLAG_SVD_GRAM and LS_FLAG_SVD_ONESIDED exclude each other");
    if (const char* why = kernel_args_bad(p.kernel, p.kappa)) return fail(ctx, LS_ERR_ARG, "create: %s", why);
    if (p.kappa > 0.0) {
        // the smallest node's screening factor exp(-kappa^2/(4 t_1^2)) must not underflow
        const double t1 = sinh(p.sinc_step) / p.t_scale;
        if (p.kappa * p.kappa / (4.0 * t1 * t1) > 600.0)
            return fail(ctx, LS_ERR_ARG, "create: kappa=%g too large for the sinc rule (t_1 = %g): its weight underflows",
                        p.kappa, t1);
    }
    ctx = new ls_ctx();
    ctx->p = p;
    ctx->st = static_cast<cudaStream_t>(stream);
    ctx->h = (p.box_hi - p.box_lo) / (double)p.N;
    for (int b = 0; b < nblocks; ++b) {
        HostBlock hb;
        hb.b = blocks[b];
        for (int a = 0; a < 3; ++a) {
            if (hb.b.L[a] < 1 || hb.b.L[a] > (1 << 20)) {
                delete ctx;
                return fail(nullptr, LS_ERR_ARG, "create: block %d has L[%d]=%lld", b, a, (long long)hb.b.L[a]);
            }
            for (int64_t k = 0; k < hb.b.L[a]; ++k) {
                int32_t m;
                if (!snap_vertex(ctx, hb.b.origin[a] + (double)k * hb.b.spacing[a], &m)) {
                    delete ctx;
                    return fail(nullptr, LS_ERR_ARG, "create: site %lld of block %d (axis %d) outside the box",
                                (long long)k, b, a);
                }
                hb.m[a].push_back(m);
            }
        }
        ctx->blocks.push_back(std::move(hb));
    }
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&ctx->num_sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) {
        delete ctx;
        return fail(nullptr, LS_ERR_CUDA, "create: no usable CUDA device (%s)", cudaGetErrorString(e));
    }
    keep_pool(dev);
    const int64_t N = p.N;
    const int R = p.R;
    int rc = LS_OK;
    {
        cudaError_t e2 = dalloc(ctx, &ctx->d_g, (int64_t)R * 2 * N);
        Scope sc_gen("genvec", ctx->st);
        const size_t gbytes = sizeof(double) * (size_t)R * 2 * N;
        const GenvecKey key{dev, N, ctx->h, R, p.sinc_step, p.t_scale, p.kernel, p.kappa,
                            (p.flags & LS_FLAG_GALERKIN) ? 1 : 0};
        bool hit = false;
        if (e2 == cudaSuccess && (p.flags & LS_FLAG_CACHE_GENVEC)) {
            std::lock_guard<std::mutex> g(g_genvec_mu);
            for (const GenvecEntry& c : genvec_cache())
                if (c.key == key) {
                    e2 = cudaMemcpyAsync(ctx->d_g, c.d, gbytes, cudaMemcpyDeviceToDevice, ctx->st);
                    hit = true;
                    break;
                }
        }
        if (e2 == cudaSuccess && !hit) {
            e2 = launch_genvec(ctx->d_g, R, N, ctx->h, p.sinc_step, p.t_scale, p.kernel, p.kappa,
                               (p.flags & LS_FLAG_GALERKIN) != 0, ctx->st);
            if (e2 == cudaSuccess && (p.flags & LS_FLAG_CACHE_GENVEC)) {
                // a new entry (the oldest goes once the cache is full); cudaFree of the evicted
                // buffer waits for the device, so no copy from it is still pending
                std::lock_guard<std::mutex> g(g_genvec_mu);
                std::deque<GenvecEntry>& cache = genvec_cache();
                if (cache.size() >= kGenvecCacheMax) {
                    cudaFree(cache.front().d);
                    cache.pop_front();
                }
                double* d = nullptr;
                e2 = cudaMalloc(&d, gbytes);
                if (e2 == cudaSuccess) e2 = cudaMemcpyAsync(d, ctx->d_g, gbytes, cudaMemcpyDeviceToDevice, ctx->st);
                if (e2 == cudaSuccess) e2 = cudaStreamSynchronize(ctx->st);   // the entry is complete before others read it
                if (e2 == cudaSuccess) cache.push_back(GenvecEntry{key, d});
                else if (d) cudaFree(d);
            }
        }
        if (e2 != cudaSuccess)
            rc = fail(ctx, e2 == cudaErrorMemoryAllocation ? LS_ERR_OOM : LS_ERR_CUDA, "create: %s", cudaGetErrorString(e2));
    }
    ctx->tucker = (p.flags & LS_FLAG_TUCKER_REF) != 0;
    if (rc == LS_OK && ctx->tucker) rc = make_reference_tucker(ctx);
    for (int l = 0; l < 3 && rc == LS_OK; ++l) {
        std::vector<int32_t> q;
        std::vector<std::vector<int32_t>> wins, keys;
        for (size_t b = 0; b < ctx->blocks.size(); ++b) {
            for (int qq = 0; qq < R; ++qq) {
                q.push_back(qq);
                wins.push_back(ctx->blocks[b].m[l]);
            }
            keys.push_back(ctx->blocks[b].m[l]);
        }
        rc = append_columns(ctx, l, q, wins);
        if (rc == LS_OK && ctx->tucker) rc = append_side(ctx, l, keys);
    }
    if (rc != LS_OK) {
        g_create_error = ctx->err;
        lattice_sum_destroy(ctx);
        return rc;
    }
    for (size_t b = 0; b < ctx->blocks.size(); ++b) {
        for (int qq = 0; qq < R; ++qq) {
            const int32_t c = (int32_t)(b * R + qq);
            for (int l = 0; l < 3; ++l) {
                ctx->tcol.push_back(c);
                ctx->mode[l].count[c] += 1;
            }
            ctx->xi.push_back(ctx->blocks[b].b.charge);
        }
        if (ctx->tucker) {
            // one Tucker term per block: its assembled side matrix is key b in every mode
            for (int l = 0; l < 3; ++l) {
                ctx->tkey.push_back((int32_t)b);
                for (int k = 0; k < ctx->r_ref; ++k) ctx->tmode[l].count[b * ctx->r_ref + k] += 1;
            }
            ctx->txi.push_back(ctx->blocks[b].b.charge);
        }
    }
    *out = ctx;
    return LS_OK;
}

int lattice_sum_add_defects(ls_ctx* ctx, const ls_defect* defects, int64_t n) {
    ls::NvtxRange nvtx_("lattice_sum_add_defects");
    if (!ctx) return fail(nullptr, LS_ERR_ARG, "add_defects: NULL context");
    if (ctx->reduced) return fail(ctx, LS_ERR_STATE, "add_defects: context already reduced");
    if (n < 0 || (n > 0 && !defects)) return fail(ctx, LS_ERR_ARG, "add_defects: bad defect array");
    const int R = ctx->p.R;
    const int nb = (int)ctx->blocks.size();
    // validate everything first so that a bad entry changes nothing; the window list of
    // defect i on axis a is kflat[koff[3 i + a] .. koff[3 i + a + 1])
    std::vector<int32_t> kflat;
    std::vector<int64_t> koff(3 * (size_t)n + 1, 0);
    kflat.reserve(3 * (size_t)n);
    std::vector<double> dxi(n);
    for (int64_t i = 0; i < n; ++i) {
        const ls_defect& d = defects[i];
        if (d.kind == LS_DEFECT_SITES) {
            if (d.block < 0 || d.block >= nb) return fail(ctx, LS_ERR_ARG, "defect %lld: block %d", (long long)i, d.block);
            const HostBlock& hb = ctx->blocks[d.block];
            for (int a = 0; a < 3; ++a) {
                if (d.extent[a] < 1 || d.site[a] < 0 || d.site[a] + d.extent[a] > hb.b.L[a])
                    return fail(ctx, LS_ERR_ARG, "defect %lld: sites out of block range on axis %d", (long long)i, a);
                for (int64_t e = 0; e < d.extent[a]; ++e) kflat.push_back(hb.m[a][d.site[a] + e]);
                koff[3 * i + a + 1] = (int64_t)kflat.size();
            }
            dxi[i] = d.charge - hb.b.charge;
        } else if (d.kind == LS_DEFECT_POINT) {
            for (int a = 0; a < 3; ++a) {
                int32_t m;
                if (!snap_vertex(ctx, d.pos[a], &m))
                    return fail(ctx, LS_ERR_ARG, "defect %lld: position outside the box", (long long)i);
                kflat.push_back(m);
                koff[3 * i + a + 1] = (int64_t)kflat.size();
            }
            dxi[i] = d.charge;
        } else {
            return fail(ctx, LS_ERR_ARG, "defect %lld: unknown kind %d", (long long)i, d.kind);
        }
    }
    std::vector<int32_t> base(3 * (size_t)n);
    for (int l = 0; l < 3; ++l) {
        ModeCols& mc = ctx->mode[l];
        std::vector<int32_t> q;
        std::vector<std::vector<int32_t>> wins, new_keys;
        for (int64_t i = 0; i < n; ++i) {
            const int32_t* w = kflat.data() + koff[3 * i + l];
            const int nw = (int)(koff[3 * i + l + 1] - koff[3 * i + l]);
            const uint64_t hk = KeyIndex::hash(w, nw);
            int32_t kidx = mc.keys.find(w, nw, hk);
            if (kidx < 0) {
                kidx = mc.keys.add(w, nw, hk);
                const std::vector<int32_t> kv(w, w + nw);
                for (int qq = 0; qq < R; ++qq) {
                    q.push_back(qq);
                    wins.push_back(kv);
                }
                new_keys.push_back(kv);
            }
            base[3 * i + l] = (int32_t)(nb * R) + kidx * R;
        }
        int rc = append_columns(ctx, l, q, wins);
        if (rc == LS_OK && ctx->tucker) rc = append_side(ctx, l, new_keys);
        if (rc != LS_OK) return rc;
    }
    // R terms a defect, one per quadrature node: term t's columns tcol[3 t + l], weight xi[t]
    const size_t t0 = ctx->xi.size();
    reserve_more(ctx->tcol, 3 * (size_t)n * R);
    reserve_more(ctx->xi, (size_t)n * R);
    ctx->tcol.resize(3 * (t0 + (size_t)n * R));
    ctx->xi.resize(t0 + (size_t)n * R);
    int32_t* tc = ctx->tcol.data() + 3 * t0;
    double* xv = ctx->xi.data() + t0;
    int32_t* cnt[3] = {ctx->mode[0].count.data(), ctx->mode[1].count.data(), ctx->mode[2].count.data()};
    for (int64_t i = 0; i < n; ++i) {
        for (int qq = 0; qq < R; ++qq) {
            for (int l = 0; l < 3; ++l) {
                const int32_t c = base[3 * i + l] + qq;
                *tc++ = c;
                cnt[l][c] += 1;
            }
            *xv++ = dxi[i];
        }
        if (ctx->tucker) {
            // one Tucker term per defect; key index = column base / R (blocks first)
            for (int l = 0; l < 3; ++l) {
                const int32_t kk = base[3 * i + l] / R;
                ctx->tkey.push_back(kk);
                for (int k = 0; k < ctx->r_ref; ++k) ctx->tmode[l].count[(int64_t)kk * ctx->r_ref + k] += 1;
            }
            ctx->txi.push_back(dxi[i]);
        }
    }
    return LS_OK;
}

}  // extern "C"

namespace {

// Scratch of one mode of one context during the reduction.
struct RedMode {
    double *G = nullptr, *L = nullptr, *pd = nullptr, *cand = nullptr, *H = nullptr, *V = nullptr, *snap = nullptr,
           *isl = nullptr, *w = nullptr, *vg = nullptr, *ytmp = nullptr, *Gz = nullptr, *Li = nullptr, *D2 = nullptr,
           *gate = nullptr;   // ||Y Y^T - I||_F before CholeskyQR (picks its first pass)
    // eigen-solver: U0 = I + F1 (first Jacobi run), S = U0^T U0, SLi, Uo, T1 = H Uo, Hp = Uo^T T1 (the
    // FP64-grade re-projection), F2 (the second run, where one is taken)
    double *U0 = nullptr, *S = nullptr, *SLi = nullptr, *Uo = nullptr, *T1 = nullptr, *Hp = nullptr, *F2 = nullptr;
    int32_t *piv = nullptr, *perm = nullptr;
    int k = 0;
    bool df = false;
};

// One context inside a (possibly batched) reduction.
struct RedState {
    ls_ctx* ctx = nullptr;
    double eps = 0.0;
    const int32_t* forced = nullptr;
    // [0, 3): pivoted Cholesky, then the eigen-solver, per mode; [3, 6): CholeskyQR per mode;
    // [6, 9): spare per-mode statuses; [9]: the exact-slice tensor-core products (never reset)
    DevStatus* d_st = nullptr;
    double* d_sel = nullptr;
    RedMode m[3];
    int sweeps[3] = {0, 0, 0};
    int64_t rotations[3] = {0, 0, 0};
    double sel[3][3] = {};
    DevStatus hs[10] = {};
    double floor_noise = 0.0;
    int64_t T = 0;
    // the non-squaring route of the FP64 path runs the Gram-route phases twice with these set:
    // kind 1 = candidate basis of the side matrix (all eigen-directions above cand_res, no
    // projection or core), kind 2 = the same for the residual rows E of the side matrix
    // (weights = the rows' norms, floor_noise given, the basis made orthogonal to reorth)
    int kind = 0;
    double cand_res[3] = {0.0, 0.0, 0.0};
    const double* reorth[3] = {nullptr, nullptr, nullptr};
    int reorth_m[3] = {0, 0, 0};
    bool drop[3] = {false, false, false};   // kind 2: no residual direction above cand_res in this mode
    // the eigen-solver's second Jacobi run is skipped: the eigenvalues are the Rayleigh quotients
    // of the FP64 re-projection H' = Uo^T H Uo and the eigenvectors Uo (the mixed path, whose
    // truncation sits far above the first run's accuracy, and the candidate bases of the
    // non-squaring route, whose accuracy the one-sided Jacobi restores)
    bool fast_eig = false;
    // the batch: red_core leaves the release (which synchronises the stream) to the caller, so that
    // the projections and cores of all contexts are queued before the first wait
    bool defer_release = false;
};

#define CUS(call)                                                                                     \
    do {                                                                                              \
        cudaError_t e_ = (call);                                                                      \
        if (e_ != cudaSuccess)                                                                        \
            return fail(R.ctx, e_ == cudaErrorMemoryAllocation ? LS_ERR_OOM : LS_ERR_CUDA, "%s: %s (%s:%d)", #call, \
                        cudaGetErrorString(e_), __FILE__, __LINE__);                                  \
    } while (0)

// terms to the device, unit vectors, weighted Gram matrices, pivoted-Cholesky jobs
int red_prepare(RedState& R, PcholJob* pj) {
    ls_ctx* ctx = R.ctx;
    cudaStream_t st = ctx->st;
    const int64_t N = ctx->p.N;
    const int64_t T = R.T = (int64_t)ctx->xi.size();
    if (R.kind != 2) {
        R.floor_noise = 8.0 * 1.1102230246251565e-16 * (double)T;   // rounding noise of the Gram matrix (trace T)
        CUS(dalloc(ctx, &ctx->d_tcol, 3 * T));
        CUS(dalloc(ctx, &ctx->d_xi, T));
        CUS(dalloc(ctx, &ctx->d_xin, T));
        CUS(upload_h2d(ctx->d_tcol, ctx->tcol.data(), 3 * T * sizeof(int32_t), st));
        count_h2d(3 * T * sizeof(int32_t));
        CUS(upload_h2d(ctx->d_xi, ctx->xi.data(), T * sizeof(double), st));
        count_h2d(T * sizeof(double));
    }
    CUS(dalloc(ctx, &R.d_st, 10));
    CUS(cudaMemsetAsync(R.d_st, 0, 10 * sizeof(DevStatus), st));
    CUS(dalloc(ctx, &R.d_sel, 9));
    const double* a[3];
    const double* w[3];
    double* G[3];
    int64_t Cs[3];
    for (int l = 0; l < 3; ++l) {
        ModeCols& mc = ctx->mode[l];
        RedMode& M = R.m[l];
        const int64_t C = Cs[l] = mc.C;
        CUS(dalloc(ctx, &ctx->d_norms[l], C));
        CUS(dalloc(ctx, &ctx->d_sigma[l], C));
        CUS(dalloc(ctx, &M.G, C * C));
        CUS(dalloc(ctx, &M.L, C * C));
        // a residual that is all rounding stops the pivoted Cholesky before its first column:
        // L = 0 then gives H = 0 and the mode is dropped
        if (R.kind == 2) CUS(cudaMemsetAsync(M.L, 0, C * C * sizeof(double), st));
        CUS(dalloc(ctx, &M.pd, C));
        CUS(dalloc(ctx, &M.cand, kPcholCand));
        CUS(dalloc(ctx, &M.piv, C));
        CUS(dalloc(ctx, &M.w, C));
        CUS(cudaMemsetAsync(ctx->d_sigma[l], 0, C * sizeof(double), st));
        if (R.kind != 2) {
            std::vector<double> wh(C);
            for (int64_t c = 0; c < C; ++c) wh[c] = sqrt((double)mc.count[c]);
            CUS(upload_h2d(M.w, wh.data(), C * sizeof(double), st));
            count_h2d(C * sizeof(double));
        }
        { Scope sc("norms", st); CUS(launch_norm_columns(mc.d_cols, C, N, ctx->d_norms[l], st)); }
        // residual rows: unit rows weighted by their norms (G = E E^T)
        if (R.kind == 2) CUS(cudaMemcpyAsync(M.w, ctx->d_norms[l], C * sizeof(double), cudaMemcpyDeviceToDevice, st));
        a[l] = mc.d_cols;
        w[l] = M.w;
        G[l] = M.G;
        // pivoted Cholesky: the energy left outside the pivot columns (<= delta) is discarded with
        // the tail; with the eps rule delta = 1e-4 eps^2 T, with forced ranks and in the passes of
        // the non-squaring route the Gram noise
        const double delta =
            (R.forced || R.kind != 0) ? (double)C * R.floor_noise : 1e-4 * R.eps * R.eps * (double)T;
        pj[l] = PcholJob{M.G, M.L, M.pd, M.cand, M.piv, R.d_st + l, C, (int)C, delta};
    }
    {
        // FP64-grade weighted Gram matrices on the tensor cores
        Scope sc("gram", st);
        std::string err;
        // the panel forms of the pivoted Cholesky read G[min(i,j)][max(i,j)] only: their Gram
        // matrices skip the tiles below the diagonal (the whole-matrix cluster form reads all)
        int upper[3];
        for (int l = 0; l < 3; ++l) upper[l] = pchol_cluster_size((int)Cs[l], (int)Cs[l]) > 0 ? 0 : 1;
        int rc = x64_gram(3, a, Cs, N, w, G, &R.d_st[9].flag, st, &err, upper);
        if (rc != LS_OK) return fail(ctx, rc, "rhosvd_reduce: Gram: %s", err.c_str());
    }
    return LS_OK;
}

// after the pivoted Cholesky (statuses in R.hs): H = L^T L and the Jacobi jobs
int red_after_pchol(RedState& R, JacobiJob* jj) {
    ls_ctx* ctx = R.ctx;
    cudaStream_t st = ctx->st;
    for (int l = 0; l < 3; ++l)
        if (R.hs[l].flag == FLAG_TIMEOUT)
            return fail(ctx, LS_ERR_TIMEOUT, "rhosvd_reduce: pivoted Cholesky barrier timed out (mode %d)", l);
    CUS(cudaMemsetAsync(R.d_st, 0, 9 * sizeof(DevStatus), st));
    // the FP32 block Jacobi and its FP64-grade re-projection for every k up to this (the block
    // form in shared memory or in one cooperative grid); beyond it the FP64 grid Jacobi
    const int kdf = 8192;
    const double* L[3];
    double* H[3];
    int64_t Cs[3];
    int ks[3];
    for (int l = 0; l < 3; ++l) {
        RedMode& M = R.m[l];
        const int k = ks[l] = M.k = std::max(1, R.hs[l].sweeps);
        CUS(dalloc(ctx, &M.H, (int64_t)k * k));
        CUS(dalloc(ctx, &M.V, (int64_t)k * k));
        CUS(dalloc(ctx, &M.snap, 6 * (k / 2 + 1)));
        CUS(dalloc(ctx, &M.perm, k));
        CUS(dalloc(ctx, &M.isl, k));
        CUS(launch_identity(M.V, k, st));
        M.df = k <= kdf;
        if (M.df)
            for (double** q : {&M.U0, &M.S, &M.SLi, &M.Uo, &M.T1, &M.Hp, &M.F2}) CUS(dalloc(ctx, q, (int64_t)k * k));
        L[l] = M.L;
        H[l] = M.H;
        Cs[l] = ctx->mode[l].C;
        // directions whose Rayleigh quotients both stay below tau = 1e-3 eps^2 T / k are discarded
        // together whatever their mixing; forced ranks resolve everything
        const double tau = (R.forced || R.kind != 0) ? 0.0 : 1e-3 * R.eps * R.eps * (double)R.T / (double)k;
        jj[l] = JacobiJob{M.H, M.V, M.snap, R.d_st + l, k, R.floor_noise, tau};
    }
    {
        // H = L^T L: FP64-grade products on the tensor cores (exact slices)
        Scope sc("pchol", st);
        std::string err;
        int rc = x64_pchol_gram(3, L, Cs, ks, Cs, H, &R.d_st[9].flag, st, &err);
        if (rc != LS_OK) return fail(ctx, rc, "rhosvd_reduce: L^T L: %s", err.c_str());
    }
    return LS_OK;
}

// eps-rank selection on the eigenvalues of H (the pivoted-Cholesky residual joins the tail)
int red_select(RedState& R) {
    ls_ctx* ctx = R.ctx;
    cudaStream_t st = ctx->st;
    {
        SortSelectJob jobs[3];
        for (int l = 0; l < 3; ++l) {
            RedMode& M = R.m[l];
            // candidate bases: every eigen-direction above cand_res (a forced rank of k, clipped)
            const int forced = R.kind != 0 ? M.k : (R.forced ? std::max(1, R.forced[l]) : 0);
            jobs[l] = SortSelectJob{M.H, M.k, forced, M.cand + kPcholCand - 1, M.perm, ctx->d_sigma[l], M.isl,
                                    R.d_sel + 3 * l};
            if (R.kind != 0) jobs[l].resolution = R.cand_res[l];
        }
        Scope sc("select", st);
        CUS(launch_sort_select(3, jobs, R.eps, R.floor_noise, st));
    }
    CUS(cudaMemcpyAsync(R.hs, R.d_st, 3 * sizeof(DevStatus), cudaMemcpyDeviceToHost, st));
    CUS(cudaMemcpyAsync(R.hs + 6, R.d_st + 6, 3 * sizeof(DevStatus), cudaMemcpyDeviceToHost, st));
    count_d2h(6 * sizeof(DevStatus));
    CUS(cudaMemcpyAsync(R.sel, R.d_sel, sizeof R.sel, cudaMemcpyDeviceToHost, st));
    count_d2h(sizeof R.sel);
    return LS_OK;
}

// after the selection (host copies ready): eigenvectors of the Gram matrices,
// the bases Y = A_w Vg Lambda^{-1/2}, and the first Gram matrix of CholeskyQR2
int red_basis(RedState& R, CholJob* cj) {
    ls_ctx* ctx = R.ctx;
    cudaStream_t st = ctx->st;
    const int64_t N = ctx->p.N;
    for (int l = 0; l < 3; ++l) {
        if (R.hs[l].flag == FLAG_TIMEOUT)
            return fail(ctx, LS_ERR_TIMEOUT, "rhosvd_reduce: Jacobi grid barrier timed out (mode %d)", l);
        if (R.hs[l].flag == FLAG_NOCONVERGE || R.hs[l].sweeps < 0)
            return fail(ctx, LS_ERR_NOCONVERGE, "rhosvd_reduce: Jacobi did not converge (mode %d)", l);
        if (R.hs[6 + l].flag == FLAG_TIMEOUT)
            return fail(ctx, LS_ERR_TIMEOUT, "rhosvd_reduce: eigen-solver Cholesky barrier timed out (mode %d)", l);
        if (R.hs[6 + l].flag == FLAG_NOT_SPD)
            return fail(ctx, LS_ERR_NOCONVERGE, "rhosvd_reduce: eigenvector orthonormalisation failed (mode %d)", l);
        R.sweeps[l] = R.hs[l].sweeps;
        ctx->r[l] = (int32_t)R.sel[l][0];
        int64_t rot = 0;
        for (int k = 0; k < R.sweeps[l] && k < 64; ++k) rot += R.hs[l].sweep_active[k];
        R.rotations[l] = rot;
    }
    const double *L[3], *U[3], *Hc[3], *vgc[3], *isl[3], *w[3], *a[3], *Yc[3];
    const int32_t* perm[3];
    double *vg[3], *Y[3], *Gz[3];
    int64_t Cs[3], kl[3];
    int ks[3], rs[3];
    for (int l = 0; l < 3; ++l) {
        ModeCols& mc = ctx->mode[l];
        RedMode& M = R.m[l];
        const int64_t C = mc.C;
        const int r = ctx->r[l];
        CUS(dalloc(ctx, &ctx->d_Z[l], (int64_t)r * N));
        CUS(dalloc(ctx, &ctx->d_P[l], (int64_t)r * C));
        CUS(dalloc(ctx, &M.Gz, (int64_t)r * r));
        CUS(dalloc(ctx, &M.Li, (int64_t)r * r));
        CUS(dalloc(ctx, &M.D2, (int64_t)r * r));
        CUS(dalloc(ctx, &M.ytmp, (int64_t)r * N));
        CUS(dalloc(ctx, &M.vg, C * M.k));
        CUS(dalloc(ctx, &M.gate, 1));
        L[l] = M.L;
        U[l] = M.V;
        Hc[l] = M.H;
        vg[l] = M.vg;
        vgc[l] = M.vg;
        isl[l] = M.isl;
        w[l] = M.w;
        a[l] = mc.d_cols;
        perm[l] = M.perm;
        Y[l] = ctx->d_Z[l];
        Yc[l] = ctx->d_Z[l];
        Gz[l] = M.Gz;
        Cs[l] = C;
        kl[l] = M.k;
        ks[l] = M.k;
        rs[l] = r;
        cj[l] = CholJob{M.Gz, M.Li, R.d_st + 3 + l, r, M.gate};
    }
    {
        // FP64-grade products on the tensor cores (exact slices)
        Scope sc("basis", st);
        std::string err;
        int rc = x64_pchol_vectors(3, L, Cs, ks, Cs, U, Hc, vg, &R.d_st[9].flag, st, &err);
        if (rc == LS_OK) rc = x64_basis(3, vgc, kl, perm, w, isl, a, Cs, N, rs, Y, &R.d_st[9].flag, st, &err);
        if (rc != LS_OK) return fail(ctx, rc, "rhosvd_reduce: basis: %s", err.c_str());
    }
    if (R.kind == 2 && R.reorth[0]) {
        // the residual's basis, made orthogonal to the first pass's: Y -= (Y Q1^T) Q1
        Scope sc("basis", st);
        double *S[3], *D[3];
        X64Mat xs[3], ys[3];
        int64_t ld[3];
        for (int l = 0; l < 3; ++l) {
            const int64_t m1 = R.reorth_m[l];
            CUS(dalloc(ctx, &S[l], (int64_t)rs[l] * m1));
            CUS(dalloc(ctx, &D[l], (int64_t)rs[l] * N));
        }
        std::string err;
        const int m1i[3] = {R.reorth_m[0], R.reorth_m[1], R.reorth_m[2]};
        const int64_t m1l[3] = {R.reorth_m[0], R.reorth_m[1], R.reorth_m[2]};
        int rc = x64_project(3, Yc, rs, R.reorth, m1l, N, S, &R.d_st[9].flag, st, &err);   // S = Y Q1^T
        for (int l = 0; l < 3; ++l) {
            xs[l] = X64Mat{S[l], rs[l], m1i[l], m1i[l], 1, nullptr};          // S: r x m1
            ys[l] = X64Mat{R.reorth[l], N, m1i[l], 1, N, nullptr};           // Q1^T: N x m1
            ld[l] = N;
        }
        if (rc == LS_OK) rc = x64_nt(3, xs, ys, D, ld, &R.d_st[9].flag, st, &err);      // D = S Q1
        if (rc != LS_OK) return fail(ctx, rc, "rhosvd_reduce: residual basis: %s", err.c_str());
        for (int l = 0; l < 3; ++l) {
            CUS(launch_sub(Y[l], D[l], (int64_t)rs[l] * N, st));
            dfree(ctx, S[l]);
            dfree(ctx, D[l]);
        }
    }
    {
        // CholeskyQR2's first pass: where Y Y^T is within kSeriesGate of I (Frobenius), the
        // series for (Y Y^T)^{-1/2} writes the transform; elsewhere the Cholesky factorisation
        // launched next does (both read the same device-side distance, so no host decision)
        Scope sc("cholqr2", st);
        const int64_t r64[3] = {rs[0], rs[1], rs[2]};
        const double* gc[3] = {Gz[0], Gz[1], Gz[2]};
        double *Li[3], *D2[3], *gate[3];
        for (int l = 0; l < 3; ++l) {
            Li[l] = R.m[l].Li;
            D2[l] = R.m[l].D2;
            gate[l] = R.m[l].gate;
        }
        std::string err;
        int rc;
        {
            Scope sg("cholqr2.gram", st);
            rc = x64_gram(3, Yc, r64, N, nullptr, Gz, &R.d_st[9].flag, st, &err);
        }
        if (rc == LS_OK) {
            Scope ss("cholqr2.series", st);
            rc = x64_lowdin(3, gc, rs, D2, Li, &R.d_st[9].flag, st, &err, gate);
        }
        if (rc != LS_OK) return fail(ctx, rc, "rhosvd_reduce: CholeskyQR: %s", err.c_str());
    }
    return LS_OK;
}

// CholeskyQR2 after the first factorisation: Y' = L^{-1} Y, G' = Y' Y'^T, and
// the second pass T = G'^{-1/2} by its series (G' = I + O(u32 cond(Y)^2))
int red_cholqr_mid(RedState& R) {
    ls_ctx* ctx = R.ctx;
    cudaStream_t st = ctx->st;
    const int64_t N = ctx->p.N;
    const double *Li[3], *src[3], *yc[3], *gc[3];
    double *dst[3], *Gz[3], *D2[3], *T[3];
    int rs[3];
    for (int l = 0; l < 3; ++l) {
        Li[l] = R.m[l].Li;
        src[l] = ctx->d_Z[l];
        dst[l] = R.m[l].ytmp;
        yc[l] = R.m[l].ytmp;
        Gz[l] = R.m[l].Gz;
        gc[l] = R.m[l].Gz;
        D2[l] = R.m[l].D2;
        T[l] = R.m[l].Li;
        rs[l] = ctx->r[l];
    }
    Scope sc("cholqr2", st);
    {
        const int64_t r64[3] = {rs[0], rs[1], rs[2]};
        std::string err;
        int rc;
        {
            Scope sa("cholqr2.apply", st);
            rc = x64_apply(3, Li, rs, src, N, dst, &R.d_st[9].flag, st, &err);
        }
        if (rc == LS_OK) {
            Scope sg("cholqr2.gram", st);
            rc = x64_gram(3, yc, r64, N, nullptr, Gz, &R.d_st[9].flag, st, &err);
        }
        if (rc != LS_OK) return fail(ctx, rc, "rhosvd_reduce: CholeskyQR: %s", err.c_str());
    }
    {
        Scope ss("cholqr2.series", st);
        std::string err;
        int rc = x64_lowdin(3, gc, rs, D2, T, &R.d_st[9].flag, st, &err);
        if (rc != LS_OK) return fail(ctx, rc, "rhosvd_reduce: CholeskyQR series: %s", err.c_str());
    }
    return LS_OK;
}

int red_project_core(RedState& R, ls_tucker_info* info);
int red_release(RedState& R, ls_tucker_info* info);

// after the second factorisation: Z = L^{-1} Y', projections, core, info
int red_finish(RedState& R, ls_tucker_info* info) {
    ls_ctx* ctx = R.ctx;
    cudaStream_t st = ctx->st;
    const int64_t N = ctx->p.N;
    {
        const double *Li[3], *src[3];
        double* dst[3];
        int rs[3];
        for (int l = 0; l < 3; ++l) {
            Li[l] = R.m[l].Li;
            src[l] = R.m[l].ytmp;
            dst[l] = ctx->d_Z[l];
            rs[l] = ctx->r[l];
        }
        Scope sc("cholqr2", st);
        Scope sa("cholqr2.apply", st);
        std::string err;
        int rc = x64_apply(3, Li, rs, src, N, dst, &R.d_st[9].flag, st, &err);
        if (rc != LS_OK) return fail(ctx, rc, "rhosvd_reduce: CholeskyQR: %s", err.c_str());
    }
    if (R.kind != 0) return red_release(R, nullptr);
    return red_project_core(R, info);
}

// (c2) projection, (c3) core, release of the scratch, status and info (Z in ctx->d_Z)
int red_core(RedState& R, ls_tucker_info* info);
int red_project_core_noproj(RedState& R, ls_tucker_info* info) { return red_core(R, info); }

int red_project_core(RedState& R, ls_tucker_info* info) {
    ls_ctx* ctx = R.ctx;
    cudaStream_t st = ctx->st;
    const int64_t N = ctx->p.N;
    {
        // (c2) projection P_l = Z_l^T A_l, both paths: FP64-grade exact-slice products on the
        // tensor cores (the dense FP64 contraction the truncation rests on)
        const double *Z[3], *a[3];
        double* P[3];
        int rs[3];
        int64_t Cs[3];
        for (int l = 0; l < 3; ++l) {
            Z[l] = ctx->d_Z[l];
            a[l] = ctx->mode[l].d_cols;
            P[l] = ctx->d_P[l];
            rs[l] = ctx->r[l];
            Cs[l] = ctx->mode[l].C;
        }
        Scope sc("project", st);
        std::string err;
        int rc = x64_project(3, Z, rs, a, Cs, N, P, &R.d_st[9].flag, st, &err);
        if (rc != LS_OK) return fail(ctx, rc, "rhosvd_reduce: projection: %s", err.c_str());
    }
    return red_core(R, info);
}

// (c3) the core from the projections in ctx->d_P, then release, statuses and info
int red_core(RedState& R, ls_tucker_info* info) {
    ls_ctx* ctx = R.ctx;
    cudaStream_t st = ctx->st;
    const int64_t T = R.T;
    { Scope sc("fold", st); CUS(launch_fold_norms(ctx->d_xi, ctx->d_tcol, T, ctx->d_norms[0], ctx->d_norms[1], ctx->d_norms[2], ctx->d_xin, st)); }
    // (c3) core: terms grouped by their mode-0 vector (counting sort on the host)
    int32_t Cs[3] = {(int32_t)ctx->mode[0].C, (int32_t)ctx->mode[1].C, (int32_t)ctx->mode[2].C};
    std::vector<int32_t> off(Cs[0] + 1, 0), perm(T);
    for (int64_t t = 0; t < T; ++t) off[ctx->tcol[3 * t] + 1] += 1;
    for (int c = 0; c < Cs[0]; ++c) off[c + 1] += off[c];
    {
        std::vector<int32_t> pos(off.begin(), off.end() - 1);
        for (int64_t t = 0; t < T; ++t) perm[pos[ctx->tcol[3 * t]]++] = (int32_t)t;
    }
    int32_t *d_perm_t = nullptr, *d_off = nullptr;
    const int64_t core_n = (int64_t)ctx->r[0] * ctx->r[1] * ctx->r[2];
    CUS(dalloc(ctx, &ctx->d_B, core_n));
    {
        Scope sc_core("core", st);
        const int64_t nn = (int64_t)ctx->r[1] * ctx->r[2];
        const int64_t w_cols = std::max<int64_t>(1, std::min<int64_t>(Cs[0], (int64_t)(32 << 20) / std::max<int64_t>(nn, 1)));
        if (ctx->p.precision == LS_MIXED) {
            // both steps on the tensor cores (two exact digits + two tails)
            std::string err;
            int rc = dt_core(ctx->d_P[0], ctx->d_P[1], ctx->d_P[2], Cs, ctx->r, ctx->d_tcol, ctx->d_xin, perm.data(),
                             off.data(), T, ctx->d_B, &R.d_st[9].flag, st, &err);
            if (rc != LS_OK) return fail(ctx, rc, "rhosvd_reduce: core: %s", err.c_str());
        } else {
            CUS(dalloc(ctx, &d_perm_t, T));
            CUS(dalloc(ctx, &d_off, Cs[0] + 1));
            CUS(upload_h2d(d_perm_t, perm.data(), T * sizeof(int32_t), st));
            count_h2d(T * sizeof(int32_t));
            CUS(upload_h2d(d_off, off.data(), (Cs[0] + 1) * sizeof(int32_t), st));
            count_h2d((Cs[0] + 1) * sizeof(int32_t));
            double *P1t = nullptr, *P2t = nullptr, *W = nullptr;
            CUS(dalloc(ctx, &P1t, (int64_t)Cs[1] * ctx->r[1]));
            CUS(dalloc(ctx, &P2t, (int64_t)Cs[2] * ctx->r[2]));
            CUS(dalloc(ctx, &W, w_cols * nn));
            CUS(launch_transpose(ctx->d_P[1], ctx->r[1], Cs[1], P1t, st));
            CUS(launch_transpose(ctx->d_P[2], ctx->r[2], Cs[2], P2t, st));
            CUS(launch_core_f64(ctx->d_P[0], P1t, P2t, Cs, ctx->r, ctx->d_tcol, ctx->d_xin, d_perm_t, d_off, W, w_cols,
                                ctx->d_B, st));
            dfree(ctx, P1t);
            dfree(ctx, P2t);
            dfree(ctx, W);
        }
    }
    dfree(ctx, d_perm_t);
    dfree(ctx, d_off);
    return R.defer_release ? LS_OK : red_release(R, info);
}

// frees the reduction scratch, reads the statuses back (synchronising the stream), checks
// them and, for a full reduction (kind 0), fills the info and marks the context reduced
int red_release(RedState& R, ls_tucker_info* info) {
    ls_ctx* ctx = R.ctx;
    cudaStream_t st = ctx->st;
    const int64_t T = R.T;
    int32_t Cs[3] = {(int32_t)ctx->mode[0].C, (int32_t)ctx->mode[1].C, (int32_t)ctx->mode[2].C};
    for (int l = 0; l < 3; ++l) {
        RedMode& M = R.m[l];
        for (void* q : {(void*)M.G, (void*)M.L, (void*)M.pd, (void*)M.cand, (void*)M.H, (void*)M.V, (void*)M.snap,
                        (void*)M.isl, (void*)M.w, (void*)M.piv, (void*)M.perm, (void*)M.vg, (void*)M.ytmp,
                        (void*)M.Gz, (void*)M.Li, (void*)M.D2, (void*)M.U0, (void*)M.S, (void*)M.SLi, (void*)M.Uo, (void*)M.T1,
                        (void*)M.Hp, (void*)M.F2, (void*)M.gate})
            dfree(ctx, q);
        const int k = M.k;
        M = RedMode{};
        M.k = k;
    }
    dfree(ctx, R.d_sel);
    R.d_sel = nullptr;
    CUS(cudaMemcpyAsync(&R.hs[3], R.d_st + 3, 3 * sizeof(DevStatus), cudaMemcpyDeviceToHost, st));
    CUS(cudaMemcpyAsync(&R.hs[9], R.d_st + 9, sizeof(DevStatus), cudaMemcpyDeviceToHost, st));
    count_d2h(4 * sizeof(DevStatus));
    double xin_norm2 = 0.0;
    if (info && R.kind == 0) {
        std::vector<double> xin(T);
        CUS(cudaMemcpyAsync(xin.data(), ctx->d_xin, T * sizeof(double), cudaMemcpyDeviceToHost, st));
        count_d2h(T * sizeof(double));
        CUS(cudaStreamSynchronize(st));
        for (double v : xin) xin_norm2 += v * v;
    } else {
        CUS(cudaStreamSynchronize(st));
    }
    dfree(ctx, R.d_st);
    R.d_st = nullptr;
    if (R.hs[9].flag == FLAG_TIMEOUT)
        return fail(ctx, LS_ERR_TIMEOUT, "rhosvd_reduce: a tensor-core product's bounded wait timed out");
    for (int l = 3; l < 6; ++l) {
        if (R.hs[l].flag == FLAG_TIMEOUT) return fail(ctx, LS_ERR_TIMEOUT, "rhosvd_reduce: Cholesky grid barrier timed out");
        if (R.hs[l].flag == FLAG_NOT_SPD && !R.drop[l - 3])
            return fail(ctx, LS_ERR_NOCONVERGE, "rhosvd_reduce: CholeskyQR2 met a non-positive pivot (mode %d)", l - 3);
    }
    if (R.kind != 0) return LS_OK;
    if (info) {
        memset(info, 0, sizeof *info);
        double ssum = 0.0;
        for (int l = 0; l < 3; ++l) {
            info->r[l] = ctx->r[l];
            info->C[l] = Cs[l];
            info->sigma_discarded[l] = sqrt(std::max(R.sel[l][1], 0.0));
            info->sigma_total[l] = sqrt(std::max(R.sel[l][2], 0.0));
            info->sweeps[l] = R.sweeps[l];
            info->rotations[l] = R.rotations[l];
            info->pivots[l] = R.m[l].k;
            // Thm A.1(d) with the resolution of the Gram route: after the eigen-solver every
            // off-diagonal entry is below the floor, so each eigenvalue is known to C * floor
            ssum += sqrt(std::max(R.sel[l][1], 0.0) + (double)Cs[l] * R.floor_noise);
        }
        info->T = T;
        info->xi_norm = sqrt(xin_norm2);
        info->bound_abs = info->xi_norm * ssum;
    }
    CUS(cudaGetLastError());
    ctx->reduced = true;
    return LS_OK;
}

// make `to` wait for the work enqueued so far on `from`
cudaError_t join(cudaStream_t to, cudaStream_t from) {
    if (to == from) return cudaSuccess;
    cudaEvent_t e;
    cudaError_t rc = cudaEventCreateWithFlags(&e, cudaEventDisableTiming);
    if (rc != cudaSuccess) return rc;
    rc = cudaEventRecord(e, from);
    if (rc == cudaSuccess) rc = cudaStreamWaitEvent(to, e, 0);
    cudaEventDestroy(e);
    return rc;
}

// Eigen-decomposition H = V diag(lambda) V^T of every mode of the batch, on s0.
// Where k fits the shared-memory solver: a first Jacobi run from H gives
// U0 = I + F1 (FP32 accuracy), U0 is orthonormalised in FP64 (Cholesky of
// U0^T U0), H' = Uo^T H Uo is formed in FP64, a second Jacobi run on the
// nearly diagonal H' gives its eigenvalues (written to the diagonal of H')
// and I + F2, and V = Uo + Uo F2; H' then takes the place of H. Both runs use
// the block Jacobi, in one cluster's shared memory where k fits and in one
// cooperative grid otherwise; beyond k = 8192 the FP64 grid Jacobi. The eps-rule tolerances: 1e-6 for the first run
// (FP32; 1e-4 where it is the mixed path's only run), 1e-10 for the second; forced ranks use the same.
int eigen_all(std::vector<RedState>& R, ls_ctx* const* ctxs, int n, const std::vector<JacobiJob>& jj, cudaStream_t s0) {
    ls_ctx* c0 = ctxs[0];
    std::vector<JacobiJob> grid;
    std::vector<DfJob> s1, s2;
    for (int i = 0; i < n; ++i)
        for (int l = 0; l < 3; ++l) {
            RedMode& M = R[i].m[l];
            const JacobiJob& J = jj[3 * i + l];
            if (!M.df) { grid.push_back(J); continue; }
            // the mixed path's single run stops at 1e-4: its Rayleigh quotients are then good to
            // about k 1e-8 relative, far inside the truncation's eps, and its basis error is second
            // order; the candidate passes keep 1e-6 (the one-sided Jacobi after them converges in
            // fewer sweeps on the more nearly orthogonal rows)
            s1.push_back(DfJob{M.H, M.k, M.T1, 1, M.U0, 1, R[i].d_st + l, J.abs_floor, J.tau,
                               (R[i].fast_eig && R[i].kind == 0) ? 1e-4 : 1e-6});
            if (!R[i].fast_eig)
                s2.push_back(DfJob{M.Hp, M.k, M.Hp, (int64_t)M.k + 1, M.F2, 0, R[i].d_st + l, J.abs_floor, J.tau, 1e-10});
        }
    auto err = [&](cudaError_t e, const char* what) {
        return fail(c0, e == cudaErrorMemoryAllocation ? LS_ERR_OOM : LS_ERR_CUDA, "rhosvd_reduce: %s: %s", what,
                    cudaGetErrorString(e));
    };
    // per context, the df modes in one grouped launch
    auto per_ctx = [&](auto&& fn) -> cudaError_t {
        for (int i = 0; i < n; ++i) {
            int nm = 0;
            RedMode* ms[3];
            for (int l = 0; l < 3; ++l)
                if (R[i].m[l].df) ms[nm++] = &R[i].m[l];
            if (nm == 0) continue;
            cudaError_t e = fn(R[i], ms, nm);
            if (e != cudaSuccess) return e;
        }
        return cudaSuccess;
    };
    cudaError_t e;
    if (!grid.empty()) {
        e = launch_jacobi_multi(grid.data(), (int)grid.size(), 60, 1e-14, c0->num_sms, s0);
        if (e != cudaSuccess) return err(e, "Jacobi launch");
    }
    if (s1.empty()) return LS_OK;
    // the block form: in one cluster's shared memory where k fits, else in one cooperative grid
    // with the matrices in global memory
    const int kblk = jacobi_blk_max_k();
    const int nsm = c0->num_sms;
    auto run_df = [kblk, nsm](const DfJob* jobs, int nj, int max_sweeps, cudaStream_t st) -> cudaError_t {
        std::vector<DfJob> small, large;
        for (int i = 0; i < nj; ++i) (jobs[i].k <= kblk ? small : large).push_back(jobs[i]);
        cudaError_t e = cudaSuccess;
        if (!small.empty()) e = launch_jacobi_blk(small.data(), (int)small.size(), max_sweeps, st);
        if (e == cudaSuccess && !large.empty())
            e = launch_jacobi_gblk(large.data(), (int)large.size(), max_sweeps, nsm, st);
        return e;
    };
    {
        Scope sc("jacobi.run1", s0);
        if ((e = run_df(s1.data(), (int)s1.size(), 60, s0)) != cudaSuccess) return err(e, "Jacobi (first run)");
    }
    {
        Scope sc_o("jacobi.ortho", s0);
        e = per_ctx([&](RedState& Rs, RedMode** ms, int nm) {
            const double *U0[3], *Sc[3], *H[3], *Tc[3], *Uc[3];
            double *S[3], *D2[3], *T[3], *Uo[3], *T1[3], *Hp[3];
            int ks[3];
            for (int j = 0; j < nm; ++j) {
                RedMode& M = *ms[j];
                U0[j] = M.U0; S[j] = M.S; Sc[j] = M.S; D2[j] = M.SLi; T[j] = M.T1; Tc[j] = M.T1;
                Uo[j] = M.Uo; Uc[j] = M.Uo; H[j] = M.H; T1[j] = M.T1; Hp[j] = M.Hp; ks[j] = M.k;
            }
            // FP64-grade products on the tensor cores (exact slices)
            int* fl = &Rs.d_st[9].flag;
            const int no[3] = {0, 0, 0}, yes[3] = {1, 1, 1};
            std::string err;
            int rc = x64_small(nm, U0, yes, U0, no, ks, S, nullptr, fl, s0, &err);            // S = U0^T U0
            if (rc == LS_OK) rc = x64_lowdin(nm, Sc, ks, D2, T, fl, s0, &err);               // T = S^{-1/2}
            if (rc == LS_OK) rc = x64_small(nm, U0, no, Tc, no, ks, Uo, nullptr, fl, s0, &err);   // Uo = U0 T
            if (rc == LS_OK) rc = x64_small(nm, H, no, Uc, no, ks, T1, nullptr, fl, s0, &err);    // T1 = H Uo
            const double* T1c[3] = {T1[0], T1[1], T1[2]};
            if (rc == LS_OK) rc = x64_small(nm, Uc, yes, T1c, no, ks, Hp, nullptr, fl, s0, &err); // H' = Uo^T T1
            return rc == LS_OK ? cudaSuccess : (rc == LS_ERR_OOM ? cudaErrorMemoryAllocation : cudaErrorLaunchFailure);
        });
        if (e != cudaSuccess) return err(e, "re-projection");
    }
    if (!s2.empty()) {
        Scope sc("jacobi.run2", s0);
        if ((e = run_df(s2.data(), (int)s2.size(), 60, s0)) != cudaSuccess) return err(e, "Jacobi (second run)");
    }
    e = per_ctx([&](RedState& Rs, RedMode** ms, int nm) {
        if (Rs.fast_eig) {
            // V = Uo; the Rayleigh quotients on the diagonal of H' are the eigenvalues
            for (int j = 0; j < nm; ++j) {
                cudaError_t ce = cudaMemcpyAsync(ms[j]->V, ms[j]->Uo, sizeof(double) * ms[j]->k * ms[j]->k,
                                                 cudaMemcpyDeviceToDevice, s0);
                if (ce != cudaSuccess) return ce;
            }
            return cudaSuccess;
        }
        const double *A[3], *B[3];
        double* out[3];
        int ks[3];
        for (int j = 0; j < nm; ++j) { A[j] = ms[j]->Uo; B[j] = ms[j]->F2; out[j] = ms[j]->V; ks[j] = ms[j]->k; }
        const int no[3] = {0, 0, 0};
        std::string err;
        const int rc = x64_small(nm, A, no, B, no, ks, out, A, &Rs.d_st[9].flag, s0, &err);   // V = Uo + Uo F2
        return rc == LS_OK ? cudaSuccess : (rc == LS_ERR_OOM ? cudaErrorMemoryAllocation : cudaErrorLaunchFailure);
    });
    if (e != cudaSuccess) return err(e, "eigenvectors");
    for (int i = 0; i < n; ++i)
        for (int l = 0; l < 3; ++l) {
            RedMode& M = R[i].m[l];
            if (M.df) std::swap(M.H, M.Hp);   // eigenvalues on the diagonal of H'
        }
    return LS_OK;
}

// The grid form of the pivoted Cholesky for the jobs beyond a cluster's shared memory,
// panel by panel: each launch takes up to kPcholPanel pivots of every unfinished job and
// leaves the panel's columns in Lp (zero past the last pivot), and the FP64-grade
// tensor-core product G -= Lp Lp^T turns G into the Schur complement the next panel
// starts from. The panel kernel reads where to continue from the device, so panels and
// products queue kPcholGroup at a time with one read-back a group (a job that ended
// takes no pivots and yields a zero panel). The panel's own updates stay in FP64.
constexpr int kPcholPanel = 64, kPcholGroup = 4;
int pchol_grid(ls_ctx* c0, std::vector<PcholJob> jobs, cudaStream_t st) {
    const int n = (int)jobs.size();
    if (n == 0) return LS_OK;
    int* d_rep = nullptr;
    double* d_lp = nullptr;
    int64_t lp_total = 0;
    for (const PcholJob& J : jobs) lp_total += J.C * kPcholPanel;
    if (cudaMallocAsync(&d_rep, sizeof(int) * 2 * n, st) != cudaSuccess ||
        cudaMallocAsync(&d_lp, sizeof(double) * lp_total, st) != cudaSuccess) {
        if (d_rep) cudaFreeAsync(d_rep, st);
        return fail(c0, LS_ERR_OOM, "rhosvd_reduce: pivoted Cholesky: out of memory");
    }
    for (int64_t j = 0, off = 0; j < n; off += jobs[j].C * kPcholPanel, ++j) jobs[j].Lp = d_lp + off;
    std::vector<int> rep(2 * n), prev(n, 0);
    std::vector<int> live(n);
    for (int j = 0; j < n; ++j) live[j] = j;
    int rc = LS_OK;
    while (!live.empty() && rc == LS_OK) {
        std::vector<PcholJob> lj;
        std::vector<const double*> L;
        std::vector<int64_t> ld, C;
        std::vector<int> k0, kb;
        std::vector<double*> S;
        std::vector<const int*> skip;
        for (int j : live) {
            skip.push_back(&jobs[j].st->done);   // the job ended: its Schur complement is not wanted
            lj.push_back(jobs[j]);
            L.push_back(jobs[j].Lp);
            ld.push_back(kPcholPanel);
            k0.push_back(0);
            kb.push_back(kPcholPanel);
            C.push_back(jobs[j].C);
            S.push_back(const_cast<double*>(jobs[j].G));
        }
        const int m = (int)lj.size();
        int64_t Cmax = 1;
        for (const PcholJob& J : lj) Cmax = std::max<int64_t>(Cmax, J.C);
        // one cluster a matrix where its rows' panel columns fit the cluster's shared memory
        const bool cl = pchol_cpanel_fits(Cmax, kPcholPanel);
        for (int g = 0; g < kPcholGroup && rc == LS_OK; ++g) {
            cudaError_t e;
            {
                Scope sc("pchol.panel", st);
                e = cl ? launch_pchol_cpanel(lj.data(), kPcholPanel, m, d_rep, st)
                       : launch_pchol_panel(lj.data(), kPcholPanel, m, c0->num_sms, d_rep, st);
            }
            if (e != cudaSuccess) {
                rc = fail(c0, LS_ERR_CUDA, "rhosvd_reduce: pivoted Cholesky panel: %s", cudaGetErrorString(e));
                break;
            }
            Scope sc("pchol.schur", st);
            std::string err;
            int r2 = x64_syrk_sub(m, L.data(), ld.data(), k0.data(), kb.data(), C.data(), S.data(),
                                  &lj[0].st->flag, st, &err, skip.data());
            if (r2 != LS_OK) rc = fail(c0, r2, "rhosvd_reduce: Schur complement: %s", err.c_str());
        }
        if (rc != LS_OK) break;
        cudaError_t e = cudaMemcpyAsync(rep.data(), d_rep, sizeof(int) * 2 * m, cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) {
            rc = fail(c0, LS_ERR_CUDA, "rhosvd_reduce: pivoted Cholesky read-back: %s", cudaGetErrorString(e));
            break;
        }
        count_d2h(sizeof(int) * 2 * m);
        std::vector<int> next;
        for (int i = 0; i < m; ++i) {
            const int j = live[i];
            // ended, or no progress in a whole group (a failed barrier, whose flag the caller reports)
            if (rep[2 * i + 1] || rep[2 * i] >= jobs[j].kmax || rep[2 * i] <= prev[j]) continue;
            prev[j] = rep[2 * i];
            next.push_back(j);
        }
        live.swap(next);
    }
    cudaFreeAsync(d_lp, st);
    cudaFreeAsync(d_rep, st);
    return rc;
}

// The reduction of n contexts: per-context phases on each context's stream;
// the cooperative steps (pivoted Cholesky, Jacobi iteration, the two Cholesky
// factorisations of CholeskyQR2) of all 3n modes as one launch each on the
// first context's stream, so that no two cooperative grids run at once.
int reduce_many(ls_ctx* const* ctxs, int n, double eps, const int32_t* forced, ls_tucker_info* infos,
                const RedState* pass = nullptr, RedState* pass_out = nullptr) {
    std::vector<RedState> R(n);
    std::vector<PcholJob> pj(3 * (size_t)n);
    std::vector<JacobiJob> jj(3 * (size_t)n);
    std::vector<CholJob> cj(3 * (size_t)n);
    ls_ctx* c0 = ctxs[0];
    cudaStream_t s0 = c0->st;
    auto gather = [&](ls_ctx* c) -> int {
        if (join(s0, c->st) != cudaSuccess) return fail(c, LS_ERR_CUDA, "rhosvd_reduce: stream join failed");
        return LS_OK;
    };
    auto scatter = [&](ls_ctx* c) -> int {
        if (join(c->st, s0) != cudaSuccess) return fail(c, LS_ERR_CUDA, "rhosvd_reduce: stream join failed");
        return LS_OK;
    };
    auto sync_all = [&]() -> int {
        for (int i = 0; i < n; ++i)
            if (cudaStreamSynchronize(ctxs[i]->st) != cudaSuccess)
                return fail(ctxs[i], LS_ERR_CUDA, "rhosvd_reduce: sync failed");
        return LS_OK;
    };
    // first CholeskyQR pass: FP32 shared-memory factorisation where r fits, FP64 grid otherwise
    auto chol_all = [&]() -> int {
        for (int i = 0; i < n; ++i)
            if (int rc = gather(ctxs[i])) return rc;
        {
            Scope sc("cholqr2", s0);
            Scope sf("cholqr2.factor", s0);
            const int rmax = chol32_max_r();
            std::vector<CholJob> small, large;
            for (const CholJob& J : cj) (J.r <= rmax ? small : large).push_back(J);
            cudaError_t e = launch_chol32_multi(small.data(), (int)small.size(), s0);
            if (e == cudaSuccess) e = launch_chol_inv_multi(large.data(), (int)large.size(), c0->num_sms, s0);
            if (e != cudaSuccess) return fail(c0, LS_ERR_CUDA, "rhosvd_reduce: Cholesky launch: %s", cudaGetErrorString(e));
        }
        for (int i = 0; i < n; ++i)
            if (int rc = scatter(ctxs[i])) return rc;
        return LS_OK;
    };
    for (int i = 0; i < n; ++i) {
        if (pass) R[i] = *pass;   // a pass of the non-squaring route (one context)
        R[i].fast_eig = R[i].kind != 0 || ctxs[i]->p.precision == LS_MIXED;
        R[i].ctx = ctxs[i];
        R[i].eps = eps;
        R[i].forced = forced;
        if (int rc = red_prepare(R[i], &pj[3 * i])) return rc;
        if (int rc = gather(ctxs[i])) return rc;
    }
    {
        // shared-memory cluster form where G and L fit, the grid form otherwise
        Scope sc("pchol", s0);
        std::vector<PcholJob> small, large;
        for (const PcholJob& J : pj) (pchol_cluster_size((int)J.C, J.kmax) > 0 ? small : large).push_back(J);
        cudaError_t e = launch_pchol_cluster(small.data(), (int)small.size(), s0);
        if (e != cudaSuccess) return fail(c0, LS_ERR_CUDA, "rhosvd_reduce: pivoted Cholesky launch: %s", cudaGetErrorString(e));
        if (int rc = pchol_grid(c0, large, s0)) return rc;
    }
    for (int i = 0; i < n; ++i) {
        if (int rc = scatter(ctxs[i])) return rc;
        if (cudaMemcpyAsync(R[i].hs, R[i].d_st, 3 * sizeof(DevStatus), cudaMemcpyDeviceToHost, ctxs[i]->st) != cudaSuccess)
            return fail(ctxs[i], LS_ERR_CUDA, "rhosvd_reduce: status read failed");
        count_d2h(3 * sizeof(DevStatus));
    }
    if (int rc = sync_all()) return rc;
    for (int i = 0; i < n; ++i) {
        if (int rc = red_after_pchol(R[i], &jj[3 * i])) return rc;
        if (int rc = gather(ctxs[i])) return rc;
    }
    {
        Scope sc("jacobi", s0);
        if (int rc = eigen_all(R, ctxs, n, jj, s0)) return rc;
    }
    for (int i = 0; i < n; ++i) {
        if (int rc = scatter(ctxs[i])) return rc;
        if (int rc = red_select(R[i])) return rc;
    }
    if (int rc = sync_all()) return rc;
    for (int i = 0; i < n; ++i)
        if (R[i].kind == 2)
            for (int l = 0; l < 3; ++l)   // nothing above the threshold: the kept energy at r = 1 is below it
                R[i].drop[l] = R[i].sel[l][2] - R[i].sel[l][1] <= R[i].cand_res[l];
    for (int i = 0; i < n; ++i)
        if (int rc = red_basis(R[i], &cj[3 * i])) return rc;
    if (int rc = chol_all()) return rc;
    for (int i = 0; i < n; ++i)
        if (int rc = red_cholqr_mid(R[i])) return rc;
    int first_err = LS_OK;
    std::vector<char> queued(n, 0);
    for (int i = 0; i < n; ++i) {
        R[i].defer_release = n > 1 && R[i].kind == 0;
        int rc = red_finish(R[i], infos ? &infos[i] : nullptr);
        queued[i] = rc == LS_OK && R[i].defer_release;
        if (rc != LS_OK && first_err == LS_OK) first_err = rc;
    }
    // the releases after every context's projection and core are queued
    for (int i = 0; i < n; ++i) {
        if (!queued[i]) continue;
        int rc = red_release(R[i], infos ? &infos[i] : nullptr);
        if (rc != LS_OK && first_err == LS_OK) first_err = rc;
    }
    if (pass_out) *pass_out = R[0];
    return first_err;
}

// a failing CUDA call inside reduce_accurate: the scratch context goes too
#define CUB(call)                                                                                  \
    do {                                                                                           \
        cudaError_t e_ = (call);                                                                   \
        if (e_ != cudaSuccess)                                                                     \
            return bail(fail(ctx, e_ == cudaErrorMemoryAllocation ? LS_ERR_OOM : LS_ERR_CUDA, "%s: %s (%s:%d)", \
                             #call, cudaGetErrorString(e_), __FILE__, __LINE__));                  \
    } while (0)

// Whether a context takes the non-squaring route: FP64 contexts by default, either
// precision on request (LS_FLAG_SVD_ONESIDED), neither with LS_FLAG_SVD_GRAM.
bool one_sided(const ls_ctx* ctx) {
    if (ctx->p.flags & LS_FLAG_SVD_GRAM) return false;
    return ctx->p.precision == LS_FP64 || (ctx->p.flags & LS_FLAG_SVD_ONESIDED);
}

// The non-squaring route (Def. 4.1 with the singular values of each side matrix itself):
//  1. the Gram route's candidate basis Q1: every eigen-direction of the weighted Gram matrix
//     1e3 times above its rounding noise 8 u T (all of them well conditioned);
//  2. the residual rows E = A_w - (A_w Q1^T) Q1 (the part of the side matrix outside Q1,
//     formed without squaring) and, by the same route on E, a basis Q2 of its range,
//     orthogonal to Q1: E's Gram matrix resolves singular values down to about
//     sqrt(u ||A|| ||E||) instead of sqrt(u) ||A||;
//  3. one-sided Jacobi on the rows of B = Q A_w^T, Q = [Q1; Q2]: the singular values and
//     the rotation M, with no product B B^T; the eps rule (or a forced rank) on those values,
//     with E's energy outside Q2 in the discarded tail;
//  4. Z = M_r Q, the leading r rotated basis vectors; then the projection and the core.
// The terms and the unit canonical vectors for the projection and the core, when the side
// matrix of the truncation is another one (the Tucker-reference variant): what the Gram
// route's first phase does for the canonical side matrix.
int prepare_terms(ls_ctx* ctx) {
    cudaStream_t st = ctx->st;
    const int64_t N = ctx->p.N;
    const int64_t T = (int64_t)ctx->xi.size();
    CU(dalloc(ctx, &ctx->d_tcol, 3 * T));
    CU(dalloc(ctx, &ctx->d_xi, T));
    CU(dalloc(ctx, &ctx->d_xin, T));
    CU(upload_h2d(ctx->d_tcol, ctx->tcol.data(), 3 * T * sizeof(int32_t), st));
    count_h2d(3 * T * sizeof(int32_t));
    CU(upload_h2d(ctx->d_xi, ctx->xi.data(), T * sizeof(double), st));
    count_h2d(T * sizeof(double));
    for (int l = 0; l < 3; ++l) {
        const int64_t C = ctx->mode[l].C;
        CU(dalloc(ctx, &ctx->d_norms[l], C));
        CU(dalloc(ctx, &ctx->d_sigma[l], C));
        CU(cudaMemsetAsync(ctx->d_sigma[l], 0, C * sizeof(double), st));
        Scope sc("norms", st);
        CU(launch_norm_columns(ctx->mode[l].d_cols, C, N, ctx->d_norms[l], st));
    }
    return LS_OK;
}

// `side` (may be NULL): a scratch context whose columns are the side matrix of the truncation,
// its rows already weighted (the Tucker-reference variant's scaled blocks), with side_T their
// total energy and Bhat the |B_hat| of Thm 4.3; NULL: the canonical side matrix of ctx itself
// (unit vectors weighted by sqrt(multiplicity)).
int reduce_accurate(ls_ctx* ctx, double eps, const int32_t* forced, ls_tucker_info* info, ls_ctx* side = nullptr,
                    double side_T = 0.0, double Bhat = 0.0) {
    cudaStream_t st = ctx->st;
    const int64_t N = ctx->p.N;
    const double u = 1.1102230246251565e-16;
    const int64_t T = (int64_t)ctx->xi.size();
    ls_ctx* sx = side ? side : ctx;
    int64_t C[3];
    for (int l = 0; l < 3; ++l) C[l] = sx->mode[l].C;
    if (side)
        if (int rc = prepare_terms(ctx)) return rc;
    // 1. candidate basis Q1 (in sx->d_Z, m1 rows)
    RedState p1, r1;
    p1.kind = side ? 2 : 1;
    const double floor1 = 8.0 * u * (side ? side_T : (double)T);
    p1.floor_noise = floor1;
    for (int l = 0; l < 3; ++l) p1.cand_res[l] = 1e3 * floor1;
    {
        ls_ctx* one[1] = {sx};
        Scope sc("svd.pass1", st);
        if (int rc = reduce_many(one, 1, eps, nullptr, nullptr, &p1, &r1)) {
            if (side && ctx->err.empty()) ctx->err = side->err;
            return rc;
        }
    }
    int m1[3];
    double tail1[3];
    for (int l = 0; l < 3; ++l) {
        m1[l] = sx->r[l];
        tail1[l] = std::max(r1.sel[l][1], 0.0);
        dfree(sx, sx->d_P[l]);
        sx->d_P[l] = nullptr;
    }
    DevStatus* ds = nullptr;   // [0]: the tensor-core products' flag; [1..3]: the one-sided Jacobi
    CU(dalloc(ctx, &ds, 4));
    CU(cudaMemsetAsync(ds, 0, 4 * sizeof(DevStatus), st));
    int* flag = &ds[0].flag;
    double* w[3];
    for (int l = 0; l < 3; ++l) {
        if (side) {
            w[l] = side->d_norms[l];   // the scratch rows are unit after the first pass; their norms weight them
            continue;
        }
        std::vector<double> wh(C[l]);
        for (int64_t c = 0; c < C[l]; ++c) wh[c] = sqrt((double)ctx->mode[l].count[c]);
        CU(dalloc(ctx, &w[l], C[l]));
        CU(upload_h2d(w[l], wh.data(), C[l] * sizeof(double), st));
        count_h2d(C[l] * sizeof(double));
    }
    // 2. residual rows E (the columns of a scratch context) and their basis Q2
    ls_ctx* e = new ls_ctx();
    e->p = ctx->p;
    e->st = st;
    e->num_sms = ctx->num_sms;
    e->h = ctx->h;
    auto bail = [&](int rc) {
        if (!e->err.empty() && ctx->err.empty()) ctx->err = e->err;
        lattice_sum_destroy(e);
        return rc;
    };
    {
        Scope sc("svd.residual", st);
        double *B1[3], *D[3], *B1m[3];
        X64Mat xs[3], ys[3];
        int64_t ld[3];
        for (int l = 0; l < 3; ++l) {
            ModeCols& em = e->mode[l];
            em.C = em.cap = C[l];
            em.count.assign(C[l], 1);
            if (dalloc(e, &em.d_cols, C[l] * N) != cudaSuccess || dalloc(ctx, &B1[l], (int64_t)m1[l] * C[l]) != cudaSuccess ||
                dalloc(ctx, &D[l], C[l] * N) != cudaSuccess)
                return bail(fail(ctx, LS_ERR_OOM, "rhosvd_reduce: out of device memory (residual rows)"));
            B1m[l] = B1[l];
            xs[l] = X64Mat{sx->d_Z[l], m1[l], N, N, 1, nullptr};        // Q1
            ys[l] = X64Mat{sx->mode[l].d_cols, C[l], N, N, 1, w[l]};    // A_w (rows)
            ld[l] = C[l];
        }
        std::string err;
        int rc = x64_nt(3, xs, ys, B1m, ld, flag, st, &err);              // B1 = Q1 A_w^T (m1 x C)
        for (int l = 0; l < 3; ++l) {
            xs[l] = X64Mat{B1[l], C[l], m1[l], 1, C[l], nullptr};        // B1^T (C x m1)
            ys[l] = X64Mat{sx->d_Z[l], N, m1[l], 1, N, nullptr};         // Q1^T (N x m1)
            ld[l] = N;
        }
        if (rc == LS_OK) rc = x64_nt(3, xs, ys, D, ld, flag, st, &err);  // D = B1^T Q1 (C x N)
        if (rc != LS_OK) return bail(fail(ctx, rc, "rhosvd_reduce: residual rows: %s", err.c_str()));
        for (int l = 0; l < 3; ++l) {
            if (launch_resid_rows(sx->mode[l].d_cols, w[l], D[l], C[l], N, e->mode[l].d_cols, st) != cudaSuccess)
                return bail(fail(ctx, LS_ERR_CUDA, "rhosvd_reduce: residual rows launch failed"));
            dfree(ctx, B1[l]);
            dfree(ctx, D[l]);
        }
    }
    // E carries the rounding dE of the two products that formed it, ||dE||_F^2 <= about
    // 2 u^2 T (m1 + 1) (each entry of B1^T Q1 to u sum_i |B1_ic| |Q1_in|, and sum_c w_c^2 = T).
    // An eigenvalue lambda of E E^T moves by about 2 sqrt(lambda) ||dE v|| (the matrix is
    // graded), so a direction is real when lambda is well above ||dE||^2; E's own Gram matrix
    // adds u ||E||^2 (||E||^2 = the first pass's discarded energy). Candidates are taken 100
    // times above floor = 8 u ||E||^2 + 64 u^2 T (m1 + 1): singular values down to about
    // 1e-13 of sigma_1 on the 16^3 lattice.
    RedState p2, r2;
    p2.kind = 2;
    p2.floor_noise = 0.0;
    for (int l = 0; l < 3; ++l) {
        const double fl = 8.0 * u * tail1[l] + 64.0 * u * u * (double)T * (double)(m1[l] + 1);
        p2.floor_noise = std::max(p2.floor_noise, fl);
        p2.cand_res[l] = 1e2 * fl;
        p2.reorth[l] = sx->d_Z[l];
        p2.reorth_m[l] = m1[l];
    }
    {
        ls_ctx* one[1] = {e};
        Scope sc("svd.pass2", st);
        if (int rc = reduce_many(one, 1, eps, nullptr, nullptr, &p2, &r2)) return bail(rc);
    }
    int m2[3], m[3];
    double tail2[3];
    for (int l = 0; l < 3; ++l) {
        m2[l] = r2.drop[l] ? 0 : (int)std::min<int64_t>(e->r[l], std::max<int64_t>(0, C[l] - m1[l]));
        tail2[l] = std::max(r2.drop[l] ? r2.sel[l][2] : r2.sel[l][1], 0.0);
        m[l] = m1[l] + m2[l];
    }
    // 3. B = Q A_w^T and its one-sided Jacobi SVD
    double *Q[3], *Bm[3], *Mr[3], *sig2[3], *isl[3], *extra = nullptr, *sel = nullptr;
    int32_t* perm[3];
    {
        Scope sc("svd.onesided", st);
        X64Mat xs[3], ys[3];
        int64_t ld[3];
        for (int l = 0; l < 3; ++l) {
            if (dalloc(ctx, &Q[l], (int64_t)m[l] * N) != cudaSuccess || dalloc(ctx, &Bm[l], (int64_t)m[l] * C[l]) != cudaSuccess ||
                dalloc(ctx, &Mr[l], (int64_t)m[l] * m[l]) != cudaSuccess || dalloc(ctx, &sig2[l], m[l]) != cudaSuccess ||
                dalloc(ctx, &isl[l], m[l]) != cudaSuccess || dalloc(ctx, &perm[l], m[l]) != cudaSuccess)
                return bail(fail(ctx, LS_ERR_OOM, "rhosvd_reduce: out of device memory (one-sided Jacobi)"));
            if (cudaMemcpyAsync(Q[l], sx->d_Z[l], (size_t)m1[l] * N * sizeof(double), cudaMemcpyDeviceToDevice, st) != cudaSuccess ||
                (m2[l] > 0 && cudaMemcpyAsync(Q[l] + (int64_t)m1[l] * N, e->d_Z[l], (size_t)m2[l] * N * sizeof(double),
                                              cudaMemcpyDeviceToDevice, st) != cudaSuccess))
                return bail(fail(ctx, LS_ERR_CUDA, "rhosvd_reduce: basis copy failed"));
            xs[l] = X64Mat{Q[l], m[l], N, N, 1, nullptr};
            ys[l] = X64Mat{sx->mode[l].d_cols, C[l], N, N, 1, w[l]};
            ld[l] = C[l];
        }
        std::string err;
        int rc = x64_nt(3, xs, ys, Bm, ld, flag, st, &err);               // B = Q A_w^T (m x C)
        if (rc != LS_OK) return bail(fail(ctx, rc, "rhosvd_reduce: B = Q A^T: %s", err.c_str()));
        unsigned* cmax = nullptr;
        if (dalloc(ctx, &cmax, 3 * 64) != cudaSuccess)
            return bail(fail(ctx, LS_ERR_OOM, "rhosvd_reduce: out of device memory (one-sided Jacobi)"));
        CUB(cudaMemsetAsync(cmax, 0, 3 * 64 * sizeof(unsigned), st));
        OsjJob jobs[3];
        for (int l = 0; l < 3; ++l)
            jobs[l] = OsjJob{Bm[l], C[l], (int)C[l], Mr[l], m[l], sig2[l], ds + 1 + l, 8.0 * u * sqrt((double)C[l]),
                             cmax + 64 * l};
        if (launch_osj(jobs, 3, 40, ctx->num_sms, st) != cudaSuccess)
            return bail(fail(ctx, LS_ERR_CUDA, "rhosvd_reduce: one-sided Jacobi launch failed"));
        dfree(ctx, cmax);
    }
    // eps rule (or forced rank) on sigma^2, with the energy outside Q in the tail
    double hsel[3][3];
    DevStatus hds[4];
    {
        Scope sc("select", st);
        if (dalloc(ctx, &extra, 3) != cudaSuccess || dalloc(ctx, &sel, 9) != cudaSuccess)
            return bail(fail(ctx, LS_ERR_OOM, "rhosvd_reduce: out of device memory (selection)"));
        CUB(upload_h2d(extra, tail2, sizeof tail2, st));
        count_h2d(sizeof tail2);
        SortSelectJob jobs[3];
        for (int l = 0; l < 3; ++l) {
            CUB(cudaMemsetAsync(ctx->d_sigma[l], 0, ctx->mode[l].C * sizeof(double), st));
            const int fr = forced ? std::max(1, std::min(forced[l], m[l])) : 0;
            jobs[l] = SortSelectJob{sig2[l], m[l], fr, extra + l, perm[l], ctx->d_sigma[l], isl[l], sel + 3 * l};
            jobs[l].dstride = 1;
            jobs[l].resolution = 0.0;
        }
        CUB(launch_sort_select(3, jobs, eps, 0.0, st));
        CUB(cudaMemcpyAsync(hsel, sel, sizeof hsel, cudaMemcpyDeviceToHost, st));
        CUB(cudaMemcpyAsync(hds, ds, sizeof hds, cudaMemcpyDeviceToHost, st));
        count_d2h(sizeof hsel + sizeof hds);
        CUB(cudaStreamSynchronize(st));
    }
    for (int l = 0; l < 4; ++l)
        if (hds[l].flag == FLAG_TIMEOUT) return bail(fail(ctx, LS_ERR_TIMEOUT, "rhosvd_reduce: a bounded wait timed out"));
    for (int l = 0; l < 3; ++l)
        if (hds[1 + l].flag == FLAG_NOCONVERGE)
            return bail(fail(ctx, LS_ERR_NOCONVERGE, "rhosvd_reduce: one-sided Jacobi did not converge (mode %d)", l));
    // 4. Z = M_r Q
    {
        Scope sc("svd.basis", st);
        double* Ms[3];
        X64Mat xs[3], ys[3];
        int64_t ld[3];
        for (int l = 0; l < 3; ++l) {
            ctx->r[l] = (int32_t)hsel[l][0];
            if (!side) dfree(ctx, ctx->d_Z[l]);
            ctx->d_Z[l] = nullptr;
            if (dalloc(ctx, &ctx->d_Z[l], (int64_t)ctx->r[l] * N) != cudaSuccess ||
                dalloc(ctx, &ctx->d_P[l], (int64_t)ctx->r[l] * ctx->mode[l].C) != cudaSuccess ||
                dalloc(ctx, &Ms[l], (int64_t)ctx->r[l] * m[l]) != cudaSuccess)
                return bail(fail(ctx, LS_ERR_OOM, "rhosvd_reduce: out of device memory (basis)"));
            CUB(launch_gather_rows(Mr[l], m[l], perm[l], ctx->r[l], nullptr, Ms[l], st));
            xs[l] = X64Mat{Ms[l], ctx->r[l], m[l], m[l], 1, nullptr};   // M_r (r x m)
            ys[l] = X64Mat{Q[l], N, m[l], 1, N, nullptr};                // Q^T (N x m)
            ld[l] = N;
        }
        std::string err;
        int rc = x64_nt(3, xs, ys, ctx->d_Z, ld, flag, st, &err);
        if (rc != LS_OK) return bail(fail(ctx, rc, "rhosvd_reduce: basis: %s", err.c_str()));
        for (int l = 0; l < 3; ++l) {
            for (void* q : {(void*)Ms[l], (void*)Bm[l], (void*)Mr[l], (void*)sig2[l], (void*)isl[l], (void*)perm[l]})
                dfree(ctx, q);
            // the range basis stays with the context (the ALS refinement restricts its SVDs to it)
            dfree(ctx, ctx->d_Q[l]);
            ctx->d_Q[l] = Q[l];
            ctx->mq[l] = m[l];
            if (!side) dfree(ctx, w[l]);
        }
        dfree(ctx, extra);
    }
    lattice_sum_destroy(e);
    // projection, core, statuses and info, as the Gram route finishes
    RedState rf;
    rf.ctx = ctx;
    rf.eps = eps;
    rf.forced = forced;
    rf.T = T;
    rf.floor_noise = 64.0 * u * u * (side ? side_T : (double)T);   // the singular values' own rounding, squared, per column
    rf.d_sel = sel;
    rf.d_st = ds;   // [0] as the products' flag slot is read at [9]: use a fresh status block
    {
        DevStatus* d10 = nullptr;
        CU(dalloc(ctx, &d10, 10));
        CU(cudaMemsetAsync(d10, 0, 10 * sizeof(DevStatus), st));
        dfree(ctx, ds);
        rf.d_st = d10;
    }
    for (int l = 0; l < 3; ++l) {
        for (int j = 0; j < 3; ++j) rf.sel[l][j] = hsel[l][j];
        rf.sweeps[l] = hds[1 + l].sweeps;
        int64_t rot = 0;
        for (int k = 0; k < hds[1 + l].sweeps && k < 64; ++k) rot += hds[1 + l].sweep_active[k];
        rf.rotations[l] = rot;
        rf.m[l].k = r1.m[l].k;
    }
    const int rc = red_project_core(rf, info);
    if (rc == LS_OK && side && info) {
        // Thm 4.3: |B_hat| in place of ||xi||, the side matrix's discarded tails
        double ssum = 0.0;
        for (int l = 0; l < 3; ++l) ssum += sqrt(std::max(hsel[l][0] > 0 ? rf.sel[l][1] : 0.0, 0.0) + (double)C[l] * rf.floor_noise);
        info->xi_norm = Bhat;
        info->bound_abs = Bhat * ssum;
    }
    return rc;
}

// The generalized RHOSVD of the Tucker-reference variant (Thm 4.3): the side matrix of mode l
// holds, for every key (a block's assembled or a defect's windowed reference Tucker vectors),
// its r_ref vectors scaled to unit Frobenius norm and weighted by sqrt(#terms using the key);
// |B_hat|^2 = ||b||^2 sum_s charge_s^2 prod_l |F_{s,l}|_F^2. The truncation then runs the
// non-squaring route on that side matrix, the projection and the core on the canonical
// vectors of the projected reference (the Tucker sum written as a canonical sum).
int reduce_tucker(ls_ctx* ctx, double eps, const int32_t* forced, ls_tucker_info* info) {
    cudaStream_t st = ctx->st;
    const int64_t N = ctx->p.N;
    const int r = ctx->r_ref;
    const int64_t S = (int64_t)ctx->txi.size();
    ls_ctx* sc = new ls_ctx();
    sc->p = ctx->p;
    sc->st = st;
    sc->num_sms = ctx->num_sms;
    sc->h = ctx->h;
    auto bail = [&](int rc) {
        if (!sc->err.empty() && ctx->err.empty()) ctx->err = sc->err;
        lattice_sum_destroy(sc);
        return rc;
    };
    std::vector<double> hn[3];
    double* nrm[3];
    double* mult[3];
    for (int l = 0; l < 3; ++l) {
        const ModeCols& tm = ctx->tmode[l];
        const int nk = (int)(tm.C / r);
        std::vector<double> mh(nk);
        for (int k = 0; k < nk; ++k) mh[k] = (double)tm.count[(int64_t)k * r];
        ModeCols& sm = sc->mode[l];
        sm.C = sm.cap = tm.C;
        sm.count.assign(tm.C, 1);
        if (dalloc(sc, &sm.d_cols, tm.C * N) != cudaSuccess || dalloc(ctx, &nrm[l], nk) != cudaSuccess ||
            dalloc(ctx, &mult[l], nk) != cudaSuccess)
            return bail(fail(ctx, LS_ERR_OOM, "rhosvd_reduce: out of device memory (Tucker side matrix)"));
        if (upload_h2d(mult[l], mh.data(), nk * sizeof(double), st) != cudaSuccess ||
            launch_block_frob(tm.d_cols, r, N, nk, mult[l], nrm[l], sm.d_cols, st) != cudaSuccess)
            return bail(fail(ctx, LS_ERR_CUDA, "rhosvd_reduce: Tucker side matrix launch failed"));
        count_h2d(nk * sizeof(double));
        hn[l].resize(nk);
    }
    for (int l = 0; l < 3; ++l)
        if (cudaMemcpyAsync(hn[l].data(), nrm[l], hn[l].size() * sizeof(double), cudaMemcpyDeviceToHost, st) != cudaSuccess)
            return bail(fail(ctx, LS_ERR_CUDA, "rhosvd_reduce: read-back failed"));
    if (cudaStreamSynchronize(st) != cudaSuccess) return bail(fail(ctx, LS_ERR_CUDA, "rhosvd_reduce: sync failed"));
    count_d2h((int64_t)(hn[0].size() + hn[1].size() + hn[2].size()) * sizeof(double));
    double bh2 = 0.0;
    for (int64_t t = 0; t < S; ++t) {
        double f = ctx->txi[t] * ctx->txi[t];
        for (int l = 0; l < 3; ++l) f *= hn[l][ctx->tkey[3 * t + l]] * hn[l][ctx->tkey[3 * t + l]];
        bh2 += f;
    }
    bh2 *= ctx->bnorm2;
    for (int l = 0; l < 3; ++l) {
        dfree(ctx, nrm[l]);
        dfree(ctx, mult[l]);
    }
    const int rc = reduce_accurate(ctx, eps, forced, info, sc, (double)S, sqrt(bh2));
    return bail(rc);
}

}  // namespace

extern "C" {

int lattice_sum_rhosvd_reduce(ls_ctx* ctx, double eps, const int32_t* forced_ranks, ls_tucker_info* info) {
    ls::NvtxRange nvtx_("lattice_sum_rhosvd_reduce");
    if (!ctx) return fail(nullptr, LS_ERR_ARG, "rhosvd_reduce: NULL context");
    if (ctx->reduced) return fail(ctx, LS_ERR_STATE, "rhosvd_reduce: already reduced");
    if (!forced_ranks && !(eps > 0.0)) return fail(ctx, LS_ERR_ARG, "rhosvd_reduce: eps must be > 0");
    ls_ctx* one[1] = {ctx};
    ls_tucker_info mine{};
    ls_tucker_info* inf = info ? info : &mine;
    const int rc = ctx->tucker     ? reduce_tucker(ctx, eps, forced_ranks, inf)
                   : one_sided(ctx) ? reduce_accurate(ctx, eps, forced_ranks, inf)
                                    : reduce_many(one, 1, eps, forced_ranks, inf);
    if (rc == LS_OK) ctx->last_info = *inf;
    // a large reduction leaves tens of GB of freed scratch in the stream-ordered pool
    // (the stream is synchronised here): when the device runs short, give it back beyond a
    // few GB, so that other allocators on the device can use it
    size_t fr = 0, tot = 0;
    if (rc == LS_OK && cudaMemGetInfo(&fr, &tot) == cudaSuccess && fr < ((size_t)32 << 30)) {
        cudaMemPool_t pool;
        int dev = 0;
        if (cudaGetDevice(&dev) == cudaSuccess && cudaDeviceGetDefaultMemPool(&pool, dev) == cudaSuccess)
            cudaMemPoolTrimTo(pool, (size_t)4 << 30);
    }
    return rc;
}

int lattice_sum_batch_reduce(ls_ctx* const* ctxs, int32_t n, double eps, ls_tucker_info* infos) {
    ls::NvtxRange nvtx_("lattice_sum_batch_reduce");
    if (!ctxs || n < 1) return fail(nullptr, LS_ERR_ARG, "batch_reduce: no contexts");
    if (!(eps > 0.0)) return fail(nullptr, LS_ERR_ARG, "batch_reduce: eps must be > 0");
    for (int i = 0; i < n; ++i) {
        if (!ctxs[i]) return fail(nullptr, LS_ERR_ARG, "batch_reduce: NULL context %d", i);
        if (ctxs[i]->reduced) return fail(ctxs[i], LS_ERR_STATE, "batch_reduce: context %d already reduced", i);
        for (int j = 0; j < i; ++j)
            if (ctxs[j] == ctxs[i]) return fail(nullptr, LS_ERR_ARG, "batch_reduce: context %d listed twice", i);
    }
    // contexts on the non-squaring route one by one, the others together
    std::vector<ls_ctx*> gram;
    std::vector<int> gi;
    int rc = LS_OK;
    for (int i = 0; i < n && rc == LS_OK; ++i) {
        if (ctxs[i]->tucker) rc = reduce_tucker(ctxs[i], eps, nullptr, infos ? &infos[i] : nullptr);
        else if (one_sided(ctxs[i])) rc = reduce_accurate(ctxs[i], eps, nullptr, infos ? &infos[i] : nullptr);
        else { gram.push_back(ctxs[i]); gi.push_back(i); }
    }
    if (rc == LS_OK && !gram.empty()) {
        std::vector<ls_tucker_info> gin(gram.size());
        rc = reduce_many(gram.data(), (int)gram.size(), eps, nullptr, infos ? gin.data() : nullptr);
        if (infos)
            for (size_t j = 0; j < gram.size(); ++j) infos[gi[j]] = gin[j];
    }
    if (rc != LS_OK) {
        for (int i = 0; i < n; ++i)
            if (!ctxs[i]->err.empty()) {
                g_create_error = ctxs[i]->err;
                break;
            }
    }
    return rc;
}

int lattice_sum_gemm_nt(const double* A, const double* B, int64_t M, int64_t N, int64_t K, double* D, void* stream) {
    if (!A || !B || !D || M < 0 || N < 0 || K < 1 || M > INT32_MAX || N > INT32_MAX)
        return fail(nullptr, LS_ERR_ARG, "gemm_nt: bad arguments");
    std::string err;
    int rc = x64_gemm_nt(A, B, M, N, K, D, static_cast<cudaStream_t>(stream), &err);
    if (rc != LS_OK) return fail(nullptr, rc, "gemm_nt: %s", err.c_str());
    return LS_OK;
}

int lattice_sum_jacobi_eig(const double* H, int32_t k, double tol, double abs_floor, int32_t form,
                           int32_t max_sweeps, double* D, double* V, int32_t* sweeps, void* stream) {
    if (!H || !D || !V || k < 1 || !(tol > 0.0) || !(abs_floor >= 0.0) || (form != 1 && form != 2) ||
        max_sweeps < 0 || max_sweeps > 60)
        return fail(nullptr, LS_ERR_ARG, "jacobi_eig: bad arguments");
    const int ms = max_sweeps ? max_sweeps : 60;
    if (form == 1 && k > jacobi_blk_max_k())
        return fail(nullptr, LS_ERR_ARG, "jacobi_eig: k = %d exceeds the cluster form (%d)", k, jacobi_blk_max_k());
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    DevStatus* ds = nullptr;
    cudaError_t e = cudaMallocAsync(&ds, sizeof(DevStatus), st);
    if (e != cudaSuccess) return fail(nullptr, LS_ERR_OOM, "jacobi_eig: %s", cudaGetErrorString(e));
    DevStatus h{};
    e = cudaMemsetAsync(ds, 0, sizeof(DevStatus), st);
    const DfJob J{H, k, D, 1, V, 1, ds, abs_floor, 0.0, tol};
    int dev = 0, nsm = 1;
    if (e == cudaSuccess) e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess) e = form == 1 ? launch_jacobi_blk(&J, 1, ms, st) : launch_jacobi_gblk(&J, 1, ms, nsm, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&h, ds, sizeof(DevStatus), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    cudaFreeAsync(ds, st);
    if (e != cudaSuccess) return fail(nullptr, LS_ERR_CUDA, "jacobi_eig: %s", cudaGetErrorString(e));
    if (sweeps) *sweeps = h.sweeps;
    if (h.flag == FLAG_TIMEOUT) return fail(nullptr, LS_ERR_TIMEOUT, "jacobi_eig: a bounded wait timed out");
    if (h.flag == FLAG_NOCONVERGE) return fail(nullptr, LS_ERR_NOCONVERGE, "jacobi_eig: no convergence in %d sweeps", ms);
    return LS_OK;
}

int lattice_sum_svd_rows(const double* B, int32_t m, int32_t C, double tol, int32_t max_sweeps, double* sig2,
                         double* M, int32_t* sweeps, int64_t* rotations, void* stream) {
    if (!B || !sig2 || !M || m < 1 || C < 1 || !(tol > 0.0) || max_sweeps < 0 || max_sweeps > 60)
        return fail(nullptr, LS_ERR_ARG, "svd_rows: bad arguments");
    const int ms = max_sweeps ? max_sweeps : 60;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    int dev = 0, nsm = 1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    double* Bw = nullptr;
    DevStatus* ds = nullptr;
    unsigned* cmax = nullptr;
    if (e == cudaSuccess) e = cudaMallocAsync(&Bw, sizeof(double) * (size_t)m * C, st);
    if (e == cudaSuccess) e = cudaMallocAsync(&ds, sizeof(DevStatus), st);
    if (e == cudaSuccess) e = cudaMallocAsync(&cmax, 64 * sizeof(unsigned), st);
    if (e != cudaSuccess) {
        if (Bw) cudaFreeAsync(Bw, st);
        if (ds) cudaFreeAsync(ds, st);
        return fail(nullptr, e == cudaErrorMemoryAllocation ? LS_ERR_OOM : LS_ERR_CUDA, "svd_rows: %s",
                    cudaGetErrorString(e));
    }
    DevStatus h{};
    e = cudaMemcpyAsync(Bw, B, sizeof(double) * (size_t)m * C, cudaMemcpyDeviceToDevice, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(ds, 0, sizeof(DevStatus), st);
    if (e == cudaSuccess) e = cudaMemsetAsync(cmax, 0, 64 * sizeof(unsigned), st);
    const OsjJob J{Bw, C, C, M, m, sig2, ds, tol, cmax};
    if (e == cudaSuccess) e = launch_osj(&J, 1, ms, nsm, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&h, ds, sizeof(DevStatus), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    cudaFreeAsync(Bw, st);
    cudaFreeAsync(ds, st);
    cudaFreeAsync(cmax, st);
    if (e != cudaSuccess) return fail(nullptr, LS_ERR_CUDA, "svd_rows: %s", cudaGetErrorString(e));
    if (sweeps) *sweeps = h.sweeps;
    if (rotations)
        for (int k = 0; k < 64; ++k) rotations[k] = k < h.sweeps ? (int64_t)h.sweep_active[k] : 0;
    if (h.flag == FLAG_TIMEOUT) return fail(nullptr, LS_ERR_TIMEOUT, "svd_rows: a bounded wait timed out");
    if (h.flag == FLAG_NOCONVERGE) return fail(nullptr, LS_ERR_NOCONVERGE, "svd_rows: no convergence in %d sweeps", ms);
    return LS_OK;
}

int lattice_sum_test_fail_alloc(int64_t n) {
    g_fail_after.store(n < 0 ? -1 : (long long)n);
    return LS_OK;
}

int lattice_sum_test_bounded_wait(int32_t absent, int64_t spin_limit, void* stream) {
    if ((absent != 0 && absent != 1) || spin_limit < 1) return fail(nullptr, LS_ERR_ARG, "test_bounded_wait: bad arguments");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    DevStatus* ds = nullptr;
    cudaError_t e = cudaMallocAsync(&ds, sizeof(DevStatus), st);
    if (e != cudaSuccess) return fail(nullptr, LS_ERR_OOM, "test_bounded_wait: %s", cudaGetErrorString(e));
    DevStatus h{};
    e = cudaMemsetAsync(ds, 0, sizeof(DevStatus), st);
    if (e == cudaSuccess) e = launch_wait_probe(ds, absent, spin_limit, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&h, ds, sizeof(DevStatus), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    cudaFreeAsync(ds, st);
    if (e != cudaSuccess) return fail(nullptr, LS_ERR_CUDA, "test_bounded_wait: %s", cudaGetErrorString(e));
    if (h.flag == FLAG_TIMEOUT) return fail(nullptr, LS_ERR_TIMEOUT, "test_bounded_wait: the wait ran out after %lld polls", (long long)spin_limit);
    return LS_OK;
}

int lattice_sum_gemm_nt_mixed(const double* A, const double* B, int64_t M, int64_t N, int64_t K, void* D,
                              int32_t out_dtype, int32_t tile_n, void* stream) {
    if (!A || !B || !D || M < 0 || N < 0 || K < 1 || M > INT32_MAX || N > INT32_MAX ||
        (out_dtype != LS_OUT_F64 && out_dtype != LS_OUT_F32))
        return fail(nullptr, LS_ERR_ARG, "gemm_nt_mixed: bad arguments");
    std::string err;
    DtOpts o;
    o.tile_n = tile_n;
    int rc = dt_gemm_nt(A, B, M, N, K, D, out_dtype == LS_OUT_F32, o, static_cast<cudaStream_t>(stream), &err);
    if (rc != LS_OK) return fail(nullptr, rc, "gemm_nt_mixed: %s", err.c_str());
    return LS_OK;
}

}  // extern "C"

namespace {

int eval_impl(ls_ctx* ctx, const int64_t* z_index, int32_t nslab, void* out_dev, int32_t out_dtype,
              std::string* tune_report) {
    if (!ctx) return fail(nullptr, LS_ERR_ARG, "eval_slab: NULL context");
    if (!ctx->reduced) return fail(ctx, LS_ERR_STATE, "eval_slab: call rhosvd_reduce first");
    if (nslab < 0 || (nslab > 0 && (!z_index || !out_dev))) return fail(ctx, LS_ERR_ARG, "eval_slab: bad arguments");
    if (out_dtype != LS_OUT_F64 && out_dtype != LS_OUT_F32) return fail(ctx, LS_ERR_ARG, "eval_slab: bad out_dtype");
    if (nslab == 0) return LS_OK;
    const int64_t N = ctx->p.N;
    std::vector<int32_t> z(nslab);
    for (int s = 0; s < nslab; ++s) {
        if (z_index[s] < 0 || z_index[s] >= N) return fail(ctx, LS_ERR_ARG, "eval_slab: z index %lld out of range", (long long)z_index[s]);
        z[s] = (int32_t)z_index[s];
    }
    cudaStream_t st = ctx->st;
    int32_t* d_z = nullptr;
    CU(dalloc(ctx, &d_z, nslab));
    CU(upload_h2d(d_z, z.data(), nslab * sizeof(int32_t), st));
    count_h2d((int64_t)(nslab * sizeof(int32_t)));
    const double* Zc[3] = {ctx->d_Z[0], ctx->d_Z[1], ctx->d_Z[2]};
    Scope sc_eval("eval", st);
    if (ctx->p.precision == LS_MIXED) {
        // the three products on the tensor cores (two exact digits + two tails)
        int rc = dt_eval(&ctx->eval_cache, Zc, ctx->r, ctx->d_B, N, d_z, nslab, out_dev, out_dtype == LS_OUT_F32,
                         DtOpts{}, st, &ctx->err, tune_report);
        dfree(ctx, d_z);
        return rc;
    }
    // FP64: slabs in chunks that bound the work buffer to ~256 MB
    const int64_t per = (int64_t)ctx->r[0] * ctx->r[1] + (int64_t)ctx->r[0] * N;
    const int chunk = (int)std::max<int64_t>(1, std::min<int64_t>(nslab, (int64_t)(32 << 20) / std::max<int64_t>(per, 1)));
    double* work = nullptr;
    CU(dalloc(ctx, &work, per * chunk));
    const size_t esz = out_dtype == LS_OUT_F32 ? 4 : 8;
    for (int s0 = 0; s0 < nslab; s0 += chunk) {
        const int ns = std::min(chunk, nslab - s0);
        char* o = static_cast<char*>(out_dev) + (size_t)s0 * N * N * esz;
        CU(launch_eval_f64(Zc, ctx->r, ctx->d_B, N, d_z + s0, ns, work, o, out_dtype == LS_OUT_F32, st));
    }
    dfree(ctx, work);
    dfree(ctx, d_z);
    return LS_OK;
}

}  // namespace

extern "C" {

int lattice_sum_eval_slab(ls_ctx* ctx, const int64_t* z_index, int32_t nslab, void* out_dev, int32_t out_dtype) {
    ls::NvtxRange nvtx_("lattice_sum_eval_slab");
    return eval_impl(ctx, z_index, nslab, out_dev, out_dtype, nullptr);
}

int lattice_sum_tune_eval(ls_ctx* ctx, const int64_t* z_index, int32_t nslab, void* out_dev, int32_t out_dtype,
                          char* report, int64_t cap) {
    ls::NvtxRange nvtx_("lattice_sum_tune_eval");
    if (!ctx) return fail(nullptr, LS_ERR_ARG, "tune_eval: NULL context");
    if (ctx->p.precision != LS_MIXED) return fail(ctx, LS_ERR_ARG, "tune_eval: the FP64 path has no tile widths to tune");
    if (cap < 0 || (cap > 0 && !report)) return fail(ctx, LS_ERR_ARG, "tune_eval: bad report buffer");
    std::string rep;
    const int rc = eval_impl(ctx, z_index, nslab, out_dev, out_dtype, &rep);
    if (rc != LS_OK) return rc;
    const std::string js = "{" + rep + "}";
    if (report && cap > 0) {
        if ((int64_t)js.size() + 1 > cap) return fail(ctx, LS_ERR_ARG, "tune_eval: report buffer of %lld bytes, need %lld",
                                                      (long long)cap, (long long)js.size() + 1);
        memcpy(report, js.c_str(), js.size() + 1);
    }
    return LS_OK;
}

int lattice_sum_als_refine(ls_ctx* ctx, int32_t sweeps, double* history, ls_tucker_info* info) {
    ls::NvtxRange nvtx_("lattice_sum_als_refine");
    if (!ctx) return fail(nullptr, LS_ERR_ARG, "als_refine: NULL context");
    if (!ctx->reduced) return fail(ctx, LS_ERR_STATE, "als_refine: call rhosvd_reduce first");
    if (sweeps < 0 || sweeps > 100) return fail(ctx, LS_ERR_ARG, "als_refine: sweeps out of range [0, 100]");
    for (int l = 0; l < 3; ++l)
        if (!ctx->d_Q[l])
            return fail(ctx, LS_ERR_STATE, "als_refine: needs the range bases of the non-squaring route "
                                           "(an LS_FP64 context, or LS_FLAG_SVD_ONESIDED)");
    cudaStream_t st = ctx->st;
    const int64_t N = ctx->p.N;
    const int64_t T = (int64_t)ctx->xi.size();
    const double u = 1.1102230246251565e-16;
    const int32_t* r = ctx->r;
    int64_t C[3];
    for (int l = 0; l < 3; ++l) C[l] = ctx->mode[l].C;
    const int* m = ctx->mq;
    Scope sc_all("als", st);
    DevStatus* ds = nullptr;   // [0]: the tensor-core products' flag, [1]: the one-sided Jacobi
    double* scal = nullptr;
    CU(dalloc(ctx, &ds, 2));
    CU(dalloc(ctx, &scal, 1));
    CU(cudaMemsetAsync(ds, 0, 2 * sizeof(DevStatus), st));
    int* flag = &ds[0].flag;
    // history[0]: ||core|| of the start
    double h0 = 0.0;
    CU(launch_sum_squares(ctx->d_B, (int64_t)r[0] * r[1] * r[2], scal, st));
    CU(cudaMemcpyAsync(&h0, scal, sizeof(double), cudaMemcpyDeviceToHost, st));
    CU(cudaStreamSynchronize(st));
    if (history) history[0] = sqrt(h0);
    // K_l = Q_l A_l^T (m_l x C_l): the unit canonical vectors in the range bases
    double* K[3];
    double* Pt[3];
    {
        X64Mat xs[3], ys[3];
        int64_t ld[3];
        for (int l = 0; l < 3; ++l) {
            CU(dalloc(ctx, &K[l], (int64_t)m[l] * C[l]));
            CU(dalloc(ctx, &Pt[l], C[l] * r[l]));
            xs[l] = X64Mat{ctx->d_Q[l], m[l], N, N, 1, nullptr};
            ys[l] = X64Mat{ctx->mode[l].d_cols, C[l], N, N, 1, nullptr};
            ld[l] = C[l];
            CU(launch_transpose(ctx->d_P[l], r[l], C[l], Pt[l], st));
        }
        std::string err;
        int rc = x64_nt(3, xs, ys, K, ld, flag, st, &err);
        if (rc != LS_OK) return fail(ctx, rc, "als_refine: %s", err.c_str());
    }
    // per mode: the terms grouped by their mode-l vector, with the columns reordered (l, m, n)
    int32_t *d_tc[3], *d_perm[3], *d_off[3];
    for (int l = 0; l < 3; ++l) {
        const int mm = l == 0 ? 1 : 0, nn = l == 2 ? 1 : 2;
        std::vector<int32_t> tc(3 * T), off(C[l] + 1, 0), perm(T);
        for (int64_t t = 0; t < T; ++t) {
            tc[3 * t] = ctx->tcol[3 * t + l];
            tc[3 * t + 1] = ctx->tcol[3 * t + mm];
            tc[3 * t + 2] = ctx->tcol[3 * t + nn];
            off[tc[3 * t] + 1] += 1;
        }
        for (int64_t c = 0; c < C[l]; ++c) off[c + 1] += off[c];
        std::vector<int32_t> pos(off.begin(), off.end() - 1);
        for (int64_t t = 0; t < T; ++t) perm[pos[tc[3 * t]]++] = (int32_t)t;
        CU(dalloc(ctx, &d_tc[l], 3 * T));
        CU(dalloc(ctx, &d_perm[l], T));
        CU(dalloc(ctx, &d_off[l], C[l] + 1));
        CU(upload_h2d(d_tc[l], tc.data(), 3 * T * sizeof(int32_t), st));
        CU(upload_h2d(d_perm[l], perm.data(), T * sizeof(int32_t), st));
        CU(upload_h2d(d_off[l], off.data(), (C[l] + 1) * sizeof(int32_t), st));
        count_h2d((3 * T + T + C[l] + 1) * sizeof(int32_t));
    }
    for (int s = 1; s <= sweeps; ++s) {
        double kept = 0.0;
        for (int l = 0; l < 3; ++l) {
            // Thm A.1(b): Y_l <- the r_l leading left singular vectors of B_l = A_l^T W_l,
            // W_l[c] = sum_{t: c_l(t) = c} xin_t P_m[:, c_m(t)] (x) P_n[:, c_n(t)]; within the range
            // basis, B_l = Q_l^T S_l with S_l = K_l W_l (m_l x r_m r_n)
            const int mm = l == 0 ? 1 : 0, nn = l == 2 ? 1 : 2;
            const int64_t w = (int64_t)r[mm] * r[nn];
            double *W = nullptr, *S = nullptr, *M = nullptr, *sig2 = nullptr, *lam = nullptr, *isl = nullptr,
                   *sel = nullptr, *Ms = nullptr;
            int32_t* pm = nullptr;
            unsigned* cmax = nullptr;
            CU(dalloc(ctx, &W, C[l] * w));
            CU(dalloc(ctx, &S, (int64_t)m[l] * w));
            CU(dalloc(ctx, &M, (int64_t)m[l] * m[l]));
            CU(dalloc(ctx, &sig2, m[l]));
            CU(dalloc(ctx, &lam, m[l]));
            CU(dalloc(ctx, &isl, m[l]));
            CU(dalloc(ctx, &pm, m[l]));
            CU(dalloc(ctx, &sel, 3));
            CU(dalloc(ctx, &cmax, 64));
            CU(dalloc(ctx, &Ms, (int64_t)r[l] * m[l]));
            CU(cudaMemsetAsync(cmax, 0, 64 * sizeof(unsigned), st));
            CU(cudaMemsetAsync(&ds[1], 0, sizeof(DevStatus), st));
            CU(launch_core_step1_f64(Pt[mm], Pt[nn], r[mm], r[nn], d_tc[l], ctx->d_xin, d_perm[l], d_off[l], 0,
                                     (int)C[l], W, st));
            std::string err;
            X64Mat xs[1] = {X64Mat{K[l], m[l], C[l], C[l], 1, nullptr}};   // K_l (m x C)
            X64Mat ys[1] = {X64Mat{W, w, C[l], 1, w, nullptr}};            // W_l^T (r_m r_n x C)
            double* D[1] = {S};
            int64_t ld[1] = {w};
            int rc = x64_nt(1, xs, ys, D, ld, flag, st, &err);
            if (rc != LS_OK) return fail(ctx, rc, "als_refine: %s", err.c_str());
            const OsjJob J{S, w, (int)w, M, m[l], sig2, &ds[1], 8.0 * u * sqrt((double)w), cmax};
            CU(launch_osj(&J, 1, 60, ctx->num_sms, st));
            SortSelectJob sj{sig2, m[l], r[l], nullptr, pm, lam, isl, sel};
            sj.dstride = 1;
            sj.resolution = 0.0;
            CU(launch_sort_select(1, &sj, 1e-300, 0.0, st));
            CU(launch_gather_rows(M, m[l], pm, r[l], nullptr, Ms, st));
            xs[0] = X64Mat{Ms, r[l], m[l], m[l], 1, nullptr};                // M_r (r x m)
            ys[0] = X64Mat{ctx->d_Q[l], N, m[l], 1, N, nullptr};             // Q^T (N x m)
            D[0] = ctx->d_Z[l];
            ld[0] = N;
            rc = x64_nt(1, xs, ys, D, ld, flag, st, &err);                   // Y_l = M_r Q_l
            const double* Zc[1] = {ctx->d_Z[l]};
            const double* ac[1] = {ctx->mode[l].d_cols};
            const int rl[1] = {r[l]};
            const int64_t Cl[1] = {C[l]};
            double* Pl[1] = {ctx->d_P[l]};
            if (rc == LS_OK) rc = x64_project(1, Zc, rl, ac, Cl, N, Pl, flag, st, &err);   // P_l = Y_l A_l^T
            if (rc != LS_OK) return fail(ctx, rc, "als_refine: %s", err.c_str());
            CU(launch_transpose(ctx->d_P[l], r[l], C[l], Pt[l], st));
            double hsel[3];
            DevStatus hd[2];
            CU(cudaMemcpyAsync(hsel, sel, sizeof hsel, cudaMemcpyDeviceToHost, st));
            CU(cudaMemcpyAsync(hd, ds, sizeof hd, cudaMemcpyDeviceToHost, st));
            count_d2h(sizeof hsel + sizeof hd);
            CU(cudaStreamSynchronize(st));
            if (hd[0].flag == FLAG_TIMEOUT || hd[1].flag == FLAG_TIMEOUT)
                return fail(ctx, LS_ERR_TIMEOUT, "als_refine: a bounded wait timed out");
            if (hd[1].flag == FLAG_NOCONVERGE)
                return fail(ctx, LS_ERR_NOCONVERGE, "als_refine: one-sided Jacobi did not converge (mode %d)", l);
            kept = std::max(hsel[2] - hsel[1], 0.0);   // ||Y_l^T B_l||^2 = the kept singular values squared
            for (void* q : {(void*)W, (void*)S, (void*)M, (void*)sig2, (void*)lam, (void*)isl, (void*)pm, (void*)sel,
                            (void*)cmax, (void*)Ms})
                dfree(ctx, q);
        }
        if (history) history[s] = sqrt(kept);
    }
    for (int l = 0; l < 3; ++l)
        for (void* q : {(void*)K[l], (void*)Pt[l], (void*)d_tc[l], (void*)d_perm[l], (void*)d_off[l]}) dfree(ctx, q);
    dfree(ctx, scal);
    dfree(ctx, ds);
    // Thm A.1(c): the core of the refined bases; the evaluation operands are rebuilt on demand
    dt_eval_free(ctx->eval_cache);
    ctx->eval_cache = nullptr;
    dfree(ctx, ctx->d_B);
    ctx->d_B = nullptr;
    ctx->reduced = false;
    RedState rf;
    rf.ctx = ctx;
    rf.T = T;
    rf.floor_noise = 0.0;
    CU(dalloc(ctx, &rf.d_st, 10));
    CU(cudaMemsetAsync(rf.d_st, 0, 10 * sizeof(DevStatus), st));
    CU(dalloc(ctx, &rf.d_sel, 9));
    for (int l = 0; l < 3; ++l) rf.sel[l][0] = r[l];
    ls_tucker_info tmp;
    const int rc = red_project_core_noproj(rf, &tmp);
    if (rc == LS_OK && info) {
        // the reduction's report still holds: ALS does not increase the error (Thm A.1(b)), so
        // the RHOSVD bound bounds the refined tensor too; sweeps = the ALS sweeps
        *info = ctx->last_info;
        for (int l = 0; l < 3; ++l) info->sweeps[l] = sweeps;
    }
    return rc;
}

int lattice_sum_galerkin(ls_ctx* ctx, const double* const* basis, int32_t nb, double* V) {
    ls::NvtxRange nvtx_("lattice_sum_galerkin");
    if (!ctx) return fail(nullptr, LS_ERR_ARG, "galerkin: NULL context");
    if (!ctx->reduced) return fail(ctx, LS_ERR_STATE, "galerkin: call rhosvd_reduce first");
    if (!basis || !basis[0] || !basis[1] || !basis[2] || nb < 1 || nb > 65535 || !V)
        return fail(ctx, LS_ERR_ARG, "galerkin: bad arguments");
    cudaStream_t st = ctx->st;
    const int64_t N = ctx->p.N;
    const int32_t* r = ctx->r;
    const int64_t npairs = (int64_t)nb * (nb + 1) / 2;
    // pairs in chunks: the Hadamard rows (np x N), the projections and Y (np x r0 r1) within ~1 GB
    const int64_t per = std::max<int64_t>(N, (int64_t)r[0] * r[1]) * 8 * 3;
    const int64_t chunk = std::max<int64_t>(1, std::min<int64_t>(npairs, ((int64_t)1 << 30) / std::max<int64_t>(per, 1)));
    std::vector<int2> hp;
    hp.reserve(npairs);
    for (int k = 0; k < nb; ++k)
        for (int m = k; m < nb; ++m) hp.push_back(make_int2(k, m));
    int2* d_pairs = nullptr;
    double *H = nullptr, *M[3] = {nullptr, nullptr, nullptr}, *Y = nullptr;
    int* flag = nullptr;
    CU(dalloc(ctx, &d_pairs, npairs));
    CU(dalloc(ctx, &H, 3 * chunk * N));
    for (int l = 0; l < 3; ++l) CU(dalloc(ctx, &M[l], chunk * r[l]));
    CU(dalloc(ctx, &Y, chunk * r[0] * r[1]));
    CU(dalloc(ctx, &flag, 1));
    CU(cudaMemsetAsync(flag, 0, sizeof(int), st));
    CU(upload_h2d(d_pairs, hp.data(), npairs * sizeof(int2), st));
    count_h2d(npairs * sizeof(int2));
    Scope sc("galerkin", st);
    for (int64_t p0 = 0; p0 < npairs; p0 += chunk) {
        const int np = (int)std::min<int64_t>(chunk, npairs - p0);
        X64Mat xs[3], ys[3];
        double* D[3];
        int64_t ld[3];
        for (int l = 0; l < 3; ++l) {
            CU(launch_hadamard_pairs(basis[l], N, d_pairs + p0, np, H + l * chunk * N, st));
            xs[l] = X64Mat{H + l * chunk * N, np, N, N, 1, nullptr};   // Hadamard rows
            ys[l] = X64Mat{ctx->d_Z[l], r[l], N, N, 1, nullptr};      // Z_l (r_l x N)
            D[l] = M[l];
            ld[l] = r[l];
        }
        std::string err;
        int rc = x64_nt(3, xs, ys, D, ld, flag, st, &err);                         // M_l = H_l Z_l^T
        xs[0] = X64Mat{M[2], np, r[2], r[2], 1, nullptr};                          // M2 (np x r2)
        ys[0] = X64Mat{ctx->d_B, (int64_t)r[0] * r[1], r[2], r[2], 1, nullptr};    // core rows (a,b)
        D[0] = Y;
        ld[0] = (int64_t)r[0] * r[1];
        if (rc == LS_OK) rc = x64_nt(1, xs, ys, D, ld, flag, st, &err);            // Y = M2 B^T
        if (rc != LS_OK) return fail(ctx, rc, "galerkin: %s", err.c_str());
        CU(launch_galerkin_contract(Y, M[0], M[1], r[0], r[1], d_pairs + p0, np, nb, V, st));
    }
    int hflag = 0;
    CU(cudaMemcpyAsync(&hflag, flag, sizeof(int), cudaMemcpyDeviceToHost, st));
    count_d2h(sizeof(int));
    CU(cudaStreamSynchronize(st));
    for (void* q : {(void*)d_pairs, (void*)H, (void*)M[0], (void*)M[1], (void*)M[2], (void*)Y, (void*)flag}) dfree(ctx, q);
    if (hflag == FLAG_TIMEOUT) return fail(ctx, LS_ERR_TIMEOUT, "galerkin: a tensor-core product's bounded wait timed out");
    return LS_OK;
}

int lattice_sum_get_factors(ls_ctx* ctx, const double** Z, const double** core, int32_t* ranks) {
    if (!ctx) return fail(nullptr, LS_ERR_ARG, "get_factors: NULL context");
    if (!ctx->reduced) return fail(ctx, LS_ERR_STATE, "get_factors: call rhosvd_reduce first");
    if (!Z || !core || !ranks) return fail(ctx, LS_ERR_ARG, "get_factors: NULL output");
    for (int l = 0; l < 3; ++l) {
        Z[l] = ctx->d_Z[l];
        ranks[l] = ctx->r[l];
    }
    *core = ctx->d_B;
    return LS_OK;
}

int lattice_sum_read(ls_ctx* ctx, int32_t what, int32_t mode, void* dst, int64_t bytes, int64_t* needed_bytes) {
    if (!ctx) return fail(nullptr, LS_ERR_ARG, "read: NULL context");
    if (mode < 0 || mode > 2) return fail(ctx, LS_ERR_ARG, "read: mode %d", mode);
    const int64_t N = ctx->p.N;
    const ModeCols& mc = ctx->mode[mode];
    const void* src = nullptr;
    int64_t need = 0;
    std::vector<int32_t> tmp_i;
    const int64_t T = (int64_t)ctx->xi.size();
    switch (what) {
        case LS_READ_GENVEC: src = ctx->d_g; need = (int64_t)ctx->p.R * 2 * N * 8; break;
        case LS_READ_COLUMNS: src = mc.d_cols; need = mc.C * N * 8; break;
        case LS_READ_NORMS: src = ctx->d_norms[mode]; need = mc.C * 8; break;
        case LS_READ_TERMS: need = 3 * T * 4; break;
        case LS_READ_XI: src = ctx->reduced ? (const void*)ctx->d_xin : nullptr; need = T * 8; break;
        case LS_READ_SIGMA: src = ctx->d_sigma[mode]; need = mc.C * 8; break;
        case LS_READ_BASIS: src = ctx->d_Z[mode]; need = (int64_t)ctx->r[mode] * N * 8; break;
        case LS_READ_PROJ: src = ctx->d_P[mode]; need = (int64_t)ctx->r[mode] * mc.C * 8; break;
        case LS_READ_CORE: src = ctx->d_B; need = (int64_t)ctx->r[0] * ctx->r[1] * ctx->r[2] * 8; break;
        case LS_READ_TUCKER_REF: src = ctx->d_t; need = (int64_t)ctx->r_ref * 2 * N * 8; break;
        default: return fail(ctx, LS_ERR_ARG, "read: unknown item %d", what);
    }
    if (needed_bytes) *needed_bytes = need;
    if (!dst) return LS_OK;
    if (bytes < need) return fail(ctx, LS_ERR_ARG, "read: buffer of %lld bytes, need %lld", (long long)bytes, (long long)need);
    if (what == LS_READ_TERMS) {
        memcpy(dst, ctx->tcol.data(), need);
        return LS_OK;
    }
    if (what == LS_READ_XI && !ctx->reduced) {
        memcpy(dst, ctx->xi.data(), need);
        return LS_OK;
    }
    if (!src) return fail(ctx, LS_ERR_STATE, "read: item %d not computed yet", what);
    CU(cudaMemcpyAsync(dst, src, need, cudaMemcpyDeviceToHost, ctx->st));
    count_d2h((int64_t)(need));
    CU(cudaStreamSynchronize(ctx->st));
    return LS_OK;
}

int lattice_sum_profile(int32_t enable) {
    Tracer& t = tracer();
    std::lock_guard<std::mutex> g(t.mu);
    if (enable) {
        for (auto& r : t.recs) {
            t.pool.push_back(r.a);
            t.pool.push_back(r.b);
        }
        t.recs.clear();
        t.kernels = 0;
        t.h2d = 0;
        t.d2h = 0;
    }
    t.on = enable != 0;
    return LS_OK;
}

int lattice_sum_profile_report(char* buf, int64_t cap, int64_t* needed_bytes) {
    Tracer& t = tracer();
    std::lock_guard<std::mutex> g(t.mu);
    struct Agg { long long launches = 0, kernels = 0; double ms = 0.0; };
    std::map<std::string, Agg> agg;
    for (auto& r : t.recs) {
        if (cudaEventSynchronize(r.b) != cudaSuccess) return fail(nullptr, LS_ERR_CUDA, "profile_report: event wait failed");
        float ms = 0.f;
        cudaEventElapsedTime(&ms, r.a, r.b);
        Agg& a = agg[r.name];
        a.launches += 1;
        a.kernels += r.kernels;
        a.ms += ms;
    }
    std::string js = "{\"steps\": {";
    bool first = true;
    char tmp[256];
    for (auto& kv : agg) {
        snprintf(tmp, sizeof tmp, "%s\"%s\": {\"launches\": %lld, \"kernels\": %lld, \"ms\": %.6f}", first ? "" : ", ",
                 kv.first.c_str(), kv.second.launches, kv.second.kernels, kv.second.ms);
        js += tmp;
        first = false;
    }
    snprintf(tmp, sizeof tmp, "}, \"kernel_launches\": %lld, \"h2d_bytes\": %lld, \"d2h_bytes\": %lld}",
             (long long)t.kernels.load(), (long long)t.h2d.load(), (long long)t.d2h.load());
    js += tmp;
    if (needed_bytes) *needed_bytes = (int64_t)js.size() + 1;
    if (!buf) return LS_OK;
    if (cap < (int64_t)js.size() + 1) return fail(nullptr, LS_ERR_ARG, "profile_report: buffer too small");
    memcpy(buf, js.c_str(), js.size() + 1);
    return LS_OK;
}

void lattice_sum_destroy(ls_ctx* ctx) {
    if (!ctx) return;
    dt_eval_free(ctx->eval_cache);
    for (void* p : ctx->allocs) cudaFreeAsync(p, ctx->st);
    ctx->allocs.clear();
    delete ctx;
}

int lattice_sum_cache_clear(void) {
    std::lock_guard<std::mutex> g(ls::g_genvec_mu);
    std::deque<ls::GenvecEntry>& cache = ls::genvec_cache();
    const int n = (int)cache.size();
    int dev0 = -1;
    cudaGetDevice(&dev0);
    bool ok = true;
    for (const ls::GenvecEntry& c : cache) {
        ok = ok && cudaSetDevice(c.key.dev) == cudaSuccess && cudaFree(c.d) == cudaSuccess;
    }
    cache.clear();
    if (dev0 >= 0) cudaSetDevice(dev0);
    if (!ok) return fail(nullptr, LS_ERR_CUDA, "cache_clear: cudaFree failed");
    return n;
}

const char* lattice_sum_last_error(const ls_ctx* ctx) {
    return ctx ? ctx->err.c_str() : g_create_error.c_str();
}

}  // extern "C"
