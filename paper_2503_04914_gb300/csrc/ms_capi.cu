// C entry points of libms.so (declared in include/ms.h): argument validation,
// handle lifetime, host<->device staging, and the permutation kernels between
// the caller's input order and the library's cell-sorted order.
#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstring>
#include <map>
#include <mutex>
#include <tuple>
#include <vector>

#include "ms_internal.cuh"

namespace {
thread_local char g_err[1024] = "";

__global__ void k_gather(const double* in, double* out, const int32_t* perm, int64_t N, int nrhs, int col) {
    const int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (s < N) out[s] = in[(int64_t)perm[s] * nrhs + col];
}
__global__ void k_scatter_in(const double* in, double* out, const int32_t* perm, int64_t N, int nrhs, int col) {
    const int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (s < N) out[(int64_t)perm[s] * nrhs + col] = in[s];
}
__global__ void k_finite(const double* a, int64_t n, int* bad) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < n && !isfinite(a[i])) atomicExch(bad, 1);
}
inline unsigned nblk(int64_t n, int bs) { return (unsigned)std::max<int64_t>(1, (n + bs - 1) / bs); }

// Device buffer freed at scope exit (host staging of the plain entry points).
struct DevBuf {
    void* p = nullptr;
    ~DevBuf() { if (p) ms_pool_free(p); }
};
ms_status dev_alloc(DevBuf& b, size_t bytes) { return ms_pool_alloc(&b.p, bytes); }

ms_status check_finite(const double* a_dev, int64_t n, cudaStream_t st, const char* what) {
    if (n == 0) return MS_OK;
    DevBuf flag;
    MS_TRY(dev_alloc(flag, sizeof(int)));
    MS_CUDA(cudaMemsetAsync(flag.p, 0, sizeof(int), st));
    k_finite<<<nblk(n, 256), 256, 0, st>>>(a_dev, n, (int*)flag.p); ms_count_launch();
    int bad = 0;
    MS_CUDA(cudaMemcpyAsync(&bad, flag.p, sizeof(int), cudaMemcpyDeviceToHost, st));
    MS_CUDA(cudaStreamSynchronize(st));
    if (bad) {
        ms_set_error(MS_ERR_NUMERIC, "%s contains non-finite values", what);
        return MS_ERR_NUMERIC;
    }
    return MS_OK;
}

ms_status validate_and_init(int d, int L, const int64_t* n_per_level, const double* h_per_level,
                            const ms_opts* opts, ms_hierarchy* h) {
    if (d < 1 || d > 3) { ms_set_error(MS_ERR_ARG, "d must be 1, 2 or 3 (got %d)", d); return MS_ERR_ARG; }
    if (L < 1 || L > MS_MAX_LEVELS) { ms_set_error(MS_ERR_ARG, "L must be in 1..%d (got %d)", MS_MAX_LEVELS, L); return MS_ERR_ARG; }
    if (!n_per_level || !h_per_level) { ms_set_error(MS_ERR_ARG, "n_per_level and h_per_level must not be NULL"); return MS_ERR_ARG; }
    ms_opts o;
    ms_default_opts(&o);
    if (opts) o = *opts;
    if (!(o.nu > 0.0) || !std::isfinite(o.nu)) { ms_set_error(MS_ERR_ARG, "nu must be positive (got %g)", o.nu); return MS_ERR_ARG; }
    WendlandPoly w;
    if (!wendland_poly(o.wendland_d, o.wendland_k, &w)) {
        ms_set_error(MS_ERR_ARG, "unsupported Wendland function phi_{%d,%d} (d in 1..3, k in 0..3)", o.wendland_d, o.wendland_k);
        return MS_ERR_ARG;
    }
    if (o.wendland_d < d) {
        ms_set_error(MS_ERR_ARG, "phi_{%d,%d} is not positive definite on R^%d (need wendland_d >= d)", o.wendland_d, o.wendland_k, d);
        return MS_ERR_ARG;
    }
    if (o.precision != MS_PREC_FP64 && o.precision != MS_PREC_MIXED) { ms_set_error(MS_ERR_ARG, "unknown precision %d", o.precision); return MS_ERR_ARG; }
    if (o.op < MS_OP_CSR || o.op > MS_OP_AUTO) { ms_set_error(MS_ERR_ARG, "unknown operator %d", o.op); return MS_ERR_ARG; }
    if (o.precond < MS_PRECOND_NONE || o.precond > MS_PRECOND_EXACT) { ms_set_error(MS_ERR_ARG, "unknown preconditioner %d", o.precond); return MS_ERR_ARG; }
    if (o.cell_split < 0 || o.cell_split > 4) { ms_set_error(MS_ERR_ARG, "cell_split must be 0..4"); return MS_ERR_ARG; }
    if (o.threads_per_row < 0 || o.threads_per_row > 32 || (o.threads_per_row & (o.threads_per_row - 1))) {
        ms_set_error(MS_ERR_ARG, "threads_per_row must be 0 or a power of two <= 32"); return MS_ERR_ARG;
    }
    if (o.autotune < 0 || o.autotune > 1) {
        ms_set_error(MS_ERR_ARG, "autotune must be 0 or 1"); return MS_ERR_ARG;
    }
    if (o.solve_ctas_per_sm < 0 || o.solve_ctas_per_sm > 2) {
        ms_set_error(MS_ERR_ARG, "solve_ctas_per_sm must be 0, 1 or 2"); return MS_ERR_ARG;
    }
    if (o.jacobi_sweeps < -1) {
        ms_set_error(MS_ERR_ARG, "jacobi_sweeps must be >= -1 (got %d)", o.jacobi_sweeps); return MS_ERR_ARG;
    }
    if (o.lower_op != MS_OP_CSR && o.lower_op != MS_OP_MATRIX_FREE) {
        ms_set_error(MS_ERR_ARG, "lower_op must be MS_OP_CSR or MS_OP_MATRIX_FREE (got %d)", o.lower_op); return MS_ERR_ARG;
    }
    if (o.lower_op == MS_OP_MATRIX_FREE && o.precision != MS_PREC_MIXED) {
        ms_set_error(MS_ERR_ARG, "lower_op = MS_OP_MATRIX_FREE needs precision = MS_PREC_MIXED (its double-float entries "
                     "use the MIXED build's offsets)");
        return MS_ERR_ARG;
    }
    h->opts = o;
    h->d = d;
    h->L = L;
    HierView& v = h->view;
    v = HierView{};
    v.d = d;
    v.L = L;
    v.w = w;
    int64_t N = 0;
    for (int l = 0; l < L; ++l) {
        if (n_per_level[l] < 1) { ms_set_error(MS_ERR_ARG, "level %d has %lld points (need >= 1)", l + 1, (long long)n_per_level[l]); return MS_ERR_ARG; }
        const double hl = h_per_level[l];
        if (!(hl > 0.0) || !std::isfinite(hl)) { ms_set_error(MS_ERR_ARG, "h of level %d must be positive (got %g)", l + 1, hl); return MS_ERR_ARG; }
        v.off[l] = N;
        N += n_per_level[l];
        v.delta[l] = o.nu * hl;
        v.dscale[l] = std::pow(v.delta[l], -(double)d);
        v.inv_delta[l] = 1.0 / v.delta[l];
    }
    v.off[L] = N;
    if (N >= (int64_t(1) << 31) - 1) { ms_set_error(MS_ERR_ARG, "too many points (%lld, limit 2^31-2)", (long long)N); return MS_ERR_ARG; }
    v.N = N;
    h->N = N;
    return MS_OK;
}

ms_status build_one(int d, int L, const int64_t* n_per_level, const double* pts_dev, const double* h_per_level,
                    const ms_opts* opts, cudaStream_t st, ms_hierarchy** out) {
    ms_hierarchy* h = new ms_hierarchy();
    ms_status s = validate_and_init(d, L, n_per_level, h_per_level, opts, h);
    if (s == MS_OK) {
        cudaError_t e = cudaGetDevice(&h->device);
        if (e == cudaSuccess) e = cudaEventCreate(&h->ev0);
        if (e == cudaSuccess) e = cudaEventCreate(&h->ev1);
        if (e != cudaSuccess) s = ms_cuda_error(e, "device / event set-up", __FILE__, __LINE__);
    }
    if (s == MS_OK) s = ms_build_impl(h, pts_dev, st);
    if (s != MS_OK) {
        ms_destroy(h);
        return s;
    }
    *out = h;
    return MS_OK;
}

// Device time of one application of the geometry-dependent operators the fit will use
// (the matrix-free FP32 A and / or the matrix-free lower blocks), 0 if it uses none.
ms_status geometry_ms(ms_hierarchy* h, cudaStream_t st, float* out) {
    *out = 0.f;
    const bool mfA = h->opts.precision == MS_PREC_MIXED && h->opts.op == MS_OP_MATRIX_FREE;
    const bool mfB = h->opts.precision == MS_PREC_MIXED && h->opts.lower_op == MS_OP_MATRIX_FREE && h->L > 1;
    if (!mfA && !mfB) return MS_OK;
    DevBuf x, y;
    MS_TRY(dev_alloc(x, sizeof(double) * h->N));
    MS_TRY(dev_alloc(y, sizeof(double) * h->N));
    MS_CUDA(cudaMemsetAsync(x.p, 0, sizeof(double) * h->N, st));
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    MS_CUDA(cudaEventCreate(&e0));
    cudaError_t ce = cudaEventCreate(&e1);
    ms_status s = ce == cudaSuccess ? MS_OK : ms_cuda_error(ce, "event", __FILE__, __LINE__);
    for (int rep = 0; rep < 2 && s == MS_OK; ++rep) {  // one untimed application, one timed
        if (rep == 1) cudaEventRecord(e0, st);
        if (mfA && s == MS_OK) s = ms_apply_impl(h, MS_APPLY_AMF32, (const double*)x.p, (double*)y.p, 1, st);
        if (mfB && s == MS_OK) s = ms_apply_impl(h, MS_APPLY_BMFDF, (const double*)x.p, (double*)y.p, 1, st);
        if (rep == 1) cudaEventRecord(e1, st);
    }
    if (s == MS_OK) {
        ce = cudaEventSynchronize(e1);
        if (ce == cudaSuccess) ce = cudaEventElapsedTime(out, e0, e1);
        if (ce != cudaSuccess) s = ms_cuda_error(ce, "geometry timing", __FILE__, __LINE__);
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    return s;
}

// (d, L, log2 N, 16 nu, wendland d, k, precision, op, lower_op) -> cell_split
using SplitKey = std::tuple<int, int, int, int, int, int, int, int, int>;
std::mutex g_split_mu;
std::map<SplitKey, int> g_split_cache;

// With opts.autotune = 1 and cell_split = 0 the first build of a hierarchy shape is made with
// cells of delta and of delta / 2; the one whose build plus one application of the fit's
// matrix-free operators takes less device time is kept (the other is destroyed) and the choice is
// cached per process by shape.  Otherwise one build.
ms_status build_common(int d, int L, const int64_t* n_per_level, const double* pts_dev, const double* h_per_level,
                       const ms_opts* opts, cudaStream_t st, ms_hierarchy** out) {
    if (!opts || !opts->autotune || opts->cell_split != 0)
        return build_one(d, L, n_per_level, pts_dev, h_per_level, opts, st, out);
    int64_t N = 0;
    for (int l = 0; l < L; ++l) N += n_per_level[l];
    int lg = 0;
    while ((int64_t(1) << (lg + 1)) <= N) ++lg;
    const SplitKey key(d, L, lg, (int)std::lround(16.0 * opts->nu), opts->wendland_d, opts->wendland_k,
                       opts->precision, opts->op, opts->lower_op);
    ms_opts o = *opts;
    int cached = 0;
    {
        std::lock_guard<std::mutex> lk(g_split_mu);
        auto it = g_split_cache.find(key);
        if (it != g_split_cache.end()) cached = it->second;
    }
    if (cached) {
        o.cell_split = cached;
        return build_one(d, L, n_per_level, pts_dev, h_per_level, &o, st, out);
    }
    ms_hierarchy* hs[2] = {nullptr, nullptr};
    float t[2] = {0.f, 0.f};
    for (int i = 0; i < 2; ++i) {
        o.cell_split = i + 1;
        ms_status s = build_one(d, L, n_per_level, pts_dev, h_per_level, &o, st, &hs[i]);
        float g = 0.f;
        if (s == MS_OK) s = geometry_ms(hs[i], st, &g);
        if (s != MS_OK) {
            if (hs[0]) ms_destroy(hs[0]);
            if (hs[1]) ms_destroy(hs[1]);
            return s;
        }
        t[i] = (float)hs[i]->build_ms + g;
    }
    const int best = t[1] < t[0] ? 1 : 0;
    ms_destroy(hs[1 - best]);
    {
        std::lock_guard<std::mutex> lk(g_split_mu);
        g_split_cache[key] = best + 1;
    }
    *out = hs[best];
    return MS_OK;
}

}  // namespace

// ---------------------------------------------------------------- internal helpers

void ms_clear_error() { g_err[0] = 0; }

void ms_set_error(ms_status st, const char* fmt, ...) {
    (void)st;
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof(g_err), fmt, ap);
    va_end(ap);
}

ms_status ms_cuda_error(cudaError_t e, const char* what, const char* file, int line) {
    const char* base = strrchr(file, '/');
    ms_set_error(MS_ERR_CUDA, "CUDA error %d (%s) in %s at %s:%d", (int)e, cudaGetErrorString(e), what,
                 base ? base + 1 : file, line);
    return e == cudaErrorMemoryAllocation ? MS_ERR_OOM : MS_ERR_CUDA;
}

// Device memory of the library comes from one memory pool per device that keeps what
// is freed (release threshold: never), so building and destroying handles repeatedly
// reuses memory instead of mapping and unmapping it on every cudaMalloc/cudaFree.
// Allocation and release are ordered on a private stream; an allocation is complete
// (usable from any stream) when ms_pool_alloc returns.  ms_pool_free must only be given
// memory that no pending work uses (callers synchronise first).
namespace {
std::mutex g_pool_mu;
struct DevPool {
    cudaMemPool_t pool = nullptr;
    cudaStream_t stream = nullptr;
};
DevPool g_pools[256];
}  // namespace

static ms_status device_pool(DevPool** out) {
    int dev = 0;
    MS_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 256) {
        ms_set_error(MS_ERR_STATE, "device ordinal %d out of range", dev);
        return MS_ERR_STATE;
    }
    std::lock_guard<std::mutex> lock(g_pool_mu);
    DevPool& dp = g_pools[dev];
    if (!dp.pool) {
        cudaMemPoolProps props{};
        props.allocType = cudaMemAllocationTypePinned;
        props.location.type = cudaMemLocationTypeDevice;
        props.location.id = dev;
        MS_CUDA(cudaMemPoolCreate(&dp.pool, &props));
        uint64_t keep = UINT64_MAX;
        MS_CUDA(cudaMemPoolSetAttribute(dp.pool, cudaMemPoolAttrReleaseThreshold, &keep));
        MS_CUDA(cudaStreamCreateWithFlags(&dp.stream, cudaStreamNonBlocking));
    }
    *out = &dp;
    return MS_OK;
}

ms_status ms_pool_alloc(void** p, size_t bytes) {
    DevPool* dp = nullptr;
    MS_TRY(device_pool(&dp));
    cudaError_t e = cudaMallocFromPoolAsync(p, std::max<size_t>(bytes, 16), dp->pool, dp->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(dp->stream);
    if (e != cudaSuccess) {
        *p = nullptr;
        ms_set_error(MS_ERR_OOM, "device allocation of %zu bytes failed: %s", bytes, cudaGetErrorString(e));
        return MS_ERR_OOM;
    }
    return MS_OK;
}

ms_status ms_tmp_alloc(void** p, size_t bytes, cudaStream_t st) {
    DevPool* dp = nullptr;
    MS_TRY(device_pool(&dp));
    const cudaError_t e = cudaMallocFromPoolAsync(p, std::max<size_t>(bytes, 16), dp->pool, st);
    if (e != cudaSuccess) {
        *p = nullptr;
        ms_set_error(MS_ERR_OOM, "device allocation of %zu bytes failed: %s", bytes, cudaGetErrorString(e));
        return MS_ERR_OOM;
    }
    return MS_OK;
}

void ms_pool_free(void* p) {
    DevPool* dp = nullptr;
    if (!p || device_pool(&dp) != MS_OK) return;
    cudaFreeAsync(p, dp->stream);
}


ms_status ms_alloc(ms_hierarchy* h, void** p, size_t bytes) {
    if (h->nallocs >= (int)(sizeof(h->allocs) / sizeof(h->allocs[0]))) {
        ms_set_error(MS_ERR_STATE, "too many device allocations in one handle");
        return MS_ERR_STATE;
    }
    MS_TRY(ms_pool_alloc(p, bytes));
    h->alloc_bytes[h->nallocs] = bytes;
    h->allocs[h->nallocs++] = *p;
    h->device_bytes += (int64_t)bytes;
    return MS_OK;
}

ms_status ms_realloc(ms_hierarchy* h, void** p, size_t bytes) {
    if (*p) {
        for (int i = 0; i < h->nallocs; ++i) {
            if (h->allocs[i] != *p) continue;
            cudaDeviceSynchronize();  // no pending work may still use the old buffer
            ms_pool_free(*p);
            h->device_bytes -= (int64_t)h->alloc_bytes[i];
            h->allocs[i] = h->allocs[h->nallocs - 1];
            h->alloc_bytes[i] = h->alloc_bytes[h->nallocs - 1];
            --h->nallocs;
            break;
        }
        *p = nullptr;
    }
    return ms_alloc(h, p, bytes);
}

void ms_gather_sorted(const double* in, double* out, const int32_t* perm, int64_t N, int nrhs, int col, cudaStream_t s) {
    k_gather<<<nblk(N, 256), 256, 0, s>>>(in, out, perm, N, nrhs, col); ms_count_launch();
}
void ms_scatter_input(const double* in, double* out, const int32_t* perm, int64_t N, int nrhs, int col, cudaStream_t s) {
    k_scatter_in<<<nblk(N, 256), 256, 0, s>>>(in, out, perm, N, nrhs, col); ms_count_launch();
}

// ---------------------------------------------------------------- C ABI

extern "C" {

void ms_default_opts(ms_opts* o) {
    if (!o) return;
    std::memset(o, 0, sizeof(*o));
    o->wendland_d = 3;
    o->wendland_k = 1;
    o->nu = 4.0;
    o->op = MS_OP_CSR;
    o->precision = MS_PREC_FP64;
    o->precond = MS_PRECOND_NONE;
}

const char* ms_last_error(void) { return g_err; }

ms_status ms_build_hierarchy(int d, int L, const int64_t* n_per_level, const double* points,
                             const double* h_per_level, const ms_opts* opts, ms_hierarchy** out) {
    g_err[0] = 0;
    if (!out || !points) { ms_set_error(MS_ERR_ARG, "points and out must not be NULL"); return MS_ERR_ARG; }
    *out = nullptr;
    {
        // validate every argument on the host before any CUDA call
        ms_hierarchy tmp;
        MS_TRY(validate_and_init(d, L, n_per_level, h_per_level, opts, &tmp));
    }
    int64_t N = 0;
    for (int l = 0; l < L; ++l) N += n_per_level[l];
    for (int64_t i = 0; i < N * d; ++i)
        if (!std::isfinite(points[i])) { ms_set_error(MS_ERR_NUMERIC, "point coordinate %lld is not finite", (long long)i); return MS_ERR_NUMERIC; }
    cudaStream_t st;
    MS_CUDA(cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking));
    DevBuf pts;
    ms_status s = dev_alloc(pts, sizeof(double) * N * d);
    if (s == MS_OK) {
        cudaError_t e = cudaMemcpyAsync(pts.p, points, sizeof(double) * N * d, cudaMemcpyHostToDevice, st);
        if (e != cudaSuccess) s = ms_cuda_error(e, "points H2D", __FILE__, __LINE__);
    }
    if (s == MS_OK) s = build_common(d, L, n_per_level, (const double*)pts.p, h_per_level, opts, st, out);
    cudaStreamSynchronize(st);
    cudaStreamDestroy(st);
    return s;
}

ms_status ms_build_hierarchy_dev(int d, int L, const int64_t* n_per_level, const double* points_dev,
                                 const double* h_per_level, const ms_opts* opts, void* stream, ms_hierarchy** out) {
    g_err[0] = 0;
    if (!out || !points_dev) { ms_set_error(MS_ERR_ARG, "points_dev and out must not be NULL"); return MS_ERR_ARG; }
    *out = nullptr;
    return build_common(d, L, n_per_level, points_dev, h_per_level, opts, (cudaStream_t)stream, out);
}

ms_status ms_fit_dev(ms_hierarchy* h, const double* f_dev, int nrhs, double rel_tol, double* alpha_dev,
                     ms_fit_stats* stats, void* stream) {
    g_err[0] = 0;
    if (!h || !f_dev || !alpha_dev) { ms_set_error(MS_ERR_ARG, "handle, f and alpha must not be NULL"); return MS_ERR_ARG; }
    if (nrhs < 1) { ms_set_error(MS_ERR_ARG, "nrhs must be >= 1 (got %d)", nrhs); return MS_ERR_ARG; }
    if (!(rel_tol > 0.0 && rel_tol < 1.0)) { ms_set_error(MS_ERR_ARG, "rel_tol must be in (0, 1) (got %g)", rel_tol); return MS_ERR_ARG; }
    cudaStream_t st = (cudaStream_t)stream;
    MS_TRY(check_finite(f_dev, h->N * (int64_t)nrhs, st, "f"));
    return ms_fit_impl(h, f_dev, nrhs, rel_tol, alpha_dev, stats, st);
}

ms_status ms_fit(ms_hierarchy* h, const double* f, int nrhs, double rel_tol, double* alpha_out, ms_fit_stats* stats) {
    g_err[0] = 0;
    if (!h || !f || !alpha_out) { ms_set_error(MS_ERR_ARG, "handle, f and alpha_out must not be NULL"); return MS_ERR_ARG; }
    if (nrhs < 1) { ms_set_error(MS_ERR_ARG, "nrhs must be >= 1 (got %d)", nrhs); return MS_ERR_ARG; }
    const size_t bytes = sizeof(double) * h->N * nrhs;
    cudaStream_t st;
    MS_CUDA(cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking));
    DevBuf fd, ad;
    ms_status s = dev_alloc(fd, bytes);
    if (s == MS_OK) s = dev_alloc(ad, bytes);
    if (s == MS_OK) {
        cudaError_t e = cudaMemcpyAsync(fd.p, f, bytes, cudaMemcpyHostToDevice, st);
        if (e != cudaSuccess) s = ms_cuda_error(e, "f H2D", __FILE__, __LINE__);
    }
    if (s == MS_OK || s >= MS_ERR_NOT_SPD) {
        if (s == MS_OK) s = ms_fit_dev(h, (const double*)fd.p, nrhs, rel_tol, (double*)ad.p, stats, st);
        if (s == MS_OK || s == MS_ERR_NOT_CONVERGED) {
            cudaError_t e = cudaMemcpyAsync(alpha_out, ad.p, bytes, cudaMemcpyDeviceToHost, st);
            if (e == cudaSuccess) e = cudaStreamSynchronize(st);
            if (e != cudaSuccess && s == MS_OK) s = ms_cuda_error(e, "alpha D2H", __FILE__, __LINE__);
        }
    }
    cudaStreamSynchronize(st);
    cudaStreamDestroy(st);
    return s;
}

ms_status ms_fit_batch_dev(ms_hierarchy* const* hs, int nh, const double* const* f_dev, double rel_tol,
                           double* const* alpha_dev, ms_fit_stats* stats, void* stream) {
    g_err[0] = 0;
    if (!hs || !f_dev || !alpha_dev || nh < 1) {
        ms_set_error(MS_ERR_ARG, "hs, f_dev and alpha_dev must not be NULL and nh >= 1 (got %d)", nh);
        return MS_ERR_ARG;
    }
    if (!(rel_tol > 0.0 && rel_tol < 1.0)) { ms_set_error(MS_ERR_ARG, "rel_tol must be in (0, 1) (got %g)", rel_tol); return MS_ERR_ARG; }
    for (int i = 0; i < nh; ++i)
        if (!hs[i] || !f_dev[i] || !alpha_dev[i]) {
            ms_set_error(MS_ERR_ARG, "hierarchy %d: handle, f and alpha must not be NULL", i);
            return MS_ERR_ARG;
        }
    return ms_fit_batch_impl(hs, nh, f_dev, rel_tol, alpha_dev, stats, (cudaStream_t)stream);
}

ms_status ms_batch_plan_create(ms_hierarchy* const* hs, int nh, const double* const* f_dev, double rel_tol,
                               double* const* alpha_dev, void* stream, ms_batch_plan** out) {
    g_err[0] = 0;
    if (!out) { ms_set_error(MS_ERR_ARG, "out must not be NULL"); return MS_ERR_ARG; }
    *out = nullptr;
    if (!hs || !f_dev || !alpha_dev || nh < 1) {
        ms_set_error(MS_ERR_ARG, "hs, f_dev and alpha_dev must not be NULL and nh >= 1 (got %d)", nh);
        return MS_ERR_ARG;
    }
    if (!(rel_tol > 0.0 && rel_tol < 1.0)) { ms_set_error(MS_ERR_ARG, "rel_tol must be in (0, 1) (got %g)", rel_tol); return MS_ERR_ARG; }
    for (int i = 0; i < nh; ++i)
        if (!hs[i] || !f_dev[i] || !alpha_dev[i]) {
            ms_set_error(MS_ERR_ARG, "hierarchy %d: handle, f and alpha must not be NULL", i);
            return MS_ERR_ARG;
        }
    return ms_batch_plan_create_impl(hs, nh, f_dev, rel_tol, alpha_dev, (cudaStream_t)stream, out);
}

ms_status ms_batch_plan_launch(ms_batch_plan* plan, void* stream, int use_graph) {
    g_err[0] = 0;
    if (!plan) { ms_set_error(MS_ERR_ARG, "plan must not be NULL"); return MS_ERR_ARG; }
    return ms_batch_plan_launch_impl(plan, (cudaStream_t)stream, use_graph ? 1 : 0);
}

ms_status ms_batch_plan_stats(ms_batch_plan* plan, void* stream, ms_fit_stats* stats) {
    g_err[0] = 0;
    if (!plan) { ms_set_error(MS_ERR_ARG, "plan must not be NULL"); return MS_ERR_ARG; }
    return ms_batch_plan_stats_impl(plan, (cudaStream_t)stream, stats, -1.f);
}

void ms_batch_plan_destroy(ms_batch_plan* plan) { ms_batch_plan_free(plan, true); }

ms_status ms_fit_batch(ms_hierarchy* const* hs, int nh, const double* const* f, double rel_tol,
                       double* const* alpha_out, ms_fit_stats* stats) {
    g_err[0] = 0;
    if (!hs || !f || !alpha_out || nh < 1) {
        ms_set_error(MS_ERR_ARG, "hs, f and alpha_out must not be NULL and nh >= 1 (got %d)", nh);
        return MS_ERR_ARG;
    }
    int64_t total = 0;
    for (int i = 0; i < nh; ++i) {
        if (!hs[i] || !f[i] || !alpha_out[i]) {
            ms_set_error(MS_ERR_ARG, "hierarchy %d: handle, f and alpha_out must not be NULL", i);
            return MS_ERR_ARG;
        }
        total += hs[i]->N;
    }
    cudaStream_t st;
    MS_CUDA(cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking));
    DevBuf fd, ad;
    ms_status s = dev_alloc(fd, sizeof(double) * total);
    if (s == MS_OK) s = dev_alloc(ad, sizeof(double) * total);
    std::vector<const double*> fp(nh);
    std::vector<double*> ap(nh);
    int64_t o = 0;
    for (int i = 0; i < nh && s == MS_OK; ++i) {
        fp[i] = (const double*)fd.p + o;
        ap[i] = (double*)ad.p + o;
        cudaError_t e = cudaMemcpyAsync((void*)fp[i], f[i], sizeof(double) * hs[i]->N, cudaMemcpyHostToDevice, st);
        if (e != cudaSuccess) s = ms_cuda_error(e, "f H2D", __FILE__, __LINE__);
        o += hs[i]->N;
    }
    if (s == MS_OK) s = ms_fit_batch_dev(hs, nh, fp.data(), rel_tol, ap.data(), stats, st);
    if (s == MS_OK || s == MS_ERR_NOT_CONVERGED) {
        for (int i = 0; i < nh; ++i) {
            cudaError_t e = cudaMemcpyAsync(alpha_out[i], ap[i], sizeof(double) * hs[i]->N, cudaMemcpyDeviceToHost, st);
            if (e != cudaSuccess) {
                if (s == MS_OK) s = ms_cuda_error(e, "alpha D2H", __FILE__, __LINE__);
                break;
            }
        }
    }
    cudaStreamSynchronize(st);
    cudaStreamDestroy(st);
    return s;
}

ms_status ms_evaluate_dev(ms_hierarchy* h, const double* alpha_dev, int nrhs, const double* query_dev, int64_t nq,
                          double* out_dev, void* stream) {
    g_err[0] = 0;
    if (!h || nrhs < 1 || nq < 0) { ms_set_error(MS_ERR_ARG, "invalid handle, nrhs or nq"); return MS_ERR_ARG; }
    if (nq > 0 && (!alpha_dev || !query_dev || !out_dev)) { ms_set_error(MS_ERR_ARG, "NULL array"); return MS_ERR_ARG; }
    return ms_evaluate_impl(h, alpha_dev, nrhs, query_dev, nq, out_dev, (cudaStream_t)stream);
}

ms_status ms_evaluate(ms_hierarchy* h, const double* alpha, int nrhs, const double* query, int64_t nq, double* out) {
    g_err[0] = 0;
    if (!h || nrhs < 1 || nq < 0) { ms_set_error(MS_ERR_ARG, "invalid handle, nrhs or nq"); return MS_ERR_ARG; }
    if (nq == 0) return MS_OK;
    if (!alpha || !query || !out) { ms_set_error(MS_ERR_ARG, "NULL array"); return MS_ERR_ARG; }
    cudaStream_t st;
    MS_CUDA(cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking));
    DevBuf ad, qd, od;
    ms_status s = dev_alloc(ad, sizeof(double) * h->N * nrhs);
    if (s == MS_OK) s = dev_alloc(qd, sizeof(double) * nq * h->d);
    if (s == MS_OK) s = dev_alloc(od, sizeof(double) * nq * nrhs);
    if (s == MS_OK) {
        cudaError_t e = cudaMemcpyAsync(ad.p, alpha, sizeof(double) * h->N * nrhs, cudaMemcpyHostToDevice, st);
        if (e == cudaSuccess) e = cudaMemcpyAsync(qd.p, query, sizeof(double) * nq * h->d, cudaMemcpyHostToDevice, st);
        if (e != cudaSuccess) s = ms_cuda_error(e, "evaluate H2D", __FILE__, __LINE__);
    }
    if (s == MS_OK) s = ms_evaluate_impl(h, (const double*)ad.p, nrhs, (const double*)qd.p, nq, (double*)od.p, st);
    if (s == MS_OK) {
        cudaError_t e = cudaMemcpyAsync(out, od.p, sizeof(double) * nq * nrhs, cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) s = ms_cuda_error(e, "evaluate D2H", __FILE__, __LINE__);
    }
    cudaStreamSynchronize(st);
    cudaStreamDestroy(st);
    return s;
}

ms_status ms_apply_dev(ms_hierarchy* h, int op, const double* x_dev, double* y_dev, int sorted_order, void* stream) {
    g_err[0] = 0;
    if (!h || !x_dev || !y_dev) { ms_set_error(MS_ERR_ARG, "NULL argument"); return MS_ERR_ARG; }
    if (op < MS_APPLY_A64 || op > MS_APPLY_BMFDF) { ms_set_error(MS_ERR_ARG, "unknown operator %d", op); return MS_ERR_ARG; }
    return ms_apply_impl(h, op, x_dev, y_dev, sorted_order, (cudaStream_t)stream);
}

ms_status ms_get_permutation(const ms_hierarchy* h, int64_t* perm_out) {
    g_err[0] = 0;
    if (!h || !perm_out) { ms_set_error(MS_ERR_ARG, "NULL argument"); return MS_ERR_ARG; }
    std::vector<int32_t> p(h->N);
    MS_CUDA(cudaMemcpy(p.data(), h->perm, sizeof(int32_t) * h->N, cudaMemcpyDeviceToHost));
    for (int64_t i = 0; i < h->N; ++i) perm_out[i] = p[i];
    return MS_OK;
}

ms_status ms_hierarchy_info(const ms_hierarchy* h, ms_info* info) {
    g_err[0] = 0;
    if (!h || !info) { ms_set_error(MS_ERR_ARG, "NULL argument"); return MS_ERR_ARG; }
    std::memset(info, 0, sizeof(*info));
    info->d = h->d;
    info->L = h->L;
    info->N = h->N;
    for (int l = 0; l < h->L; ++l) {
        info->n_per_level[l] = h->view.off[l + 1] - h->view.off[l];
        info->delta[l] = h->view.delta[l];
    }
    info->nnz_A = h->A.nnz;
    info->nnz_B = h->B.nnz;
    info->device_bytes = h->device_bytes;
    info->build_ms = h->build_ms;
    for (int l = 0; l < h->L; ++l) info->tpr_A[l] = ms_tpr_of(h, l);
    info->pc_basis = h->pc.nbasis;
    info->cell_split = h->opts.cell_split > 0 ? h->opts.cell_split : 1;
    info->solve_ctas_per_sm = h->opts.solve_ctas_per_sm == 1 ? 1 : 2;
    return MS_OK;
}

ms_status ms_trim_memory(void) {
    g_err[0] = 0;
    DevPool* dp = nullptr;
    MS_TRY(device_pool(&dp));
    MS_CUDA(cudaStreamSynchronize(dp->stream));  // frees are ordered on the pool's stream
    MS_CUDA(cudaMemPoolTrimTo(dp->pool, 0));
    return MS_OK;
}

void ms_destroy(ms_hierarchy* h) {
    if (!h) return;
    cudaDeviceSynchronize();  // the handle's memory returns to the pool: no work may still use it
    for (ms_batch_plan* p : h->plans) ms_batch_plan_detach(p, h);
    for (int i = 0; i < h->nallocs; ++i) ms_pool_free(h->allocs[i]);
    if (h->ev0) cudaEventDestroy(h->ev0);
    if (h->ev1) cudaEventDestroy(h->ev1);
    delete h;
}

}  // extern "C"

// ---------------------------------------------------------------- launch counter

#include <atomic>
namespace {
std::atomic<uint64_t> g_launches{0};
}
void ms_count_launch(unsigned n) { g_launches.fetch_add(n, std::memory_order_relaxed); }
extern "C" uint64_t ms_launch_count(void) { return g_launches.load(std::memory_order_relaxed); }
