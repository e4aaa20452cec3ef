// The fit of one hierarchy: one persistent cooperative launch per batch of right-hand
// sides (the kernel and its schedule are in ms_solve_dev.cuh), the stand-alone mat-vecs and the
// allocation-free fit.
#include <algorithm>
#include <cmath>
#include <map>
#include <mutex>
#include <tuple>
#include <vector>

#include "ms_solve_dev.cuh"

namespace {

// f (input order, [N][nrhs], columns col0..col0+R-1) -> [N][RW] in sorted order (padding 0),
// and back for alpha.
__global__ void k_gather_wide(const double* in, double* out, const int32_t* perm, int64_t N, int nrhs, int col0,
                              int R, int RW) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= N * RW) return;
    const int64_t row = i / RW;
    const int r = (int)(i % RW);
    out[i] = r < R ? in[(int64_t)perm[row] * nrhs + col0 + r] : 0.0;
}
__global__ void k_scatter_wide(const double* in, double* out, const int32_t* perm, int64_t N, int nrhs, int col0,
                               int R, int RW) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= N * RW) return;
    const int64_t row = i / RW;
    const int r = (int)(i % RW);
    if (r < R) out[(int64_t)perm[row] * nrhs + col0 + r] = in[i];
}

// ---------------------------------------------------------------- stand-alone mat-vecs

template <typename TV, typename TX, typename TA>
__global__ void k_spmv(const int64_t* rp, const int32_t* col, const TV* val, const TX* x, double* y, int64_t N,
                       int S, const double* sub, double sign) {
    const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    const int spw = 32 / S;
    const int64_t row = warp * spw + lane / S;
    const bool ok = row < N;
    int64_t s = 0, e = 0;
    if (ok) { s = rp[row]; e = rp[row + 1]; }
    const TA v = csr_row_vec<TV, TX, TA>(col, val, x, s, e, lane & (S - 1), S);
    if (ok && (lane & (S - 1)) == 0) y[row] = sub ? sub[row] + sign * (double)v : (double)v;
}

// y = D_L x matrix-free: one warp per cell of every level.
__global__ void k_mf_apply(MFView v, const float* x, double* y, int tpp, int64_t total_cells) {
    const int64_t gw = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    if (gw >= total_cells) return;  // warp-uniform
    int l = 0;
    while (l + 1 < v.L && gw >= v.lv[l + 1].cell_off) ++l;
    const int64_t cell = gw - v.lv[l].cell_off;
    mf_cells_any(v, l, cell, cell + 1, 0, 1, tpp, x, [&](int64_t row, float val) { y[row] = (double)val; });
}

// y = D_L x matrix-free, staged form: one CTA per cell of every level (mf_cell_staged); a cell
// of more than the CTA's 128 points takes the warp form on the CTA's first warp.
__global__ void __launch_bounds__(128) k_mf_apply_staged(MFView v, const float* x, double* y, int tpp) {
    __shared__ float4 stage[kMfStage];
    const int64_t gc = blockIdx.x;
    int l = 0;
    while (l + 1 < v.L && gc >= v.lv[l + 1].cell_off) ++l;
    const int64_t cell = gc - v.lv[l].cell_off;
    auto emit = [&](int64_t row, float val) { y[row] = (double)val; };
    if (!mf_cell_staged_any(v, l, cell, x, stage, emit) && threadIdx.x < 32)
        mf_cells_any(v, l, cell, cell + 1, 0, 1, tpp, x, emit);
}

__global__ void k_to_f32(const double* in, float* out, int64_t n) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < n) out[i] = (float)in[i];
}

// x split into double-float parts hi + lo
__global__ void k_split_ff(const double* in, float* hi, float* lo, int64_t n) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < n) {
        const ff t = ff_from_double(in[i]);
        hi[i] = t.hi;
        lo[i] = t.lo;
    }
}

// FP32 constants of the matrix-free lower blocks: the Wendland polynomial and delta_j^-d.
struct LowerF32 {
    float c[4];
    float ds[MS_MAXL];
};

// y = (T_L - D_L) x matrix-free: S lanes per row; row s of level k sums the entries of every
// level j < k (lower_row_mf, level j's frame of s set up in FP64), rows of level 0 get 0.
template <bool FF>
__global__ void k_lower_mf_apply(const __grid_constant__ HierView v, const float* W, const float* Wlo,
                                 const int32_t* cellid, const __grid_constant__ FFLevels ffl,
                                 const __grid_constant__ LowerF32 lf, const float* xhi, const float* xlo, double* y,
                                 int S) {
    const int64_t gw = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    const int64_t row = gw * (32 / S) + lane / S;
    const int sl = lane & (S - 1);
    const bool ok = row < v.N;
    ff acc = {0.0f, 0.0f};
    if (ok) {
        const int k = level_of_row(v.off, v.L, row);
        for (int j = 0; j < k; ++j) {
            const Frame f = frame_of(v, j, point_at(v, row));
            const ff part = lower_row_mf_any<FF>(v, W, Wlo, cellid, ffl, lf.c, lf.ds[j], j, f, xhi, xlo, sl, S);
            acc = FF ? ff_add(acc, part) : ff{acc.hi + part.hi, 0.0f};
        }
    }
    if (FF) {
        acc = ff_group_sum(acc, S);
    } else {
        for (int o = S >> 1; o > 0; o >>= 1) acc.hi += __shfl_xor_sync(0xffffffffu, acc.hi, o);
    }
    if (ok && sl == 0) y[row] = FF ? ff_to_double(acc) : (double)acc.hi;
}

// Several blocks of right-hand sides of one hierarchy in ONE cooperative launch: the grid is
// split into P equal partitions of consecutive CTAs, partition p = CTAs [p G / P, (p + 1) G / P)
// runs the whole schedule of eq. split for block p (args[p]: its own work vectors, reductions
// and barrier words), the same device code as a single fit.  The blocks' small, latency-bound
// phases then overlap instead of running one launch after another.
__host__ __device__ inline int part_first_cta(int p, int G, int P) { return (int)(((long long)p * G) / P); }

template <int MODE, bool WIDE>
__global__ void __launch_bounds__(kBS, 2) k_fit_parts(const SolveArgs* __restrict__ args, int P) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    Shared& sh = *reinterpret_cast<Shared*>(smem_raw);
    __shared__ int pid;
    if (threadIdx.x == 0) {
        const int G = gridDim.x, b = blockIdx.x;
        int p = (int)(((long long)b * P) / G);
        while (p + 1 < P && part_first_cta(p + 1, G, P) <= b) ++p;
        while (p > 0 && part_first_cta(p, G, P) > b) --p;
        pid = p;
        sh.cta = b - part_first_cta(p, G, P);
        sh.nb = part_first_cta(p + 1, G, P) - part_first_cta(p, G, P);
    }
    __syncthreads();
    fit_body<MODE, WIDE>(args[pid], sh);
}

const void* parts_kernel(bool mixed, bool wide) {
    if (wide) return mixed ? (const void*)k_fit_parts<1, true> : (const void*)k_fit_parts<0, true>;
    return mixed ? (const void*)k_fit_parts<1, false> : (const void*)k_fit_parts<0, false>;
}

constexpr int kMaxParts = 16;  // blocks of right-hand sides per launch

// Per-block counters of a partitioned launch, carved from h->pbuf (256-byte aligned pieces).
struct PartCounters {
    unsigned* bar;
    int* status;
    int64_t* iters;
    int* refines;
    double* bytes;
    unsigned long long* prof;
    int* pcfb;
};
constexpr size_t pad256b(size_t b) { return (b + 255) / 256 * 256; }
constexpr size_t kPartBytes = pad256b(sizeof(unsigned) * kBarWords) + pad256b(sizeof(int)) +
                              pad256b(sizeof(int64_t) * MS_MAXL) + pad256b(sizeof(int) * MS_MAXL) +
                              pad256b(sizeof(double)) + pad256b(sizeof(unsigned long long) * kProf) +
                              pad256b(sizeof(int) * 2);
PartCounters part_counters(const ms_hierarchy* h, int p) {
    unsigned char* b = static_cast<unsigned char*>(h->pbuf) + (size_t)p * kPartBytes;
    PartCounters c;
    c.bar = reinterpret_cast<unsigned*>(b);
    b += pad256b(sizeof(unsigned) * kBarWords);
    c.status = reinterpret_cast<int*>(b);
    b += pad256b(sizeof(int));
    c.iters = reinterpret_cast<int64_t*>(b);
    b += pad256b(sizeof(int64_t) * MS_MAXL);
    c.refines = reinterpret_cast<int*>(b);
    b += pad256b(sizeof(int) * MS_MAXL);
    c.bytes = reinterpret_cast<double*>(b);
    b += pad256b(sizeof(double));
    c.prof = reinterpret_cast<unsigned long long*>(b);
    b += pad256b(sizeof(unsigned long long) * kProf);
    c.pcfb = reinterpret_cast<int*>(b);
    return c;
}

ms_status ensure_parts(ms_hierarchy* h, int P) {
    if (h->pbuf && h->pbuf_parts >= P) return MS_OK;
    MS_TRY(ms_realloc(h, &h->pbuf, kPartBytes * (size_t)P));
    MS_TRY(ms_realloc(h, &h->d_args, sizeof(SolveArgs) * (size_t)P));
    h->pbuf_parts = P;
    return MS_OK;
}

// The solve kernel for a precision and a CTAs-per-SM choice (opts.solve_ctas_per_sm;
// 0 = automatic = 2: measured on GB300 at 1.4M points, 2 CTAs per SM (64 registers)
// fit 21% (FP64) and 24% (MIXED, learned preconditioner) faster than 1 (128 registers)).
int ctas_per_sm(const ms_opts& o) {
    if (o.solve_ctas_per_sm == 1 || o.solve_ctas_per_sm == 2) return o.solve_ctas_per_sm;
    return 2;
}

const void* fit_kernel(bool mixed, int minb, bool wide = false) {
    if (wide) return mixed ? (const void*)k_fit<1, 2, true> : (const void*)k_fit<0, 2, true>;
    if (mixed) return minb == 1 ? (const void*)k_fit<1, 1, false> : (const void*)k_fit<1, 2, false>;
    return minb == 1 ? (const void*)k_fit<0, 1, false> : (const void*)k_fit<0, 2, false>;
}

// Cooperative grid of the solve kernel: min(per_sm, minb) CTAs on every SM.
ms_status fit_blocks(bool mixed, int minb, int dev, int* blocks, bool wide = false) {
    const void* fn = fit_kernel(mixed, minb, wide);
    // the per-CTA state is above the default 48 KB of dynamic shared memory
    MS_CUDA(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sizeof(Shared)));
    int sms = 0, per_sm = 0;
    MS_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    MS_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, kBS, sizeof(Shared)));
    if (per_sm < 1) {
        ms_set_error(MS_ERR_CUDA, "solve kernel cannot be resident on an SM");
        return MS_ERR_CUDA;
    }
    *blocks = std::min(sms * std::min(per_sm, minb), kMaxGroups * kGroup);
    return MS_OK;
}

}  // namespace

// ---------------------------------------------------------------- host side

ms_status ms_ensure_workspace(ms_hierarchy* h, int R) {
    if (h->f && h->ws_rhs >= R) return MS_OK;
    if (!h->plans.empty()) {
        ms_set_error(MS_ERR_STATE, "the work space must grow to %d right-hand sides, but a batch plan holds it "
                     "(destroy the plan first)", R);
        return MS_ERR_STATE;
    }
    const int64_t n = h->N * (int64_t)R;
    MS_TRY(ms_realloc(h, (void**)&h->f, sizeof(double) * n));
    MS_TRY(ms_realloc(h, (void**)&h->beta, sizeof(double) * n));
    MS_TRY(ms_realloc(h, (void**)&h->x, sizeof(double) * n));
    MS_TRY(ms_realloc(h, (void**)&h->r, sizeof(double) * n));
    MS_TRY(ms_realloc(h, (void**)&h->p, sizeof(double) * n));
    MS_TRY(ms_realloc(h, (void**)&h->q, sizeof(double) * n));
    MS_TRY(ms_realloc(h, (void**)&h->s, sizeof(double) * n));
    if (!h->tmp64) MS_TRY(ms_alloc(h, (void**)&h->tmp64, sizeof(double) * h->N));
    if (h->opts.precision == MS_PREC_MIXED) {
        MS_TRY(ms_realloc(h, (void**)&h->x32, sizeof(float) * n));
        MS_TRY(ms_realloc(h, (void**)&h->r32, sizeof(float) * n));
        MS_TRY(ms_realloc(h, (void**)&h->p32, sizeof(float) * n));
        MS_TRY(ms_realloc(h, (void**)&h->q32, sizeof(float) * n));
        MS_TRY(ms_realloc(h, (void**)&h->s32, sizeof(float) * n));
        if (h->opts.precond != MS_PRECOND_NONE) {
            MS_TRY(ms_realloc(h, (void**)&h->u32, sizeof(float) * n));
            MS_TRY(ms_realloc(h, (void**)&h->u1_32, sizeof(float) * n));
        }
    }
    int dev = 0;
    MS_CUDA(cudaGetDevice(&dev));
    MS_TRY(fit_blocks(h->opts.precision == MS_PREC_MIXED, ctas_per_sm(h->opts), dev, &h->solve_blocks));
    h->mf_tpp = h->mf_tpp_tuned > 0 ? h->mf_tpp_tuned : mf_tpp_for(h);
    const int V = R * h->L;
    MS_TRY(ms_realloc(h, (void**)&h->part, sizeof(double) * kAcc * V * h->solve_blocks));
    MS_TRY(ms_realloc(h, (void**)&h->gpart, sizeof(double) * kMaxGroups * kAcc * V));
    MS_TRY(ms_realloc(h, (void**)&h->scal, sizeof(double) * kAcc * V));
    MS_TRY(ms_realloc(h, (void**)&h->resid, sizeof(double) * V));
    if (!h->bar) {
        MS_TRY(ms_alloc(h, (void**)&h->bar, sizeof(unsigned) * kBarWords));
        MS_TRY(ms_alloc(h, (void**)&h->status, sizeof(int)));
        MS_TRY(ms_alloc(h, (void**)&h->iters, sizeof(int64_t) * MS_MAXL));
        MS_TRY(ms_alloc(h, (void**)&h->refines, sizeof(int) * MS_MAXL));
        MS_TRY(ms_alloc(h, (void**)&h->bytes, sizeof(double)));
        MS_TRY(ms_alloc(h, (void**)&h->prof, sizeof(unsigned long long) * kProf));
        MS_TRY(ms_alloc(h, (void**)&h->pcfb, sizeof(int) * 2));
    }
    h->ws_rhs = R;
    return MS_OK;
}

// ---------------------------------------------------------------- autotuner
//
// The CSR mat-vec of a level gives each row S lanes (S a power of two); the rule
// tpr_for (about 16 entries a lane) is a good guess but the best S depends on the
// row count, the entries per row and the precision.  With opts.autotune = 1 the first
// fit of a handle times a stand-in for the solve kernel's mat-vec phase (k_tune_matvec:
// the solve grid, 256-row chunks dealt round-robin to the CTAs, S lanes per row) on
// every level of at least kTuneMinRows rows for S = 1, 2, ..., 32 (matrix-free
// operator: the lanes per target point, 1 to 8, over all levels) and keeps the
// fastest.  Choices are cached for the process, keyed by the level's shape, so later
// handles of the same shape skip the timing.

int ms_tpr_of(const ms_hierarchy* h, int l) {
    if (h->opts.threads_per_row > 0) return h->opts.threads_per_row;
    if (h->tprA_tuned[l] > 0) return h->tprA_tuned[l];
    const int64_t n = h->view.off[l + 1] - h->view.off[l];
    return tpr_for((double)(h->rpA_lv[l + 1] - h->rpA_lv[l]) / (double)std::max<int64_t>(n, 1));
}

namespace {

template <typename TV, typename TX>
__global__ void __launch_bounds__(kBS) k_tune_matvec(const int64_t* rp, const int32_t* col, const TV* val,
                                                     const TX* x, TX* y, int64_t r0, int64_t r1, int S) {
    const int64_t nch = (r1 - r0 + kChunk - 1) / kChunk;
    for (int64_t c = blockIdx.x; c < nch; c += gridDim.x) {
        const int64_t a0 = r0 + c * kChunk, a1 = min(a0 + (int64_t)kChunk, r1);
        rows_by_subwarp(a0, a1, S, [&](int64_t row, bool ok, int sl) {
            int64_t s = 0, e = 0;
            if (ok) { s = rp[row]; e = rp[row + 1]; }
            const TX v = csr_row<TV, TX, TX>(col, val, x, s, e, sl, S);
            if (ok && sl == 0) y[row] = v;
        });
    }
}

constexpr int64_t kTuneMinRows = 4096;
constexpr int kTuneWarm = 2, kTuneReps = 5;

// (op, d, wendland d, wendland k, mixed, log2 rows, entries per row rounded) -> lanes
using TuneKey = std::tuple<int, int, int, int, int, int, int>;
std::mutex g_tune_mu;
std::map<TuneKey, int> g_tune_cache;

TuneKey tune_key(const ms_hierarchy* h, int64_t rows, double per_row) {
    int lg = 0;
    while ((int64_t(1) << (lg + 1)) <= rows) ++lg;
    return TuneKey(h->opts.op, h->d, h->opts.wendland_d, h->opts.wendland_k,
                   h->opts.precision == MS_PREC_MIXED ? 1 : 0, lg, (int)std::lround(per_row));
}

// Time `launch` kTuneReps times after kTuneWarm untimed runs; milliseconds in *ms.
template <typename F>
ms_status time_launches(cudaStream_t st, cudaEvent_t e0, cudaEvent_t e1, F launch, float* ms) {
    for (int i = 0; i < kTuneWarm; ++i) launch();
    MS_CUDA(cudaEventRecord(e0, st));
    for (int i = 0; i < kTuneReps; ++i) launch();
    MS_CUDA(cudaEventRecord(e1, st));
    MS_CUDA(cudaEventSynchronize(e1));
    MS_CUDA(cudaGetLastError());
    MS_CUDA(cudaEventElapsedTime(ms, e0, e1));
    return MS_OK;
}

ms_status autotune_run(ms_hierarchy* h, cudaStream_t st, cudaEvent_t e0, cudaEvent_t e1) {
    const bool mixed = h->opts.precision == MS_PREC_MIXED;
    const int64_t N = h->N;
    float* x32 = h->r32;  // scratch: the fit overwrites every work vector before it reads it
    MS_CUDA(cudaMemsetAsync(h->r, 0, sizeof(double) * N, st));
    if (mixed) MS_CUDA(cudaMemsetAsync(x32, 0, sizeof(float) * N, st));
    if (h->opts.op == MS_OP_MATRIX_FREE) {
        if (!mixed) return MS_OK;  // the FP64 fit reads the CSR matrix
        const int64_t rows = N;
        const TuneKey key = tune_key(h, rows, (double)h->total_cells);
        {
            std::lock_guard<std::mutex> g(g_tune_mu);
            auto it = g_tune_cache.find(key);
            if (it != g_tune_cache.end()) { h->mf_tpp_tuned = it->second; return MS_OK; }
        }
        const MFView v = make_mfview(h);
        int best = 0;
        float best_ms = 0.f;
        for (int t = 1; t <= 8; t <<= 1) {
            float ms = 0.f;
            MS_TRY(time_launches(st, e0, e1, [&] {
                k_mf_apply<<<nblk(h->total_cells * 32, 256), 256, 0, st>>>(v, x32, h->q, t, h->total_cells);
                ms_count_launch();
            }, &ms));
            if (best == 0 || ms < best_ms) { best = t; best_ms = ms; }
        }
        h->mf_tpp_tuned = best;
        std::lock_guard<std::mutex> g(g_tune_mu);
        g_tune_cache[key] = best;
        return MS_OK;
    }
    for (int l = 0; l < h->L; ++l) {
        const int64_t r0 = h->view.off[l], n = h->view.off[l + 1] - r0;
        if (n < kTuneMinRows) continue;
        const double per_row = (double)(h->rpA_lv[l + 1] - h->rpA_lv[l]) / (double)n;
        const TuneKey key = tune_key(h, n, per_row);
        {
            std::lock_guard<std::mutex> g(g_tune_mu);
            auto it = g_tune_cache.find(key);
            if (it != g_tune_cache.end()) { h->tprA_tuned[l] = it->second; continue; }
        }
        int best = 0;
        float best_ms = 0.f;
        const int blocks = std::max(h->solve_blocks, 1);
        for (int S = 1; S <= 32; S <<= 1) {
            float ms = 0.f;
            MS_TRY(time_launches(st, e0, e1, [&] {
                if (mixed)
                    k_tune_matvec<float, float><<<blocks, kBS, 0, st>>>(h->A.rp, h->A.col, h->A.v32, x32, h->q32,
                                                                         r0, r0 + n, S);
                else
                    k_tune_matvec<double, double><<<blocks, kBS, 0, st>>>(h->A.rp, h->A.col, h->A.v64, h->r, h->q,
                                                                           r0, r0 + n, S);
                ms_count_launch();
            }, &ms));
            if (best == 0 || ms < best_ms) { best = S; best_ms = ms; }
        }
        h->tprA_tuned[l] = best;
        std::lock_guard<std::mutex> g(g_tune_mu);
        g_tune_cache[key] = best;
    }
    return MS_OK;
}

}  // namespace

// Runs the autotuner once per handle (after a build, when opts.autotune = 1).
ms_status ms_autotune(ms_hierarchy* h, cudaStream_t st) {
    if (!h->opts.autotune || h->tuned) return MS_OK;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    MS_CUDA(cudaEventCreate(&e0));
    if (cudaEventCreate(&e1) != cudaSuccess) {
        cudaEventDestroy(e0);
        ms_set_error(MS_ERR_CUDA, "cudaEventCreate failed");
        return MS_ERR_CUDA;
    }
    const ms_status s = autotune_run(h, st, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (s != MS_OK) return s;
    h->tuned = true;
    h->mf_tpp = h->mf_tpp_tuned > 0 ? h->mf_tpp_tuned : h->mf_tpp;
    return MS_OK;
}

namespace {

// CTAs per SM of the solve kernel in use; re-sizes the per-CTA reduction buffer when the
// cooperative grid changes.
ms_status set_solve_ctas(ms_hierarchy* h, int c) {
    h->opts.solve_ctas_per_sm = c;
    if (!h->f) return MS_OK;  // sized by the next fit's work space
    int dev = 0, blocks = 0;
    MS_CUDA(cudaGetDevice(&dev));
    MS_TRY(fit_blocks(h->opts.precision == MS_PREC_MIXED, c, dev, &blocks));
    if (blocks > h->solve_blocks)
        MS_TRY(ms_realloc(h, (void**)&h->part, sizeof(double) * kAcc * (size_t)h->ws_rhs * h->L * blocks));
    h->solve_blocks = blocks;
    return MS_OK;
}

// (d, L, log2 N, wendland d, k, precision, precond, op, lower_op, several rhs) -> CTAs per SM
using CtaKey = std::tuple<int, int, int, int, int, int, int, int, int, int>;
std::map<CtaKey, int> g_cta_cache;

}  // namespace

ms_status fit_impl_inner(ms_hierarchy* h, const double* f_dev, int nrhs, double rel_tol, double* alpha_dev,
                         ms_fit_stats* stats, cudaStream_t st);

// With opts.autotune = 1 and solve_ctas_per_sm = 0, the first fit of a hierarchy shape runs
// once with 1 CTA per SM (up to 128 registers a thread) and once with 2 (up to 64), keeps the
// faster kernel time for the handle and caches it per process by shape; the call returns the
// second run's result (both are fits to rel_tol).
#ifdef MS_CTA_PROF
// Diagnostic build only: the per-CTA timelines of the last single-hierarchy solve launch.
extern "C" int ms_debug_cta_prof(unsigned long long* out, int n) {
    const size_t b = sizeof(unsigned long long) * kProf * (size_t)std::min(std::max(n, 0), 1024);
    return cudaMemcpyFromSymbol(out, g_cta_prof, b) == cudaSuccess ? 0 : 1;
}
#endif

ms_status ms_fit_impl(ms_hierarchy* h, const double* f_dev, int nrhs, double rel_tol, double* alpha_dev,
                      ms_fit_stats* stats, cudaStream_t st) {
    if (!(h->opts.autotune && h->opts.solve_ctas_per_sm == 0))
        return fit_impl_inner(h, f_dev, nrhs, rel_tol, alpha_dev, stats, st);
    int lg = 0;
    while ((int64_t(1) << (lg + 1)) <= h->N) ++lg;
    const CtaKey key(h->d, h->L, lg, h->opts.wendland_d, h->opts.wendland_k, h->opts.precision, h->opts.precond,
                     h->opts.op, h->opts.lower_op, nrhs > 1 ? 1 : 0);
    int cached = 0;
    {
        // (the lock is released before the fit: the fit's lane tuning takes the same mutex)
        std::lock_guard<std::mutex> lk(g_tune_mu);
        auto it = g_cta_cache.find(key);
        if (it != g_cta_cache.end()) cached = it->second;
    }
    if (cached) {
        MS_TRY(set_solve_ctas(h, cached));
        return fit_impl_inner(h, f_dev, nrhs, rel_tol, alpha_dev, stats, st);
    }
    ms_fit_stats s1{}, s2{};
    MS_TRY(set_solve_ctas(h, 1));
    ms_status r = fit_impl_inner(h, f_dev, nrhs, rel_tol, alpha_dev, &s1, st);
    if (r != MS_OK) {
        h->opts.solve_ctas_per_sm = 0;
        return r;
    }
    MS_TRY(set_solve_ctas(h, 2));
    r = fit_impl_inner(h, f_dev, nrhs, rel_tol, alpha_dev, &s2, st);
    const int best = s1.fit_ms < s2.fit_ms ? 1 : 2;
    MS_TRY(set_solve_ctas(h, best));
    if (r == MS_OK) {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        g_cta_cache[key] = best;
    }
    if (stats) *stats = s2;
    return r;
}

ms_status fit_impl_inner(ms_hierarchy* h, const double* f_dev, int nrhs, double rel_tol, double* alpha_dev,
                         ms_fit_stats* stats, cudaStream_t st) {
    const int Rmax = rhs_per_launch(h, nrhs);
    const bool wide = wide_layout(h, nrhs, ctas_per_sm(h->opts));
    int RWmax = 1;
    while (RWmax < Rmax) RWmax <<= 1;
    MS_TRY(ms_ensure_workspace(h, wide ? RWmax : Rmax));
    const int L = h->L;
    const int64_t N = h->N;
    const bool mixed = h->opts.precision == MS_PREC_MIXED;
    if (mixed && h->opts.op != MS_OP_MATRIX_FREE && !h->A.v32) {
        ms_set_error(MS_ERR_STATE, "MIXED fit needs FP32 values (build with precision = MS_PREC_MIXED)");
        return MS_ERR_STATE;
    }
    if (h->opts.precond != MS_PRECOND_NONE) {
        if (!mixed) {
            ms_set_error(MS_ERR_ARG, "a preconditioner needs precision = MS_PREC_MIXED (it acts on the FP32 inner CG)");
            return MS_ERR_ARG;
        }
        MS_TRY(ms_pc_build(h, h->opts.precond, st));
    }
    MS_TRY(ms_autotune(h, st));

    ms_status result = MS_OK;
    int launches = 0;
    float total_ms = 0.f;
    double bytes = 0.0;
    std::vector<int64_t> it_sum(MS_MAXL, 0);
    std::vector<int> ref_sum(MS_MAXL, 0);
    std::vector<double> res_max(MS_MAXL, 0.0);
    double phase[kProf] = {};
    int fallbacks = 0, f64_fallbacks = 0;
    int dstat = 0;
    int solve_launches = 0, rhs_launch = 0;
    // blocks of at most Rmax right-hand sides; with 2 CTAs per SM up to kMaxParts blocks share one
    // partitioned launch (k_fit_parts), within a bound on the work vectors' size
    const int width = wide ? RWmax : Rmax;
    const int nblocks = (nrhs + Rmax - 1) / Rmax;
    int Pmax = 1;
    if (nblocks > 1 && ctas_per_sm(h->opts) == 2) {
        const int64_t cap = std::max<int64_t>(1, (int64_t)(256ll << 20) / std::max<int64_t>(1, (int64_t)width * N));
        Pmax = (int)std::min<int64_t>({(int64_t)nblocks, (int64_t)kMaxParts, cap, (int64_t)h->solve_blocks / 8});
        Pmax = std::max(Pmax, 1);
    }
    if (Pmax > 1) {
        MS_TRY(ms_ensure_workspace(h, width * Pmax));
        MS_TRY(ensure_parts(h, Pmax));
    }
    const int Vs = Rmax * L;  // virtual levels of a full block (the carving stride)
    for (int col0 = 0; col0 < nrhs;) {
        const int P = std::min(Pmax, (nrhs - col0 + Rmax - 1) / Rmax);
        int grid = h->solve_blocks;
        if (wide) MS_TRY(fit_blocks(mixed, 2, h->device, &grid, true));
        if (P > 1) {
            int g2 = 0;
            const void* fn = parts_kernel(mixed, wide);
            MS_CUDA(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sizeof(Shared)));
            int sms = 0, per_sm = 0;
            MS_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, h->device));
            MS_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, kBS, sizeof(Shared)));
            g2 = sms * std::min(per_sm, 2);
            grid = std::min(grid, g2);
        }
        grid = std::min(grid, h->solve_blocks);  // the reduction buffers hold solve_blocks CTAs
        std::vector<SolveArgs> as(P);
        std::vector<int> Rs(P);
        for (int p = 0; p < P; ++p) {
            const int cb = col0 + p * Rmax;
            const int R = std::min(Rmax, nrhs - cb);
            Rs[p] = R;
            SolveArgs& a = as[p];
            fill_args(h, rel_tol, R, a, wide, grid / P);
            const int64_t vo = (int64_t)p * width * N;  // this block's work vectors
            auto off64 = [&](double* q) { return q ? q + vo : q; };
            auto off32 = [&](float* q) { return q ? q + vo : q; };
            a.f = off64(h->f); a.beta = off64(h->beta); a.x = off64(h->x); a.r = off64(h->r);
            a.p = off64(h->p); a.q = off64(h->q); a.s = off64(h->s);
            a.x32 = off32(h->x32); a.r32 = off32(h->r32); a.p32 = off32(h->p32); a.q32 = off32(h->q32);
            a.s32 = off32(h->s32); a.u32 = off32(h->u32); a.u1_32 = off32(h->u1_32);
            if (P == 1) {
                a.part = h->part; a.gpart = h->gpart; a.scal = h->scal; a.resid = h->resid;
                a.bar = h->bar; a.status = h->status; a.iters = h->iters; a.refines = h->refines;
                a.bytes = h->bytes; a.prof = h->prof; a.pcfb = h->pcfb;
            } else {
                a.part = h->part + (size_t)kAcc * Vs * part_first_cta(p, grid, P);
                a.gpart = h->gpart + (size_t)p * kMaxGroups * kAcc * Vs;
                a.scal = h->scal + (size_t)p * kAcc * Vs;
                a.resid = h->resid + (size_t)p * Vs;
                const PartCounters c = part_counters(h, p);
                a.bar = c.bar; a.status = c.status; a.iters = c.iters; a.refines = c.refines;
                a.bytes = c.bytes; a.prof = c.prof; a.pcfb = c.pcfb;
            }
            if (wide) {
                k_gather_wide<<<nblk(N * a.RW, 256), 256, 0, st>>>(f_dev, h->f + vo, h->perm, N, nrhs, cb, R, a.RW);
                ms_count_launch();
                ++launches;
            } else {
                for (int r = 0; r < R; ++r) {
                    ms_gather_sorted(f_dev, h->f + vo + (int64_t)r * N, h->perm, N, nrhs, cb + r, st);
                    ++launches;
                }
            }
            MS_CUDA(cudaMemsetAsync(a.bar, 0, sizeof(unsigned) * kBarWords, st));
            MS_CUDA(cudaMemsetAsync(a.status, 0, sizeof(int), st));
            MS_CUDA(cudaMemsetAsync(a.resid, 0, sizeof(double) * a.V, st));
        }
        if (P > 1) MS_CUDA(cudaMemcpyAsync(h->d_args, as.data(), sizeof(SolveArgs) * P, cudaMemcpyHostToDevice, st));
        MS_CUDA(cudaEventRecord(h->ev0, st));
        if (P == 1) {
            void* args[] = {&as[0]};
            MS_CUDA(cudaLaunchCooperativeKernel(fit_kernel(mixed, ctas_per_sm(h->opts), wide), dim3(grid), dim3(kBS),
                                                args, sizeof(Shared), st));
        } else {
            const SolveArgs* da = static_cast<const SolveArgs*>(h->d_args);
            int np = P;
            void* args[] = {&da, &np};
            MS_CUDA(cudaLaunchCooperativeKernel(parts_kernel(mixed, wide), dim3(grid), dim3(kBS), args,
                                                sizeof(Shared), st));
        }
        ms_count_launch();
        MS_CUDA(cudaEventRecord(h->ev1, st));
        ++launches;
        ++solve_launches;
        rhs_launch = std::max(rhs_launch, nrhs - col0 < P * Rmax ? nrhs - col0 : P * Rmax);
        for (int p = 0; p < P; ++p) {
            const SolveArgs& a = as[p];
            const int cb = col0 + p * Rmax;
            if (wide) {
                k_scatter_wide<<<nblk(N * a.RW, 256), 256, 0, st>>>(a.x, alpha_dev, h->perm, N, nrhs, cb, Rs[p], a.RW);
                ms_count_launch();
                ++launches;
            } else {
                for (int r = 0; r < Rs[p]; ++r) {
                    ms_scatter_input(a.x + (int64_t)r * N, alpha_dev, h->perm, N, nrhs, cb + r, st);
                    ++launches;
                }
            }
        }
        MS_CUDA(cudaGetLastError());
        int tcs = 0;  // the tensor-core network that made the learned rows
        if (h->pc.tcstat && h->opts.precond == MS_PRECOND_LEARNED)
            MS_CUDA(cudaMemcpyAsync(&tcs, h->pc.tcstat, sizeof(int), cudaMemcpyDeviceToHost, st));
        std::vector<int> pst(P, 0), pfb(2 * P, 0);
        std::vector<int64_t> pit((size_t)P * MS_MAXL, 0);
        std::vector<int> pref((size_t)P * MS_MAXL, 0);
        std::vector<double> pres((size_t)P * Vs, 0.0), pb(P, 0.0);
        std::vector<unsigned long long> ppr((size_t)P * kProf, 0);
        for (int p = 0; p < P; ++p) {
            const SolveArgs& a = as[p];
            MS_CUDA(cudaMemcpyAsync(&pst[p], a.status, sizeof(int), cudaMemcpyDeviceToHost, st));
            MS_CUDA(cudaMemcpyAsync(&pit[(size_t)p * MS_MAXL], a.iters, sizeof(int64_t) * MS_MAXL,
                                    cudaMemcpyDeviceToHost, st));
            MS_CUDA(cudaMemcpyAsync(&pref[(size_t)p * MS_MAXL], a.refines, sizeof(int) * MS_MAXL,
                                    cudaMemcpyDeviceToHost, st));
            MS_CUDA(cudaMemcpyAsync(&pres[(size_t)p * Vs], a.resid, sizeof(double) * a.V, cudaMemcpyDeviceToHost, st));
            MS_CUDA(cudaMemcpyAsync(&pb[p], a.bytes, sizeof(double), cudaMemcpyDeviceToHost, st));
            MS_CUDA(cudaMemcpyAsync(&ppr[(size_t)p * kProf], a.prof, sizeof(unsigned long long) * kProf,
                                    cudaMemcpyDeviceToHost, st));
            MS_CUDA(cudaMemcpyAsync(&pfb[2 * p], a.pcfb, sizeof(int) * 2, cudaMemcpyDeviceToHost, st));
        }
        MS_CUDA(cudaStreamSynchronize(st));
        if (tcs != 0 && result == MS_OK) {
            result = (ms_status)tcs;
            ms_set_error(result, "a wait for the tensor-core network's MMAs ran out (the learned rows are not valid)");
        }
        float ms = 0.f;
        MS_CUDA(cudaEventElapsedTime(&ms, h->ev0, h->ev1));
        total_ms += ms;
        for (int i = 0; i < kProf; ++i) phase[i] += 1e-6 * (double)ppr[i];  // block 0's first CTA
        for (int p = 0; p < P; ++p) {
            bytes += pb[p];
            fallbacks += pfb[2 * p];
            f64_fallbacks += pfb[2 * p + 1];
            for (int l = 0; l < L; ++l) {
                it_sum[l] += pit[(size_t)p * MS_MAXL + l];
                ref_sum[l] += pref[(size_t)p * MS_MAXL + l];
                for (int r = 0; r < Rs[p]; ++r) res_max[l] = std::max(res_max[l], pres[(size_t)p * Vs + r * L + l]);
            }
            if (pst[p] != 0) dstat = dstat ? dstat : pst[p];
            if (pst[p] != 0 && result == MS_OK) {
                result = (ms_status)pst[p];
                ms_set_error(result, "device status %d during the fit of right-hand sides %d..%d", pst[p],
                             col0 + p * Rmax, col0 + p * Rmax + Rs[p] - 1);
            }
        }
        col0 += std::min(nrhs - col0, P * Rmax);
    }
    if (stats) {
        *stats = ms_fit_stats{};
        stats->L = L;
        stats->sweeps = ms_sweeps_of(h);
        for (int l = 0; l < L; ++l) {
            stats->cg_iterations[l] = it_sum[l];
            stats->refinements[l] = ref_sum[l];
            stats->rel_residual[l] = res_max[l];
        }
        stats->device_status = dstat;
        stats->fit_ms = total_ms;
        stats->matvec_bytes = bytes;
        stats->kernel_launches = launches;
        stats->solve_launches = solve_launches;
        stats->rhs_per_launch = rhs_launch;
        stats->precond_fallbacks = fallbacks;
        stats->fp64_fallbacks = f64_fallbacks;
        for (int i = 0; i < kProf; ++i) stats->phase_ms[i] = phase[i];
    }
    return result;
}

ms_status ms_apply_impl(ms_hierarchy* h, int op, const double* x_dev, double* y_dev, int sorted, cudaStream_t st) {
    MS_TRY(ms_ensure_workspace(h, std::max(h->ws_rhs, 1)));
    const int64_t N = h->N;
    const double* xs = x_dev;
    double* ys = y_dev;
    if (!sorted) {
        ms_gather_sorted(x_dev, h->tmp64, h->perm, N, 1, 0, st);
        xs = h->tmp64;
        ys = h->q;
    }
    if ((op == MS_APPLY_B64 || op == MS_APPLY_B32) && h->opts.lower_op == MS_OP_MATRIX_FREE) {
        ms_set_error(MS_ERR_ARG, "B is not stored (built with lower_op = MS_OP_MATRIX_FREE): use MS_APPLY_BMF32 or "
                     "MS_APPLY_BMFDF");
        return MS_ERR_ARG;
    }
    const DevCSR& M = (op == MS_APPLY_A64 || op == MS_APPLY_A32 || op == MS_APPLY_AMF32) ? h->A : h->B;
    const double avg = (double)M.nnz / (double)std::max<int64_t>(N, 1);
    const int S = (op <= MS_APPLY_AMF32 && h->opts.threads_per_row > 0) ? h->opts.threads_per_row : tpr_for(avg);
    const unsigned blocks = nblk(N * (int64_t)S, 256);
    switch (op) {
    case MS_APPLY_A64:
    case MS_APPLY_B64:
        k_spmv<double, double, double><<<blocks, 256, 0, st>>>(M.rp, M.col, M.v64, xs, ys, N, S, nullptr, 1.0);
        ms_count_launch();
        break;
    case MS_APPLY_A32:
    case MS_APPLY_B32: {
        if (!M.v32) {
            ms_set_error(MS_ERR_ARG, "FP32 values were not built (build with precision = MS_PREC_MIXED)");
            return MS_ERR_ARG;
        }
        float* x32 = reinterpret_cast<float*>(h->r);  // scratch: N floats fit in an N-double buffer
        k_to_f32<<<nblk(N, 256), 256, 0, st>>>(xs, x32, N);
        ms_count_launch();
        k_spmv<float, float, float><<<blocks, 256, 0, st>>>(M.rp, M.col, M.v32, x32, ys, N, S, nullptr, 1.0);
        ms_count_launch();
        break;
    }
    case MS_APPLY_AMF32: {
        float* x32 = reinterpret_cast<float*>(h->r);
        k_to_f32<<<nblk(N, 256), 256, 0, st>>>(xs, x32, N);
        ms_count_launch();
        const MFView v = make_mfview(h);
        k_mf_apply_staged<<<(unsigned)h->total_cells, 128, 0, st>>>(v, x32, ys, h->mf_tpp);
        ms_count_launch();
        break;
    }
    case MS_APPLY_BMF32:
    case MS_APPLY_BMFDF: {
        const bool dff = op == MS_APPLY_BMFDF;
        if (dff && !h->Wlo) {
            ms_set_error(MS_ERR_ARG, "MS_APPLY_BMFDF needs the double-float offsets of a MIXED build");
            return MS_ERR_ARG;
        }
        float* xhi = reinterpret_cast<float*>(h->r);  // scratch: 2 N floats fit in an N-double buffer
        float* xlo = xhi + N;
        if (dff) k_split_ff<<<nblk(N, 256), 256, 0, st>>>(xs, xhi, xlo, N);
        else k_to_f32<<<nblk(N, 256), 256, 0, st>>>(xs, xhi, N);
        ms_count_launch();
        HierView v = h->view;
        LowerF32 lf{};
        for (int i = 0; i < 4; ++i) lf.c[i] = (float)v.w.c[i];
        for (int l = 0; l < h->L; ++l) lf.ds[l] = (float)v.dscale[l];
        const FFLevels ffl = make_fflevels(v);
        const int Sl = 8;
        const unsigned nb = nblk(N * (int64_t)Sl, 256);
        if (dff)
            k_lower_mf_apply<true><<<nb, 256, 0, st>>>(v, h->W, h->Wlo, h->cellid, ffl, lf, xhi, xlo, ys, Sl);
        else
            k_lower_mf_apply<false><<<nb, 256, 0, st>>>(v, h->W, h->Wlo, h->cellid, ffl, lf, xhi, nullptr, ys, Sl);
        ms_count_launch();
        break;
    }
    default:
        ms_set_error(MS_ERR_ARG, "operator %d is not available", op);
        return MS_ERR_ARG;
    }
    MS_CUDA(cudaGetLastError());
    if (!sorted) ms_scatter_input(ys, y_dev, h->perm, N, 1, 0, st);
    MS_CUDA(cudaGetLastError());
    return MS_OK;
}

// ---------------------------------------------------------------- allocation-free fit
//
// ms_fit_dev gives the handle a work space on its first call (cudaMalloc).
// Some callers cannot allow that at fit time: applications whose device memory
// is already fully reserved by another allocator or pool (a fresh cudaMalloc
// would fail), latency-critical loops that must not call the allocator
// (cudaMalloc and cudaFree can synchronise the device), and processes whose
// device-memory budget is fixed at start-up.  ms_fit_static_dev serves them:
// it runs the same solve kernel, with its work space (solve vectors, reduction
// partials, barrier words, status and counters) in the fixed device array
// below instead of memory the call allocates.  The array belongs to the loaded
// module, so every GPU that loads libms.so holds it until the process exits.

#include <mutex>

namespace {

constexpr int64_t kStaticMaxPoints = 65536;  // largest hierarchy (total points) the array serves
constexpr int kStaticMaxBlocks = 1024;       // largest cooperative grid it serves
constexpr size_t pad256(size_t b) { return (b + 255) / 256 * 256; }
constexpr size_t kStaticVec64 = pad256(sizeof(double) * kStaticMaxPoints);
constexpr size_t kStaticVec32 = pad256(sizeof(float) * kStaticMaxPoints);
constexpr size_t kStaticPart = pad256(sizeof(double) * kAcc * MS_MAXL * kStaticMaxBlocks);
constexpr size_t kStaticGpart = pad256(sizeof(double) * kMaxGroups * kAcc * MS_MAXL);
constexpr size_t kStaticSmall = 4096;  // barrier words, status, per-level counters, residuals, sums
constexpr size_t kStaticBytes =
    7 * kStaticVec64 + 5 * kStaticVec32 + kStaticPart + kStaticGpart + kStaticSmall;
static_assert(kStaticBytes == 5820416, "the header documents the array as about 5.6 MiB (5,820,416 bytes)");

}  // namespace

static __device__ __align__(256) unsigned char g_fit_scratch[kStaticBytes];

namespace {

std::mutex g_scratch_mu;
void* g_scratch_addr[256] = {};

// Device address of g_fit_scratch on device `dev` (which must be current),
// looked up once per device and cached for the process.  In host code the name
// g_fit_scratch is only a host-side stand-in: it must never be handed to a kernel.
// A cudaDeviceReset ends the context the cached address belongs to; like every
// handle of that device, the cache is then invalid (the library does not support
// use across a reset).
ms_status fit_scratch_address(int dev, unsigned char** out) {
    if (dev < 0 || dev >= 256) {
        ms_set_error(MS_ERR_STATE, "device ordinal %d out of range", dev);
        return MS_ERR_STATE;
    }
    std::lock_guard<std::mutex> lock(g_scratch_mu);
    if (!g_scratch_addr[dev]) {
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_fit_scratch);
        if (e != cudaSuccess) return ms_cuda_error(e, "cudaGetSymbolAddress(g_fit_scratch)", __FILE__, __LINE__);
        g_scratch_addr[dev] = p;
    }
    *out = static_cast<unsigned char*>(g_scratch_addr[dev]);
    return MS_OK;
}

}  // namespace

extern "C" ms_status ms_fit_static_dev(ms_hierarchy* h, const double* f_dev, double rel_tol, double* alpha_dev,
                                       ms_fit_stats* stats, void* stream) {
    ms_clear_error();
    if (!h || !f_dev || !alpha_dev) {
        ms_set_error(MS_ERR_ARG, "handle, f and alpha must not be NULL");
        return MS_ERR_ARG;
    }
    if (!(rel_tol > 0.0 && rel_tol < 1.0)) {
        ms_set_error(MS_ERR_ARG, "rel_tol must be in (0, 1) (got %g)", rel_tol);
        return MS_ERR_ARG;
    }
    if (h->N > kStaticMaxPoints) {
        ms_set_error(MS_ERR_ARG, "hierarchy has %lld points; the allocation-free fit serves at most %lld",
                     (long long)h->N, (long long)kStaticMaxPoints);
        return MS_ERR_ARG;
    }
    const bool mixed = h->opts.precision == MS_PREC_MIXED;
    if (mixed && h->opts.op != MS_OP_MATRIX_FREE && !h->A.v32) {
        ms_set_error(MS_ERR_STATE, "MIXED fit needs FP32 values (build with precision = MS_PREC_MIXED)");
        return MS_ERR_STATE;
    }
    if (h->opts.precond != MS_PRECOND_NONE) {
        ms_set_error(MS_ERR_STATE, "the allocation-free fit does not apply a preconditioner (precond must be NONE)");
        return MS_ERR_STATE;
    }
    int dev = 0;
    MS_CUDA(cudaGetDevice(&dev));
    if (dev != h->device) {
        ms_set_error(MS_ERR_STATE, "the handle belongs to device %d but device %d is current", h->device, dev);
        return MS_ERR_STATE;
    }
    unsigned char* base = nullptr;
    MS_TRY(fit_scratch_address(dev, &base));
    cudaStream_t st = (cudaStream_t)stream;

    int blocks = 0;
    const int minb = ctas_per_sm(h->opts);
    MS_TRY(fit_blocks(mixed, minb, dev, &blocks));
    blocks = std::min(blocks, kStaticMaxBlocks);

    // carve the fixed array
    unsigned char* c = base;
    double* v64[7];
    for (int i = 0; i < 7; ++i, c += kStaticVec64) v64[i] = reinterpret_cast<double*>(c);
    float* v32[5];
    for (int i = 0; i < 5; ++i, c += kStaticVec32) v32[i] = reinterpret_cast<float*>(c);
    double* part = reinterpret_cast<double*>(c);
    c += kStaticPart;
    double* gpart = reinterpret_cast<double*>(c);
    c += kStaticGpart;
    unsigned char* small = c;
    int* status = reinterpret_cast<int*>(small + 64);                      // [1]
    int64_t* iters = reinterpret_cast<int64_t*>(small + 128);              // [MS_MAXL]
    int* refines = reinterpret_cast<int*>(small + 128 + 8 * MS_MAXL);      // [MS_MAXL]
    double* resid = reinterpret_cast<double*>(small + 128 + 12 * MS_MAXL); // [MS_MAXL]
    double* bytes = reinterpret_cast<double*>(small + 128 + 20 * MS_MAXL); // [1]
    double* scal = reinterpret_cast<double*>(small + 1024);                // [kAcc][MS_MAXL]
    unsigned* bar = reinterpret_cast<unsigned*>(small + 2560);             // [kBarWords]
    // the array keeps the previous call's contents: clear what must start at zero
    MS_CUDA(cudaMemsetAsync(small, 0, kStaticSmall, st));

    const int L = h->L;
    SolveArgs a{};
    fill_args(h, rel_tol, 1, a, false, blocks);  // the chunking ms_fit_dev uses on the same grid
    a.f = v64[0]; a.beta = v64[1]; a.x = v64[2]; a.r = v64[3]; a.p = v64[4]; a.q = v64[5]; a.s = v64[6];
    a.x32 = v32[0]; a.r32 = v32[1]; a.p32 = v32[2]; a.q32 = v32[3]; a.s32 = v32[4];
    a.part = part; a.gpart = gpart; a.scal = scal; a.bar = bar; a.status = status;
    a.iters = iters; a.refines = refines; a.resid = resid; a.bytes = bytes;
    a.prof = reinterpret_cast<unsigned long long*>(small + 2048);  // [kProf]
    a.pcfb = reinterpret_cast<int*>(small + 3072);                 // [2]
    a.pc = 0;  // the allocation-free fit runs without a preconditioner (checked above)
    // lanes per target point of the matrix-free operator as ms_fit_dev chooses them, also on a
    // handle that has never been fitted
    a.mf_tpp = h->mf_tpp_tuned > 0 ? h->mf_tpp_tuned : mf_tpp_for(h);

    ms_gather_sorted(f_dev, v64[0], h->perm, h->N, 1, 0, st);
    void* args[] = {&a};
    MS_CUDA(cudaEventRecord(h->ev0, st));
    MS_CUDA(cudaLaunchCooperativeKernel(fit_kernel(mixed, minb), dim3(blocks), dim3(kBS), args, sizeof(Shared), st));
    ms_count_launch();
    MS_CUDA(cudaEventRecord(h->ev1, st));
    ms_scatter_input(a.x, alpha_dev, h->perm, h->N, 1, 0, st);
    MS_CUDA(cudaGetLastError());

    int dstat = 0;
    int64_t it[MS_MAXL];
    int ref[MS_MAXL];
    double res[MS_MAXL], b = 0.0;
    unsigned long long pr[kProf];
    int fb[2] = {0, 0};
    MS_CUDA(cudaMemcpyAsync(&dstat, status, sizeof(int), cudaMemcpyDeviceToHost, st));
    MS_CUDA(cudaMemcpyAsync(it, iters, sizeof(it), cudaMemcpyDeviceToHost, st));
    MS_CUDA(cudaMemcpyAsync(ref, refines, sizeof(ref), cudaMemcpyDeviceToHost, st));
    MS_CUDA(cudaMemcpyAsync(res, resid, sizeof(res), cudaMemcpyDeviceToHost, st));
    MS_CUDA(cudaMemcpyAsync(&b, bytes, sizeof(double), cudaMemcpyDeviceToHost, st));
    MS_CUDA(cudaMemcpyAsync(pr, a.prof, sizeof(pr), cudaMemcpyDeviceToHost, st));
    MS_CUDA(cudaMemcpyAsync(fb, a.pcfb, sizeof(fb), cudaMemcpyDeviceToHost, st));
    MS_CUDA(cudaStreamSynchronize(st));
    float ms = 0.f;
    MS_CUDA(cudaEventElapsedTime(&ms, h->ev0, h->ev1));
    if (stats) {
        *stats = ms_fit_stats{};
        stats->L = L;
        stats->sweeps = a.sweeps;
        for (int l = 0; l < L; ++l) {
            stats->cg_iterations[l] = it[l];
            stats->refinements[l] = ref[l];
            stats->rel_residual[l] = res[l];
        }
        stats->device_status = dstat;
        stats->fit_ms = ms;
        stats->matvec_bytes = b;
        stats->kernel_launches = 3;
        stats->solve_launches = 1;
        stats->rhs_per_launch = 1;
        stats->precond_fallbacks = fb[0];
        stats->fp64_fallbacks = fb[1];
        for (int i = 0; i < kProf; ++i) stats->phase_ms[i] = 1e-6 * (double)pr[i];
    }
    if (dstat != 0) {
        ms_set_error((ms_status)dstat, "device status %d during the allocation-free fit", dstat);
        return (ms_status)dstat;
    }
    return MS_OK;
}

// ---------------------------------------------------------------- bounded-wait self-test

namespace {

// One CTA in a partition of `pretend` CTAs enters the solve kernel's grid barrier; the
// others never arrive.
__global__ void __launch_bounds__(kBS) k_wait_selftest(const __grid_constant__ SolveArgs a, unsigned pretend) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    Shared& sh = *reinterpret_cast<Shared*>(smem_raw);
    if (threadIdx.x == 0) {
        sh.cta = 0;
        sh.nb = (int)pretend;
        sh.tprev = ms_globaltimer();
        for (int k = 0; k < kProf; ++k) sh.pt[k] = 0ull;
    }
    __syncthreads();
    gsync(a, sh);
}

}  // namespace

extern "C" ms_status ms_wait_selftest(double timeout_s, int peer_timed_out, int* device_status, double* waited_s) {
    if (!device_status || !(timeout_s > 0.0 && timeout_s <= 10.0)) {
        ms_set_error(MS_ERR_ARG, "timeout_s must be in (0, 10] and device_status non-NULL");
        return MS_ERR_ARG;
    }
    struct Buf {
        void* p = nullptr;
        cudaEvent_t e0 = nullptr, e1 = nullptr;
        ~Buf() {
            if (p) cudaFree(p);
            if (e0) cudaEventDestroy(e0);
            if (e1) cudaEventDestroy(e1);
        }
    } b;
    const size_t bar_bytes = sizeof(unsigned) * kBarWords;
    MS_CUDA(cudaMalloc(&b.p, bar_bytes + sizeof(int)));
    MS_CUDA(cudaMemset(b.p, 0, bar_bytes + sizeof(int)));
    int* status = reinterpret_cast<int*>(static_cast<char*>(b.p) + bar_bytes);
    if (peer_timed_out) {
        const int t = MS_ERR_TIMEOUT;
        MS_CUDA(cudaMemcpy(status, &t, sizeof(int), cudaMemcpyHostToDevice));
    }
    SolveArgs a{};
    a.bar = static_cast<unsigned*>(b.p);
    a.status = status;
    a.timeout_ns = (unsigned long long)(timeout_s * 1e9);
    MS_CUDA(cudaFuncSetAttribute(k_wait_selftest, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sizeof(Shared)));
    MS_CUDA(cudaEventCreate(&b.e0));
    MS_CUDA(cudaEventCreate(&b.e1));
    MS_CUDA(cudaEventRecord(b.e0, 0));
    k_wait_selftest<<<1, kBS, sizeof(Shared), 0>>>(a, 2u);
    ms_count_launch();
    MS_CUDA(cudaGetLastError());
    MS_CUDA(cudaEventRecord(b.e1, 0));
    MS_CUDA(cudaEventSynchronize(b.e1));
    float ms = 0.f;
    MS_CUDA(cudaEventElapsedTime(&ms, b.e0, b.e1));
    MS_CUDA(cudaMemcpy(device_status, status, sizeof(int), cudaMemcpyDeviceToHost));
    if (waited_s) *waited_s = 1e-3 * (double)ms;
    return MS_OK;
}
