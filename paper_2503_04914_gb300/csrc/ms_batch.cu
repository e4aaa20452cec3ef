// Batched fit of several independent hierarchies in ONE persistent cooperative
// launch.  The grid is split into partitions of consecutive CTAs, one per
// hierarchy, sized in proportion to the hierarchy's work (its A nonzeros plus
// points); every partition runs the whole schedule of eq. split for its
// hierarchy (the same device code as the single fit) with a grid barrier and
// reductions of its own, so small hierarchies do not wait on large ones and a
// barrier among a few CTAs costs far less than one among all of them.
#include <algorithm>
#include <cmath>
#include <numeric>
#include <vector>

#include "ms_solve_dev.cuh"

namespace {

// Partition g = the CTAs [cta0[g], cta0[g + 1]).
template <int MODE>
__global__ void __launch_bounds__(kBS, 2) k_fit_multi(const SolveArgs* __restrict__ args,
                                                      const int* __restrict__ cta0, int ng) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    Shared& sh = *reinterpret_cast<Shared*>(smem_raw);
    __shared__ int part_id;
    if (threadIdx.x == 0) {
        int lo = 0, hi = ng - 1;  // the last g with cta0[g] <= blockIdx.x
        while (lo < hi) {
            const int mid = (lo + hi + 1) / 2;
            if (cta0[mid] <= (int)blockIdx.x) lo = mid;
            else hi = mid - 1;
        }
        part_id = lo;
        sh.cta = (int)blockIdx.x - cta0[lo];
        sh.nb = cta0[lo + 1] - cta0[lo];
    }
    __syncthreads();
    fit_body<MODE>(args[part_id], sh);
}

// Zero every partition's barrier words, status and residuals (block g: hierarchy g).
__global__ void k_batch_reset(const SolveArgs* args) {
    const SolveArgs& a = args[blockIdx.x];
    for (int i = threadIdx.x; i < kBarWords; i += blockDim.x) a.bar[i] = 0u;
    for (int i = threadIdx.x; i < a.V; i += blockDim.x) a.resid[i] = 0.0;
    if (threadIdx.x == 0) *a.status = 0;
}

// Per-hierarchy results gathered into one array (one device-to-host copy).
struct BatchStat {
    int status, pcfb, f64fb;
    double bytes;
    long long iters[MS_MAXL];
    int refines[MS_MAXL];
    double resid[MS_MAXL];
    unsigned long long prof[kProf];
};

__global__ void k_batch_stats(const SolveArgs* args, BatchStat* out) {
    const SolveArgs& a = args[blockIdx.x];
    BatchStat& o = out[blockIdx.x];
    const int t = threadIdx.x;
    if (t < a.L) {
        o.iters[t] = a.iters[t];
        o.refines[t] = a.refines[t];
        o.resid[t] = a.resid[t];
    }
    if (t < kProf) o.prof[t] = a.prof[t];
    if (t == 0) {
        o.status = *a.status;
        o.pcfb = a.pcfb[0];
        o.f64fb = a.pcfb[1];
        o.bytes = *a.bytes;
    }
}

const void* multi_kernel(bool mixed) { return mixed ? (const void*)k_fit_multi<1> : (const void*)k_fit_multi<0>; }

// CTAs of one launch: 2 per SM (the kernel's register budget), at most kMaxGroups * kGroup.
ms_status multi_blocks(bool mixed, int dev, int* blocks) {
    const void* fn = multi_kernel(mixed);
    MS_CUDA(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sizeof(Shared)));
    int sms = 0, per_sm = 0;
    MS_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    MS_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, kBS, sizeof(Shared)));
    if (per_sm < 1) {
        ms_set_error(MS_ERR_CUDA, "batched solve kernel cannot be resident on an SM");
        return MS_ERR_CUDA;
    }
    *blocks = std::min(sms * std::min(per_sm, 2), kMaxGroups * kGroup);
    return MS_OK;
}

// Split `total` CTAs among the hierarchies in proportion to their work: at least one
// each, at most cap[i] (the size of hierarchy i's reduction buffers).  Requires
// work.size() <= total.
std::vector<int> partition(const std::vector<double>& work, const std::vector<int>& cap, int total) {
    const size_t n = work.size();
    const double sum = std::accumulate(work.begin(), work.end(), 0.0);
    std::vector<double> want(n);
    std::vector<int> c(n);
    long used = 0;
    for (size_t i = 0; i < n; ++i) {
        want[i] = sum > 0 ? total * work[i] / sum : (double)total / n;
        c[i] = std::max(1, std::min(cap[i], (int)want[i]));
        used += c[i];
    }
    // lifting tiny shares to one CTA can overshoot: take back from the largest
    while (used > total) {
        const size_t i = std::max_element(c.begin(), c.end()) - c.begin();
        --c[i];
        --used;
    }
    // hand out the rest by the largest shortfall
    while (used < total) {
        size_t best = n;
        double gap = 0.0;
        for (size_t i = 0; i < n; ++i)
            if (c[i] < cap[i] && want[i] - c[i] > gap) {
                gap = want[i] - c[i];
                best = i;
            }
        if (best == n) break;
        ++c[best];
        ++used;
    }
    return c;
}

struct StreamBuf {
    void* p = nullptr;
    cudaStream_t s = nullptr;
    ~StreamBuf() { if (p) cudaFreeAsync(p, s); }
};

}  // namespace

ms_status ms_fit_batch_impl(ms_hierarchy* const* hs, int nh, const double* const* f_dev, double rel_tol,
                            double* const* alpha_dev, ms_fit_stats* stats, cudaStream_t st) {
    int dev = 0;
    MS_CUDA(cudaGetDevice(&dev));
    const bool mixed = hs[0]->opts.precision == MS_PREC_MIXED;
    for (int i = 0; i < nh; ++i) {
        ms_hierarchy* h = hs[i];
        if (h->device != dev) {
            ms_set_error(MS_ERR_STATE, "hierarchy %d belongs to device %d but device %d is current", i, h->device, dev);
            return MS_ERR_STATE;
        }
        if ((h->opts.precision == MS_PREC_MIXED) != mixed) {
            ms_set_error(MS_ERR_ARG, "all hierarchies of a batch must have the same precision (hierarchy %d differs)", i);
            return MS_ERR_ARG;
        }
        if (mixed && h->opts.op != MS_OP_MATRIX_FREE && !h->A.v32) {
            ms_set_error(MS_ERR_STATE, "hierarchy %d: MIXED fit needs FP32 values", i);
            return MS_ERR_STATE;
        }
        if (h->opts.precond != MS_PRECOND_NONE && !mixed) {
            ms_set_error(MS_ERR_ARG, "hierarchy %d: a preconditioner needs precision = MS_PREC_MIXED", i);
            return MS_ERR_ARG;
        }
        MS_TRY(ms_ensure_workspace(h, 1));
        if (h->opts.precond != MS_PRECOND_NONE) MS_TRY(ms_pc_build(h, h->opts.precond, st));
    }
    int total = 0;
    MS_TRY(multi_blocks(mixed, dev, &total));

    std::vector<BatchStat> hst(nh);
    float kernel_ms = 0.f;
    int launches = 0;
    ms_status result = MS_OK;
    // waves of at most `total` hierarchies (one CTA each at least)
    for (int w0 = 0; w0 < nh; w0 += total) {
        const int n = std::min(total, nh - w0);
        std::vector<double> work(n);
        std::vector<int> cap(n);
        std::vector<SolveArgs> args(n);
        for (int i = 0; i < n; ++i) {
            ms_hierarchy* h = hs[w0 + i];
            work[i] = (double)h->A.nnz + 4.0 * (double)h->N;
            cap[i] = h->solve_blocks;
            SolveArgs& a = args[i];
            fill_args(h, rel_tol, 1, a);
            a.f = h->f; a.beta = h->beta; a.x = h->x; a.r = h->r; a.p = h->p; a.q = h->q; a.s = h->s;
            a.x32 = h->x32; a.r32 = h->r32; a.p32 = h->p32; a.q32 = h->q32; a.s32 = h->s32;
            a.u32 = h->u32; a.u1_32 = h->u1_32;
            a.part = h->part; a.gpart = h->gpart; a.scal = h->scal; a.bar = h->bar; a.status = h->status;
            a.iters = h->iters; a.refines = h->refines; a.resid = h->resid; a.bytes = h->bytes; a.prof = h->prof;
            a.pcfb = h->pcfb;
        }
        const std::vector<int> cnt = partition(work, cap, total);
        std::vector<int> cta0(n + 1, 0);
        for (int i = 0; i < n; ++i) cta0[i + 1] = cta0[i] + cnt[i];
        const int grid = cta0[n];

        StreamBuf dargs, dcta, dstat;
        dargs.s = dcta.s = dstat.s = st;
        MS_CUDA(cudaMallocAsync(&dargs.p, sizeof(SolveArgs) * n, st));
        MS_CUDA(cudaMallocAsync(&dcta.p, sizeof(int) * (n + 1), st));
        MS_CUDA(cudaMallocAsync(&dstat.p, sizeof(BatchStat) * n, st));
        MS_CUDA(cudaMemcpyAsync(dargs.p, args.data(), sizeof(SolveArgs) * n, cudaMemcpyHostToDevice, st));
        MS_CUDA(cudaMemcpyAsync(dcta.p, cta0.data(), sizeof(int) * (n + 1), cudaMemcpyHostToDevice, st));
        for (int i = 0; i < n; ++i) {
            ms_hierarchy* h = hs[w0 + i];
            ms_gather_sorted(f_dev[w0 + i], h->f, h->perm, h->N, 1, 0, st);
            ++launches;
        }
        k_batch_reset<<<n, 128, 0, st>>>((const SolveArgs*)dargs.p);
        ms_count_launch();
        ++launches;
        const SolveArgs* pa = (const SolveArgs*)dargs.p;
        const int* pc = (const int*)dcta.p;
        int ng = n;
        void* kargs[] = {&pa, &pc, &ng};
        MS_CUDA(cudaEventRecord(hs[0]->ev0, st));
        MS_CUDA(cudaLaunchCooperativeKernel(multi_kernel(mixed), dim3(grid), dim3(kBS), kargs, sizeof(Shared), st));
        ms_count_launch();
        ++launches;
        MS_CUDA(cudaEventRecord(hs[0]->ev1, st));
        for (int i = 0; i < n; ++i) {
            ms_hierarchy* h = hs[w0 + i];
            ms_scatter_input(h->x, alpha_dev[w0 + i], h->perm, h->N, 1, 0, st);
            ++launches;
        }
        k_batch_stats<<<n, 64, 0, st>>>((const SolveArgs*)dargs.p, (BatchStat*)dstat.p);
        ms_count_launch();
        ++launches;
        MS_CUDA(cudaGetLastError());
        MS_CUDA(cudaMemcpyAsync(hst.data() + w0, dstat.p, sizeof(BatchStat) * n, cudaMemcpyDeviceToHost, st));
        MS_CUDA(cudaStreamSynchronize(st));
        float ms = 0.f;
        MS_CUDA(cudaEventElapsedTime(&ms, hs[0]->ev0, hs[0]->ev1));
        kernel_ms += ms;
    }
    for (int i = 0; i < nh; ++i) {
        const BatchStat& b = hst[i];
        if (b.status != 0 && result == MS_OK) {
            result = (ms_status)b.status;
            ms_set_error(result, "device status %d in the fit of hierarchy %d of the batch", b.status, i);
        }
        if (!stats) continue;
        ms_fit_stats& s = stats[i];
        s = ms_fit_stats{};
        const ms_hierarchy* h = hs[i];
        s.L = h->L;
        s.sweeps = h->opts.jacobi_sweeps > 0 ? h->opts.jacobi_sweeps : std::max(h->L - 1, 0);
        for (int l = 0; l < h->L; ++l) {
            s.cg_iterations[l] = b.iters[l];
            s.refinements[l] = b.refines[l];
            s.rel_residual[l] = b.resid[l];
        }
        s.precond_fallbacks = b.pcfb;
        s.fp64_fallbacks = b.f64fb;
        s.device_status = b.status;
        s.fit_ms = kernel_ms;  // the batch's launches, shared by all its hierarchies
        s.matvec_bytes = b.bytes;
        s.kernel_launches = launches;
        for (int k = 0; k < kProf; ++k) s.phase_ms[k] = 1e-6 * (double)b.prof[k];
    }
    return result;
}
