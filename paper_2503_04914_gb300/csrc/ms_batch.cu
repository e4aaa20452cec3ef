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

// Input/output binding of one hierarchy of a plan: its right-hand side and
// coefficients (caller's device buffers, input order) and its sorted work vectors.
struct BatchIO {
    const double* f;
    double* alpha;
    const int32_t* perm;  // sorted position -> input index
    double* fs;           // the hierarchy's sorted right-hand side (work vector f)
    const double* xs;     // the hierarchy's sorted solution (work vector x)
    int64_t N;
};

// f -> sorted work vector, every hierarchy of a wave in one launch (blockIdx.y = hierarchy).
__global__ void k_batch_gather(const BatchIO* io) {
    const BatchIO& b = io[blockIdx.y];
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < b.N; i += (int64_t)gridDim.x * blockDim.x)
        b.fs[i] = b.f[b.perm[i]];
}

// sorted solution -> alpha in input order.
__global__ void k_batch_scatter(const BatchIO* io) {
    const BatchIO& b = io[blockIdx.y];
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < b.N; i += (int64_t)gridDim.x * blockDim.x)
        b.alpha[b.perm[i]] = b.xs[i];
}

constexpr int kPlanLaunchesPerWave = 5;  // gather, reset, solve, scatter, stats

}  // namespace

// A prepared batch: every host-side step of the batched fit done once, the device
// arguments uploaded, so that a launch only enqueues kernels.
struct ms_batch_plan {
    int dev = 0;
    bool mixed = false;
    int nh = 0;
    std::vector<ms_hierarchy*> hs;
    std::vector<int> w0;    // hierarchies [w0[w], w0[w + 1]) form wave w
    std::vector<int> grid;  // CTAs of wave w
    std::vector<int> coff;  // wave w's partition offsets start at d_cta + coff[w]
    unsigned gather_x = 1;  // grid.x of the gather / scatter launches
    void* mem = nullptr;    // one pool allocation holding the arrays below
    SolveArgs* d_args = nullptr;  // [nh]
    BatchIO* d_io = nullptr;      // [nh]
    BatchStat* d_stat = nullptr;  // [nh]
    int* d_cta = nullptr;
    cudaStream_t cap = nullptr;   // private stream for graph capture
    cudaGraphExec_t exec = nullptr;
    bool valid = true;            // false once a hierarchy of the plan was destroyed
};

namespace {

size_t pad256(size_t b) { return (b + 255) / 256 * 256; }

// Enqueue every wave on st; e0/e1 (nullable) bracket the solve launches.
ms_status plan_enqueue(const ms_batch_plan* p, cudaStream_t st, cudaEvent_t e0, cudaEvent_t e1) {
    const void* fn = multi_kernel(p->mixed);
    const int nw = (int)p->grid.size();
    for (int w = 0; w < nw; ++w) {
        const int a0 = p->w0[w], n = p->w0[w + 1] - a0;
        k_batch_gather<<<dim3(p->gather_x, n), 256, 0, st>>>(p->d_io + a0);
        k_batch_reset<<<n, 128, 0, st>>>(p->d_args + a0);
        const SolveArgs* pa = p->d_args + a0;
        const int* pc = p->d_cta + p->coff[w];
        int ng = n;
        void* kargs[] = {&pa, &pc, &ng};
        if (e0 && w == 0) MS_CUDA(cudaEventRecord(e0, st));
        MS_CUDA(cudaLaunchCooperativeKernel(fn, dim3(p->grid[w]), dim3(kBS), kargs, sizeof(Shared), st));
        if (e1 && w == nw - 1) MS_CUDA(cudaEventRecord(e1, st));
        k_batch_scatter<<<dim3(p->gather_x, n), 256, 0, st>>>(p->d_io + a0);
        k_batch_stats<<<n, 64, 0, st>>>(p->d_args + a0, p->d_stat + a0);
        MS_CUDA(cudaGetLastError());
    }
    return MS_OK;
}

int plan_launches(const ms_batch_plan* p) { return kPlanLaunchesPerWave * (int)p->grid.size(); }

}  // namespace

// device_sync: wait for every launch of the plan first (the caller has not synchronised).
void ms_batch_plan_free(ms_batch_plan* p, bool device_sync) {
    if (!p) return;
    if (device_sync) cudaDeviceSynchronize();
    if (p->exec) cudaGraphExecDestroy(p->exec);
    if (p->cap) cudaStreamDestroy(p->cap);
    if (p->mem) ms_pool_free(p->mem);
    for (ms_hierarchy* h : p->hs)
        if (h) h->plans.erase(std::remove(h->plans.begin(), h->plans.end(), p), h->plans.end());
    delete p;
}

void ms_batch_plan_detach(ms_batch_plan* p, const ms_hierarchy* h) {
    for (ms_hierarchy*& q : p->hs)
        if (q == h) q = nullptr;
    p->valid = false;
}

ms_status ms_batch_plan_create_impl(ms_hierarchy* const* hs, int nh, const double* const* f_dev, double rel_tol,
                                    double* const* alpha_dev, cudaStream_t st, ms_batch_plan** out) {
    *out = nullptr;
    int dev = 0;
    MS_CUDA(cudaGetDevice(&dev));
    const bool mixed = hs[0]->opts.precision == MS_PREC_MIXED;
    {
        std::vector<const ms_hierarchy*> sorted(hs, hs + nh);
        std::sort(sorted.begin(), sorted.end());
        if (std::adjacent_find(sorted.begin(), sorted.end()) != sorted.end()) {
            ms_set_error(MS_ERR_ARG, "a hierarchy appears twice in the batch (they would share work space)");
            return MS_ERR_ARG;
        }
    }
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
        MS_TRY(ms_autotune(h, st));
    }
    int total = 0;
    MS_TRY(multi_blocks(mixed, dev, &total));

    ms_batch_plan* p = new ms_batch_plan();
    p->dev = dev;
    p->mixed = mixed;
    p->nh = nh;
    std::vector<SolveArgs> args(nh);
    std::vector<BatchIO> io(nh);
    std::vector<int> cta;
    int64_t maxN = 1;
    // waves of at most `total` hierarchies (one CTA each at least)
    for (int a0 = 0; a0 < nh; a0 += total) {
        const int n = std::min(total, nh - a0);
        std::vector<double> work(n);
        std::vector<int> cap(n);
        for (int i = 0; i < n; ++i) {
            ms_hierarchy* h = hs[a0 + i];
            work[i] = (double)h->A.nnz + 4.0 * (double)h->N;
            cap[i] = h->solve_blocks;
            SolveArgs& a = args[a0 + i];
            fill_args(h, rel_tol, 1, a);
            a.f = h->f; a.beta = h->beta; a.x = h->x; a.r = h->r; a.p = h->p; a.q = h->q; a.s = h->s;
            a.x32 = h->x32; a.r32 = h->r32; a.p32 = h->p32; a.q32 = h->q32; a.s32 = h->s32;
            a.u32 = h->u32; a.u1_32 = h->u1_32;
            a.part = h->part; a.gpart = h->gpart; a.scal = h->scal; a.bar = h->bar; a.status = h->status;
            a.iters = h->iters; a.refines = h->refines; a.resid = h->resid; a.bytes = h->bytes; a.prof = h->prof;
            a.pcfb = h->pcfb;
            io[a0 + i] = BatchIO{f_dev[a0 + i], alpha_dev[a0 + i], h->perm, h->f, h->x, h->N};
            maxN = std::max(maxN, h->N);
        }
        const std::vector<int> cnt = partition(work, cap, total);
        p->w0.push_back(a0);
        p->coff.push_back((int)cta.size());
        int c = 0;
        cta.push_back(0);
        for (int i = 0; i < n; ++i) cta.push_back(c += cnt[i]);
        p->grid.push_back(c);
    }
    p->w0.push_back(nh);
    p->gather_x = (unsigned)std::min<int64_t>((maxN + 255) / 256, 2048);
    const size_t bA = pad256(sizeof(SolveArgs) * nh), bI = pad256(sizeof(BatchIO) * nh),
                 bS = pad256(sizeof(BatchStat) * nh), bC = pad256(sizeof(int) * cta.size());
    ms_status s = ms_pool_alloc(&p->mem, bA + bI + bS + bC);
    if (s == MS_OK) {
        unsigned char* m = (unsigned char*)p->mem;
        p->d_args = (SolveArgs*)m;
        p->d_io = (BatchIO*)(m + bA);
        p->d_stat = (BatchStat*)(m + bA + bI);
        p->d_cta = (int*)(m + bA + bI + bS);
        cudaError_t e = cudaMemcpyAsync(p->d_args, args.data(), sizeof(SolveArgs) * nh, cudaMemcpyHostToDevice, st);
        if (e == cudaSuccess) e = cudaMemcpyAsync(p->d_io, io.data(), sizeof(BatchIO) * nh, cudaMemcpyHostToDevice, st);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(p->d_cta, cta.data(), sizeof(int) * cta.size(), cudaMemcpyHostToDevice, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);  // the host arrays go out of scope
        if (e != cudaSuccess) s = ms_cuda_error(e, "batch plan upload", __FILE__, __LINE__);
    }
    p->hs.assign(hs, hs + nh);
    for (ms_hierarchy* h : p->hs) h->plans.push_back(p);
    if (s != MS_OK) {
        ms_batch_plan_free(p, true);
        return s;
    }
    *out = p;
    return MS_OK;
}

ms_status ms_batch_plan_launch_impl(ms_batch_plan* p, cudaStream_t st, int use_graph) {
    int dev = 0;
    MS_CUDA(cudaGetDevice(&dev));
    if (dev != p->dev) {
        ms_set_error(MS_ERR_STATE, "the plan belongs to device %d but device %d is current", p->dev, dev);
        return MS_ERR_STATE;
    }
    if (!p->valid) {
        ms_set_error(MS_ERR_STATE, "a hierarchy of the plan was destroyed");
        return MS_ERR_STATE;
    }
    if (!use_graph) {
        MS_TRY(plan_enqueue(p, st, nullptr, nullptr));
        ms_count_launch((unsigned)plan_launches(p));
        return MS_OK;
    }
    if (!p->exec) {
        // capture the launch sequence once on a private stream, then replay it
        if (!p->cap) MS_CUDA(cudaStreamCreateWithFlags(&p->cap, cudaStreamNonBlocking));
        MS_CUDA(cudaStreamBeginCapture(p->cap, cudaStreamCaptureModeThreadLocal));
        const ms_status s = plan_enqueue(p, p->cap, nullptr, nullptr);
        cudaGraph_t g = nullptr;
        const cudaError_t e = cudaStreamEndCapture(p->cap, &g);
        if (s != MS_OK || e != cudaSuccess) {
            if (g) cudaGraphDestroy(g);
            if (s != MS_OK) return s;
            return ms_cuda_error(e, "capture of the batched fit", __FILE__, __LINE__);
        }
        const cudaError_t ei = cudaGraphInstantiate(&p->exec, g, 0);
        cudaGraphDestroy(g);
        if (ei != cudaSuccess) {
            p->exec = nullptr;
            return ms_cuda_error(ei, "instantiation of the batched-fit graph", __FILE__, __LINE__);
        }
    }
    MS_CUDA(cudaGraphLaunch(p->exec, st));
    ms_count_launch((unsigned)plan_launches(p));
    return MS_OK;
}

// Read the per-hierarchy results of the last launch (waits for st).  kernel_ms < 0: no timing.
ms_status ms_batch_plan_stats_impl(ms_batch_plan* p, cudaStream_t st, ms_fit_stats* stats, float kernel_ms) {
    if (!p->valid) {
        ms_set_error(MS_ERR_STATE, "a hierarchy of the plan was destroyed");
        return MS_ERR_STATE;
    }
    std::vector<BatchStat> hst(p->nh);
    MS_CUDA(cudaMemcpyAsync(hst.data(), p->d_stat, sizeof(BatchStat) * p->nh, cudaMemcpyDeviceToHost, st));
    MS_CUDA(cudaStreamSynchronize(st));
    ms_status result = MS_OK;
    for (int i = 0; i < p->nh; ++i) {
        const BatchStat& b = hst[i];
        if (b.status != 0 && result == MS_OK) {
            result = (ms_status)b.status;
            ms_set_error(result, "device status %d in the fit of hierarchy %d of the batch", b.status, i);
        }
        if (!stats) continue;
        ms_fit_stats& s = stats[i];
        s = ms_fit_stats{};
        const ms_hierarchy* h = p->hs[i];
        s.L = h->L;
        s.sweeps = ms_sweeps_of(h);
        for (int l = 0; l < h->L; ++l) {
            s.cg_iterations[l] = b.iters[l];
            s.refinements[l] = b.refines[l];
            s.rel_residual[l] = b.resid[l];
        }
        s.precond_fallbacks = b.pcfb;
        s.fp64_fallbacks = b.f64fb;
        s.device_status = b.status;
        s.fit_ms = kernel_ms > 0.f ? kernel_ms : 0.0;  // the batch's solve launches, shared by all its hierarchies
        s.matvec_bytes = b.bytes;
        s.kernel_launches = plan_launches(p);
        s.solve_launches = (int32_t)p->grid.size();
        s.rhs_per_launch = 1;
        for (int k = 0; k < kProf; ++k) s.phase_ms[k] = 1e-6 * (double)b.prof[k];
    }
    return result;
}

ms_status ms_fit_batch_impl(ms_hierarchy* const* hs, int nh, const double* const* f_dev, double rel_tol,
                            double* const* alpha_dev, ms_fit_stats* stats, cudaStream_t st) {
    ms_batch_plan* p = nullptr;
    MS_TRY(ms_batch_plan_create_impl(hs, nh, f_dev, rel_tol, alpha_dev, st, &p));
    ms_status s = plan_enqueue(p, st, hs[0]->ev0, hs[0]->ev1);
    if (s == MS_OK) {
        ms_count_launch((unsigned)plan_launches(p));
        const cudaError_t e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) s = ms_cuda_error(e, "batched fit", __FILE__, __LINE__);
    }
    if (s == MS_OK) {
        float ms = -1.f;
        if (cudaEventElapsedTime(&ms, hs[0]->ev0, hs[0]->ev1) != cudaSuccess) ms = -1.f;
        s = ms_batch_plan_stats_impl(p, st, stats, ms);
    }
    ms_batch_plan_free(p, s != MS_OK);
    return s;
}
