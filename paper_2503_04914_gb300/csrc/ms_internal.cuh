// Internal definitions shared by the CUDA translation units of libms.so.
//
// Data layout in device memory (all levels concatenated, coarse to fine):
//   * points are stored "sorted": within each level, by the Morton code of
//     their cell in that level's uniform grid (cell size delta_l / cell_split),
//     ties broken by input index.  X is SoA: X[a * N + s] is coordinate a of
//     sorted point s.  perm[s] is the input index of sorted point s.
//   * cell_start is an exclusive prefix sum of points per cell over the
//     cells of all levels (level l's cells start at grid[l].cell_off); the
//     points of cell g are sorted positions [cell_start[g], cell_start[g+1]).
//   * A (block diagonal) and B (strictly lower blocks) are CSR over sorted
//     rows: int64 row offsets, int32 global sorted column indices, FP64 values
//     and optional FP32 values.  Row s of B holds the blocks j = 1..k-1 of its
//     level k in increasing j.
#pragma once

#include <cstdint>
#include <vector>

#include <cuda_fp16.h>
#include <cstdio>
#include <cuda_runtime.h>
#include <cuda/atomic>

#include "../../include/ms.h"

#define MS_MAXL MS_MAX_LEVELS

// ------------------------------------------------------------------ kernel

// phi(r) = (1-r)^e * (c0 + c1 r + c2 r^2 + c3 r^3) for r < 1, else 0.
struct WendlandPoly {
    int e;
    int k;          // degree of the polynomial factor
    double c[4];
};

// Wendland phi_{d,k}, l = floor(d/2)+k+1 (Wendland's closed forms, k = 0..3).
static inline bool wendland_poly(int wd, int wk, WendlandPoly* w) {
    if (wd < 1 || wd > 3 || wk < 0 || wk > 3) return false;
    const double l = wd / 2 + wk + 1;
    w->e = (int)l + wk;
    w->k = wk;
    w->c[0] = w->c[1] = w->c[2] = w->c[3] = 0.0;
    switch (wk) {
    case 0: w->c[0] = 1.0; break;
    case 1: w->c[0] = 1.0; w->c[1] = l + 1.0; break;
    case 2: w->c[0] = 3.0; w->c[1] = 3.0 * l + 6.0; w->c[2] = l * l + 4.0 * l + 3.0; break;
    case 3:
        w->c[0] = 15.0; w->c[1] = 15.0 * l + 45.0; w->c[2] = 6.0 * l * l + 36.0 * l + 45.0;
        w->c[3] = l * l * l + 9.0 * l * l + 23.0 * l + 15.0;
        break;
    }
    return true;
}

// wendland_eval in FP32 from coefficients already converted to float (each conversion from
// FP64 is an FP64-pipe instruction, scarce on this GPU).
__device__ __forceinline__ float wendland_eval_f(const WendlandPoly& w, const float* c, float r) {
    if (!(r < 1.0f)) return 0.0f;
    const float s = 1.0f - r, s2 = s * s, s4 = s2 * s2;
    float pw;
    switch (w.e) {
    case 4: pw = s4; break;
    case 6: pw = s4 * s2; break;
    case 8: pw = s4 * s4; break;
    default: {
        pw = 1.0f;
        for (int i = 0; i < w.e; ++i) pw *= s;
    }
    }
    float p = c[w.k];
    for (int i = w.k - 1; i >= 0; --i) p = p * r + c[i];
    return pw * p;
}

template <typename T>
__device__ __forceinline__ T wendland_eval(const WendlandPoly& w, T r) {
    if (!(r < T(1))) return T(0);  // compact support: phi vanishes for r >= 1
    const T s = T(1) - r;
    // (1 - r)^e by squaring (e = 3..11 for the supported (d, k); fewer multiplications,
    // which matter where T = double: FP64 issue is scarce on this GPU)
    const T s2 = s * s, s4 = s2 * s2;
    T pw;
    switch (w.e) {
    case 4: pw = s4; break;
    case 6: pw = s4 * s2; break;
    case 8: pw = s4 * s4; break;
    default: {
        pw = T(1);
        for (int i = 0; i < w.e; ++i) pw *= s;
    }
    }
    // Horner from the degree k: the zero leading coefficients cost FP64 issue and leave the
    // value unchanged (0 * r + 0 = 0 exactly)
    T p = T(w.c[w.k]);
    for (int i = w.k - 1; i >= 0; --i) p = p * r + T(w.c[i]);
    return pw * p;
}

// ------------------------------------------------------------------ grids

struct LevelGrid {
    double lo[3];      // grid origin (level bounding-box minimum)
    double inv_cell;   // 1 / cell size
    double cell;       // cell size
    float cod;         // cell size / delta (a power of 2)
    int G[3];          // cells per axis (1 for unused axes)
    int bits;          // Morton bits per axis (P = 2^bits >= max G)
    int64_t cell_off;  // first global cell id of the level
    int64_t ncells;    // P^d
};

__host__ __device__ __forceinline__ uint32_t spread2(uint32_t v) {  // 16 -> 32 bits, 1 gap
    v &= 0x0000ffffu;
    v = (v | (v << 8)) & 0x00ff00ffu;
    v = (v | (v << 4)) & 0x0f0f0f0fu;
    v = (v | (v << 2)) & 0x33333333u;
    v = (v | (v << 1)) & 0x55555555u;
    return v;
}
__host__ __device__ __forceinline__ uint32_t spread3(uint32_t v) {  // 10 -> 30 bits, 2 gaps
    v &= 0x000003ffu;
    v = (v | (v << 16)) & 0x030000ffu;
    v = (v | (v << 8)) & 0x0300f00fu;
    v = (v | (v << 4)) & 0x030c30c3u;
    v = (v | (v << 2)) & 0x09249249u;
    return v;
}
__host__ __device__ __forceinline__ uint32_t morton(int d, int cx, int cy, int cz) {
    if (d == 1) return (uint32_t)cx;
    if (d == 2) return spread2((uint32_t)cx) | (spread2((uint32_t)cy) << 1);
    return spread3((uint32_t)cx) | (spread3((uint32_t)cy) << 1) | (spread3((uint32_t)cz) << 2);
}

// Everything a kernel needs to know about the hierarchy (passed by value).
struct HierView {
    int d, L, R;                // R = neighbour cell radius (cells searched: (2R+1)^d)
    int64_t N;
    int64_t off[MS_MAXL + 1];   // level row offsets
    double delta[MS_MAXL];
    double dscale[MS_MAXL];     // delta^-d
    double inv_delta[MS_MAXL];  // 1 / delta (correctly rounded, as the device's 1.0 / delta)
    LevelGrid grid[MS_MAXL];
    WendlandPoly w;
    const double* X;            // [d][N] sorted coordinates
    const int32_t* cell_start;  // [total cells + 1]
};

__device__ __forceinline__ int level_of_row(const int64_t* off, int L, int64_t row) {
    int l = 0;
    while (l + 1 < L && row >= off[l + 1]) ++l;
    return l;
}

// Cell coordinate of coordinate value v on axis a of grid g.  Not clamped to
// the grid (callers skip or clamp out-of-range cells) but kept within
// [-4, G+4] so that far-away query points cannot overflow the conversion.
__device__ __forceinline__ int cell_coord(const LevelGrid& g, int a, double v) {
    double u = floor((v - g.lo[a]) * g.inv_cell);
    u = fmin(fmax(u, -4.0), (double)g.G[a] + 4.0);
    return (int)u;
}

// Calls visit(p, r2) for every sorted point p of level j with |x_p - y|^2 < delta_j^2
// (the (2R+1)^d cells around y's cell in level j's grid, FP64 distances).
template <typename F>
__device__ __forceinline__ void for_each_neighbour(const HierView& v, int j, const double* y, F&& visit) {
    const LevelGrid& g = v.grid[j];
    const double d2 = v.delta[j] * v.delta[j];
    int c[3] = {0, 0, 0};
    for (int a = 0; a < v.d; ++a) c[a] = cell_coord(g, a, y[a]);
    const int R = v.R;
    const int rz = v.d >= 3 ? R : 0, ry = v.d >= 2 ? R : 0;
    for (int dz = -rz; dz <= rz; ++dz) {
        const int cz = c[2] + dz;
        if (cz < 0 || cz >= g.G[2]) continue;
        for (int dy = -ry; dy <= ry; ++dy) {
            const int cy = c[1] + dy;
            if (cy < 0 || cy >= g.G[1]) continue;
            for (int dx = -R; dx <= R; ++dx) {
                const int cx = c[0] + dx;
                if (cx < 0 || cx >= g.G[0]) continue;
                const int64_t gid = g.cell_off + morton(v.d, cx, cy, cz);
                const int32_t s = v.cell_start[gid], e = v.cell_start[gid + 1];
                for (int32_t p = s; p < e; ++p) {
                    double r2 = 0.0;
                    for (int a = 0; a < v.d; ++a) {
                        const double t = v.X[a * v.N + p] - y[a];
                        r2 = fma(t, t, r2);
                    }
                    if (r2 < d2) visit(p, r2);
                }
            }
        }
    }
}

// ------------------------------------------------------------------ errors (host)

struct MsError {
    ms_status st;
};
void ms_set_error(ms_status st, const char* fmt, ...);
void ms_clear_error();  // empties this thread's last-error message (entry of every C-ABI call)
// Jacobi sweeps of a fit: opts.jacobi_sweeps > 0 as given, 0 = L - 1 (exact, Theorem 9), -1 = none
// (the fit returns D_L^{-1} f, the block-diagonal solve of eq. split alone)
inline int ms_sweeps_of(const ms_hierarchy* h);
void ms_count_launch(unsigned n = 1);  // process-wide kernel launch counter
ms_status ms_cuda_error(cudaError_t e, const char* what, const char* file, int line);

#define MS_CUDA(call)                                                            \
    do {                                                                         \
        cudaError_t e__ = (call);                                                \
        if (e__ != cudaSuccess) return ms_cuda_error(e__, #call, __FILE__, __LINE__); \
    } while (0)

#define MS_TRY(call)                         \
    do {                                     \
        ms_status s__ = (call);              \
        if (s__ != MS_OK) return s__;        \
    } while (0)

// ------------------------------------------------------------------ device helpers

__device__ __forceinline__ unsigned long long ms_globaltimer() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Deterministic block sum (fixed shuffle tree, then warp 0 over the warp sums).
// Result is valid in every thread.  `scratch` holds >= BS/32 doubles.
template <int BS>
__device__ __forceinline__ double block_sum(double v, double* scratch) {
    v = warp_sum(v);
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    __syncthreads();
    if (lane == 0) scratch[w] = v;
    __syncthreads();
    double t = (lane < BS / 32) ? scratch[lane] : 0.0;
    t = warp_sum(t);
    return t;
}

// ------------------------------------------------------------------ host-side handle

struct DevCSR {
    int64_t* rp = nullptr;   // [N+1]
    int32_t* col = nullptr;  // [nnz]
    double* v64 = nullptr;   // [nnz]
    float* v32 = nullptr;    // [nnz] (MIXED only)
    int64_t nnz = 0;
};

// Factorised sparse-approximate-inverse preconditioner M = G^T G of the level CGs
// (rows: self + up to kPcK nearest preceding same-level neighbours within delta).
constexpr int kPcK = 16;
constexpr int kPcOut = kPcK + 1;
constexpr int kPcHidden = 64;
// candidate rows the network predicts per point (the row is their FSAI-optimal combination)
constexpr int kPcMaxBasis = 16;
constexpr int kPcBasisDefault = 16;

struct Precond {
    int n_in = 0, n_params = 0;
    int nbasis = kPcBasisDefault;  // candidate rows per point (network outputs: 17 nbasis)
    bool trained = false;        // network weights present
    int built_kind = 0;          // kind of G currently built (0 = none)
    float* theta = nullptr;      // [n_params] FP32 master weights (W1,b1,W2,b2,W3,b3)
    float* theta_bf = nullptr;   // [n_params] the same rounded to BF16 (stored as float)
    float* adam_m = nullptr;
    float* adam_v = nullptr;
    float* musig = nullptr;      // [2 * kPcOut] standardisation of the scale-free targets
    int32_t* nbr = nullptr;      // [N][kPcK] pattern neighbours (sorted positions, -1 = none)
    int32_t* gcol = nullptr;     // [kPcOut][N] row pattern of G (slot 0 = self, -1 = none; slot-major)
    __half* gval = nullptr;      // [kPcOut][N] scale-free rows ghat (G = delta_l^{d/2} ghat), FP16
    int64_t* gt_rp = nullptr;    // [N+1] rows of G^T (in-pattern)
    int32_t* gt_col = nullptr;   // [nnz] source rows
    __half* gt_val = nullptr;    // [nnz] ghat^T values, FP16
    int64_t gt_nnz = 0;
    int fp32_weights = 0;
    int* tcstat = nullptr;       // status of the tensor-core network (MS_ERR_TIMEOUT if a wait ran out)
    int augment = 4;                     // extra training patches per point (last training)
    uint64_t seed = 2503049140ull;       // seed of the last training
};

struct ms_hierarchy {
    int device = 0;
    Precond pc;
    float *u32 = nullptr, *u1_32 = nullptr;  // preconditioned-CG work vectors [ws_rhs][N]
    int d = 0, L = 0;
    int64_t N = 0;
    ms_opts opts{};
    HierView view{};             // X / cell_start pointers filled
    int64_t total_cells = 0;
    double* X = nullptr;         // [d][N] sorted
    int32_t* perm = nullptr;     // sorted -> input
    int32_t* cell_start = nullptr;
    float* W = nullptr;          // [d][N] FP32 offsets from the own cell corner, in units of delta_l
    float* Wlo = nullptr;        // [d][N] their low parts (W + Wlo: about 48 bits; MIXED builds)
    int32_t* cellid = nullptr;   // [N] level-local Morton cell of each sorted point
    int mf_tpp = 2;              // matrix-free lanes per target point
    DevCSR A, B;
    int32_t* Bseg = nullptr;     // [L][N] start of column level j's segment in each B row (offset from rpB)
    // lower_op = MATRIX_FREE: the build's frames of every row in the levels up to its own, kept for
    // the fit's lower-block updates (row s of level k, level j <= k at frame_base[k] + (s - off[k]) (k + 1) + j)
    void* frames = nullptr;
    int64_t frame_base[MS_MAXL + 1] = {};
    int64_t Bblk[MS_MAXL][MS_MAXL] = {};  // entries of block B_kj
    int64_t rpA_lv[MS_MAXL + 1] = {};     // A.rp / B.rp at the level boundaries (host copies)
    int64_t rpB_lv[MS_MAXL + 1] = {};
    // solver work space (sorted order; vectors hold ws_rhs right-hand sides, [ws_rhs][N])
    int ws_rhs = 0;
    double *f = nullptr, *beta = nullptr, *x = nullptr, *r = nullptr, *p = nullptr, *q = nullptr, *s = nullptr;
    float *x32 = nullptr, *r32 = nullptr, *p32 = nullptr, *q32 = nullptr, *s32 = nullptr;
    double* part = nullptr;      // reduction partials
    double* gpart = nullptr;     // group sums of the partials
    double* scal = nullptr;      // published grid sums
    unsigned long long* prof = nullptr;  // device timeline of the solve kernel
    int* pcfb = nullptr;                 // preconditioner fallbacks of the last fit
    // several blocks of right-hand sides in one launch: per-block barrier words, status and counters
    // (pbuf, for pbuf_parts blocks) and the blocks' solve arguments (d_args)
    void* pbuf = nullptr;
    int pbuf_parts = 0;
    void* d_args = nullptr;
    unsigned* bar = nullptr;     // barrier words
    int* status = nullptr;       // device status
    int64_t* iters = nullptr;    // per-level iteration counters
    int* refines = nullptr;
    double* resid = nullptr;
    double* bytes = nullptr;
    double* tmp64 = nullptr;     // [N] scratch (permutations)
    int solve_blocks = 0;        // cooperative grid size
    int tprA_tuned[MS_MAXL] = {};  // autotuned CSR lanes per row of A_l (0 = by rule)
    int mf_tpp_tuned = 0;          // autotuned matrix-free lanes per point (0 = by rule)
    bool tuned = false;
    std::vector<struct ms_batch_plan*> plans;  // live batch plans that hold pointers to the work space
    int64_t device_bytes = 0;
    double build_ms = 0.0;
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;
    void* allocs[96];
    size_t alloc_bytes[96];
    int nallocs = 0;
};

inline int ms_sweeps_of(const ms_hierarchy* h) {
    if (h->opts.jacobi_sweeps > 0) return h->opts.jacobi_sweeps;
    return h->opts.jacobi_sweeps < 0 ? 0 : (h->L > 1 ? h->L - 1 : 0);
}

ms_status ms_alloc(ms_hierarchy* h, void** p, size_t bytes);
// library memory pool of the current device (ms_capi.cu)
ms_status ms_pool_alloc(void** p, size_t bytes);
void ms_pool_free(void* p);
// Scratch memory ordered on stream st from the same pool (kept mapped when freed, so that
// repeated builds do not map and unmap their temporaries); free with cudaFreeAsync on st.
ms_status ms_tmp_alloc(void** p, size_t bytes, cudaStream_t st);
// free *p (if it is one of the handle's allocations) and allocate `bytes` in its place
ms_status ms_realloc(ms_hierarchy* h, void** p, size_t bytes);
ms_status ms_build_impl(ms_hierarchy* h, const double* points_dev, cudaStream_t s);
ms_status ms_fit_impl(ms_hierarchy* h, const double* f_dev, int nrhs, double rel_tol, double* alpha_dev,
                      ms_fit_stats* stats, cudaStream_t s);
ms_status ms_apply_impl(ms_hierarchy* h, int op, const double* x_dev, double* y_dev, int sorted, cudaStream_t s);
ms_status ms_evaluate_impl(ms_hierarchy* h, const double* alpha_dev, int nrhs, const double* q_dev, int64_t nq,
                           double* out_dev, cudaStream_t s);

// batched fit of several hierarchies in one launch (ms_batch.cu)
ms_status ms_fit_batch_impl(ms_hierarchy* const* hs, int nh, const double* const* f_dev, double rel_tol,
                            double* const* alpha_dev, ms_fit_stats* stats, cudaStream_t st);

// CSR lanes per row of A_l used by the solve (ms_solve.cu)
int ms_tpr_of(const ms_hierarchy* h, int l);

// solve work space for R right-hand sides (ms_solve.cu)
ms_status ms_ensure_workspace(ms_hierarchy* h, int R);

// learned / exact FSAI preconditioner (ms_precond.cu): build G and G^T for `kind`
ms_status ms_pc_build(ms_hierarchy* h, int kind, cudaStream_t s);
// prepared batched fits (ms_batch.cu)
struct ms_batch_plan;
ms_status ms_batch_plan_create_impl(ms_hierarchy* const* hs, int nh, const double* const* f_dev, double rel_tol,
                                    double* const* alpha_dev, cudaStream_t st, ms_batch_plan** out);
ms_status ms_batch_plan_launch_impl(ms_batch_plan* p, cudaStream_t st, int use_graph);
ms_status ms_batch_plan_stats_impl(ms_batch_plan* p, cudaStream_t st, ms_fit_stats* stats, float kernel_ms);
void ms_batch_plan_free(ms_batch_plan* p, bool device_sync);
void ms_batch_plan_detach(ms_batch_plan* p, const ms_hierarchy* h);  // h is being destroyed
// with opts.autotune = 1: choose the mat-vec lanes per row of each level once (ms_solve.cu)
ms_status ms_autotune(ms_hierarchy* h, cudaStream_t st);

// permutation helpers (ms_capi.cu)
void ms_gather_sorted(const double* in, double* out, const int32_t* perm, int64_t N, int nrhs, int col, cudaStream_t s);
void ms_scatter_input(const double* in, double* out, const int32_t* perm, int64_t N, int nrhs, int col, cudaStream_t s);
