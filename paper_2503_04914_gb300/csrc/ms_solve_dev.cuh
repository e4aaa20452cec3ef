// Device side of the fit (shared by the single-hierarchy and the batched solve kernels).
#pragma once
// The fit: eq. split of Section 3 solved on the device in ONE persistent
// cooperative kernel per batch of right-hand sides.
//
//   T'_L beta = f   by Jacobi sweeps (eq. jacobi, Theorem 9), beta_0 = f;
//   D_L alpha = beta by per-level conjugate gradients (Theorem 8,
//                    eq. blockdiagonal_levelwise), all levels in flight together.
//
// Sweep m (0-based) of the Jacobi iteration solves A_l t_l = beta_l for the
// levels l = m..L-2 together (warm-started from the previous sweep; level m,
// whose beta is final, to the requested tolerance, the others to the
// intermediate tolerance), then recomputes beta_k = f_k - sum_{j<k} B_kj t_j for
// the rows of levels k = m+1..L-1.  Levels below m already hold their final t
// (their beta cannot change any more) and are not re-solved; rows of levels
// <= m are not recomputed (they would reproduce the same values).  A final
// solve over all levels gives alpha_l = A_l^{-1} beta_l and certifies every
// level's FP64 true residual.
//
// Several right-hand sides share one launch: every (right-hand side, level)
// pair is a "virtual level" v = r L + l with its own CG scalars; the matrix is
// shared and the vectors are stored right-hand-side-major ([R][N]).
//
// Level solves: CG in the single-reduction form of Chronopoulos and Gear
// (w = A u, then r.u, w.u and r.r in one reduction; p = u + beta p,
// s = w + beta s, x += alpha p, r -= alpha s, u = M r or u = r), which is CG's
// recurrence with one grid-wide reduction and two grid barriers per
// iteration (four with the preconditioner).  FP64 dots are reduced
// deterministically: per-CTA partials (a shared-memory block sum), then, inside
// the grid barrier, the last CTA of each group of 16 sums its group's partials
// and the last group leader sums the group sums, in fixed orders, and publishes
// them, so all CTAs take the same convergence decisions.  Stopping:
// |beta_l - A_l x| <= tol |beta_l| in FP64 (true residual, re-checked after
// the recursive residual has converged).
//   FP64 mode : CG on FP64 vectors with the FP64 CSR values.
//   MIXED mode: iterative refinement: outer FP64 true residual r = b - A x
//               (FP64 CSR), inner CG on FP32 vectors with FP32 CSR values (or
//               matrix-free FP32 entries) and FP32 accumulation (FP64 dots and
//               scalars) for A d = r/|r|, then x += |r| d in FP64.
// Grid barriers are bounded; on a time-out every CTA returns and the host
// reports MS_ERR_TIMEOUT.
#include <algorithm>
#include <cmath>
#include <vector>

#include "ms_geom.cuh"
#include "ms_internal.cuh"
#include "ms_matfree.cuh"

namespace {

constexpr int kBS = 512;     // threads per CTA of the solve kernel
constexpr int kChunk = 256;  // rows per work chunk (chunks never straddle levels)
constexpr int kNW = kBS / 32;
constexpr int kAcc = 3;      // accumulators per phase
constexpr int kMaxV = 256;   // virtual levels (right-hand side, level) per launch
constexpr int kLCells = 128;   // cells of the staged box
constexpr int kGroup = 16;           // CTAs per first-level barrier counter
constexpr int kMaxGroups = 64;       // <= 1024 CTAs
constexpr int kBarWords = 2 + kMaxGroups;  // top count, generation, group counters
// phase categories of the device timeline (ms_fit_stats.phase_ms)
enum { kPrfResid = 0, kPrfMatvec = 1, kPrfUpdate = 2, kPrfBarrier = 3, kPrfLower = 4, kPrfOther = 5,
       kPrfScalar = 6, kProf = 8 };

struct SolveArgs {
    int L, R, V;       // levels, right-hand sides of this launch, V = R L virtual levels
    int RW;            // wide layout: lanes (vector elements) per row, a power of 2 >= R; 0 = RHS-major
    int crow;          // rows per work chunk
    int crowl[MS_MAXL];  // rows per work chunk of each level (right-hand-side-major layout)
    int64_t N;         // points
    int C;             // chunks per right-hand side
    int64_t off[MS_MAXL + 1];
    int coff[MS_MAXL + 1];       // chunk offsets per level (within one right-hand side)
    int64_t nnzA[MS_MAXL], nnzB[MS_MAXL];
    int tprA[MS_MAXL], tprB[MS_MAXL];
    const int64_t* Arp;
    const int32_t* Acol;
    const double* Av64;
    const float* Av32;
    const int64_t* Brp;
    const int32_t* Bcol;
    const double* Bv64;
    const int32_t* Bseg;       // [L][N] start of column level j's segment in each B row
    int lower_inc;             // sweep m subtracts B_km t_m only (see k_fit)
    // matrix-free lower blocks (lower_mf = 1, MIXED builds): B_km t_m recomputed in
    // double-float from the geometry (the build stores no B)
    int lower_mf;
    int tprLmf[MS_MAXL];       // lanes per row of the update from level m
    const Frame* frames;       // the build's frames: row s of level k, level j <= k at
    int64_t fbase[MS_MAXL + 1];  // fbase[k] + (s - off[k]) (k + 1) + j
    HierView hv;
    FFLevels ffl;
    const float* Wlo;          // [d][N] low parts of the in-cell offsets
    int64_t nnzBm[MS_MAXL];    // entries of the blocks B_km, k > m
    int tprBm[MS_MAXL];
    const double* f;                       // [R][N]
    double *beta, *x, *r, *p, *q, *s;      // [R][N]; q holds w = A u
    float *x32, *r32, *p32, *q32, *s32;    // [R][N]
    double* part;      // [kAcc][V][CTAs] per-CTA partial sums
    double* gpart;     // [kMaxGroups][kAcc][V] group sums
    double* scal;      // [kAcc][V] grid sums published inside the barrier
    unsigned* bar;     // [kBarWords]
    int* status;
    int64_t* iters;    // [MS_MAXL] summed over the right-hand sides
    int* refines;      // [MS_MAXL] summed over the right-hand sides
    double* resid;     // [V]
    double* bytes;     // [1]
    unsigned long long* prof;  // [kProf] nanoseconds CTA 0 spent per phase category
    int sweeps, max_iters, max_outer;
    double tol, inter_tol, inner_tol;
    unsigned long long timeout_ns;
    int mf;            // MIXED inner mat-vec is matrix-free
    int mf_tpp;        // lanes per target point of the matrix-free mat-vec
    MFView mfv;
    // MIXED inner CG preconditioned with M = G^T G (pc = 1)
    int pc;
    const int32_t* gcol;   // [kPcOut][N] (slot-major: slot k of consecutive rows is contiguous)
    const __half* gval;    // [kPcOut][N] scale-free rows ghat (FP16)
    const int64_t* gt_rp;  // rows of G^T
    const int32_t* gt_col;
    const __half* gt_val;
    float pcs[MS_MAXL];    // delta_l^d: G^T G = delta_l^d ghat^T ghat on level l
    float *u32, *u1_32;    // [R][N]
    int* pcfb;             // [2] levels that fell back to plain CG, to FP64 inner CG
};

// Per-CTA shared state of the solve (identical in every CTA), in dynamic shared memory.
struct Shared {
    double red[kAcc][kBS];
    double acc[kAcc][kMaxV];
    double out[kAcc][kMaxV];
    double bb[kMaxV], alpha[kMaxV], beta[kMaxV], tol[kMaxV], scale[kMaxV], target[kMaxV], gam[kMaxV];
    int act[kMaxV], oact[kMaxV], zero[kMaxV], first[kMaxV], pcoff[kMaxV], fresh[kMaxV];
    int it_solve[kMaxV];
    int32_t lq[kNW][64];    // per-warp candidate queues of the matrix-free lower update
    int32_t lqd[kNW][64];   // their cells' displacements
    // staged matrix-free lower update (lower_chunk_staged; the points' positions go to red)
    int32_t lcoff[kLCells + 1];  // first staged point of each box cell (x fastest, then y, then z)
    int32_t lps[kLCells];        // the cell's first point (index into the sorted points)
    int32_t lbox[8];           // box origin (3), extent (3), cells, fits
    int32_t lred[kNW][6];      // per-warp minima and maxima of the rows' cells
    int refines[kMaxV];
    int f64[kMaxV];         // MIXED: the level's inner CG runs in FP64 (FP32 refinement stalled)
    int f64n[kMaxV];        // levels switched to FP64
    double prevres[kMaxV];  // MIXED: true residual of the previous outer round
    int fb[kMaxV];          // preconditioner fall-backs
    long long it_total[kMaxV];
    double vbytes[kMaxV];   // algorithmic bytes moved, per virtual level
    double bytes;           // bytes of the lower-block updates
    int last, glast, ok;
    int cta, nb;            // this CTA's index in its partition, CTAs in the partition
    unsigned mine;
    unsigned long long pt[kProf];
    unsigned long long tprev;
};

#ifdef MS_CTA_PROF
// Diagnostic build (-DMS_CTA_PROF): every CTA keeps the timeline, and each CTA's totals per
// category are left in g_cta_prof for ms_debug_cta_prof (load balance between CTAs).
__device__ unsigned long long g_cta_prof[1024][kProf];
#endif

// Device timeline: CTA 0's thread 0 charges the time since the previous mark to `cat`.
__device__ __forceinline__ void prof(Shared& sh, int cat) {
#ifdef MS_CTA_PROF
    if (threadIdx.x == 0) {
#else
    if (sh.cta == 0 && threadIdx.x == 0) {
#endif
        const unsigned long long now = ms_globaltimer();
        sh.pt[cat] += now - sh.tprev;
        sh.tprev = now;
    }
}

// y = sum_k val[k] * x[col[k]] over one CSR row, by a sub-warp of S lanes
// (sl = lane within the sub-warp); the result is valid in every lane.  All 32
// lanes of the warp must call it (invalid rows pass e = s).
// The matrix (col, val) is read-only for the whole kernel and may use the
// non-coherent path; x is written by other CTAs between phases and must not
// (no __restrict__ on it).  The loop is unrolled by 4 with independent loads so
// that a lane keeps several gathers in flight (small levels are latency-bound).
// The per-lane partial sums are combined by shuffles in a fixed order.  (Inside the
// solve kernel this form measured faster than the 128-bit form below: with four
// entries a lane per group the latter leaves fewer independent gathers in flight and
// needs more registers than the kernel's 64.)
template <typename TV, typename TX, typename TA>
__device__ __forceinline__ TA csr_row(const int32_t* __restrict__ col, const TV* __restrict__ val,
                                      const TX* x, int64_t s, int64_t e, int sl, int S) {
    TA acc = TA(0);
    int64_t k = s + sl;
    for (; k + 3 * S < e; k += 4 * S) {
        const int32_t c0 = __ldg(col + k), c1 = __ldg(col + k + S), c2 = __ldg(col + k + 2 * S),
                      c3 = __ldg(col + k + 3 * S);
        const TV v0 = __ldg(val + k), v1 = __ldg(val + k + S), v2 = __ldg(val + k + 2 * S), v3 = __ldg(val + k + 3 * S);
        const TX x0 = x[c0], x1 = x[c1], x2 = x[c2], x3 = x[c3];
        acc += (TA)v0 * (TA)x0;
        acc += (TA)v1 * (TA)x1;
        acc += (TA)v2 * (TA)x2;
        acc += (TA)v3 * (TA)x3;
    }
    for (; k < e; k += S) acc += (TA)__ldg(val + k) * (TA)x[__ldg(col + k)];
    for (int o = S >> 1; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    return acc;
}

// The same sum with 128-bit loads (used by the stand-alone mat-vec): FP32 and FP64 values
// are read four entries at a time (int4 columns, float4 / 2 x double2 values); the entries
// from the first multiple of 4 at or after s are split into groups of four, group g to lane
// g mod S, and the (at most 3) entries before that boundary and after the last full group go
// to the lanes one by one (lane sl takes every S-th of them).  The CSR arrays start on
// 16-byte boundaries (the build checks it).
template <typename TV, typename TX, typename TA>
__device__ __forceinline__ TA csr_row_vec(const int32_t* __restrict__ col, const TV* __restrict__ val,
                                          const TX* x, int64_t s, int64_t e, int sl, int S) {
    static_assert(sizeof(TV) == 4 || sizeof(TV) == 8, "FP32 or FP64 values");
    TA acc = TA(0);
    const int64_t a = min(e, (s + 3) & ~int64_t(3));  // 16-byte boundary of the columns
    for (int64_t k = s + sl; k < a; k += S) acc += (TA)__ldg(val + k) * (TA)x[__ldg(col + k)];
    const int64_t ng = (e - a) >> 2;                  // full groups of four from a
    const int4* c4 = reinterpret_cast<const int4*>(col + a);
    for (int64_t g = sl; g < ng; g += S) {
        const int4 c = __ldg(c4 + g);
        TA v0, v1, v2, v3;
        if constexpr (sizeof(TV) == 4) {
            const float4 v = __ldg(reinterpret_cast<const float4*>(val + a) + g);
            v0 = (TA)v.x; v1 = (TA)v.y; v2 = (TA)v.z; v3 = (TA)v.w;
        } else {
            const double2 u = __ldg(reinterpret_cast<const double2*>(val + a) + 2 * g);
            const double2 w = __ldg(reinterpret_cast<const double2*>(val + a) + 2 * g + 1);
            v0 = (TA)u.x; v1 = (TA)u.y; v2 = (TA)w.x; v3 = (TA)w.y;
        }
        const TX x0 = x[c.x], x1 = x[c.y], x2 = x[c.z], x3 = x[c.w];
        acc += v0 * (TA)x0;
        acc += v1 * (TA)x1;
        acc += v2 * (TA)x2;
        acc += v3 * (TA)x3;
    }
    for (int64_t t = a + 4 * ng + sl; t < e; t += S) acc += (TA)__ldg(val + t) * (TA)x[__ldg(col + t)];
    for (int o = S >> 1; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    return acc;
}

// A work chunk: rows [r0, r1) of level l for right-hand side rhs (vectors at offset vb).
struct Chunk {
    int v, l;
    int64_t r0, r1, vb;
};

// Add the block's thread-local accumulators into sh.acc[k][cur]: values are
// staged in shared memory and summed by one warp per accumulator in a fixed
// order (few FP64 instructions; deterministic).
template <int K>
__device__ __forceinline__ void flush_acc(Shared& sh, double* acc, int cur) {
#pragma unroll
    for (int k = 0; k < K; ++k) {
        sh.red[k][threadIdx.x] = acc[k];
        acc[k] = 0.0;
    }
    __syncthreads();
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (w < K) {
        double t = 0.0;
#pragma unroll
        for (int j = 0; j < kBS / 32; ++j) t += sh.red[w][lane + 32 * j];
        t = warp_sum(t);
        if (lane == 0) sh.acc[w][cur] += t;
    }
    __syncthreads();
}

// Run body(chunk, acc) over this CTA's chunks whose virtual level passes sel(v);
// thread-local accumulators are block-reduced into sh.acc[k][v] and the per-CTA
// sums of all virtual levels are written to the partials array.
template <int K, typename Sel, typename Body>
__device__ __forceinline__ void run_phase(const SolveArgs& a, Shared& sh, Sel sel, Body body) {
    if (K > 0) {
        for (int i = threadIdx.x; i < kAcc * kMaxV; i += kBS) (&sh.acc[0][0])[i] = 0.0;
        __syncthreads();
    }
    double acc[K > 0 ? K : 1];
#pragma unroll
    for (int k = 0; k < (K > 0 ? K : 1); ++k) acc[k] = 0.0;
    int cur = -1;
    // Global chunk g = rhs * C + c goes to CTA g mod sh.nb; the CTA walks its
    // chunks in increasing g, level by level, and jumps over levels that sel() rejects.
    const int nb = sh.nb, C = a.C;
    int first = sh.cta;  // first chunk of this CTA within the current right-hand side
    for (int rhs = 0; rhs < a.R; ++rhs) {
        int l = 0;
        for (int c = first; c < C;) {
            while (c >= a.coff[l + 1]) ++l;
            const int v = rhs * a.L + l;
            if (!sel(v)) {
                const int e = a.coff[l + 1];
                c += (e - c + nb - 1) / nb * nb;
                continue;
            }
            if (K > 0 && v != cur) {
                if (cur >= 0) flush_acc<K>(sh, acc, cur);
                cur = v;
            }
            Chunk ch;
            ch.l = l;
            ch.v = v;
            ch.vb = (int64_t)rhs * a.N;
            ch.r0 = a.off[l] + (int64_t)(c - a.coff[l]) * a.crowl[l];
            ch.r1 = min(ch.r0 + (int64_t)a.crowl[l], a.off[l + 1]);
            body(ch, acc);
            c += nb;
        }
        // chunks of the next right-hand side: rhs * C + c == sh.cta (mod nb)
        first = (first - C % nb + nb) % nb;
    }
    if (K > 0) {
        if (cur >= 0) flush_acc<K>(sh, acc, cur);
        for (int i = threadIdx.x; i < K * a.V; i += kBS) {
            const int k = i / a.V, v = i % a.V;
            a.part[((size_t)k * a.V + v) * sh.nb + sh.cta] = sh.acc[k][v];
        }
    }
}

// Waiting side of a grid barrier (thread 0 spins on the generation word, bounded),
// then, with K > 0, every CTA copies the published sums into sh.out.
template <int K>
__device__ __forceinline__ bool gsync_finish(const SolveArgs& a, Shared& sh) {
    int ok = 1;
    if (!sh.last && threadIdx.x == 0) {
        cuda::atomic_ref<unsigned, cuda::thread_scope_device> g(a.bar[1]);
        cuda::atomic_ref<int, cuda::thread_scope_device> st(*a.status);
        const unsigned long long t0 = ms_globaltimer();
        unsigned spins = 0;
        while (g.load(cuda::memory_order_acquire) == sh.mine) {
            if ((++spins & 255u) == 0u) {
                if (st.load(cuda::memory_order_relaxed) == MS_ERR_TIMEOUT) { ok = 0; break; }
                if (ms_globaltimer() - t0 > a.timeout_ns) {
                    int expect = 0;
                    st.compare_exchange_strong(expect, (int)MS_ERR_TIMEOUT, cuda::memory_order_relaxed);
                    if (expect != 0) st.store((int)MS_ERR_TIMEOUT, cuda::memory_order_relaxed);
                    ok = 0;
                    break;
                }
            }
            __nanosleep(32);
        }
    }
    // No status load after the release (it would add an L2 round trip to every barrier):
    // a CTA that timed out never arrives at the next barrier, whose waiters see the
    // recorded time-out within 256 polls and leave.
    if (threadIdx.x == 0) sh.ok = ok;  // a separate flag: sh.last may still be read by lagging warps
    __syncthreads();
    if (!sh.ok) return false;
    if (K > 0) {
        const int npair = K * a.V;
        for (int i = threadIdx.x; i < npair; i += kBS) {
            const int k = i / a.V, v = i % a.V;
            sh.out[k][v] = __ldcg(a.scal + i);
        }
        __syncthreads();
    }
    prof(sh, kPrfBarrier);
    return true;
}

// Release by the last CTA to arrive (thread 0): reset the counter, advance the generation.
__device__ __forceinline__ void gsync_release(const SolveArgs& a, Shared& sh) {
    if (threadIdx.x == 0) {
        cuda::atomic_ref<unsigned, cuda::thread_scope_device> g(a.bar[1]);
        cuda::atomic_ref<unsigned, cuda::thread_scope_device> c(a.bar[0]);
        c.store(0u, cuda::memory_order_relaxed);
        g.store(sh.mine + 1u, cuda::memory_order_release);
    }
}

// Grid barrier; with K > 0 it also reduces the per-CTA partials of the K V sums,
// publishes them in a.scal before releasing the other CTAs, and every CTA then
// copies the sums into sh.out.  Arrival is one counter for all CTAs (measured on
// GB300 with 304 CTAs: 2.3 us per barrier against 4.9 us for a two-level arrival,
// whose extra atomic costs a round trip).  With few partials (K V nb <= 16384
// values, K V <= the CTA's threads) the last CTA to arrive sums them itself over a fixed
// segmentation of the CTAs; more partials (wide multi-RHS launches, or many virtual
// levels on a small grid partition) take a two-level arrival in which
// the last CTA of each group of kGroup sums its group and the last group leader sums
// the groups.  Both orders are fixed, so every run gives the same sums.  Every wait
// is bounded: past timeout_ns it records MS_ERR_TIMEOUT and returns false; a waiting
// CTA also returns false once it sees that another CTA has recorded a time-out.
template <int K>
__device__ bool gsync_reduce(const SolveArgs& a, Shared& sh) {
    const unsigned nb = sh.nb;
    const int npair = K * a.V;
    // (the one-CTA summation gives every sum at least one thread: npair <= kBS)
    if ((long)npair * nb <= 16384 && npair <= kBS) {
        __syncthreads();
        if (threadIdx.x == 0) {
            cuda::atomic_ref<unsigned, cuda::thread_scope_device> g(a.bar[1]);
            cuda::atomic_ref<unsigned, cuda::thread_scope_device> c(a.bar[0]);
            sh.mine = g.load(cuda::memory_order_relaxed);
            sh.last = c.fetch_add(1u, cuda::memory_order_acq_rel) == nb - 1;
        }
        __syncthreads();
        if (sh.last) {
            if (K > 0) {
                // S segments of the CTAs per sum, one thread each, then the S segment sums
                // in order (staged in sh.red, which no phase uses across a barrier)
                const int S = max(1, min(kBS / max(npair, 1), (int)nb));
                const int t = threadIdx.x;
                if (t < npair * S) {
                    const int i = t / S, sg = t % S;
                    const unsigned b0 = (unsigned)((long)sg * nb / S), b1 = (unsigned)((long)(sg + 1) * nb / S);
                    const double* src = a.part + (size_t)i * nb;
                    double acc = 0.0;
                    for (unsigned b = b0; b < b1; ++b) acc += __ldcg(src + b);
                    sh.red[0][t] = acc;
                }
                __syncthreads();
                for (int i = t; i < npair; i += kBS) {
                    double acc = 0.0;
                    for (int sg = 0; sg < S; ++sg) acc += sh.red[0][i * S + sg];
                    __stcg(a.scal + i, acc);
                }
                __syncthreads();
            }
            gsync_release(a, sh);
        }
        return gsync_finish<K>(a, sh);
    }
    const unsigned grp = (unsigned)sh.cta / kGroup;
    const unsigned ngrp = (nb + kGroup - 1) / kGroup;
    __syncthreads();
    if (threadIdx.x == 0) {
        cuda::atomic_ref<unsigned, cuda::thread_scope_device> g(a.bar[1]);
        cuda::atomic_ref<unsigned, cuda::thread_scope_device> gc(a.bar[2 + grp]);
        sh.mine = g.load(cuda::memory_order_relaxed);
        const unsigned gsize = min((unsigned)kGroup, nb - grp * kGroup);
        sh.glast = gc.fetch_add(1u, cuda::memory_order_acq_rel) == gsize - 1;
        if (sh.glast) gc.store(0u, cuda::memory_order_relaxed);
        sh.last = 0;
    }
    __syncthreads();
    if (sh.glast) {
        if (K > 0) {  // group sums, in CTA order
            const unsigned b0 = grp * kGroup, b1 = min(nb, b0 + kGroup);
            for (int i = threadIdx.x; i < npair; i += kBS) {
                const double* src = a.part + (size_t)i * nb;
                double acc = 0.0;
                for (unsigned b = b0; b < b1; ++b) acc += __ldcg(src + b);
                __stcg(a.gpart + (size_t)grp * kAcc * a.V + i, acc);
            }
            __syncthreads();
        }
        if (threadIdx.x == 0) {
            cuda::atomic_ref<unsigned, cuda::thread_scope_device> c(a.bar[0]);
            sh.last = c.fetch_add(1u, cuda::memory_order_acq_rel) == ngrp - 1;
        }
        __syncthreads();
    }
    if (sh.last) {
        if (K > 0) {  // grid sums, in group order
            for (int i = threadIdx.x; i < npair; i += kBS) {
                double acc = 0.0;
                for (unsigned gi = 0; gi < ngrp; ++gi) acc += __ldcg(a.gpart + (size_t)gi * kAcc * a.V + i);
                __stcg(a.scal + i, acc);
            }
        }
        __syncthreads();
        gsync_release(a, sh);
    }
    return gsync_finish<K>(a, sh);
}

__device__ __forceinline__ bool gsync(const SolveArgs& a, Shared& sh) { return gsync_reduce<0>(a, sh); }

// Rows [r0, r1) of a chunk, one sub-warp of S lanes per row; fn(row, valid, sl).
template <typename Fn>
__device__ __forceinline__ void rows_by_subwarp(int64_t r0, int64_t r1, int S, Fn fn) {
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int spw = 32 / S;
    const int64_t n = r1 - r0;
    for (int64_t base = (int64_t)w * spw; base < n; base += (int64_t)kNW * spw) {
        const int64_t row = r0 + base + lane / S;
        fn(row, row < r1, lane & (S - 1));
    }
}


// ---------------------------------------------------------------- wide (SpMM) layout
//
// The right-hand sides of a launch stored row-major: element (row, r) at row * RW + r,
// RW = the power of 2 >= R.  Thread t works for right-hand side t % RW in every phase
// (kBS and 32 are multiples of RW).  In a mat-vec phase the RW lanes of a row read its
// matrix entries once (the same address in every lane: one broadcast load) and gather RW
// consecutive vector elements per column, so a CSR read serves all right-hand sides.
// Chunks of a.crow = 512 / RW rows hold one element per thread.

template <int K>
__device__ __forceinline__ void flush_wide(const SolveArgs& a, Shared& sh, double* acc, int l) {
#pragma unroll
    for (int k = 0; k < K; ++k) {
        sh.red[k][threadIdx.x] = acc[k];
        acc[k] = 0.0;
    }
    __syncthreads();
    const int RW = a.RW;
    for (int i = threadIdx.x; i < K * RW; i += kBS) {
        const int k = i / RW, r = i % RW;
        double t = 0.0;
        for (int j = r; j < kBS; j += RW) t += sh.red[k][j];
        if (r < a.R) sh.acc[k][r * a.L + l] += t;
    }
    __syncthreads();
}

// body(l, r0, r1, acc) over this CTA's chunks of the levels where sel(r L + l) holds for
// some right-hand side r; per-CTA sums as in run_phase.
template <int K, typename Sel, typename Body>
__device__ __forceinline__ void run_phase_wide(const SolveArgs& a, Shared& sh, Sel sel, Body body) {
    if (K > 0) {
        for (int i = threadIdx.x; i < kAcc * kMaxV; i += kBS) (&sh.acc[0][0])[i] = 0.0;
        __syncthreads();
    }
    double acc[K > 0 ? K : 1];
#pragma unroll
    for (int k = 0; k < (K > 0 ? K : 1); ++k) acc[k] = 0.0;
    int cur = -1;
    const int nb = sh.nb, C = a.C;
    int l = 0, lsel = -1;
    bool lok = false;
    for (int c = sh.cta; c < C;) {
        while (c >= a.coff[l + 1]) ++l;
        if (l != lsel) {
            lsel = l;
            lok = false;
            for (int r = 0; r < a.R; ++r) lok |= sel(r * a.L + l);
        }
        if (!lok) {
            c += (a.coff[l + 1] - c + nb - 1) / nb * nb;
            continue;
        }
        if (K > 0 && l != cur) {
            if (cur >= 0) flush_wide<K>(a, sh, acc, cur);
            cur = l;
        }
        const int64_t r0 = a.off[l] + (int64_t)(c - a.coff[l]) * a.crow;
        const int64_t r1 = min(r0 + (int64_t)a.crow, a.off[l + 1]);
        body(l, r0, r1, acc);
        c += nb;
    }
    if (K > 0) {
        if (cur >= 0) flush_wide<K>(a, sh, acc, cur);
        for (int i = threadIdx.x; i < K * a.V; i += kBS) {
            const int k = i / a.V, v = i % a.V;
            a.part[((size_t)k * a.V + v) * sh.nb + sh.cta] = sh.acc[k][v];
        }
    }
}

// Elements (row, r) of rows [r0, r1): fn(row, i = row * RW + r); r = this thread's lane.
template <typename Fn>
__device__ __forceinline__ void elems_wide(const SolveArgs& a, int64_t r0, int64_t r1, Fn fn) {
    const int RW = a.RW;
    const int64_t n = (r1 - r0) * RW;
    for (int64_t e = threadIdx.x; e < n; e += kBS) {
        const int64_t row = r0 + e / RW;
        fn(row, row * RW + (e % RW));
    }
}

// Rows [r0, r1), RW lanes per row (32 / RW rows per warp): fn(row) for this thread's row.
template <typename Fn>
__device__ __forceinline__ void rows_wide(const SolveArgs& a, int64_t r0, int64_t r1, Fn fn) {
    const int RW = a.RW;
    const int rpw = 32 / RW;
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int64_t base = r0 + (int64_t)w * rpw; base < r1; base += (int64_t)kNW * rpw) {
        const int64_t row = base + lane / RW;
        if (row < r1) fn(row);
    }
}

// sum_k val[k] * x[col[k] * RW + r] over [s, e): the row's entries read by all RW lanes.
template <typename TV, typename TX, typename TA>
__device__ __forceinline__ TA csr_row_wide(const int32_t* __restrict__ col, const TV* __restrict__ val,
                                           const TX* x, int64_t s, int64_t e, int r, int RW) {
    TA acc = TA(0);
    int64_t k = s;
    for (; k + 3 < e; k += 4) {
        const int32_t c0 = __ldg(col + k), c1 = __ldg(col + k + 1), c2 = __ldg(col + k + 2), c3 = __ldg(col + k + 3);
        const TV v0 = __ldg(val + k), v1 = __ldg(val + k + 1), v2 = __ldg(val + k + 2), v3 = __ldg(val + k + 3);
        const TX x0 = x[(int64_t)c0 * RW + r], x1 = x[(int64_t)c1 * RW + r], x2 = x[(int64_t)c2 * RW + r],
                 x3 = x[(int64_t)c3 * RW + r];
        acc += (TA)v0 * (TA)x0;
        acc += (TA)v1 * (TA)x1;
        acc += (TA)v2 * (TA)x2;
        acc += (TA)v3 * (TA)x3;
    }
    for (; k < e; ++k) acc += (TA)__ldg(val + k) * (TA)x[(int64_t)__ldg(col + k) * RW + r];
    return acc;
}

// ---------------------------------------------------------------- level solve

// Solve A_l x_l = beta_l for the levels [l0, l1) of every right-hand side, x warm.
// tight_all: every level to a.tol, else only level l0 to a.tol and the others to
// a.inter_tol.
// Decisions after an FP64 true residual (P1), one thread per virtual level: converged,
// zero right-hand side, non-finite, out of iterations, or one more refinement round
// (with its stopping target; MIXED levels whose rounds stall switch to FP64 inner CG).
// Sets my_any / my_zero for the caller's block vote.
template <int MODE>
__device__ __forceinline__ void decide_outer(const SolveArgs& a, Shared& sh, bool first_outer, int& my_any,
                                             int& my_zero) {
    const int tid = threadIdx.x;
    const int V = a.V, L = a.L;
    my_any = 0;
    my_zero = 0;
    for (int v = tid; v < V; v += kBS) {
        if (!sh.oact[v]) continue;
        const int l = v % L;
        const double rr = sh.out[0][v];
        if (first_outer) sh.bb[v] = sh.out[1][v];
        const double bb = sh.bb[v];
        sh.vbytes[v] += (double)a.nnzA[l] * 12.0 + (double)(a.off[l + 1] - a.off[l]) * 32.0;
        if (!isfinite(rr) || !isfinite(bb)) {
            sh.oact[v] = 0;
            if (sh.cta == 0) atomicCAS(a.status, 0, (int)MS_ERR_NUMERIC);
            continue;
        }
        if (bb == 0.0) {  // zero right-hand side: the solution is zero
            sh.zero[v] = 1;
            sh.oact[v] = 0;
            my_zero = 1;
            if (sh.cta == 0) a.resid[v] = 0.0;
            continue;
        }
        const double res = sqrt(rr / bb);
        if (sh.cta == 0) a.resid[v] = res;
        if (res <= sh.tol[v]) {
            sh.oact[v] = 0;
            continue;
        }
        if (sh.it_solve[v] >= a.max_iters) {
            sh.oact[v] = 0;
            if (sh.cta == 0) atomicCAS(a.status, 0, (int)MS_ERR_NOT_CONVERGED);
            continue;
        }
        // MIXED: an outer round that did not halve the true residual means the FP32 inner
        // CG stalls on this level (conditioning beyond FP32): run its inner CG in FP64
        if (MODE == 1 && !sh.f64[v] && res > 0.5 * sh.prevres[v]) {
            sh.f64[v] = 1;
            sh.f64n[v] += 1;
        }
        sh.prevres[v] = res;
        my_any = 1;
        sh.refines[v] += 1;
        sh.act[v] = 1;
        sh.first[v] = 1;
        if (MODE == 0 || sh.f64[v]) {
            // recursive-residual target, with margin below the true-residual tolerance
            sh.target[v] = 0.25 * sh.tol[v] * sh.tol[v] * bb;
        } else {
            sh.scale[v] = 1.0 / sqrt(rr);
            const double need = 0.5 * sh.tol[v] * sqrt(bb) * sh.scale[v];
            const double t = fmax(a.inner_tol, fmin(need, 1.0));
            sh.target[v] = t * t;
        }
    }
}

// Decisions after the mat-vec and its dots, one thread per active virtual level: the
// CG step sizes, convergence of the recursive residual, break-downs (preconditioner
// fall-back, curvature loss, not SPD).  Returns whether this thread's levels go on.
template <int MODE>
__device__ __forceinline__ int decide_inner(const SolveArgs& a, Shared& sh, bool use_pc) {
    const int tid = threadIdx.x;
    const int V = a.V, L = a.L;
    int my_go = 0;
    for (int v = tid; v < V; v += kBS) {
        if (!sh.act[v]) continue;
        const int l = v % L;
        const double gam = sh.out[0][v], del = sh.out[1][v], rho = sh.out[2][v];
        const bool dbl = MODE == 0 || sh.f64[v];
        const bool lpc = use_pc && !sh.pcoff[v] && !dbl;
        const double n = (double)(a.off[l + 1] - a.off[l]);
        sh.vbytes[v] += (double)a.nnzA[l] * (dbl ? 12.0 : 8.0) + n * (dbl ? 32.0 : (lpc ? 24.0 : 20.0));
        if (lpc) sh.vbytes[v] += n * (2.0 * kPcOut * 10.0 + 16.0);
        if (!isfinite(gam) || !isfinite(del) || !isfinite(rho)) {
            sh.act[v] = 0;
            sh.oact[v] = 0;
            if (sh.cta == 0) atomicCAS(a.status, 0, (int)MS_ERR_NUMERIC);
            continue;
        }
        if (rho <= sh.target[v] || sh.it_solve[v] >= a.max_iters) {
            sh.act[v] = 0;  // converged (recursive residual) or capped
            continue;
        }
        if (lpc && !(gam > 0.0)) {
            // r^T M r <= 0 cannot happen for an SPD M: treat the preconditioner as
            // broken and fall back to plain CG from the current iterate
            sh.pcoff[v] = 1;
            sh.fb[v] += 1;
            sh.act[v] = 0;
            continue;
        }
        double al, be;
        if (sh.first[v]) {
            be = 0.0;
            al = del > 0.0 ? gam / del : -1.0;
        } else {
            be = gam / sh.gam[v];
            const double den = del - be * gam / sh.alpha[v];
            al = den > 0.0 ? gam / den : -1.0;
        }
        if (!(al > 0.0)) {
            if (MODE == 1 && !sh.first[v]) {  // (FP32, or an FP64 fallback level)
                // lost curvature in the FP32 recurrence (cancellation on an ill-conditioned
                // level): end this inner solve; the FP64 true residual restarts it
                sh.act[v] = 0;
                continue;
            }
            if (lpc) {  // u^T A u <= 0 at a restart: the preconditioner is unusable here
                sh.pcoff[v] = 1;
                sh.fb[v] += 1;
                sh.act[v] = 0;
                continue;
            }
            // p^T A p <= 0 at a restart: A_l is not positive definite in floating point
            sh.act[v] = 0;
            sh.oact[v] = 0;
            if (sh.cta == 0) atomicCAS(a.status, 0, (int)MS_ERR_NOT_SPD);
            continue;
        }
        sh.fresh[v] = sh.first[v];  // the update must not read the old p, s
        sh.first[v] = 0;
        sh.alpha[v] = al;
        sh.beta[v] = be;
        sh.gam[v] = gam;
        sh.it_solve[v] += 1;
        sh.it_total[v] += 1;
        sh.vbytes[v] += n * (dbl ? 72.0 : 36.0);
        my_go = 1;
    }
    return my_go;
}

template <int MODE>
__device__ bool solve_levels(const SolveArgs& a, Shared& sh, int l0, int l1, bool tight_all) {
    const int tid = threadIdx.x;
    const int V = a.V, L = a.L;
    for (int v = tid; v < kMaxV; v += kBS) {
        const int l = v % L;
        sh.oact[v] = (v < V && l >= l0 && l < l1) ? 1 : 0;
        sh.act[v] = 0;
        sh.zero[v] = 0;
        sh.pcoff[v] = 0;
        sh.prevres[v] = INFINITY;
        sh.it_solve[v] = 0;
        sh.tol[v] = (tight_all || l == l0) ? a.tol : a.inter_tol;
    }
    __syncthreads();
    bool first_outer = true;
    for (int outer = 0; outer < a.max_outer; ++outer) {
        // ---- P1: FP64 true residual r = b - A x (FP64 CSR)
        run_phase<2>(a, sh, [&](int v) { return sh.oact[v] != 0; }, [&](const Chunk& ch, double* acc) {
            const int S = a.tprA[ch.l];
            const double* xv = a.x + ch.vb;
            rows_by_subwarp(ch.r0, ch.r1, S, [&](int64_t row, bool ok, int sl) {
                int64_t s = 0, e = 0;
                if (ok) { s = a.Arp[row]; e = a.Arp[row + 1]; }
                const double y = csr_row<double, double, double>(a.Acol, a.Av64, xv, s, e, sl, S);
                if (ok && sl == 0) {
                    const double b = a.beta[ch.vb + row];
                    const double ri = b - y;
                    a.r[ch.vb + row] = ri;
                    acc[0] += ri * ri;
                    acc[1] += b * b;
                }
            });
        });
        prof(sh, kPrfResid);
        if (!gsync_reduce<2>(a, sh)) return false;
        // decisions: one thread per virtual level
        int my_any = 0, my_zero = 0;
        decide_outer<MODE>(a, sh, first_outer, my_any, my_zero);
        const bool any = __syncthreads_or(my_any) != 0;
        const bool anyzero = __syncthreads_or(my_zero) != 0;
        prof(sh, kPrfScalar);
        first_outer = false;
        {
            if (anyzero) {
                run_phase<0>(a, sh, [&](int v) { return sh.zero[v] != 0; }, [&](const Chunk& ch, double*) {
                    for (int64_t row = ch.r0 + tid; row < ch.r1; row += kBS) a.x[ch.vb + row] = 0.0;
                });
                prof(sh, kPrfOther);
                // other CTAs read these rows in the next phases
                if (!gsync(a, sh)) return false;
                for (int v = tid; v < kMaxV; v += kBS) sh.zero[v] = 0;
                __syncthreads();
            }
        }
        if (!any) break;

        if (MODE == 1) {
            // ---- P2: r32 = r / |r|, x32 = 0
            run_phase<0>(a, sh, [&](int v) { return sh.act[v] != 0 && !sh.f64[v]; }, [&](const Chunk& ch, double*) {
                const double sc = sh.scale[ch.v];
                for (int64_t row = ch.r0 + tid; row < ch.r1; row += kBS) {
                    a.r32[ch.vb + row] = (float)(a.r[ch.vb + row] * sc);
                    a.x32[ch.vb + row] = 0.f;
                }
            });
            for (int v = tid; v < V; v += kBS)
                if (sh.act[v] && !sh.f64[v]) sh.vbytes[v] += (double)(a.off[v % L + 1] - a.off[v % L]) * 16.0;
            prof(sh, kPrfOther);
            if (!gsync(a, sh)) return false;
        }

        // ---- inner CG iterations (single-reduction form; preconditioned with
        //      M = G^T G in MIXED mode when a.pc: u = M r, otherwise u = r)
        for (;;) {
            const bool use_pc = MODE == 1 && a.pc;
            if (use_pc) {
                // G1: u1 = ghat r  (row pattern: self + preceding neighbours; the level's
                //     factor delta^d of G^T G is applied in G2)
                run_phase<0>(a, sh, [&](int v) { return sh.act[v] != 0 && !sh.pcoff[v] && !sh.f64[v]; },
                             [&](const Chunk& ch, double*) {
                                 // two lanes per row (slots k = half, half + 2, ...), all threads busy
                                 const float* rv = a.r32 + ch.vb;
                                 const int half = tid & 1;
                                 for (int64_t base = ch.r0; base < ch.r1; base += kBS / 2) {
                                     const int64_t row = base + (tid >> 1);
                                     float acc = 0.f;
                                     if (row < ch.r1) {
#pragma unroll
                                         for (int k = half; k < kPcOut; k += 2) {
                                             const int32_t c = __ldg(a.gcol + k * a.N + row);
                                             if (c >= 0) acc = fmaf(__half2float(__ldg(a.gval + k * a.N + row)), rv[c], acc);
                                         }
                                     }
                                     acc += __shfl_xor_sync(0xffffffffu, acc, 1);
                                     if (row < ch.r1 && half == 0) a.u1_32[ch.vb + row] = acc;
                                 }
                             });
                prof(sh, kPrfOther);
                if (!gsync(a, sh)) return false;
                // G2: u = delta^d ghat^T u1 = G^T G r
                run_phase<0>(a, sh, [&](int v) { return sh.act[v] != 0 && !sh.pcoff[v] && !sh.f64[v]; },
                             [&](const Chunk& ch, double*) {
                                 const float* u1 = a.u1_32 + ch.vb;
                                 rows_by_subwarp(ch.r0, ch.r1, 2, [&](int64_t row, bool ok, int sl) {
                                     int64_t s = 0, e = 0;
                                     if (ok) { s = __ldg(a.gt_rp + row); e = __ldg(a.gt_rp + row + 1); }
                                     const float y = csr_row<__half, float, float>(a.gt_col, a.gt_val, u1, s, e, sl, 2);
                                     if (ok && sl == 0) a.u32[ch.vb + row] = a.pcs[ch.l] * y;
                                 });
                             });
                prof(sh, kPrfOther);
                if (!gsync(a, sh)) return false;
            }
            // M: w = A u; gamma = r.u, delta = w.u, rho = r.r
            run_phase<3>(a, sh, [&](int v) { return sh.act[v] != 0; }, [&](const Chunk& ch, double* acc) {
                if (MODE == 0 || sh.f64[ch.v]) {
                    const int S = a.tprA[ch.l];
                    const double* rv = a.r + ch.vb;
                    rows_by_subwarp(ch.r0, ch.r1, S, [&](int64_t row, bool ok, int sl) {
                        int64_t s = 0, e = 0;
                        if (ok) { s = a.Arp[row]; e = a.Arp[row + 1]; }
                        const double y = csr_row<double, double, double>(a.Acol, a.Av64, rv, s, e, sl, S);
                        if (ok && sl == 0) {
                            const double ri = rv[row];
                            a.q[ch.vb + row] = y;
                            acc[0] += ri * ri;
                            acc[1] += ri * y;
                            acc[2] += ri * ri;
                        }
                    });
                    return;
                }
                const float* uin = ((use_pc && !sh.pcoff[ch.v]) ? a.u32 : a.r32) + ch.vb;
                const float* rv = a.r32 + ch.vb;
                float* qv = a.q32 + ch.vb;
                if (a.mf) {
                    // matrix-free: the cells whose first point lies in [r0, r1)
                    const MFLevel& g = a.mfv.lv[ch.l];
                    int64_t cfirst = a.mfv.cellid[ch.r0];
                    if (a.mfv.cell_start[g.cell_off + cfirst] < ch.r0) ++cfirst;
                    const int64_t cend = (int64_t)a.mfv.cellid[ch.r1 - 1] + 1;
                    mf_cells_any(a.mfv, ch.l, cfirst, cend, tid >> 5, kNW, a.mf_tpp, uin,
                                 [&](int64_t row, float y) {
                                     const float ri = rv[row], ui = uin[row];
                                     qv[row] = y;
                                     acc[0] += (double)ri * (double)ui;
                                     acc[1] += (double)ui * (double)y;
                                     acc[2] += (double)(ri * ri);
                                 });
                    return;
                }
                const int S = a.tprA[ch.l];
                rows_by_subwarp(ch.r0, ch.r1, S, [&](int64_t row, bool ok, int sl) {
                    int64_t s = 0, e = 0;
                    if (ok) { s = a.Arp[row]; e = a.Arp[row + 1]; }
                    const float y = csr_row<float, float, float>(a.Acol, a.Av32, uin, s, e, sl, S);
                    if (ok && sl == 0) {
                        const float ri = rv[row], ui = uin[row];
                        qv[row] = y;
                        acc[0] += (double)ri * (double)ui;
                        acc[1] += (double)ui * (double)y;
                        acc[2] += (double)(ri * ri);
                    }
                });
            });
            prof(sh, kPrfMatvec);
            if (!gsync_reduce<3>(a, sh)) return false;
            const int my_go = decide_inner<MODE>(a, sh, use_pc);
            const bool go = __syncthreads_or(my_go) != 0;
            prof(sh, kPrfScalar);
            if (!go) break;
            // E: p = u + beta p; s = w + beta s; x += alpha p; r -= alpha s
            run_phase<0>(a, sh, [&](int v) { return sh.act[v] != 0; }, [&](const Chunk& ch, double*) {
                const double al = sh.alpha[ch.v], be = sh.beta[ch.v];
                // first iteration: p = u, s = w (the old p, s are not read: they may
                // hold anything, and 0 * NaN would poison the recurrence)
                const bool fr = sh.fresh[ch.v] != 0;
                const int64_t vb = ch.vb;
                if (MODE == 0 || sh.f64[ch.v]) {
                    for (int64_t row = ch.r0 + tid; row < ch.r1; row += kBS) {
                        const int64_t i = vb + row;
                        const double ri = a.r[i];
                        const double pi = fr ? ri : ri + be * a.p[i];
                        const double si = fr ? a.q[i] : a.q[i] + be * a.s[i];
                        a.p[i] = pi;
                        a.s[i] = si;
                        a.x[i] += al * pi;
                        a.r[i] = ri - al * si;
                    }
                    return;
                }
                const float af = (float)al, bf = (float)be;
                if (use_pc && !sh.pcoff[ch.v]) {
                    // u = M r is its own vector, so the (p, x) and (s, r) halves of a row are
                    // independent: threads [0, kBS/2) update p and x, threads [kBS/2, kBS)
                    // update s and r, and all threads are busy on a chunk of kBS/2 rows
                    const bool px = tid < kBS / 2;
                    const int t2 = px ? tid : tid - kBS / 2;
                    for (int64_t row = ch.r0 + t2; row < ch.r1; row += kBS / 2) {
                        const int64_t i = vb + row;
                        if (px) {
                            const float pi = fr ? a.u32[i] : fmaf(bf, a.p32[i], a.u32[i]);
                            a.p32[i] = pi;
                            a.x32[i] = fmaf(af, pi, a.x32[i]);
                        } else {
                            const float si = fr ? a.q32[i] : fmaf(bf, a.s32[i], a.q32[i]);
                            a.s32[i] = si;
                            a.r32[i] = fmaf(-af, si, a.r32[i]);
                        }
                    }
                    return;
                }
                for (int64_t row = ch.r0 + tid; row < ch.r1; row += kBS) {
                    const int64_t i = vb + row;
                    const float ri = a.r32[i];
                    const float pi = fr ? ri : fmaf(bf, a.p32[i], ri);
                    const float si = fr ? a.q32[i] : fmaf(bf, a.s32[i], a.q32[i]);
                    a.p32[i] = pi;
                    a.s32[i] = si;
                    a.x32[i] = fmaf(af, pi, a.x32[i]);
                    a.r32[i] = fmaf(-af, si, ri);
                }
            });
            prof(sh, kPrfUpdate);
            if (!gsync(a, sh)) return false;
        }

        if (MODE == 1) {
            // ---- P3: x += |r| d  (FP64)
            run_phase<0>(a, sh, [&](int v) { return sh.oact[v] != 0 && sh.scale[v] > 0.0 && !sh.f64[v]; },
                         [&](const Chunk& ch, double*) {
                             const double inv = 1.0 / sh.scale[ch.v];
                             for (int64_t row = ch.r0 + tid; row < ch.r1; row += kBS)
                                 a.x[ch.vb + row] += (double)a.x32[ch.vb + row] * inv;
                         });
            for (int v = tid; v < V; v += kBS)
                if (sh.oact[v] && !sh.f64[v]) sh.vbytes[v] += (double)(a.off[v % L + 1] - a.off[v % L]) * 20.0;
            prof(sh, kPrfOther);
            if (!gsync(a, sh)) return false;
        }
    }
    // levels still active after max_outer rounds did not reach the tolerance
    if (sh.cta == 0)
        for (int v = tid; v < V; v += kBS)
            if (sh.oact[v]) atomicCAS(a.status, 0, (int)MS_ERR_NOT_CONVERGED);
    __syncthreads();
    return true;
}


// solve_levels for the wide layout (no preconditioner, CSR operators).
template <int MODE>
__device__ bool solve_levels_wide(const SolveArgs& a, Shared& sh, int l0, int l1, bool tight_all) {
    const int tid = threadIdx.x;
    const int V = a.V, L = a.L, RW = a.RW;
    const int rl = tid % RW;  // this thread's right-hand side
    const bool rok = rl < a.R;
    for (int v = tid; v < kMaxV; v += kBS) {
        const int l = v % L;
        sh.oact[v] = (v < V && l >= l0 && l < l1) ? 1 : 0;
        sh.act[v] = 0;
        sh.zero[v] = 0;
        sh.pcoff[v] = 0;
        sh.prevres[v] = INFINITY;
        sh.it_solve[v] = 0;
        sh.tol[v] = (tight_all || l == l0) ? a.tol : a.inter_tol;
    }
    __syncthreads();
    bool first_outer = true;
    for (int outer = 0; outer < a.max_outer; ++outer) {
        // ---- P1: FP64 true residual r = b - A x (FP64 CSR)
        run_phase_wide<2>(a, sh, [&](int v) { return sh.oact[v] != 0; },
                          [&](int l, int64_t r0, int64_t r1, double* acc) {
                              if (!(rok && sh.oact[rl * L + l])) return;
                              rows_wide(a, r0, r1, [&](int64_t row) {
                                  const double y = csr_row_wide<double, double, double>(
                                      a.Acol, a.Av64, a.x, a.Arp[row], a.Arp[row + 1], rl, RW);
                                  const int64_t i = row * RW + rl;
                                  const double b = a.beta[i];
                                  const double ri = b - y;
                                  a.r[i] = ri;
                                  acc[0] += ri * ri;
                                  acc[1] += b * b;
                              });
                          });
        prof(sh, kPrfResid);
        if (!gsync_reduce<2>(a, sh)) return false;
        int my_any = 0, my_zero = 0;
        decide_outer<MODE>(a, sh, first_outer, my_any, my_zero);
        const bool any = __syncthreads_or(my_any) != 0;
        const bool anyzero = __syncthreads_or(my_zero) != 0;
        prof(sh, kPrfScalar);
        first_outer = false;
        if (anyzero) {
            run_phase_wide<0>(a, sh, [&](int v) { return sh.zero[v] != 0; },
                              [&](int l, int64_t r0, int64_t r1, double*) {
                                  if (!(rok && sh.zero[rl * L + l])) return;
                                  elems_wide(a, r0, r1, [&](int64_t, int64_t i) { a.x[i] = 0.0; });
                              });
            prof(sh, kPrfOther);
            if (!gsync(a, sh)) return false;
            for (int v = tid; v < kMaxV; v += kBS) sh.zero[v] = 0;
            __syncthreads();
        }
        if (!any) break;

        if (MODE == 1) {
            // ---- P2: r32 = r / |r|, x32 = 0
            run_phase_wide<0>(a, sh, [&](int v) { return sh.act[v] != 0 && !sh.f64[v]; },
                              [&](int l, int64_t r0, int64_t r1, double*) {
                                  const int v = rl * L + l;
                                  if (!(rok && sh.act[v] && !sh.f64[v])) return;
                                  const double sc = sh.scale[v];
                                  elems_wide(a, r0, r1, [&](int64_t, int64_t i) {
                                      a.r32[i] = (float)(a.r[i] * sc);
                                      a.x32[i] = 0.f;
                                  });
                              });
            for (int v = tid; v < V; v += kBS)
                if (sh.act[v] && !sh.f64[v]) sh.vbytes[v] += (double)(a.off[v % L + 1] - a.off[v % L]) * 16.0;
            prof(sh, kPrfOther);
            if (!gsync(a, sh)) return false;
        }

        // ---- inner CG iterations (single-reduction form, u = r)
        for (;;) {
            // M: w = A r; gamma = r.r, delta = w.r, rho = r.r
            run_phase_wide<3>(a, sh, [&](int v) { return sh.act[v] != 0; },
                              [&](int l, int64_t r0, int64_t r1, double* acc) {
                                  const int v = rl * L + l;
                                  if (!(rok && sh.act[v])) return;
                                  if (MODE == 0 || sh.f64[v]) {
                                      rows_wide(a, r0, r1, [&](int64_t row) {
                                          const double y = csr_row_wide<double, double, double>(
                                              a.Acol, a.Av64, a.r, a.Arp[row], a.Arp[row + 1], rl, RW);
                                          const int64_t i = row * RW + rl;
                                          const double ri = a.r[i];
                                          a.q[i] = y;
                                          acc[0] += ri * ri;
                                          acc[1] += ri * y;
                                          acc[2] += ri * ri;
                                      });
                                  } else {
                                      rows_wide(a, r0, r1, [&](int64_t row) {
                                          const float y = csr_row_wide<float, float, float>(
                                              a.Acol, a.Av32, a.r32, a.Arp[row], a.Arp[row + 1], rl, RW);
                                          const int64_t i = row * RW + rl;
                                          const float ri = a.r32[i];
                                          a.q32[i] = y;
                                          acc[0] += (double)ri * (double)ri;
                                          acc[1] += (double)ri * (double)y;
                                          acc[2] += (double)(ri * ri);
                                      });
                                  }
                              });
            prof(sh, kPrfMatvec);
            if (!gsync_reduce<3>(a, sh)) return false;
            const int my_go = decide_inner<MODE>(a, sh, false);
            const bool go = __syncthreads_or(my_go) != 0;
            prof(sh, kPrfScalar);
            if (!go) break;
            // E: p = r + beta p; s = w + beta s; x += alpha p; r -= alpha s
            run_phase_wide<0>(a, sh, [&](int v) { return sh.act[v] != 0; },
                              [&](int l, int64_t r0, int64_t r1, double*) {
                                  const int v = rl * L + l;
                                  if (!(rok && sh.act[v])) return;
                                  const double al = sh.alpha[v], be = sh.beta[v];
                                  const bool fr = sh.fresh[v] != 0;
                                  if (MODE == 0 || sh.f64[v]) {
                                      elems_wide(a, r0, r1, [&](int64_t, int64_t i) {
                                          const double ri = a.r[i];
                                          const double pi = fr ? ri : ri + be * a.p[i];
                                          const double si = fr ? a.q[i] : a.q[i] + be * a.s[i];
                                          a.p[i] = pi;
                                          a.s[i] = si;
                                          a.x[i] += al * pi;
                                          a.r[i] = ri - al * si;
                                      });
                                  } else {
                                      const float af = (float)al, bf = (float)be;
                                      elems_wide(a, r0, r1, [&](int64_t, int64_t i) {
                                          const float ri = a.r32[i];
                                          const float pi = fr ? ri : fmaf(bf, a.p32[i], ri);
                                          const float si = fr ? a.q32[i] : fmaf(bf, a.s32[i], a.q32[i]);
                                          a.p32[i] = pi;
                                          a.s32[i] = si;
                                          a.x32[i] = fmaf(af, pi, a.x32[i]);
                                          a.r32[i] = fmaf(-af, si, ri);
                                      });
                                  }
                              });
            prof(sh, kPrfUpdate);
            if (!gsync(a, sh)) return false;
        }

        if (MODE == 1) {
            // ---- P3: x += |r| d  (FP64)
            run_phase_wide<0>(a, sh, [&](int v) { return sh.oact[v] != 0 && sh.scale[v] > 0.0 && !sh.f64[v]; },
                              [&](int l, int64_t r0, int64_t r1, double*) {
                                  const int v = rl * L + l;
                                  if (!(rok && sh.oact[v] && sh.scale[v] > 0.0 && !sh.f64[v])) return;
                                  const double inv = 1.0 / sh.scale[v];
                                  elems_wide(a, r0, r1, [&](int64_t, int64_t i) { a.x[i] += (double)a.x32[i] * inv; });
                              });
            for (int v = tid; v < V; v += kBS)
                if (sh.oact[v] && !sh.f64[v]) sh.vbytes[v] += (double)(a.off[v % L + 1] - a.off[v % L]) * 20.0;
            prof(sh, kPrfOther);
            if (!gsync(a, sh)) return false;
        }
    }
    if (sh.cta == 0)
        for (int v = tid; v < V; v += kBS)
            if (sh.oact[v]) atomicCAS(a.status, 0, (int)MS_ERR_NOT_CONVERGED);
    __syncthreads();
    return true;
}

// beta_k -= B_km t_m for the rows [r0, r1) of one chunk of level k > m, with the coarse
// level's points staged in shared memory: the box of level-m cells within R cells of the
// rows' cells is found (a block min/max of the rows' frames), the FP32 positions in the box
// of its points are copied once (box cell by box cell, x fastest; axis by axis into the
// reduction scratch sh.red, which no phase keeps across a barrier, so the CTA's shared
// memory and the L1 share left to the mat-vecs stay as they are), and then a warp per row
// tests the points of its (2R+1)^d cells from shared memory: the cells of one (z, y) line of
// the box are contiguous there, so a row reads (2R+1)^(d-1) ranges, with no dependent
// global loads between them.  Survivors of the FP32 test (the band of the per-warp form,
// r^2 <= 1 + 1e-4; the positions' rounding, ~1e-6, is far inside it) are queued with their
// cell and their double-float entries ff_entry_dc computed 32 at a time; the entries and
// their order are those of lower_row_mf_warp (the queue holds the survivors in the same
// order), so the sums agree with it up to the rare candidate at r ~ 1 that one FP32 test
// keeps and the other drops (its entry is 0).  Returns false, with nothing written, when
// the box has more than kLCells cells or more points than the scratch holds (the caller
// then takes the per-warp form).  Called by every thread of the CTA with the same chunk.
template <int D, int E, int K>
__device__ __forceinline__ bool lower_chunk_staged(const SolveArgs& a, Shared& sh, const Chunk& ch, int m) {
    constexpr int kCap = (int)(sizeof(sh.red) / sizeof(float)) / D;  // staged points
    float* const sp = reinterpret_cast<float*>(&sh.red[0][0]);        // axis ax at sp + ax kCap
    const int tid = threadIdx.x, wid = tid >> 5, lane = tid & 31;
    const HierView& v = a.hv;
    const LevelGrid& g = v.grid[m];
    const int R = v.R, k = ch.l;
    const Frame* frm = a.frames + a.fbase[k] + m;  // frame of row r in level m: frm[(r - off[k]) (k + 1)]
    // 1. the rows' cells: block minima and maxima
    int lo[3] = {0x7fffffff, 0x7fffffff, 0x7fffffff}, hi[3] = {-0x7fffffff, -0x7fffffff, -0x7fffffff};
    for (int64_t row = ch.r0 + tid; row < ch.r1; row += kBS) {
        const Frame* f = frm + (row - a.off[k]) * (k + 1);
#pragma unroll
        for (int ax = 0; ax < D; ++ax) {
            const int c = f->c[ax];
            lo[ax] = min(lo[ax], c);
            hi[ax] = max(hi[ax], c);
        }
    }
#pragma unroll
    for (int ax = 0; ax < D; ++ax) {
        for (int o = 16; o > 0; o >>= 1) {
            lo[ax] = min(lo[ax], __shfl_xor_sync(0xffffffffu, lo[ax], o));
            hi[ax] = max(hi[ax], __shfl_xor_sync(0xffffffffu, hi[ax], o));
        }
    }
    if (lane == 0) {
#pragma unroll
        for (int ax = 0; ax < D; ++ax) {
            sh.lred[wid][ax] = lo[ax];
            sh.lred[wid][3 + ax] = hi[ax];
        }
    }
    __syncthreads();
    if (tid == 0) {
        int ncell = 1, fits = 1;
        for (int ax = 0; ax < 3; ++ax) {
            int blo = 0, n = 1;
            if (ax < D) {
                int l0 = 0x7fffffff, h0 = -0x7fffffff;
                for (int w = 0; w < kNW; ++w) {
                    l0 = min(l0, sh.lred[w][ax]);
                    h0 = max(h0, sh.lred[w][3 + ax]);
                }
                blo = max(l0 - R, 0);
                const int bhi = min(h0 + R, g.G[ax] - 1);
                n = bhi - blo + 1;
                if (n <= 0) n = 0;
                if (n > 255) fits = 0;
            }
            sh.lbox[ax] = blo;
            sh.lbox[3 + ax] = n;
            ncell = fits ? ncell * n : 0;
            if (ncell > kLCells) fits = 0;
        }
        sh.lbox[6] = fits ? ncell : 0;
        sh.lbox[7] = fits;
    }
    __syncthreads();
    if (!sh.lbox[7]) {
        __syncthreads();  // every thread has read lbox before the caller's next chunk rewrites it
        return false;
    }
    const int ncell = sh.lbox[6];
    const int blo0 = sh.lbox[0], blo1 = sh.lbox[1], blo2 = sh.lbox[2];
    const int n0 = sh.lbox[3], n1 = sh.lbox[4];
    // 2. the box cells' first points and point counts, then their offsets (one warp scans)
    for (int c = tid; c < ncell; c += kBS) {
        const int cx = blo0 + c % n0, cy = blo1 + (c / n0) % n1, cz = blo2 + c / (n0 * n1);
        const int64_t gid = g.cell_off + morton(D, cx, D >= 2 ? cy : 0, D >= 3 ? cz : 0);
        const int32_t ps = __ldg(v.cell_start + gid);
        sh.lps[c] = ps;
        sh.lcoff[c + 1] = __ldg(v.cell_start + gid + 1) - ps;
    }
    __syncthreads();
    if (wid == 0) {
        int carry = 0;
        for (int b0 = 0; b0 < ncell; b0 += 32) {
            const int c = b0 + lane;
            int t = c < ncell ? sh.lcoff[c + 1] : 0;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int u = __shfl_up_sync(0xffffffffu, t, o);
                if (lane >= o) t += u;
            }
            if (c < ncell) sh.lcoff[c + 1] = carry + t;
            carry += __shfl_sync(0xffffffffu, t, 31);
        }
        if (lane == 0) sh.lcoff[0] = 0;
    }
    __syncthreads();
    const int total = sh.lcoff[ncell];
    if (total > kCap) {
        __syncthreads();
        return false;
    }
    // 3. the points' positions in the box (units of delta_m), a warp per box cell
    const float cod = g.cod;
    const int64_t N = v.N;
    const float* W = a.mfv.W;
    for (int c = wid; c < ncell; c += kNW) {
        const int r[3] = {c % n0, (c / n0) % n1, c / (n0 * n1)};
        const int32_t ps = sh.lps[c], np = sh.lcoff[c + 1] - sh.lcoff[c];
        const int o = sh.lcoff[c];
#pragma unroll
        for (int ax = 0; ax < D; ++ax) {
            const float b = __fmul_rn(small_int_to_float(r[ax]), cod);
            for (int t = lane; t < np; t += 32) sp[ax * kCap + o + t] = __fadd_rn(b, __ldg(W + ax * N + ps + t));
        }
    }
    __syncthreads();
    // 4. a warp per row
    const float* xh = a.p32 + ch.vb;
    const float* xl = a.s32 + ch.vb;
    int32_t* q = sh.lq[wid];    // survivors: staged index
    int32_t* qc = sh.lqd[wid];  // and box cell | x << 8 | y << 16 | z << 24 (box coordinates)
    for (int64_t row = ch.r0 + wid; row < ch.r1; row += kNW) {
        const Frame f = frm[(row - a.off[k]) * (k + 1)];
        const int bl[3] = {blo0, blo1, blo2};
        float Y[3] = {0.0f, 0.0f, 0.0f};
        int rlo[3] = {0, 0, 0}, rhi[3] = {0, 0, 0};  // the row's cells in box coordinates
#pragma unroll
        for (int ax = 0; ax < D; ++ax) {
            Y[ax] = __fadd_rn(__fmul_rn(small_int_to_float(f.c[ax] - bl[ax]), cod), f.fr[ax]);
            rlo[ax] = max(f.c[ax] - R, 0) - bl[ax];
            rhi[ax] = min(f.c[ax] + R, g.G[ax] - 1) - bl[ax];
        }
        ff acc = {0.0f, 0.0f};
        int qn = 0;  // queued survivors (warp-uniform)
        auto entry = [&](int i, int32_t cd) {
            const int c = cd & 255;
            const int32_t p = sh.lps[c] + (i - sh.lcoff[c]);
            const int dcs[3] = {((cd >> 8) & 255) + blo0 - f.c[0], ((cd >> 16) & 255) + blo1 - f.c[1],
                                ((cd >> 24) & 255) + blo2 - f.c[2]};
            acc = ff_add(acc, ff_mul(ff_entry_dc<E, K>(v, W, a.Wlo, a.ffl, m, p, f, dcs), {xh[p], xl[p]}));
        };
        for (int zr = rlo[2]; zr <= rhi[2]; ++zr) {
            for (int yr = rlo[1]; yr <= rhi[1]; ++yr) {
                if (rlo[0] > rhi[0]) continue;
                const int line = (zr * n1 + yr) * n0;
                const int s = sh.lcoff[line + rlo[0]], e = sh.lcoff[line + rhi[0] + 1];
                const int32_t yz = (yr << 16) | (zr << 24);
                for (int b0 = s; b0 < e; b0 += 32) {
                    const int i = b0 + lane;
                    bool pass = false;
                    int xr = rlo[0];
                    if (i < e) {
                        float t = __fsub_rn(sp[i], Y[0]);
                        float qq = t * t;
                        if (D >= 2) { t = __fsub_rn(sp[kCap + i], Y[1]); qq = fmaf(t, t, qq); }
                        if (D >= 3) { t = __fsub_rn(sp[2 * kCap + i], Y[2]); qq = fmaf(t, t, qq); }
                        pass = qq <= 1.0f + 1e-4f;
                        for (int x = rlo[0] + 1; x <= rhi[0]; ++x) xr += i >= sh.lcoff[line + x];
                    }
                    const unsigned mask = __ballot_sync(0xffffffffu, pass);
                    if (pass) {
                        const int slot = qn + __popc(mask & ((1u << lane) - 1u));
                        q[slot] = i;
                        qc[slot] = (line + xr) | (xr << 8) | yz;
                    }
                    qn += __popc(mask);
                    if (qn >= 32) {
                        __syncwarp();
                        entry(q[lane], qc[lane]);
                        __syncwarp();
                        if (lane < qn - 32) {
                            q[lane] = q[32 + lane];
                            qc[lane] = qc[32 + lane];
                        }
                        qn -= 32;
                        __syncwarp();
                    }
                }
            }
        }
        __syncwarp();
        if (lane < qn) entry(q[lane], qc[lane]);
        __syncwarp();
        const ff sum = ff_group_sum(acc, 32);
        if (lane == 0) a.beta[ch.vb + row] -= ff_to_double(sum);
    }
    __syncthreads();  // the staged points stay until every warp is done with them
    return true;
}

// lower_chunk_staged for the hierarchy's (d, Wendland exponent and degree), with the same
// specialisations as lower_row_mf_warp_any.
__device__ __forceinline__ bool lower_chunk_staged_any(const SolveArgs& a, Shared& sh, const Chunk& ch, int m) {
    const int e = a.hv.w.e, kk = a.hv.w.k;
    if (a.hv.d == 2) {
        if (e == 4 && kk == 1) return lower_chunk_staged<2, 4, 1>(a, sh, ch, m);
        if (e == 6 && kk == 2) return lower_chunk_staged<2, 6, 2>(a, sh, ch, m);
        return lower_chunk_staged<2, 0, 0>(a, sh, ch, m);
    }
    if (a.hv.d == 3) {
        if (e == 4 && kk == 1) return lower_chunk_staged<3, 4, 1>(a, sh, ch, m);
        if (e == 6 && kk == 2) return lower_chunk_staged<3, 6, 2>(a, sh, ch, m);
        return lower_chunk_staged<3, 0, 0>(a, sh, ch, m);
    }
    return lower_chunk_staged<1, 0, 0>(a, sh, ch, m);
}

// The whole schedule of eq. split for one hierarchy, run by the CTAs [0, sh.nb) of a
// partition (sh.cta: this CTA's index in it).
template <int MODE, bool WIDE = false>
__device__ __forceinline__ void fit_body(const SolveArgs& a, Shared& sh) {
    const int tid = threadIdx.x;
    for (int v = tid; v < kMaxV; v += kBS) {
        sh.it_total[v] = 0;
        sh.refines[v] = 0;
        sh.fb[v] = 0;
        sh.f64[v] = 0;
        sh.f64n[v] = 0;
        sh.vbytes[v] = 0.0;
        sh.scale[v] = 0.0;
    }
    if (tid == 0) {
        sh.bytes = 0.0;
        for (int i = 0; i < kProf; ++i) sh.pt[i] = 0ull;
        sh.tprev = ms_globaltimer();
    }
    __syncthreads();
    const int L = a.L;
    // beta_0 = f, x = 0
    if (WIDE) {
        const int rl = tid % a.RW;
        run_phase_wide<0>(a, sh, [](int) { return true; }, [&](int, int64_t r0, int64_t r1, double*) {
            elems_wide(a, r0, r1, [&](int64_t, int64_t i) {
                a.beta[i] = rl < a.R ? a.f[i] : 0.0;
                a.x[i] = 0.0;
            });
        });
    } else {
        run_phase<0>(a, sh, [](int) { return true; }, [&](const Chunk& ch, double*) {
            for (int64_t row = ch.r0 + tid; row < ch.r1; row += kBS) {
                a.beta[ch.vb + row] = a.f[ch.vb + row];
                a.x[ch.vb + row] = 0.0;
            }
        });
    }
    prof(sh, kPrfOther);
    if (!gsync(a, sh)) return;
    // With inter_tol >= 1 (default) sweep m iterates level m only: the levels above it
    // still hold t = 0, which passes their residual test at once, so their FP64 residuals
    // are not computed either.
    const bool skip = a.inter_tol >= 1.0;
    for (int m = 0; m < a.sweeps; ++m) {
        if (m <= L - 2) {
            if (!(WIDE ? solve_levels_wide<MODE>(a, sh, m, skip ? m + 1 : L - 1, false)
                       : solve_levels<MODE>(a, sh, m, skip ? m + 1 : L - 1, false)))
                return;
        }
        if (WIDE && m + 1 <= L - 1) {
            // lower-block update in the wide layout: every right-hand side of a row at once
            const int rl = tid % a.RW;
            const int32_t* seg0 = a.Bseg + (int64_t)m * a.N;
            run_phase_wide<0>(a, sh, [&](int v) { return v % L >= m + 1; }, [&](int, int64_t r0, int64_t r1, double*) {
                if (rl >= a.R) return;
                rows_wide(a, r0, r1, [&](int64_t row) {
                    const int64_t b = a.Brp[row];
                    const int64_t i = row * a.RW + rl;
                    if (a.lower_inc) {
                        const double y = csr_row_wide<double, double, double>(
                            a.Bcol, a.Bv64, a.x, b + __ldg(seg0 + row), b + __ldg(seg0 + a.N + row), rl, a.RW);
                        a.beta[i] -= y;
                    } else {
                        const double y = csr_row_wide<double, double, double>(a.Bcol, a.Bv64, a.x, b, a.Brp[row + 1],
                                                                              rl, a.RW);
                        a.beta[i] = a.f[i] - y;
                    }
                });
            });
            if (tid == 0) {
                if (a.lower_inc) {
                    sh.bytes += (double)a.nnzBm[m] * 12.0 + (double)(a.off[L] - a.off[m + 1]) * (16.0 + 16.0 * a.R);
                } else {
                    for (int l = m + 1; l < L; ++l)
                        sh.bytes += (double)a.nnzB[l] * 12.0 + (double)(a.off[l + 1] - a.off[l]) * (8.0 + 24.0 * a.R);
                }
            }
            prof(sh, kPrfLower);
            if (!gsync(a, sh)) return;
        } else if (MODE == 1 && m + 1 <= L - 1 && a.lower_inc && a.lower_mf) {  // (MIXED builds only)
            // beta_k -= B_km t_m with B's entries recomputed: t_m split into double-float
            // parts (p32, s32: free between level solves), then one S-lane group per row of
            // levels k = m+1..L-1 sums its entries in double-float (the entries' arithmetic is
            // that of the stored B of a MIXED build) and subtracts the sum in FP64.
            run_phase<0>(a, sh, [&](int v) { return v % L == m; }, [&](const Chunk& ch, double*) {
                for (int64_t row = ch.r0 + tid; row < ch.r1; row += kBS) {
                    const ff t = ff_from_double(a.x[ch.vb + row]);
                    a.p32[ch.vb + row] = t.hi;
                    a.s32[ch.vb + row] = t.lo;
                }
            });
            prof(sh, kPrfLower);
            if (!gsync(a, sh)) return;
            run_phase<0>(a, sh, [&](int v) { return v % L >= m + 1; }, [&](const Chunk& ch, double*) {
                // level m's points around the chunk staged in shared memory when they fit
                if (lower_chunk_staged_any(a, sh, ch, m)) return;
                // else a warp per row: its frame in level m's grid from the build, the candidates
                // of the (2R+1)^d cells around it tested in FP32 and compacted (lower_row_mf_warp)
                const int wid = tid >> 5, lane = tid & 31;
                const float* xh = a.p32 + ch.vb;
                const float* xl = a.s32 + ch.vb;
                const int k = ch.l;
                for (int64_t row = ch.r0 + wid; row < ch.r1; row += kNW) {
                    const Frame f = a.frames[a.fbase[k] + (row - a.off[k]) * (k + 1) + m];
                    const ff acc = ff_group_sum(lower_row_mf_warp_any(a.hv, a.mfv.W, a.Wlo, a.mfv.cellid, a.ffl, m, f,
                                                                      xh, xl, lane, sh.lq[wid], sh.lqd[wid]),
                                                32);
                    if (lane == 0) a.beta[ch.vb + row] -= ff_to_double(acc);
                }
            });
            if (tid == 0)
                sh.bytes += a.R * ((double)(a.off[L] - a.off[m + 1]) * (16.0 + 36.0) +
                                   (double)(a.off[m + 1] - a.off[m]) * (16.0 + 8.0 + 4.0 * 2.0 * a.hv.d));
            prof(sh, kPrfLower);
            if (!gsync(a, sh)) return;
        } else if (m + 1 <= L - 1 && a.lower_inc) {
            // beta_k -= B_km t_m for the rows of levels k = m+1..L-1 (FP64).  When
            // intermediate levels are not iterated (inter_tol >= 1) t_m is the only
            // level solution that changed since beta was last updated (levels above m
            // still hold t = 0), so only the blocks B_km are read: every block of B
            // once over the whole fit.
            run_phase<0>(a, sh, [&](int v) { return v % L >= m + 1; }, [&](const Chunk& ch, double*) {
                const int S = a.tprBm[m];
                const double* xv = a.x + ch.vb;
                const int32_t* seg0 = a.Bseg + (int64_t)m * a.N;
                const int32_t* seg1 = seg0 + a.N;
                rows_by_subwarp(ch.r0, ch.r1, S, [&](int64_t row, bool ok, int sl) {
                    int64_t s = 0, e = 0;
                    if (ok) {
                        const int64_t b = a.Brp[row];
                        s = b + __ldg(seg0 + row);
                        e = b + __ldg(seg1 + row);
                    }
                    const double y = csr_row<double, double, double>(a.Bcol, a.Bv64, xv, s, e, sl, S);
                    if (ok && sl == 0) a.beta[ch.vb + row] -= y;
                });
            });
            if (tid == 0)
                sh.bytes += a.R * ((double)a.nnzBm[m] * 12.0 + (double)(a.off[L] - a.off[m + 1]) * 32.0);
            prof(sh, kPrfLower);
            if (!gsync(a, sh)) return;
        } else if (m + 1 <= L - 1) {
            // beta_k = f_k - sum_{j<k} B_kj t_j for the rows of levels k = m+1..L-1 (FP64)
            run_phase<0>(a, sh, [&](int v) { return v % L >= m + 1; }, [&](const Chunk& ch, double*) {
                const int S = a.tprB[ch.l];
                const double* xv = a.x + ch.vb;
                rows_by_subwarp(ch.r0, ch.r1, S, [&](int64_t row, bool ok, int sl) {
                    int64_t s = 0, e = 0;
                    if (ok) { s = a.Brp[row]; e = a.Brp[row + 1]; }
                    const double y = csr_row<double, double, double>(a.Bcol, a.Bv64, xv, s, e, sl, S);
                    if (ok && sl == 0) a.beta[ch.vb + row] = a.f[ch.vb + row] - y;
                });
            });
            if (tid == 0)
                for (int l = m + 1; l < L; ++l)
                    sh.bytes += a.R * ((double)a.nnzB[l] * 12.0 + (double)(a.off[l + 1] - a.off[l]) * 32.0);
            prof(sh, kPrfLower);
            if (!gsync(a, sh)) return;
        }
    }
    if (!(WIDE ? solve_levels_wide<MODE>(a, sh, 0, L, true) : solve_levels<MODE>(a, sh, 0, L, true))) return;
#ifdef MS_CTA_PROF
    if (tid == 0 && sh.cta < 1024)
        for (int i = 0; i < kProf; ++i) g_cta_prof[sh.cta][i] = sh.pt[i];
#endif
    if (sh.cta == 0 && tid == 0) {
        for (int l = 0; l < L; ++l) {
            long long it = 0;
            int rf = 0;
            for (int r = 0; r < a.R; ++r) {
                it += sh.it_total[r * L + l];
                rf += sh.refines[r * L + l];
            }
            a.iters[l] = it;
            a.refines[l] = rf;
        }
        double b = sh.bytes;
        int fb = 0, f64n = 0;
        for (int v = 0; v < a.V; ++v) {
            b += sh.vbytes[v];
            fb += sh.fb[v];
            f64n += sh.f64n[v];
        }
        a.bytes[0] = b;
        for (int i = 0; i < kProf; ++i) a.prof[i] = sh.pt[i];
        a.pcfb[0] = fb;
        a.pcfb[1] = f64n;
    }
}

// The persistent solve kernel of one hierarchy.  MINB: CTAs per SM the kernel is
// compiled for (1: up to 128 registers a thread, 2: up to 64).  WIDE: the right-hand
// sides in the row-major (SpMM) layout.
template <int MODE, int MINB, bool WIDE>
__global__ void __launch_bounds__(kBS, MINB) k_fit(const __grid_constant__ SolveArgs a) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    Shared& sh = *reinterpret_cast<Shared*>(smem_raw);
    if (threadIdx.x == 0) {
        sh.cta = blockIdx.x;
        sh.nb = gridDim.x;
    }
    __syncthreads();
    fit_body<MODE, WIDE>(a, sh);
}

// ---------------------------------------------------------------- host helpers

inline unsigned nblk(int64_t n, int bs) { return (unsigned)std::max<int64_t>(1, (n + bs - 1) / bs); }

// Sub-warp width for CSR rows of avg_nnz entries: about 16 entries per lane
// keeps enough independent loads in flight per lane (measured on GB300: 4 lanes
// for ~50-entry rows run 2.5x faster than 16).
int tpr_for(double avg_nnz) {
    int S = 1;
    while (S < 32 && S * 16 < avg_nnz) S <<= 1;
    return S;
}

MFView make_mfview(const ms_hierarchy* h) {
    MFView v{};
    v.d = h->d;
    v.L = h->L;
    v.N = h->N;
    v.E = h->view.w.e;
    for (int i = 0; i < 4; ++i) v.c[i] = (float)h->view.w.c[i];
    v.W = h->W;
    v.cellid = h->cellid;
    v.cell_start = h->cell_start;
    for (int l = 0; l < h->L; ++l) {
        const LevelGrid& g = h->view.grid[l];
        MFLevel& m = v.lv[l];
        for (int a = 0; a < 3; ++a) m.G[a] = g.G[a];
        m.R = h->view.R;
        m.cod = (float)(g.cell / h->view.delta[l]);
        m.dscale = (float)h->view.dscale[l];
        m.cell_off = g.cell_off;
        m.ncells = g.ncells;
    }
    return v;
}

// Lanes per target point of the matrix-free mat-vec: about one warp per cell of the finest level.
int mf_tpp_for(const ms_hierarchy* h) {
    const LevelGrid& g = h->view.grid[h->L - 1];
    const double occupied = (double)g.G[0] * g.G[1] * g.G[2];
    const double per_cell = (double)(h->view.off[h->L] - h->view.off[h->L - 1]) / std::max(occupied, 1.0);
    int t = 1;
    while (t < 8 && per_cell * t * 2 <= 32.0) t <<= 1;
    return t;
}

// Fill the solve arguments that depend only on the hierarchy, the options and R.
// wide: the right-hand sides of the launch in the row-major (SpMM) layout, RW lanes per row.
// ncta > 0 (the CTAs of the launch or partition): a level with fewer rows than ncta chunks of 256
// takes chunks of max(32, the power of 2 >= its rows / ncta) rows, so its rows spread over more
// CTAs (a CTA handles at most one of its chunks); larger levels keep 256 rows a chunk, which keeps
// the element-wise phases' threads busy.  0: 256 rows for every level.
void fill_args(const ms_hierarchy* h, double rel_tol, int R, SolveArgs& a, bool wide = false, int ncta = 0) {
    const int64_t* rpA = h->rpA_lv;
    const int64_t* rpB = h->rpB_lv;
    a.mf = (h->opts.precision == MS_PREC_MIXED && h->opts.op == MS_OP_MATRIX_FREE) ? 1 : 0;
    a.mf_tpp = h->mf_tpp;
    a.mfv = make_mfview(h);
    a.pc = (h->opts.precision == MS_PREC_MIXED && h->opts.precond != MS_PRECOND_NONE) ? 1 : 0;
    a.gcol = h->pc.gcol;
    a.gval = h->pc.gval;
    a.gt_rp = h->pc.gt_rp;
    a.gt_col = h->pc.gt_col;
    a.gt_val = h->pc.gt_val;
    for (int l = 0; l < h->L; ++l) a.pcs[l] = (float)std::pow(h->view.delta[l], (double)h->d);
    const int L = h->L;
    a.L = L;
    a.R = R;
    a.V = R * L;
    a.N = h->N;
    a.RW = 0;
    if (wide) {
        a.RW = 1;
        while (a.RW < R) a.RW <<= 1;
    }
    a.crow = wide ? kBS / a.RW : kChunk;
    for (int l = 0; l < L; ++l) {
        int cr = a.crow;
        const int64_t n = h->view.off[l + 1] - h->view.off[l];
        if (!wide && ncta > 0 && n < (int64_t)ncta * kChunk) {
            cr = 32;
            while (cr < kChunk && (int64_t)cr * ncta < n) cr <<= 1;
        }
        a.crowl[l] = cr;
    }
    int64_t c = 0;
    for (int l = 0; l <= L; ++l) {
        a.off[l] = h->view.off[l];
        a.coff[l] = (int)c;
        if (l < L) c += (h->view.off[l + 1] - h->view.off[l] + a.crowl[l] - 1) / a.crowl[l];
    }
    a.C = (int)c;
    for (int l = 0; l < L; ++l) {
        const int64_t n = h->view.off[l + 1] - h->view.off[l];
        a.nnzA[l] = rpA[l + 1] - rpA[l];
        a.nnzB[l] = rpB[l + 1] - rpB[l];
        a.tprA[l] = h->opts.threads_per_row > 0 ? h->opts.threads_per_row
                    : h->tprA_tuned[l] > 0       ? h->tprA_tuned[l]
                                                 : tpr_for((double)a.nnzA[l] / n);
        a.tprB[l] = tpr_for((double)a.nnzB[l] / n);
    }
    a.Arp = h->A.rp; a.Acol = h->A.col; a.Av64 = h->A.v64; a.Av32 = h->A.v32;
    a.Brp = h->B.rp; a.Bcol = h->B.col; a.Bv64 = h->B.v64;
    a.Bseg = h->Bseg;
    a.lower_mf = (h->opts.precision == MS_PREC_MIXED && h->opts.lower_op == MS_OP_MATRIX_FREE) ? 1 : 0;
    a.hv = h->view;
    a.hv.X = h->X;
    a.hv.cell_start = h->cell_start;
    a.ffl = make_fflevels(h->view);
    a.Wlo = h->Wlo;
    for (int m = 0; m < L; ++m) a.tprLmf[m] = lower_mf_lanes(h->view, m);
    a.frames = static_cast<const Frame*>(h->frames);
    for (int l = 0; l <= L; ++l) a.fbase[l] = h->frame_base[l];
    if (!a.frames) a.lower_mf = 0;  // (a handle built with stored B)
    for (int m = 0; m < L; ++m) {
        int64_t nb = 0;
        for (int k = m + 1; k < L; ++k) nb += h->Bblk[k][m];
        const int64_t rows = h->view.off[L] - h->view.off[std::min(m + 1, L)];
        a.nnzBm[m] = nb;
        a.tprBm[m] = tpr_for(rows > 0 ? (double)nb / rows : 1.0);
    }
    const bool mixed = h->opts.precision == MS_PREC_MIXED;
    a.sweeps = ms_sweeps_of(h);
    a.max_iters = h->opts.max_iters > 0 ? h->opts.max_iters : 20000;
    a.max_outer = mixed ? 40 : 8;
    a.tol = rel_tol;
    a.inter_tol = h->opts.inter_tol > 0 ? std::max(h->opts.inter_tol, rel_tol) : 1.0;
    a.inner_tol = h->opts.inner_tol > 0 ? h->opts.inner_tol : 1e-4;
    a.lower_inc = (a.inter_tol >= 1.0 && (a.Bseg || a.lower_mf)) ? 1 : 0;
    a.timeout_ns = 4000000000ull;
}

// Right-hand sides per launch: every (right-hand side, level) pair is a virtual level.
int rhs_per_launch(const ms_hierarchy* h, int nrhs) { return std::max(1, std::min(nrhs, std::min(32, kMaxV / h->L))); }

// Several right-hand sides take the wide (SpMM) layout when the level operators are CSR
// without a preconditioner and the solve kernel runs 2 CTAs per SM.
bool wide_layout(const ms_hierarchy* h, int nrhs, int minb) {
    return nrhs > 1 && minb == 2 && h->opts.precond == MS_PRECOND_NONE &&
           !(h->opts.precision == MS_PREC_MIXED && h->opts.op == MS_OP_MATRIX_FREE) &&
           h->opts.lower_op != MS_OP_MATRIX_FREE;
}

}  // namespace
