// Hierarchy build: per-level uniform-cell binning and CSR assembly of the
// level blocks A_l = Phi_{delta_l}(X_l, X_l) and the strictly lower blocks
// B_kj = Phi_{delta_j}(X_k, X_j), k > j (Section 3, definition of B and eq. mas;
// Assumption 1, eq. kernelscaling for Phi_delta = delta^-d phi(|.|/delta)).
//
// Binning (replaces the kd-tree of Section 5.3): the cell size of level l is
// delta_l / cell_split, so every neighbour within delta_l of a point lies in the
// (2R+1)^d cells around its cell, R = cell_split.  Cells are numbered by the
// Morton code of their integer coordinates; points are counting-sorted by
// (level, cell) and, inside a cell, ranked by input index, which makes the
// sorted order (and every later summation order) deterministic.
#include <algorithm>
#include <cmath>
#include <vector>

#include "ms_ff.cuh"
#include "ms_internal.cuh"
#include "ms_matfree.cuh"
#include "ms_scan.cuh"

namespace {

constexpr int kBboxBlocks = 64;

// ---------------------------------------------------------------- bounding boxes

// partial[(l * kBboxBlocks + b) * 7 + {0..2: min, 3..5: max, 6: non-finite count}]
__global__ void k_bbox(const double* pts, int d, const int64_t* off_dev, int L, double* partial) {
    const int l = blockIdx.y;
    const int64_t s = off_dev[l], e = off_dev[l + 1];
    double mn[3] = {INFINITY, INFINITY, INFINITY}, mx[3] = {-INFINITY, -INFINITY, -INFINITY};
    double bad = 0.0;
    for (int64_t i = s + blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < e;
         i += (int64_t)gridDim.x * blockDim.x) {
        for (int a = 0; a < d; ++a) {
            const double v = pts[i * d + a];
            if (!isfinite(v)) bad += 1.0;
            mn[a] = fmin(mn[a], v);
            mx[a] = fmax(mx[a], v);
        }
    }
    __shared__ double sh[256];
    for (int k = 0; k < 7; ++k) {
        double v = k < 3 ? mn[k] : (k < 6 ? mx[k - 3] : bad);
        sh[threadIdx.x] = v;
        __syncthreads();
        for (int o = blockDim.x / 2; o > 0; o >>= 1) {
            if (threadIdx.x < o) {
                const double a = sh[threadIdx.x], b = sh[threadIdx.x + o];
                sh[threadIdx.x] = k < 3 ? fmin(a, b) : (k < 6 ? fmax(a, b) : a + b);
            }
            __syncthreads();
        }
        if (threadIdx.x == 0) partial[(l * kBboxBlocks + blockIdx.x) * 7 + k] = sh[0];
        __syncthreads();
    }
}

// ---------------------------------------------------------------- binning

__global__ void k_cell_keys(const double* pts, HierView v, int32_t* key, int32_t* count) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= v.N) return;
    const int l = level_of_row(v.off, v.L, i);
    const LevelGrid& g = v.grid[l];
    int c[3] = {0, 0, 0};
    for (int a = 0; a < v.d; ++a) {
        int ca = cell_coord(g, a, pts[i * v.d + a]);
        c[a] = min(max(ca, 0), g.G[a] - 1);
    }
    const int32_t gid = (int32_t)(g.cell_off + morton(v.d, c[0], c[1], c[2]));
    key[i] = gid;
    atomicAdd(&count[gid], 1);
}

__global__ void k_scatter(const int32_t* key, const int32_t* cell_start, int32_t* cursor, int32_t* tmp, int64_t N) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= N) return;
    const int32_t g = key[i];
    const int32_t pos = cell_start[g] + atomicAdd(&cursor[g], 1);
    tmp[pos] = (int32_t)i;
}

// Final position of each point: cell start + number of points of the same cell
// with a smaller input index.
__global__ void k_rank(const int32_t* key, const int32_t* cell_start, const int32_t* tmp, int32_t* perm, int64_t N) {
    const int64_t pos = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (pos >= N) return;
    const int32_t i = tmp[pos];
    const int32_t g = key[i];
    const int32_t s = cell_start[g], e = cell_start[g + 1];
    int32_t rank = 0;
    for (int32_t j = s; j < e; ++j) rank += (tmp[j] < i);
    perm[s + rank] = i;
}

__global__ void k_gather_points(const double* pts, const int32_t* perm, double* X, int d, int64_t N) {
    const int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (s >= N) return;
    const int64_t i = perm[s];
    for (int a = 0; a < d; ++a) X[a * N + s] = pts[i * d + a];
}

// Matrix-free geometry of each sorted point: its level-local Morton cell and its
// offset from that cell's corner in units of delta_l (FP32).
__global__ void k_mf_coords(HierView v, float* W, float* Wlo, int32_t* cellid) {
    const int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (s >= v.N) return;
    const int l = level_of_row(v.off, v.L, s);
    const LevelGrid& g = v.grid[l];
    const double inv_delta = 1.0 / v.delta[l];
    int c[3] = {0, 0, 0};
    for (int a = 0; a < v.d; ++a) {
        const double x = v.X[a * v.N + s];
        c[a] = min(max(cell_coord(g, a, x), 0), g.G[a] - 1);
        const double t = (x - (g.lo[a] + (double)c[a] * g.cell)) * inv_delta;
        const float hi = (float)t;
        W[a * v.N + s] = hi;
        if (Wlo) Wlo[a * v.N + s] = (float)(t - (double)hi);  // W + Wlo: t to about 48 bits
    }
    cellid[s] = (int32_t)morton(v.d, c[0], c[1], c[2]);
}


// ---------------------------------------------------------------- CSR assembly
//
// One warp per row s (level k).  For each column level j (j = k for A, j < k for
// B) the warp walks the (2R+1)^d cells around s's cell in level j's grid; its
// lanes take a cell's points 32 at a time.  The test |x_p - x_s| < delta_j is
// taken in FP32 first, from cell-relative coordinates in units of delta_j (the
// cell offset plus the FP32 in-cell offsets W), whose error is ~1e-6 of delta_j^2;
// only candidates within 1e-4 of the boundary are re-tested in FP64
// (fma-accumulated r^2 < delta_j^2), so the pattern is exactly the FP64 one.
// The FP64 values are computed for the entries only (FP64 is scarce on this GPU).

// Position of y relative to level j's grid: cell c[a] and the offset from that
// cell's corner in units of delta_j.  Lane a < d computes axis a.
struct Frame {
    int c[3];
    float fr[3];
    float frlo[3];  // fr + frlo: the offset to about 48 bits (double-float entries)
};

struct Pt {
    double x, y, z;
};

__device__ __forceinline__ Pt point_at(const HierView& v, int64_t s) {
    Pt q{v.X[s], 0.0, 0.0};
    if (v.d >= 2) q.y = v.X[v.N + s];
    if (v.d >= 3) q.z = v.X[2 * v.N + s];
    return q;
}

// |x_p - y|^2 in FP64, accumulated axis by axis with fma
__device__ __forceinline__ double dist2(const HierView& v, int64_t p, const Pt& y) {
    double u = v.X[p] - y.x;
    double r2 = fma(u, u, 0.0);
    if (v.d >= 2) { u = v.X[v.N + p] - y.y; r2 = fma(u, u, r2); }
    if (v.d >= 3) { u = v.X[2 * v.N + p] - y.z; r2 = fma(u, u, r2); }
    return r2;
}

// Frame of y in level j's grid, all axes (FP64 set-up: one lane per level calls it).
__device__ __forceinline__ Frame frame_of(const HierView& v, int j, const Pt& y) {
    const LevelGrid& g = v.grid[j];
    Frame f{};
    const double ya[3] = {y.x, y.y, y.z};
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        if (a < v.d) {
            f.c[a] = cell_coord(g, a, ya[a]);
            const double t = (ya[a] - (g.lo[a] + (double)f.c[a] * g.cell)) * v.inv_delta[j];
            f.fr[a] = (float)t;
            f.frlo[a] = (float)(t - (double)f.fr[a]);
        }
    }
    return f;
}

// Lane `src`'s frame (src may differ between lanes; every lane must take part).
__device__ __forceinline__ Frame frame_from(const Frame& mine, int src) {
    Frame f;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        f.c[a] = __shfl_sync(0xffffffffu, mine.c[a], src);
        f.fr[a] = __shfl_sync(0xffffffffu, mine.fr[a], src);
        f.frlo[a] = __shfl_sync(0xffffffffu, mine.frlo[a], src);
    }
    return f;
}

// ---------------------------------------------------------------- double-float entries
//
// With precision = MIXED the stored FP64 entries are evaluated in double-float arithmetic
// (ms_ff.cuh) from the points' cell-relative offsets W + Wlo, exact to about 48 bits:
// relative errors near 1e-14 instead of 1e-16, far inside what the mixed path promises
// (its inner solves run in FP32), at about 3 FP64 instructions per entry (the final
// conversion) instead of about 30.

// Per-level constants: cell size / delta and delta^-d as double-floats.
struct FFLevels {
    ff cod[MS_MAXL];
    ff ds[MS_MAXL];
};

// phi(r) for the Wendland closed form w in double-float; 0 for r >= 1.
__device__ __forceinline__ ff ff_wendland(const WendlandPoly& w, ff r) {
    if (!(r.hi < 1.0f || (r.hi == 1.0f && r.lo < 0.0f))) return {0.0f, 0.0f};
    const ff s = ff_add({1.0f, 0.0f}, ff_neg(r));
    const ff s2 = ff_sqr(s), s4 = ff_sqr(s2);
    ff pw;
    switch (w.e) {
    case 4: pw = s4; break;
    case 6: pw = ff_mul(s4, s2); break;
    case 8: pw = ff_sqr(s4); break;
    default: {
        pw = {1.0f, 0.0f};
        for (int i = 0; i < w.e; ++i) pw = ff_mul(pw, s);
    }
    }
    ff p = ff_from_double(w.c[w.k]);
    for (int i = w.k - 1; i >= 0; --i) p = ff_add(ff_mul(p, r), ff_from_double(w.c[i]));
    return ff_mul(pw, p);
}

// delta_j^-d phi(|x_p - y| / delta_j) for point p of level j (cell cp, offsets W + Wlo) and
// y's frame f in level j's grid: the scaled offset on axis a is
// (cp_a - c_a) cod + (W_a + Wlo_a) - (fr_a + frlo_a).
__device__ __forceinline__ double ff_entry(const HierView& v, const float* __restrict__ W,
                                           const float* __restrict__ Wlo, const int32_t* __restrict__ cellid,
                                           const FFLevels& ffl, int j, int32_t p, const Frame& f) {
    int cp[3];
    demorton(v.d, (uint32_t)__ldg(cellid + p), cp);
    ff r2 = {0.0f, 0.0f};
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        if (a < v.d) {
            const ff cell = ff_mul(ffl.cod[j], {(float)(cp[a] - f.c[a]), 0.0f});
            const ff w = {__ldg(W + a * v.N + p), __ldg(Wlo + a * v.N + p)};
            const ff t = ff_add(ff_add(cell, w), ff_neg({f.fr[a], f.frlo[a]}));
            r2 = ff_add(r2, ff_sqr(t));
        }
    }
    return ff_to_double(ff_mul(ffl.ds[j], ff_wendland(v.w, ff_sqrt(r2))));
}

// Offset (units of delta) of a neighbour cell displaced by `dc` cells, seen from a point at
// fractional offset fr in its own cell; both CSR kernels take it from here so that they
// make the same decisions.
__device__ __forceinline__ float cell_offset(int dc, float cod, float fr) { return __fsub_rn(__fmul_rn((float)dc, cod), fr); }

// |x_p - y| < delta_j for candidate p in the neighbour cell with offsets (c0, c1, c2): FP32
// test on the cell-relative coordinates W (units of delta_j), the FP64 distance inside a band
// of 1e-4 around the support boundary.  Rounded operation by operation (no contraction), so
// every caller gets the same answer.
__device__ __forceinline__ bool within(const HierView& v, const float* __restrict__ W, int32_t p, float c0, float c1,
                                       float c2, const Pt& y, double d2) {
    float t = __fadd_rn(c0, __ldg(W + p));
    float qq = __fmul_rn(t, t);
    if (v.d >= 2) { t = __fadd_rn(c1, __ldg(W + v.N + p)); qq = __fmaf_rn(t, t, qq); }
    if (v.d >= 3) { t = __fadd_rn(c2, __ldg(W + 2 * v.N + p)); qq = __fmaf_rn(t, t, qq); }
    if (qq < 1.0f - 1e-4f) return true;
    if (qq <= 1.0f + 1e-4f) return dist2(v, p, y) < d2;
    return false;
}

// visit(p, in, mask): called by all 32 lanes for every group of up to 32
// candidates p; `in` = p is a neighbour, mask = ballot of `in`.  f: y's frame in
// level j's grid.  The (2R+1)^d cells around f's cell are taken 32 at a time (lane q
// looks up cell q's point range); their points form one list in cell order (dx
// fastest, then dy, dz; points in sorted order within a cell), which the warp walks 32
// candidates per step with every lane busy (cells hold ~16 points, so a step per cell
// would leave half the lanes idle and repeat the per-cell work in every lane).
template <typename F>
__device__ __forceinline__ void warp_neighbours(const HierView& v, const float* __restrict__ W, int j,
                                                const Frame& f, const Pt& y, int lane, F&& visit) {
    const LevelGrid& g = v.grid[j];
    const float cod = g.cod;
    const double d2 = v.delta[j] * v.delta[j];
    const int R = v.R, side = 2 * R + 1;
    const int nc = v.d == 1 ? side : (v.d == 2 ? side * side : side * side * side);
    for (int q0 = 0; q0 < nc; q0 += 32) {
        const int q = q0 + lane;
        int start = 0, cnt = 0;
        float o0 = 0.f, o1 = 0.f, o2 = 0.f;
        if (q < nc) {
            const int dx = q % side - R;
            const int dy = v.d >= 2 ? (q / side) % side - R : 0;
            const int dz = v.d >= 3 ? q / (side * side) - R : 0;
            const int cx = f.c[0] + dx, cy = f.c[1] + dy, cz = f.c[2] + dz;
            if (cx >= 0 && cx < g.G[0] && cy >= 0 && cy < g.G[1] && cz >= 0 && cz < g.G[2]) {
                const int64_t gid = g.cell_off + morton(v.d, cx, cy, cz);
                start = __ldg(v.cell_start + gid);
                cnt = __ldg(v.cell_start + gid + 1) - start;
            }
            o0 = cell_offset(dx, cod, f.fr[0]);
            o1 = cell_offset(dy, cod, f.fr[1]);
            o2 = cell_offset(dz, cod, f.fr[2]);
        }
        int incl = cnt;  // inclusive prefix of the cells' point counts over the lanes
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int t = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += t;
        }
        const int total = __shfl_sync(0xffffffffu, incl, 31);
        for (int b = 0; b < total; b += 32) {
            const int i = b + lane;
            // cell of candidate i: the number of cells whose inclusive prefix is <= i
            // (branch-free binary search over the lanes; every lane takes every step)
            int cq = 0;
#pragma unroll
            for (int st = 16; st >= 1; st >>= 1) {
                const int pv = __shfl_sync(0xffffffffu, incl, cq + st - 1);
                if (pv <= i) cq += st;
            }
            const int cs = __shfl_sync(0xffffffffu, start, cq);
            const int ce = __shfl_sync(0xffffffffu, incl, cq) - __shfl_sync(0xffffffffu, cnt, cq);
            const float c0 = __shfl_sync(0xffffffffu, o0, cq);
            const float c1 = __shfl_sync(0xffffffffu, o1, cq);
            const float c2 = __shfl_sync(0xffffffffu, o2, cq);
            const int32_t p = cs + (i - ce);
            const bool in = i < total && within(v, W, p, c0, c1, c2, y, d2);
            visit(p, in, __ballot_sync(0xffffffffu, in));
        }
    }
}

constexpr int kCsrBS = 256;  // 8 rows per block

// Entries of row s: one warp per row, one lane per (column level j, neighbour cell) pair
// at a time, each lane walking its cell's points (the count needs no positions, so no
// compaction across lanes).
__global__ void __launch_bounds__(kCsrBS, 4) k_csr_count(HierView v, const float* __restrict__ W, int32_t* cntA,
                                                       int32_t* cntB) {
    const int64_t s = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (s >= v.N) return;  // warp-uniform
    const int k = level_of_row(v.off, v.L, s);
    const Pt y = point_at(v, s);
    // lane j <= k holds y's frame in level j's grid
    Frame mine{};
    if (lane <= k) mine = frame_of(v, lane, y);
    const int R = v.R, side = 2 * R + 1;
    const int nc = v.d == 1 ? side : (v.d == 2 ? side * side : side * side * side);
    const int pairs = (k + 1) * nc;
    int32_t na = 0, nb = 0;
    for (int t0 = 0; t0 < pairs; t0 += 32) {
        const int t = t0 + lane;
        const int j = min(t / nc, k);  // lanes past the last pair read a valid frame and skip
        Frame f;
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            f.c[a] = __shfl_sync(0xffffffffu, mine.c[a], j);
            f.fr[a] = __shfl_sync(0xffffffffu, mine.fr[a], j);
        }
        if (t >= pairs) continue;
        const LevelGrid& g = v.grid[j];
        const int q = t - j * nc;
        const int dx = q % side - R;
        const int dy = v.d >= 2 ? (q / side) % side - R : 0;
        const int dz = v.d >= 3 ? q / (side * side) - R : 0;
        const int cx = f.c[0] + dx, cy = f.c[1] + dy, cz = f.c[2] + dz;
        if (cx < 0 || cx >= g.G[0] || cy < 0 || cy >= g.G[1] || cz < 0 || cz >= g.G[2]) continue;
        const int64_t gid = g.cell_off + morton(v.d, cx, cy, cz);
        const int32_t ps = __ldg(v.cell_start + gid), pe = __ldg(v.cell_start + gid + 1);
        const float o0 = cell_offset(dx, g.cod, f.fr[0]);
        const float o1 = cell_offset(dy, g.cod, f.fr[1]);
        const float o2 = cell_offset(dz, g.cod, f.fr[2]);
        const double d2 = v.delta[j] * v.delta[j];
        int32_t n = 0;
        for (int32_t p = ps; p < pe; ++p) n += within(v, W, p, o0, o1, o2, y, d2) ? 1 : 0;
        if (j == k) na += n;
        else nb += n;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        na += __shfl_xor_sync(0xffffffffu, na, o);
        nb += __shfl_xor_sync(0xffffffffu, nb, o);
    }
    if (lane == 0) {
        cntA[s] = na;
        cntB[s] = nb;
    }
}

// Also records, for the rows of level k, where each column level's segment of
// the B row starts: Bseg[j][s] = offset from rpB[s] of the first entry of
// column level j (j = 0..k; Bseg[k][s] = the row length).  The columns are
// found first (FP32 test, compacted by ballot); the FP64 values then take all
// 32 lanes over the row's entries.
// FF: entries in double-float arithmetic (MIXED builds), else FP64.
template <bool FF>
__global__ void __launch_bounds__(kCsrBS, 4) k_csr_fill(const __grid_constant__ HierView v, const float* __restrict__ W,
                                                      const float* __restrict__ Wlo, const int32_t* __restrict__ cellid,
                                                      const __grid_constant__ FFLevels ffl, const int64_t* rpA,
                                                      int32_t* colA, double* valA, float* valA32, const int64_t* rpB,
                                                      int32_t* colB, double* valB, float* valB32, int32_t* Bseg) {
    const int64_t s = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (s >= v.N) return;  // warp-uniform
    const unsigned below = (1u << lane) - 1u;
    const int k = level_of_row(v.off, v.L, s);
    const Pt y = point_at(v, s);
    Frame mine{};
    if (lane <= k) mine = frame_of(v, lane, y);
    auto emit = [&](int j, int64_t& pos, int32_t* col) {
        warp_neighbours(v, W, j, frame_from(mine, j), y, lane, [&](int32_t p, bool in, unsigned m) {
            if (in) col[pos + __popc(m & below)] = p;
            pos += __popc(m);
        });
    };
    const int64_t a0 = rpA[s];
    int64_t pa = a0;
    emit(k, pa, colA);
    const int64_t b0 = rpB[s];
    int64_t pb = b0;
    for (int j = 0; j < k; ++j) {
        if (lane == 0) Bseg[(int64_t)j * v.N + s] = (int32_t)(pb - b0);
        emit(j, pb, colB);
    }
    if (lane == 0) Bseg[(int64_t)k * v.N + s] = (int32_t)(pb - b0);
    __syncwarp();  // the columns written by the other lanes are read below
    if (FF) {
        const Frame fk = frame_from(mine, k);
        for (int64_t i = a0 + lane; i < pa; i += 32) {
            const double value = ff_entry(v, W, Wlo, cellid, ffl, k, colA[i], fk);
            valA[i] = value;
            if (valA32) valA32[i] = (float)value;
        }
        // every lane takes part in each step (the frame of the entry's level comes by shuffle)
        for (int64_t i0 = b0; i0 < pb; i0 += 32) {
            const int64_t i = i0 + lane;
            const bool ok = i < pb;
            const int32_t p = ok ? colB[i] : (int32_t)v.off[0];
            const int j = level_of_row(v.off, v.L, p);
            const Frame fj = frame_from(mine, j);
            if (ok) {
                const double value = ff_entry(v, W, Wlo, cellid, ffl, j, p, fj);
                valB[i] = value;
                if (valB32) valB32[i] = (float)value;
            }
        }
        return;
    }
    {
        const double inv = v.inv_delta[k], sc = v.dscale[k];
        for (int64_t i = a0 + lane; i < pa; i += 32) {
            const double value = sc * wendland_eval<double>(v.w, sqrt(dist2(v, colA[i], y)) * inv);
            valA[i] = value;
            if (valA32) valA32[i] = (float)value;
        }
    }
    for (int64_t i = b0 + lane; i < pb; i += 32) {
        const int32_t p = colB[i];
        const int j = level_of_row(v.off, v.L, p);
        const double value = v.dscale[j] * wendland_eval<double>(v.w, sqrt(dist2(v, p, y)) * v.inv_delta[j]);
        valB[i] = value;
        if (valB32) valB32[i] = (float)value;
    }
}

// A.rp and B.rp at the level boundaries: out[l] = rpA[off[l]], out[L + 1 + l] = rpB[off[l]].
__global__ void k_level_rows(HierView v, const int64_t* rpA, const int64_t* rpB, int64_t* out) {
    const int l = threadIdx.x;
    if (l <= v.L) {
        out[l] = rpA[v.off[l]];
        out[v.L + 1 + l] = rpB[v.off[l]];
    }
}

// Entries of every block B_kj (k > j): out[k * L + j].
__global__ void k_block_nnz(const int32_t* Bseg, const int64_t* rpB, HierView v, unsigned long long* out) {
    __shared__ unsigned long long sh[MS_MAXL * MS_MAXL];
    const int L = v.L;
    for (int i = threadIdx.x; i < L * L; i += blockDim.x) sh[i] = 0ull;
    __syncthreads();
    const int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (s < v.N) {
        const int k = level_of_row(v.off, L, s);
        for (int j = 0; j < k; ++j) {
            const int32_t e = Bseg[(int64_t)(j + 1) * v.N + s], b = Bseg[(int64_t)j * v.N + s];
            if (e > b) atomicAdd(&sh[k * L + j], (unsigned long long)(e - b));
        }
    }
    __syncthreads();
    for (int i = threadIdx.x; i < L * L; i += blockDim.x)
        if (sh[i]) atomicAdd(&out[i], sh[i]);
}

inline unsigned nblk(int64_t n, int bs) { return (unsigned)std::max<int64_t>(1, (n + bs - 1) / bs); }

}  // namespace

// ---------------------------------------------------------------- host build

ms_status ms_build_impl(ms_hierarchy* h, const double* pts, cudaStream_t st) {
    HierView& v = h->view;
    const int d = h->d, L = h->L;
    const int64_t N = h->N;

    std::vector<void*> temps;
    auto talloc = [&](void** p, size_t bytes) -> ms_status {
        cudaError_t e = cudaMallocAsync(p, std::max<size_t>(bytes, 16), st);
        if (e != cudaSuccess) {
            ms_set_error(MS_ERR_OOM, "device allocation of %zu bytes failed: %s", bytes, cudaGetErrorString(e));
            return MS_ERR_OOM;
        }
        temps.push_back(*p);
        return MS_OK;
    };
    struct Freer {
        std::vector<void*>& t;
        cudaStream_t s;
        ~Freer() { for (void* p : t) cudaFreeAsync(p, s); }
    } freer{temps, st};

    MS_CUDA(cudaEventRecord(h->ev0, st));

    // 1. level bounding boxes (and a finiteness check)
    int64_t* off_dev = nullptr;
    double* part = nullptr;
    MS_TRY(talloc((void**)&off_dev, sizeof(int64_t) * (L + 1)));
    MS_TRY(talloc((void**)&part, sizeof(double) * L * kBboxBlocks * 7));
    MS_CUDA(cudaMemcpyAsync(off_dev, v.off, sizeof(int64_t) * (L + 1), cudaMemcpyHostToDevice, st));
    k_bbox<<<dim3(kBboxBlocks, L), 256, 0, st>>>(pts, d, off_dev, L, part); ms_count_launch();
    MS_CUDA(cudaGetLastError());
    std::vector<double> hp((size_t)L * kBboxBlocks * 7);
    MS_CUDA(cudaMemcpyAsync(hp.data(), part, sizeof(double) * hp.size(), cudaMemcpyDeviceToHost, st));
    MS_CUDA(cudaStreamSynchronize(st));

    const int split = h->opts.cell_split > 0 ? h->opts.cell_split : 1;
    v.R = split;
    int64_t cells = 0;
    for (int l = 0; l < L; ++l) {
        double lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
        double bad = 0;
        for (int b = 0; b < kBboxBlocks; ++b) {
            const double* q = &hp[((size_t)l * kBboxBlocks + b) * 7];
            for (int a = 0; a < d; ++a) { lo[a] = std::min(lo[a], q[a]); hi[a] = std::max(hi[a], q[3 + a]); }
            bad += q[6];
        }
        if (bad > 0) {
            ms_set_error(MS_ERR_NUMERIC, "level %d has non-finite point coordinates", l + 1);
            return MS_ERR_NUMERIC;
        }
        LevelGrid& g = v.grid[l];
        double cell = v.delta[l] / split;
        const int max_bits = d == 1 ? 30 : (d == 2 ? 15 : 10);
        int bits = 0;
        for (int tries = 0; tries < 64; ++tries) {
            int gmax = 1;
            for (int a = 0; a < 3; ++a) {
                g.G[a] = 1;
                if (a < d) {
                    const double ext = (hi[a] - lo[a]) / cell;
                    g.G[a] = (int)std::max(1.0, std::ceil(std::min(ext, 1e9)));
                    gmax = std::max(gmax, g.G[a]);
                }
            }
            bits = 0;
            while ((1 << bits) < gmax) ++bits;
            if (bits <= max_bits && (int64_t(1) << (bits * d)) <= (int64_t(1) << 27)) break;
            cell *= 2.0;  // too many cells: coarser grid, still covers delta with radius R
        }
        for (int a = 0; a < 3; ++a) g.lo[a] = a < d ? lo[a] : 0.0;
        g.cell = cell;
        g.inv_cell = 1.0 / cell;
        g.cod = (float)(cell / v.delta[l]);
        g.bits = bits;
        g.ncells = int64_t(1) << (bits * d);
        g.cell_off = cells;
        cells += g.ncells;
    }
    h->total_cells = cells;
    if (cells >= (int64_t(1) << 31) - 1) {
        ms_set_error(MS_ERR_ARG, "too many grid cells (%lld)", (long long)cells);
        return MS_ERR_ARG;
    }

    // 2. counting sort by (level, Morton cell), ranked by input index inside a cell
    int32_t *key, *count, *cursor, *tmp, *tile;
    MS_TRY(talloc((void**)&key, sizeof(int32_t) * N));
    MS_TRY(talloc((void**)&count, sizeof(int32_t) * cells));
    MS_TRY(talloc((void**)&cursor, sizeof(int32_t) * cells));
    MS_TRY(talloc((void**)&tmp, sizeof(int32_t) * N));
    const int64_t maxn = std::max<int64_t>(N, cells) + 1;
    MS_TRY(talloc((void**)&tile, sizeof(int64_t) * ((maxn + kScanTile - 1) / kScanTile + 2)));
    MS_TRY(ms_alloc(h, (void**)&h->cell_start, sizeof(int32_t) * (cells + 1)));
    MS_TRY(ms_alloc(h, (void**)&h->perm, sizeof(int32_t) * N));
    MS_TRY(ms_alloc(h, (void**)&h->X, sizeof(double) * d * N));
    MS_CUDA(cudaMemsetAsync(count, 0, sizeof(int32_t) * cells, st));
    MS_CUDA(cudaMemsetAsync(cursor, 0, sizeof(int32_t) * cells, st));
    v.X = h->X;
    v.cell_start = h->cell_start;
    k_cell_keys<<<nblk(N, 256), 256, 0, st>>>(pts, v, key, count); ms_count_launch();
    exclusive_scan<int32_t, int32_t>(count, cells, h->cell_start, tile, st);
    k_scatter<<<nblk(N, 256), 256, 0, st>>>(key, h->cell_start, cursor, tmp, N); ms_count_launch();
    k_rank<<<nblk(N, 256), 256, 0, st>>>(key, h->cell_start, tmp, h->perm, N); ms_count_launch();
    k_gather_points<<<nblk(N, 256), 256, 0, st>>>(pts, h->perm, h->X, d, N); ms_count_launch();
    MS_CUDA(cudaGetLastError());
    // double-float entries (MIXED) also need the low parts of the offsets
    const bool ffvals = h->opts.precision == MS_PREC_MIXED;
    float* Wlo = nullptr;
    MS_TRY(ms_alloc(h, (void**)&h->W, sizeof(float) * d * N));
    MS_TRY(ms_alloc(h, (void**)&h->cellid, sizeof(int32_t) * N));
    if (ffvals) MS_TRY(talloc((void**)&Wlo, sizeof(float) * d * N));
    k_mf_coords<<<nblk(N, 256), 256, 0, st>>>(v, h->W, Wlo, h->cellid); ms_count_launch();
    MS_CUDA(cudaGetLastError());

    // 3. CSR of A (diagonal blocks) and B (strictly lower blocks)
    int32_t *cntA, *cntB;
    MS_TRY(talloc((void**)&cntA, sizeof(int32_t) * N));
    MS_TRY(talloc((void**)&cntB, sizeof(int32_t) * N));
    MS_TRY(ms_alloc(h, (void**)&h->A.rp, sizeof(int64_t) * (N + 1)));
    MS_TRY(ms_alloc(h, (void**)&h->B.rp, sizeof(int64_t) * (N + 1)));
    k_csr_count<<<nblk(N * 32, kCsrBS), kCsrBS, 0, st>>>(v, h->W, cntA, cntB); ms_count_launch();
    exclusive_scan<int32_t, int64_t>(cntA, N, h->A.rp, (int64_t*)tile, st);
    exclusive_scan<int32_t, int64_t>(cntB, N, h->B.rp, (int64_t*)tile, st);
    MS_CUDA(cudaGetLastError());
    int64_t nnz[2];
    MS_CUDA(cudaMemcpyAsync(&nnz[0], h->A.rp + N, sizeof(int64_t), cudaMemcpyDeviceToHost, st));
    MS_CUDA(cudaMemcpyAsync(&nnz[1], h->B.rp + N, sizeof(int64_t), cudaMemcpyDeviceToHost, st));
    MS_CUDA(cudaStreamSynchronize(st));
    h->A.nnz = nnz[0];
    h->B.nnz = nnz[1];
    // FP32 CSR values serve the MIXED inner CG unless it runs matrix-free
    const bool fp32 = h->opts.precision == MS_PREC_MIXED && h->opts.op != MS_OP_MATRIX_FREE;
    MS_TRY(ms_alloc(h, (void**)&h->A.col, sizeof(int32_t) * h->A.nnz));
    MS_TRY(ms_alloc(h, (void**)&h->A.v64, sizeof(double) * h->A.nnz));
    if (fp32) MS_TRY(ms_alloc(h, (void**)&h->A.v32, sizeof(float) * h->A.nnz));
    MS_TRY(ms_alloc(h, (void**)&h->B.col, sizeof(int32_t) * h->B.nnz));
    MS_TRY(ms_alloc(h, (void**)&h->B.v64, sizeof(double) * h->B.nnz));
    // the fit updates beta with FP64 B values only; FP32 B values serve MS_APPLY_B32 on request
    if (h->opts.lower_fp32) MS_TRY(ms_alloc(h, (void**)&h->B.v32, sizeof(float) * h->B.nnz));
    MS_TRY(ms_alloc(h, (void**)&h->Bseg, sizeof(int32_t) * (size_t)L * N));
    FFLevels ffl{};
    for (int l = 0; l < L; ++l) {
        ffl.cod[l] = ff_from_double(v.grid[l].cell / v.delta[l]);
        ffl.ds[l] = ff_from_double(v.dscale[l]);
    }
    if (ffvals)
        k_csr_fill<true><<<nblk(N * 32, kCsrBS), kCsrBS, 0, st>>>(v, h->W, Wlo, h->cellid, ffl, h->A.rp, h->A.col,
                                                                  h->A.v64, h->A.v32, h->B.rp, h->B.col, h->B.v64,
                                                                  h->B.v32, h->Bseg);
    else
        k_csr_fill<false><<<nblk(N * 32, kCsrBS), kCsrBS, 0, st>>>(v, h->W, nullptr, h->cellid, ffl, h->A.rp,
                                                                   h->A.col, h->A.v64, h->A.v32, h->B.rp, h->B.col,
                                                                   h->B.v64, h->B.v32, h->Bseg);
    ms_count_launch();
    unsigned long long* blk;
    MS_TRY(talloc((void**)&blk, sizeof(unsigned long long) * L * L));
    MS_CUDA(cudaMemsetAsync(blk, 0, sizeof(unsigned long long) * L * L, st));
    k_block_nnz<<<nblk(N, 256), 256, 0, st>>>(h->Bseg, h->B.rp, v, blk); ms_count_launch();
    MS_CUDA(cudaGetLastError());
    std::vector<unsigned long long> hb((size_t)L * L);
    MS_CUDA(cudaMemcpyAsync(hb.data(), blk, sizeof(unsigned long long) * L * L, cudaMemcpyDeviceToHost, st));
    int64_t* lvrows;
    MS_TRY(talloc((void**)&lvrows, sizeof(int64_t) * 2 * (L + 1)));
    k_level_rows<<<1, 64, 0, st>>>(v, h->A.rp, h->B.rp, lvrows); ms_count_launch();
    MS_CUDA(cudaGetLastError());
    std::vector<int64_t> hl(2 * (L + 1));
    MS_CUDA(cudaMemcpyAsync(hl.data(), lvrows, sizeof(int64_t) * hl.size(), cudaMemcpyDeviceToHost, st));
    MS_CUDA(cudaEventRecord(h->ev1, st));
    MS_CUDA(cudaStreamSynchronize(st));
    float ms = 0.f;
    MS_CUDA(cudaEventElapsedTime(&ms, h->ev0, h->ev1));
    h->build_ms = ms;
    for (int k = 0; k < L; ++k)
        for (int j = 0; j < L; ++j) h->Bblk[k][j] = (int64_t)hb[(size_t)k * L + j];
    for (int l = 0; l <= L; ++l) {
        h->rpA_lv[l] = hl[l];
        h->rpB_lv[l] = hl[L + 1 + l];
    }
    return MS_OK;
}
