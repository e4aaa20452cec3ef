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
#include "ms_geom.cuh"

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
// One warp per row s (level k).  Its candidates are the (2R+1)^d cells around s's
// cell in the grid of every column level j <= k (j = k for A, j < k for B); the
// lanes take one (level, cell) pair each and walk that cell's points.  The count
// kernel stores every pair's count; the fill scans them to place each lane's
// columns and writes the same entries in the same order.  The test |x_p - x_s| < delta_j is
// taken in FP32 first, from cell-relative coordinates in units of delta_j (the
// cell offset plus the FP32 in-cell offsets W), whose error is ~1e-6 of delta_j^2;
// only candidates within 1e-4 of the boundary are re-tested in FP64
// (fma-accumulated r^2 < delta_j^2), so the pattern is exactly the FP64 one.
// The FP64 values are computed for the entries only (FP64 is scarce on this GPU).

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

constexpr int kCsrBS = 256;  // 8 rows per block

// Candidate cells of row s: the (2R+1)^d cells around y's cell in each level j <= k, as
// pairs t = j nc + q (q: dx fastest, then dy, dz).  Pair t of row s has slot
// PairLayout::base[k] + (s - off[k]) (k + 1) nc + t in the per-pair count array.
struct PairLayout {
    int64_t base[MS_MAXL];
    int nc;
    // Frames: row s of level k has its frames in levels 0..k at fbase[k] + (s - off[k]) (k + 1) + j
    // (fbase[L] = all frames).
    int64_t fbase[MS_MAXL + 1];
    double d2[MS_MAXL];  // delta_j^2, rounded as the FP64 product delta_j * delta_j
};

// Every row's frames in the levels up to its own, one thread per (row, level).  Set up in
// the count and again in the fill by lanes 0..k of a row's warp, the frames took about 34
// FP64 instructions per row with a few lanes active each, and GB300's FP64 pipe holds a warp
// instruction about 19 cycles whatever its active lanes: most of the count kernel's time.
// Here every lane is busy and each frame is set up once.
__global__ void k_frames(const __grid_constant__ HierView v, const __grid_constant__ PairLayout pl, Frame* F) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= pl.fbase[v.L]) return;
    int k = 0;
    while (k + 1 < v.L && i >= pl.fbase[k + 1]) ++k;
    const int64_t r = i - pl.fbase[k];
    const int64_t row = r / (k + 1);
    const int j = (int)(r - row * (k + 1));
    F[i] = frame_of(v, j, point_at(v, v.off[k] + row));
}

// The points [ps, pe) and the cell offsets (units of delta_j) of pair q of level j, seen
// from y's frame f in level j's grid; false when the cell lies outside the grid.
__device__ __forceinline__ bool pair_cell(const HierView& v, int j, int q, const Frame& f, int32_t& ps, int32_t& pe,
                                          float& o0, float& o1, float& o2) {
    const LevelGrid& g = v.grid[j];
    const int R = v.R, side = 2 * R + 1;
    const int dx = q % side - R;
    const int dy = v.d >= 2 ? (q / side) % side - R : 0;
    const int dz = v.d >= 3 ? q / (side * side) - R : 0;
    const int cx = f.c[0] + dx, cy = f.c[1] + dy, cz = f.c[2] + dz;
    if (cx < 0 || cx >= g.G[0] || cy < 0 || cy >= g.G[1] || cz < 0 || cz >= g.G[2]) return false;
    const int64_t gid = g.cell_off + morton(v.d, cx, cy, cz);
    ps = __ldg(v.cell_start + gid);
    pe = __ldg(v.cell_start + gid + 1);
    o0 = cell_offset(dx, g.cod, f.fr[0]);
    o1 = cell_offset(dy, g.cod, f.fr[1]);
    o2 = cell_offset(dz, g.cod, f.fr[2]);
    return true;
}

// Entries of row s: one warp per row, one lane per (column level j, neighbour cell) pair
// at a time, each lane walking its cell's points.  Also stores each pair's count, from
// which the fill places its columns.
__global__ void __launch_bounds__(kCsrBS, 4) k_csr_count(const __grid_constant__ HierView v, const float* __restrict__ W,
                                                       const __grid_constant__ PairLayout pl,
                                                       const Frame* __restrict__ F, int32_t* cntA, int32_t* cntB,
                                                       int32_t* pcnt, int onlyA) {
    const int64_t s = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (s >= v.N) return;  // warp-uniform
    const int k = level_of_row(v.off, v.L, s);
    const Pt y = point_at(v, s);
    // lane j <= k holds y's frame in level j's grid
    Frame mine{};
    if (lane <= k) mine = F[pl.fbase[k] + (s - v.off[k]) * (k + 1) + lane];
    const int nc = pl.nc;
    const int pairs = (k + 1) * nc;
    int32_t* pc = pcnt + pl.base[k] + (s - v.off[k]) * pairs;
    int32_t na = 0, nb = 0;
    // the lower-block pairs (levels j < k; none with onlyA, when B is not stored): a lane per
    // pair walking its cell's points
    const int pairsB = onlyA ? 0 : k * nc;
    for (int t0 = 0; t0 < pairsB; t0 += 32) {
        const int t = t0 + lane;
        const int j = min(t / nc, k);  // lanes past the last pair read a valid frame and skip
        const Frame f = frame_from(mine, j);
        if (t >= pairsB) continue;
        int32_t ps = 0, pe = 0;
        float o0 = 0.f, o1 = 0.f, o2 = 0.f;
        int32_t n = 0;
        if (pair_cell(v, j, t - j * nc, f, ps, pe, o0, o1, o2)) {
            const double d2 = pl.d2[j];
            for (int32_t p = ps; p < pe; ++p) n += within(v, W, p, o0, o1, o2, y, d2) ? 1 : 0;
        }
        pc[t] = n;
        nb += n;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) nb += __shfl_xor_sync(0xffffffffu, nb, o);
    // the row's own level: the warp walks each neighbour cell together (a lane per point)
    {
        const Frame fk = frame_from(mine, k);
        const double d2 = pl.d2[k];
        for (int q = 0; q < nc; ++q) {
            int32_t ps = 0, pe = 0;
            float o0 = 0.f, o1 = 0.f, o2 = 0.f;
            int32_t n = 0;
            if (pair_cell(v, k, q, fk, ps, pe, o0, o1, o2))
                for (int32_t p0 = ps; p0 < pe; p0 += 32) {
                    const int32_t p = p0 + lane;
                    n += __popc(__ballot_sync(0xffffffffu, p < pe && within(v, W, p, o0, o1, o2, y, d2)));
                }
            if (lane == 0) pc[k * nc + q] = n;
            na += n;
        }
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
// FF: entries in double-float arithmetic (MIXED builds), else FP64.  E, K: the Wendland
// exponent and degree when compiled for them (0: taken from v.w).
template <bool FF, int E, int K>
__global__ void __launch_bounds__(kCsrBS, 4) k_csr_fill(const __grid_constant__ HierView v, const float* __restrict__ W,
                                                      const float* __restrict__ Wlo, const int32_t* __restrict__ cellid,
                                                      const __grid_constant__ FFLevels ffl,
                                                      const __grid_constant__ PairLayout pl,
                                                      const Frame* __restrict__ F,
                                                      const int32_t* __restrict__ pcnt, const int64_t* rpA,
                                                      int32_t* colA, double* valA, float* valA32, const int64_t* rpB,
                                                      int32_t* colB, double* valB, float* valB32, int32_t* Bseg,
                                                      int onlyA) {
    const int64_t s = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (s >= v.N) return;  // warp-uniform
    const int k = level_of_row(v.off, v.L, s);
    const Pt y = point_at(v, s);
    Frame mine{};
    if (lane <= k) mine = F[pl.fbase[k] + (s - v.off[k]) * (k + 1) + lane];
    // Columns: lane per (level, cell) pair as in the count; a warp scan of the stored pair
    // counts (A pairs and B pairs separately, in pair order) gives every lane the position
    // of its cell's first entry, so the columns come out in the order of the pairs (B: level
    // by level), points in cell order, and the count's decisions are repeated exactly.
    const int nc = pl.nc;
    const int pairs = (k + 1) * nc;
    const int32_t* pc = pcnt + pl.base[k] + (s - v.off[k]) * pairs;
    const int64_t a0 = rpA[s], b0 = rpB[s];
    int64_t pa = a0, pb = b0;
    // the lower-block pairs (levels j < k): a lane per pair, placed by a warp scan of the counts
    const int pairsB = onlyA ? 0 : k * nc;
    for (int t0 = 0; t0 < pairsB; t0 += 32) {
        const int t = t0 + lane;
        const bool ok = t < pairsB;
        const int j = min(t / nc, k);
        const Frame f = frame_from(mine, j);
        const int32_t n = ok ? __ldg(pc + t) : 0;
        int32_t ib = n;  // inclusive scan over the lanes
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int32_t ub = __shfl_up_sync(0xffffffffu, ib, o);
            if (lane >= o) ib += ub;
        }
        const int32_t tb = __shfl_sync(0xffffffffu, ib, 31);
        const int q = t - j * nc;
        // first pair of a column level j < k: its segment of the B row starts here
        if (ok && q == 0 && Bseg) Bseg[(int64_t)j * v.N + s] = (int32_t)(pb + ib - n - b0);
        if (ok && n > 0) {
            int32_t ps = 0, pe = 0;
            float o0 = 0.f, o1 = 0.f, o2 = 0.f;
            pair_cell(v, j, q, f, ps, pe, o0, o1, o2);
            const double d2 = pl.d2[j];
            int64_t pos = pb + ib - n;
            for (int32_t p = ps; p < pe; ++p)
                if (within(v, W, p, o0, o1, o2, y, d2)) colB[pos++] = p;
        }
        pb += tb;
    }
    // the row's own level: the warp walks each neighbour cell together and places the columns
    // by ballot, in the same order (pairs in order, points in cell order) and with the same
    // decisions as the count
    {
        const Frame fk = frame_from(mine, k);
        const double d2 = pl.d2[k];
        for (int q = 0; q < nc; ++q) {
            int32_t ps = 0, pe = 0;
            float o0 = 0.f, o1 = 0.f, o2 = 0.f;
            if (!pair_cell(v, k, q, fk, ps, pe, o0, o1, o2)) continue;
            for (int32_t p0 = ps; p0 < pe; p0 += 32) {
                const int32_t p = p0 + lane;
                const bool hit = p < pe && within(v, W, p, o0, o1, o2, y, d2);
                const unsigned m = __ballot_sync(0xffffffffu, hit);
                if (hit) colA[pa + __popc(m & ((1u << lane) - 1u))] = p;
                pa += __popc(m);
            }
        }
    }
    if (lane == 0 && Bseg) Bseg[(int64_t)k * v.N + s] = (int32_t)(pb - b0);
    __syncwarp();  // the columns written by the other lanes are read below
    if (FF) {
        const Frame fk = frame_from(mine, k);
        for (int64_t i = a0 + lane; i < pa; i += 32) {
            const ff value = ff_entry<E, K>(v, W, Wlo, cellid, ffl, k, colA[i], fk);
            valA[i] = ff_to_double(value);
            if (valA32) valA32[i] = value.hi;  // the FP32 value nearest to hi + lo (|lo| <= ulp(hi) / 2)
        }
        // every lane takes part in each step (the frame of the entry's level comes by shuffle)
        for (int64_t i0 = b0; i0 < pb; i0 += 32) {
            const int64_t i = i0 + lane;
            const bool ok = i < pb;
            const int32_t p = ok ? colB[i] : (int32_t)v.off[0];
            const int j = level_of_row(v.off, v.L, p);
            const Frame fj = frame_from(mine, j);
            if (ok) {
                const ff value = ff_entry<E, K>(v, W, Wlo, cellid, ffl, j, p, fj);
                valB[i] = ff_to_double(value);
                if (valB32) valB32[i] = value.hi;
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
        MS_TRY(ms_tmp_alloc(p, bytes, st));
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
    MS_TRY(ms_alloc(h, (void**)&h->W, sizeof(float) * d * N));
    MS_TRY(ms_alloc(h, (void**)&h->cellid, sizeof(int32_t) * N));
    if (ffvals) MS_TRY(ms_alloc(h, (void**)&h->Wlo, sizeof(float) * d * N));
    float* Wlo = h->Wlo;
    k_mf_coords<<<nblk(N, 256), 256, 0, st>>>(v, h->W, Wlo, h->cellid); ms_count_launch();
    MS_CUDA(cudaGetLastError());

    // 3. CSR of A (diagonal blocks) and B (strictly lower blocks)
    int32_t *cntA, *cntB, *pcnt = nullptr;
    MS_TRY(talloc((void**)&cntA, sizeof(int32_t) * N));
    MS_TRY(talloc((void**)&cntB, sizeof(int32_t) * N));
    MS_TRY(ms_alloc(h, (void**)&h->A.rp, sizeof(int64_t) * (N + 1)));
    MS_TRY(ms_alloc(h, (void**)&h->B.rp, sizeof(int64_t) * (N + 1)));
    // per-(row, level, cell) counts: rows of level k have (k + 1) nc pairs
    PairLayout pl{};
    {
        const int side = 2 * v.R + 1;
        pl.nc = d == 1 ? side : (d == 2 ? side * side : side * side * side);
        int64_t tot = 0, ftot = 0;
        for (int l = 0; l < L; ++l) {
            pl.base[l] = tot;
            pl.fbase[l] = ftot;
            tot += (v.off[l + 1] - v.off[l]) * (int64_t)(l + 1) * pl.nc;
            ftot += (v.off[l + 1] - v.off[l]) * (int64_t)(l + 1);
            pl.d2[l] = v.delta[l] * v.delta[l];
        }
        pl.fbase[L] = ftot;
        int32_t* pc = nullptr;
        MS_TRY(talloc((void**)&pc, sizeof(int32_t) * tot));
        pcnt = pc;
    }
    Frame* frames = nullptr;
    // lower_op = MATRIX_FREE: the handle keeps the frames (36 bytes per (row, level) pair, instead
    // of B's 12 bytes per entry) for the fit's lower-block updates
    const bool keep_frames = h->opts.lower_op == MS_OP_MATRIX_FREE;
    if (keep_frames) {
        MS_TRY(ms_alloc(h, (void**)&frames, sizeof(Frame) * pl.fbase[L]));
        h->frames = frames;
        for (int l = 0; l <= L; ++l) h->frame_base[l] = pl.fbase[l];
    } else {
        MS_TRY(talloc((void**)&frames, sizeof(Frame) * pl.fbase[L]));
    }
    k_frames<<<nblk(pl.fbase[L], 256), 256, 0, st>>>(v, pl, frames); ms_count_launch();
    // lower_op = MATRIX_FREE: the fit recomputes B's entries, the build stores A only
    const int onlyA = h->opts.lower_op == MS_OP_MATRIX_FREE ? 1 : 0;
    if (onlyA) MS_CUDA(cudaMemsetAsync(cntB, 0, sizeof(int32_t) * N, st));
    k_csr_count<<<nblk(N * 32, kCsrBS), kCsrBS, 0, st>>>(v, h->W, pl, frames, cntA, cntB, pcnt, onlyA);
    ms_count_launch();
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
    if (!onlyA) MS_TRY(ms_alloc(h, (void**)&h->Bseg, sizeof(int32_t) * (size_t)L * N));
    // the solve's CSR rows read columns and values four entries at a time (128-bit loads from
    // the first multiple of 4 of a row): the arrays must start on 16-byte boundaries
    for (const void* q : {(const void*)h->A.col, (const void*)h->A.v64, (const void*)h->A.v32, (const void*)h->B.col,
                          (const void*)h->B.v64, (const void*)h->B.v32})
        if (reinterpret_cast<uintptr_t>(q) % 16 != 0) {
            ms_set_error(MS_ERR_STATE, "a CSR array is not 16-byte aligned");
            return MS_ERR_STATE;
        }
    FFLevels ffl{};
    for (int l = 0; l < L; ++l) {
        ffl.cod[l] = ff_from_double(v.grid[l].cell / v.delta[l]);
        ffl.ds[l] = ff_from_double(v.dscale[l]);
    }
    for (int i = 0; i < 4; ++i) ffl.c[i] = ff_from_double(v.w.c[i]);
    {
        // phi_{d,1} has (e, k) = (floor(d/2) + 3, 1) and phi_{d,2} (floor(d/2) + 5, 2): (4, 1) and (6, 2)
        // for d = 2, 3 get their own straight-line code
        auto fill = ffvals ? (v.w.e == 4 && v.w.k == 1   ? k_csr_fill<true, 4, 1>
                              : v.w.e == 6 && v.w.k == 2 ? k_csr_fill<true, 6, 2>
                                                         : k_csr_fill<true, 0, 0>)
                           : k_csr_fill<false, 0, 0>;
        fill<<<nblk(N * 32, kCsrBS), kCsrBS, 0, st>>>(v, h->W, Wlo, h->cellid, ffl, pl, frames, pcnt, h->A.rp, h->A.col,
                                                      h->A.v64, h->A.v32, h->B.rp, h->B.col, h->B.v64, h->B.v32,
                                                      h->Bseg, onlyA);
    }
    ms_count_launch();
    unsigned long long* blk;
    MS_TRY(talloc((void**)&blk, sizeof(unsigned long long) * L * L));
    MS_CUDA(cudaMemsetAsync(blk, 0, sizeof(unsigned long long) * L * L, st));
    if (!onlyA) {
        k_block_nnz<<<nblk(N, 256), 256, 0, st>>>(h->Bseg, h->B.rp, v, blk);
        ms_count_launch();
    }
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
