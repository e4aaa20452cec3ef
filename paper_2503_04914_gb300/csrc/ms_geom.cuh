// Geometry of the level grids shared by the CSR build and the matrix-free lower blocks:
// frames of a point in a level's cell grid, the double-float entries of the MIXED build,
// and the matrix-free rows of the strictly lower blocks B_kj = Phi_{delta_j}(X_k, X_j)
// (Section 3, definition of B; Assumption 1, eq. kernelscaling).
#pragma once

#include "ms_ff.cuh"
#include "ms_internal.cuh"
#include "ms_matfree.cuh"

namespace {

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

// Frame of y in level j's grid, all axes (FP64 set-up; k_frames calls it once per (row, level)).
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

// Per-level constants (cell size / delta, delta^-d) and the Wendland polynomial's
// coefficients as double-floats, converted once on the host: a conversion from FP64 costs
// FP64 instructions, which is what this path avoids.
struct FFLevels {
    ff cod[MS_MAXL];
    ff ds[MS_MAXL];
    ff c[4];
};

// phi(r) for the Wendland closed form w in double-float; 0 for r >= 1.  E, K: the exponent
// and the degree as compile-time constants (0: read them from w).
template <int E, int K>
__device__ __forceinline__ ff ff_wendland(const WendlandPoly& w, const ff* c, ff r) {
    if (!(r.hi < 1.0f || (r.hi == 1.0f && r.lo < 0.0f))) return {0.0f, 0.0f};
    const ff s = ff_add({1.0f, 0.0f}, ff_neg(r));
    const ff s2 = ff_sqr(s), s4 = ff_sqr(s2);
    const int e = E > 0 ? E : w.e;
    ff pw;
    if (e == 4) pw = s4;
    else if (e == 6) pw = ff_mul(s4, s2);
    else if (e == 8) pw = ff_sqr(s4);
    else {
        pw = {1.0f, 0.0f};
        for (int i = 0; i < e; ++i) pw = ff_mul(pw, s);
    }
    const int k = E > 0 ? K : w.k;
    ff p = c[k];
#pragma unroll
    for (int i = 3; i >= 1; --i)
        if (i <= k) p = ff_add(ff_mul(p, r), c[i - 1]);
    return ff_mul(pw, p);
}

// delta_j^-d phi(|x_p - y| / delta_j) for point p of level j (cell cp, offsets W + Wlo) and
// y's frame f in level j's grid: the scaled offset on axis a is
// (cp_a - c_a) cod + (W_a + Wlo_a) - (fr_a + frlo_a).  cod_exact: cod is a float, so the cell
// term is an exact FP32 product.
template <int E, int K>
__device__ __forceinline__ ff ff_entry(const HierView& v, const float* __restrict__ W,
                                           const float* __restrict__ Wlo, const int32_t* __restrict__ cellid,
                                           const FFLevels& ffl, int j, int32_t p, const Frame& f) {
    int cp[3];
    demorton(v.d, (uint32_t)__ldg(cellid + p), cp);
    const bool cod_exact = ffl.cod[j].lo == 0.0f;
    ff r2 = {0.0f, 0.0f};
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        if (a < v.d) {
            const ff w = {__ldg(W + a * v.N + p), __ldg(Wlo + a * v.N + p)};
            const float dc = small_int_to_float(cp[a] - f.c[a]);
            ff t;
            if (cod_exact) {
                t = ff_sum3(__fmul_rn(dc, ffl.cod[j].hi), w, {f.fr[a], f.frlo[a]});
            } else {
                t = ff_add(ff_add(ff_mul(ffl.cod[j], {dc, 0.0f}), w), ff_neg({f.fr[a], f.frlo[a]}));
            }
            r2 = a == 0 ? ff_sqr(t) : ff_add(r2, ff_sqr(t));
        }
    }
    return ff_mul(ffl.ds[j], ff_wendland<E, K>(v.w, ffl.c, ff_sqrt(r2)));
}

// ff_entry for a point p known to lie in the cell displaced by dcs[a] cells from f's cell (the
// candidate loops know it): the same arithmetic without the cell id's load and Morton decode.
template <int E, int K>
__device__ __forceinline__ ff ff_entry_dc(const HierView& v, const float* __restrict__ W,
                                          const float* __restrict__ Wlo, const FFLevels& ffl, int j, int32_t p,
                                          const Frame& f, const int* dcs) {
    const bool cod_exact = ffl.cod[j].lo == 0.0f;
    ff r2 = {0.0f, 0.0f};
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        if (a < v.d) {
            const ff w = {__ldg(W + a * v.N + p), __ldg(Wlo + a * v.N + p)};
            const float dc = small_int_to_float(dcs[a]);
            ff t;
            if (cod_exact) {
                t = ff_sum3(__fmul_rn(dc, ffl.cod[j].hi), w, {f.fr[a], f.frlo[a]});
            } else {
                t = ff_add(ff_add(ff_mul(ffl.cod[j], {dc, 0.0f}), w), ff_neg({f.fr[a], f.frlo[a]}));
            }
            r2 = a == 0 ? ff_sqr(t) : ff_add(r2, ff_sqr(t));
        }
    }
    return ff_mul(ffl.ds[j], ff_wendland<E, K>(v.w, ffl.c, ff_sqrt(r2)));
}

// Offset (units of delta) of a neighbour cell displaced by `dc` cells, seen from a point at
// fractional offset fr in its own cell; both CSR kernels take it from here so that they
// make the same decisions.
__device__ __forceinline__ float cell_offset(int dc, float cod, float fr) {
    return __fsub_rn(__fmul_rn(small_int_to_float(dc), cod), fr);
}


// The per-level double-float constants of a hierarchy (host side: a conversion from FP64
// costs FP64 instructions on the device).
inline FFLevels make_fflevels(const HierView& v) {
    FFLevels f{};
    for (int l = 0; l < v.L; ++l) {
        f.cod[l] = ff_from_double(v.grid[l].cell / v.delta[l]);
        f.ds[l] = ff_from_double(v.dscale[l]);
    }
    for (int i = 0; i < 4; ++i) f.c[i] = ff_from_double(v.w.c[i]);
    return f;
}

// ---------------------------------------------------------------- matrix-free lower blocks
//
// sum_p B(y, p) x_p over the points p of level j within delta_j of y (a point of a finer
// level, given by its frame f in level j's grid): the paper's lower-block mat-vec (McV of
// Section 5.3) with the entries recomputed instead of read.  The lanes sl = 0..S-1 of a group
// stride over each candidate cell's points (the (2R+1)^d cells around f's cell); the caller
// reduces over the group.  A candidate whose FP32 scaled distance exceeds 1 + 1e-4 is skipped
// (its entry is zero: phi vanishes for r >= 1, and the FP32 error is far below the band).
//   FF: the double-float entry ff_entry (the arithmetic, and so the value, of the stored
//       B of a MIXED build) times x_p = xhi_p + xlo_p, accumulated in double-float;
//   else: the FP32 entry delta_j^-d phi(r) (r through the hardware reciprocal square root)
//       times x_p = xhi_p, accumulated in FP32 (the result's lo part stays 0).
template <int D, int E, int K, bool FF>
__device__ __forceinline__ ff lower_row_mf(const HierView& v, const float* __restrict__ W,
                                           const float* __restrict__ Wlo, const int32_t* __restrict__ cellid,
                                           const FFLevels& ffl, const float* fc, float dsj, int j, const Frame& f,
                                           const float* xhi, const float* xlo, int sl, int S) {
    const LevelGrid& g = v.grid[j];
    const int R = v.R;
    const int rz = D >= 3 ? R : 0, ry = D >= 2 ? R : 0;
    const int64_t N = v.N;
    ff acc = {0.0f, 0.0f};
    for (int dz = -rz; dz <= rz; ++dz) {
        const int cz = f.c[2] + dz;
        if (D >= 3 && (cz < 0 || cz >= g.G[2])) continue;
        const float o2 = D >= 3 ? cell_offset(dz, g.cod, f.fr[2]) : 0.0f;
        for (int dy = -ry; dy <= ry; ++dy) {
            const int cy = f.c[1] + dy;
            if (D >= 2 && (cy < 0 || cy >= g.G[1])) continue;
            const float o1 = D >= 2 ? cell_offset(dy, g.cod, f.fr[1]) : 0.0f;
            for (int dx = -R; dx <= R; ++dx) {
                const int cx = f.c[0] + dx;
                if (cx < 0 || cx >= g.G[0]) continue;
                const float o0 = cell_offset(dx, g.cod, f.fr[0]);
                const int64_t gid = g.cell_off + morton(D, cx, D >= 2 ? cy : 0, D >= 3 ? cz : 0);
                const int32_t ps = __ldg(v.cell_start + gid), pe = __ldg(v.cell_start + gid + 1);
                for (int32_t p = ps + sl; p < pe; p += S) {
                    float t = o0 + __ldg(W + p);
                    float qq = t * t;
                    if (D >= 2) { t = o1 + __ldg(W + N + p); qq = fmaf(t, t, qq); }
                    if (D >= 3) { t = o2 + __ldg(W + 2 * N + p); qq = fmaf(t, t, qq); }
                    if (qq > 1.0f + 1e-4f) continue;
                    if (FF) {
                        const ff e = ff_entry<E, K>(v, W, Wlo, cellid, ffl, j, p, f);
                        acc = ff_add(acc, ff_mul(e, {xhi[p], xlo[p]}));
                    } else {
                        const float r = qq * rsqrtf(fmaxf(qq, 1e-30f));
                        acc.hi = fmaf(dsj * mf_phi<E>(fminf(r, 1.0f), fc, v.w.e), xhi[p], acc.hi);
                    }
                }
            }
        }
    }
    return acc;
}

// Dispatch on (d, Wendland exponent and degree): phi_{d,1} = (4, 1), phi_{d,2} = (6, 2) for
// d = 2, 3 get their own code, the rest the generic loops.
template <bool FF>
__device__ __forceinline__ ff lower_row_mf_any(const HierView& v, const float* W, const float* Wlo,
                                               const int32_t* cellid, const FFLevels& ffl, const float* fc, float dsj,
                                               int j, const Frame& f, const float* xhi, const float* xlo, int sl,
                                               int S) {
    const int e = v.w.e, k = v.w.k;
    if (v.d == 2) {
        if (e == 4 && k == 1) return lower_row_mf<2, 4, 1, FF>(v, W, Wlo, cellid, ffl, fc, dsj, j, f, xhi, xlo, sl, S);
        if (e == 6 && k == 2) return lower_row_mf<2, 6, 2, FF>(v, W, Wlo, cellid, ffl, fc, dsj, j, f, xhi, xlo, sl, S);
        return lower_row_mf<2, 0, 0, FF>(v, W, Wlo, cellid, ffl, fc, dsj, j, f, xhi, xlo, sl, S);
    }
    if (v.d == 3) {
        if (e == 4 && k == 1) return lower_row_mf<3, 4, 1, FF>(v, W, Wlo, cellid, ffl, fc, dsj, j, f, xhi, xlo, sl, S);
        if (e == 6 && k == 2) return lower_row_mf<3, 6, 2, FF>(v, W, Wlo, cellid, ffl, fc, dsj, j, f, xhi, xlo, sl, S);
        return lower_row_mf<3, 0, 0, FF>(v, W, Wlo, cellid, ffl, fc, dsj, j, f, xhi, xlo, sl, S);
    }
    return lower_row_mf<1, 0, 0, FF>(v, W, Wlo, cellid, ffl, fc, dsj, j, f, xhi, xlo, sl, S);
}

// The same sum by a whole warp with the candidates compacted: every lane tests one candidate
// of a cell at a time (FP32), the survivors are appended to the warp's queue q (64 entries in
// shared memory), and whenever 32 are queued every lane computes one double-float entry, so the
// entries' arithmetic runs on full warps whatever fraction of the candidates survives.  Returns
// the lane's partial sum (the caller sums over the warp).  Every lane of the warp must call it.
template <int D, int E, int K>
__device__ __forceinline__ ff lower_row_mf_warp(const HierView& v, const float* __restrict__ W,
                                                const float* __restrict__ Wlo, const int32_t* __restrict__ cellid,
                                                const FFLevels& ffl, int j, const Frame& f, const float* xhi,
                                                const float* xlo, int lane, int32_t* q, int32_t* qd) {
    const LevelGrid& g = v.grid[j];
    const int R = v.R;
    const int rz = D >= 3 ? R : 0, ry = D >= 2 ? R : 0;
    const int64_t N = v.N;
    ff acc = {0.0f, 0.0f};
    int qn = 0;  // queued candidates (warp-uniform)
    for (int dz = -rz; dz <= rz; ++dz) {
        const int cz = f.c[2] + dz;
        if (D >= 3 && (cz < 0 || cz >= g.G[2])) continue;
        const float o2 = D >= 3 ? cell_offset(dz, g.cod, f.fr[2]) : 0.0f;
        for (int dy = -ry; dy <= ry; ++dy) {
            const int cy = f.c[1] + dy;
            if (D >= 2 && (cy < 0 || cy >= g.G[1])) continue;
            const float o1 = D >= 2 ? cell_offset(dy, g.cod, f.fr[1]) : 0.0f;
            for (int dx = -R; dx <= R; ++dx) {
                const int cx = f.c[0] + dx;
                if (cx < 0 || cx >= g.G[0]) continue;
                const float o0 = cell_offset(dx, g.cod, f.fr[0]);
                const int32_t code = (dx + 4) | ((dy + 4) << 4) | ((dz + 4) << 8);  // the cell's displacement
                const int64_t gid = g.cell_off + morton(D, cx, D >= 2 ? cy : 0, D >= 3 ? cz : 0);
                const int32_t ps = __ldg(v.cell_start + gid), pe = __ldg(v.cell_start + gid + 1);
                for (int32_t base = ps; base < pe; base += 32) {
                    const int32_t p = base + lane;
                    bool pass = false;
                    if (p < pe) {
                        float t = o0 + __ldg(W + p);
                        float qq = t * t;
                        if (D >= 2) { t = o1 + __ldg(W + N + p); qq = fmaf(t, t, qq); }
                        if (D >= 3) { t = o2 + __ldg(W + 2 * N + p); qq = fmaf(t, t, qq); }
                        pass = qq <= 1.0f + 1e-4f;
                    }
                    const unsigned mask = __ballot_sync(0xffffffffu, pass);
                    if (pass) {
                        const int slot = qn + __popc(mask & ((1u << lane) - 1u));
                        q[slot] = p;
                        qd[slot] = code;
                    }
                    qn += __popc(mask);
                    if (qn >= 32) {
                        __syncwarp();
                        const int32_t pp = q[lane], cd = qd[lane];
                        const int dcs[3] = {(cd & 15) - 4, ((cd >> 4) & 15) - 4, ((cd >> 8) & 15) - 4};
                        acc = ff_add(acc, ff_mul(ff_entry_dc<E, K>(v, W, Wlo, ffl, j, pp, f, dcs), {xhi[pp], xlo[pp]}));
                        __syncwarp();
                        if (lane < qn - 32) {
                            q[lane] = q[32 + lane];
                            qd[lane] = qd[32 + lane];
                        }
                        qn -= 32;
                        __syncwarp();
                    }
                }
            }
        }
    }
    __syncwarp();
    if (lane < qn) {
        const int32_t pp = q[lane], cd = qd[lane];
        const int dcs[3] = {(cd & 15) - 4, ((cd >> 4) & 15) - 4, ((cd >> 8) & 15) - 4};
        acc = ff_add(acc, ff_mul(ff_entry_dc<E, K>(v, W, Wlo, ffl, j, pp, f, dcs), {xhi[pp], xlo[pp]}));
    }
    __syncwarp();
    return acc;
}

__device__ __forceinline__ ff lower_row_mf_warp_any(const HierView& v, const float* W, const float* Wlo,
                                                    const int32_t* cellid, const FFLevels& ffl, int j, const Frame& f,
                                                    const float* xhi, const float* xlo, int lane, int32_t* q,
                                                    int32_t* qd) {
    const int e = v.w.e, k = v.w.k;
    if (v.d == 2) {
        if (e == 4 && k == 1) return lower_row_mf_warp<2, 4, 1>(v, W, Wlo, cellid, ffl, j, f, xhi, xlo, lane, q, qd);
        if (e == 6 && k == 2) return lower_row_mf_warp<2, 6, 2>(v, W, Wlo, cellid, ffl, j, f, xhi, xlo, lane, q, qd);
        return lower_row_mf_warp<2, 0, 0>(v, W, Wlo, cellid, ffl, j, f, xhi, xlo, lane, q, qd);
    }
    if (v.d == 3) {
        if (e == 4 && k == 1) return lower_row_mf_warp<3, 4, 1>(v, W, Wlo, cellid, ffl, j, f, xhi, xlo, lane, q, qd);
        if (e == 6 && k == 2) return lower_row_mf_warp<3, 6, 2>(v, W, Wlo, cellid, ffl, j, f, xhi, xlo, lane, q, qd);
        return lower_row_mf_warp<3, 0, 0>(v, W, Wlo, cellid, ffl, j, f, xhi, xlo, lane, q, qd);
    }
    return lower_row_mf_warp<1, 0, 0>(v, W, Wlo, cellid, ffl, j, f, xhi, xlo, lane, q, qd);
}

// Double-float sum over the S lanes of a group (every lane of the warp must call it).
__device__ __forceinline__ ff ff_group_sum(ff a, int S) {
    for (int o = S >> 1; o > 0; o >>= 1) {
        const ff b = {__shfl_xor_sync(0xffffffffu, a.hi, o), __shfl_xor_sync(0xffffffffu, a.lo, o)};
        a = ff_add(a, b);
    }
    return a;
}

// Lanes per row of the matrix-free lower update from level j: about 16 candidates a lane.
inline int lower_mf_lanes(const HierView& v, int j) {
    const LevelGrid& g = v.grid[j];
    const double cells = (double)g.G[0] * g.G[1] * g.G[2];
    const int side = 2 * v.R + 1;
    const double nc = v.d == 1 ? side : (v.d == 2 ? side * side : side * side * side);
    const double cand = nc * (double)(v.off[j + 1] - v.off[j]) / (cells > 0 ? cells : 1.0);
    int S = 1;
    while (S < 32 && S * 16 < cand) S <<= 1;
    return S;
}

}  // namespace
