// Matrix-free FP32 block-diagonal mat-vec y_l = A_l x_l (Section 3: A_l is
// Phi_{delta_l}(X_l, X_l); Assumption 1: Phi_delta = delta^-d phi(|.|/delta)),
// the GB300 counterpart of the paper's kd-tree mat-vec "AMV" (Section 5.3,
// Algorithm 1).  Entries are recomputed from FP32 point offsets instead of
// being read from a CSR matrix, so the kernel is bound by the FP32/MUFU pipes
// rather than by HBM.
//
// Geometry: points are sorted by the Morton code of their cell (cell size
// delta_l / cell_split); every delta-neighbour of a point lies in the (2R+1)^d
// cells around its cell.  Each point stores its offset from its own cell's
// corner in units of delta_l (FP32, |offset| < cell/delta), so the scaled
// distance to a point in the neighbour cell displaced by (dx,dy,dz) cells is
// |(dx,dy,dz) * cell/delta + w_j - w_i|: small numbers, about 1e-7 relative
// accuracy for r = |x_i - x_j| / delta_l.
//
// Work split: one warp per target cell; TPP lanes per target point (32/TPP
// targets per pass); the TPP lanes of a target split every neighbour cell's
// candidates, so all target groups of the warp read the same TPP candidates
// at each step (broadcast loads from L1).  Evaluation is branch-free:
// s = max(1 - r, 0) makes entries beyond the support exactly zero.
#pragma once

#include "ms_internal.cuh"

__host__ __device__ __forceinline__ uint32_t compact2(uint32_t v) {  // inverse of spread2
    v &= 0x55555555u;
    v = (v | (v >> 1)) & 0x33333333u;
    v = (v | (v >> 2)) & 0x0f0f0f0fu;
    v = (v | (v >> 4)) & 0x00ff00ffu;
    v = (v | (v >> 8)) & 0x0000ffffu;
    return v;
}
__host__ __device__ __forceinline__ uint32_t compact3(uint32_t v) {  // inverse of spread3
    v &= 0x09249249u;
    v = (v | (v >> 2)) & 0x030c30c3u;
    v = (v | (v >> 4)) & 0x0300f00fu;
    v = (v | (v >> 8)) & 0x030000ffu;
    v = (v | (v >> 16)) & 0x000003ffu;
    return v;
}
__host__ __device__ __forceinline__ void demorton(int d, uint32_t code, int* c) {
    if (d == 1) { c[0] = (int)code; c[1] = c[2] = 0; return; }
    if (d == 2) { c[0] = (int)compact2(code); c[1] = (int)compact2(code >> 1); c[2] = 0; return; }
    c[0] = (int)compact3(code);
    c[1] = (int)compact3(code >> 1);
    c[2] = (int)compact3(code >> 2);
}

// FP32 view of one level's operator.
struct MFLevel {
    int G[3];
    int R;            // neighbour cell radius
    float cod;        // cell size / delta
    float dscale;     // delta^-d
    int64_t cell_off; // first global cell id of the level
    int64_t ncells;
};

struct MFView {
    int d, L;
    int64_t N;
    int E;             // Wendland exponent (phi = (1-r)^E * poly(r))
    float c[4];        // polynomial coefficients
    const float* W;    // [d][N] offsets in units of delta (sorted order)
    const int32_t* cellid;      // [N] level-local Morton cell of each sorted point
    const int32_t* cell_start;  // global cell -> first sorted point
    MFLevel lv[MS_MAXL];
};

// phi(r) = max(1-r,0)^E * (c0 + c1 r + c2 r^2 + c3 r^3); E = 4 and E = 6 (phi_{.,1}, phi_{.,2})
// are specialised, E = 0 selects the generic loop over the runtime exponent erun.
template <int E>
__device__ __forceinline__ float mf_phi(float r, const float* c, int erun) {
    const float s = fmaxf(1.0f - r, 0.0f);
    float pw, p;
    if (E == 4) {
        const float s2 = s * s;
        pw = s2 * s2;
        p = fmaf(c[1], r, c[0]);
    } else if (E == 6) {
        const float s2 = s * s;
        pw = s2 * s2 * s2;
        p = fmaf(fmaf(c[2], r, c[1]), r, c[0]);
    } else {
        pw = 1.0f;
        for (int i = 0; i < erun; ++i) pw *= s;
        p = fmaf(fmaf(fmaf(c[3], r, c[2]), r, c[1]), r, c[0]);
    }
    return pw * p;
}

// Sum over the neighbour cells of (cx,cy,cz) in level lv of phi(r_ij) * x_j for the
// target offset wi; lanes of one TPP group stride over each cell's candidates.
template <int D, int E>
__device__ __forceinline__ float mf_gather(const MFView& v, const MFLevel& g, const int* cc, const float* wi,
                                           const float* x, int sub, int TPP) {
    float acc = 0.0f;
    const int R = g.R;
    const int rz = D >= 3 ? R : 0, ry = D >= 2 ? R : 0;
    const float* Wx = v.W;
    const float* Wy = v.W + v.N;
    const float* Wz = v.W + 2 * v.N;
    for (int dz = -rz; dz <= rz; ++dz) {
        const int cz = cc[2] + dz;
        if (D >= 3 && (cz < 0 || cz >= g.G[2])) continue;
        const float oz = D >= 3 ? (float)dz * g.cod - wi[2] : 0.0f;
        for (int dy = -ry; dy <= ry; ++dy) {
            const int cy = cc[1] + dy;
            if (D >= 2 && (cy < 0 || cy >= g.G[1])) continue;
            const float oy = D >= 2 ? (float)dy * g.cod - wi[1] : 0.0f;
            for (int dx = -R; dx <= R; ++dx) {
                const int cx = cc[0] + dx;
                if (cx < 0 || cx >= g.G[0]) continue;
                const float ox = (float)dx * g.cod - wi[0];
                const int64_t gid = g.cell_off + morton(D, cx, cy, cz);
                const int32_t s = v.cell_start[gid], e = v.cell_start[gid + 1];
                // phi(r) x_j for candidate j: r = r2 / sqrt(r2) through the hardware reciprocal
                // square root (FP32 entries need no correctly rounded sqrt); r2 = 0 gives r = 0
                auto term = [&](float wx, float wy, float wz, float xj) {
                    const float ex = wx + ox;
                    float r2 = ex * ex;
                    if (D >= 2) {
                        const float ey = wy + oy;
                        r2 = fmaf(ey, ey, r2);
                    }
                    if (D >= 3) {
                        const float ez = wz + oz;
                        r2 = fmaf(ez, ez, r2);
                    }
                    const float r = r2 * rsqrtf(fmaxf(r2, 1e-30f));
                    acc = fmaf(mf_phi<E>(r, v.c, v.E), xj, acc);
                };
                // four candidates' loads issued before their arithmetic (the loop is latency-bound
                // otherwise); the terms are still added in candidate order
                int32_t j = s + sub;
                for (; j + 3 * TPP < e; j += 4 * TPP) {
                    float wx[4], wy[4] = {0.f, 0.f, 0.f, 0.f}, wz[4] = {0.f, 0.f, 0.f, 0.f}, xj[4];
#pragma unroll
                    for (int u = 0; u < 4; ++u) {
                        const int32_t jj = j + u * TPP;
                        wx[u] = Wx[jj];
                        if (D >= 2) wy[u] = Wy[jj];
                        if (D >= 3) wz[u] = Wz[jj];
                        xj[u] = x[jj];
                    }
#pragma unroll
                    for (int u = 0; u < 4; ++u) term(wx[u], wy[u], wz[u], xj[u]);
                }
                for (; j < e; j += TPP) term(Wx[j], D >= 2 ? Wy[j] : 0.f, D >= 3 ? Wz[j] : 0.f, x[j]);
            }
        }
    }
    return acc;
}

// y_i = delta^-d sum_j phi(r_ij) x_j for every point i of the level-local cells
// [c0, c1) of level l: one warp per cell (warp w of nw handles cells c0+w, c0+w+nw, ...).
// emit(row, value) is called once per row by the group's leading lane.
template <int D, int E, typename Emit>
__device__ __forceinline__ void mf_cells(const MFView& v, int l, int64_t c0, int64_t c1, int w, int nw, int TPP,
                                         const float* x, Emit emit) {
    const MFLevel& g = v.lv[l];
    const int lane = threadIdx.x & 31;
    const int sub = lane & (TPP - 1);
    const int per = 32 / TPP;
    for (int64_t cell = c0 + w; cell < c1; cell += nw) {
        const int32_t cs = v.cell_start[g.cell_off + cell], ce = v.cell_start[g.cell_off + cell + 1];
        if (cs == ce) continue;
        int cc[3];
        demorton(D, (uint32_t)cell, cc);
        for (int32_t t0 = cs; t0 < ce; t0 += per) {
            const int32_t t = t0 + lane / TPP;
            const bool ok = t < ce;
            float wi[3] = {0.f, 0.f, 0.f};
            if (ok) {
                wi[0] = v.W[t];
                if (D >= 2) wi[1] = v.W[v.N + t];
                if (D >= 3) wi[2] = v.W[2 * v.N + t];
            }
            float acc = ok ? mf_gather<D, E>(v, g, cc, wi, x, sub, TPP) : 0.0f;
            for (int o = TPP >> 1; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
            if (ok && sub == 0) emit((int64_t)t, acc * g.dscale);
        }
    }
}

// ---------------------------------------------------------------- staged form (one CTA per cell)
//
// y_i = delta^-d sum_j phi(r_ij) x_j for the points i of one cell, with the candidates j of the
// (2R+1)^d neighbour cells staged in shared memory: each as a float4 (its offset from the target
// cell's corner in units of delta, W_j + (c_j - c) cod per axis, and x_j), written once by the
// whole CTA and then read by every target as a broadcast 128-bit load, so the inner loop has no
// index arithmetic or global loads.  TPP threads share a target (the largest power of 2 with
// TPP n_targets <= blockDim, at most 32) and stride over the staged candidates; the partial sums
// are combined by shuffles in a fixed order.  A neighbourhood larger than the stage is processed
// in rounds (each thread keeps its target's sum).  Returns false, without writing, for a cell of
// more than blockDim points (the caller takes the warp form for it).
constexpr int kMfStage = 1024;  // staged candidates (16 KB)

template <int D, int E, typename Emit>
__device__ __forceinline__ bool mf_cell_staged(const MFView& v, int l, int64_t cell, const float* x, float4* stage,
                                               Emit emit) {
    const MFLevel& g = v.lv[l];
    const int tid = threadIdx.x, nthr = blockDim.x;
    const int32_t ts = v.cell_start[g.cell_off + cell], te = v.cell_start[g.cell_off + cell + 1];
    const int nt = te - ts;
    if (nt == 0) return true;
    if (nt > nthr) return false;
    int tpp = 1;
    while (tpp < 32 && 2 * tpp * nt <= nthr) tpp *= 2;
    const int sub = tid & (tpp - 1);
    const int32_t ti = ts + tid / tpp;
    const bool ok = tid / tpp < nt;
    float wi[3] = {0.f, 0.f, 0.f};
    if (ok)
        for (int a = 0; a < D; ++a) wi[a] = v.W[a * v.N + ti];
    int cc[3];
    demorton(D, (uint32_t)cell, cc);
    const int R = g.R;
    const int rz = D >= 3 ? R : 0, ry = D >= 2 ? R : 0;
    float acc = 0.f;
    int n = 0;  // staged so far (uniform in the CTA)
    auto consume = [&]() {
        __syncthreads();
        if (ok) {
#pragma unroll 4
            for (int k = sub; k < n; k += tpp) {
                const float4 c = stage[k];
                const float ex = c.x - wi[0];
                float r2 = ex * ex;
                if (D >= 2) {
                    const float ey = c.y - wi[1];
                    r2 = fmaf(ey, ey, r2);
                }
                if (D >= 3) {
                    const float ez = c.z - wi[2];
                    r2 = fmaf(ez, ez, r2);
                }
                const float r = r2 * rsqrtf(fmaxf(r2, 1e-30f));
                acc = fmaf(mf_phi<E>(r, v.c, v.E), c.w, acc);
            }
        }
        __syncthreads();
        n = 0;
    };
    for (int dz = -rz; dz <= rz; ++dz) {
        const int cz = cc[2] + dz;
        if (D >= 3 && (cz < 0 || cz >= g.G[2])) continue;
        for (int dy = -ry; dy <= ry; ++dy) {
            const int cy = cc[1] + dy;
            if (D >= 2 && (cy < 0 || cy >= g.G[1])) continue;
            for (int dx = -R; dx <= R; ++dx) {
                const int cx = cc[0] + dx;
                if (cx < 0 || cx >= g.G[0]) continue;
                const int64_t gid = g.cell_off + morton(D, cx, cy, cz);
                const int32_t s = v.cell_start[gid], e = v.cell_start[gid + 1];
                const float ox = (float)dx * g.cod, oy = (float)dy * g.cod, oz = (float)dz * g.cod;
                for (int32_t j0 = s; j0 < e;) {
                    if (n == kMfStage) consume();
                    const int take = min(e - j0, kMfStage - n);
                    for (int k = tid; k < take; k += nthr) {
                        const int32_t j = j0 + k;
                        stage[n + k] = make_float4(v.W[j] + ox, D >= 2 ? v.W[v.N + j] + oy : 0.f,
                                                   D >= 3 ? v.W[2 * v.N + j] + oz : 0.f, x[j]);
                    }
                    n += take;
                    j0 += take;
                }
            }
        }
    }
    if (n > 0) consume();
    for (int o = tpp >> 1; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if (ok && sub == 0) emit((int64_t)ti, acc * g.dscale);
    return true;
}

template <typename Emit>
__device__ __forceinline__ bool mf_cell_staged_any(const MFView& v, int l, int64_t cell, const float* x,
                                                   float4* stage, Emit emit) {
    if (v.d == 2) {
        if (v.E == 4) return mf_cell_staged<2, 4>(v, l, cell, x, stage, emit);
        if (v.E == 6) return mf_cell_staged<2, 6>(v, l, cell, x, stage, emit);
        return mf_cell_staged<2, 0>(v, l, cell, x, stage, emit);
    }
    if (v.d == 3) {
        if (v.E == 4) return mf_cell_staged<3, 4>(v, l, cell, x, stage, emit);
        if (v.E == 6) return mf_cell_staged<3, 6>(v, l, cell, x, stage, emit);
        return mf_cell_staged<3, 0>(v, l, cell, x, stage, emit);
    }
    return mf_cell_staged<1, 0>(v, l, cell, x, stage, emit);
}

// Dispatch on (d, Wendland exponent) to the specialised loop.
template <typename Emit>
__device__ __forceinline__ void mf_cells_any(const MFView& v, int l, int64_t c0, int64_t c1, int w, int nw, int TPP,
                                             const float* x, Emit emit) {
    if (v.d == 2) {
        if (v.E == 4) mf_cells<2, 4>(v, l, c0, c1, w, nw, TPP, x, emit);
        else if (v.E == 6) mf_cells<2, 6>(v, l, c0, c1, w, nw, TPP, x, emit);
        else mf_cells<2, 0>(v, l, c0, c1, w, nw, TPP, x, emit);
    } else if (v.d == 3) {
        if (v.E == 4) mf_cells<3, 4>(v, l, c0, c1, w, nw, TPP, x, emit);
        else if (v.E == 6) mf_cells<3, 6>(v, l, c0, c1, w, nw, TPP, x, emit);
        else mf_cells<3, 0>(v, l, c0, c1, w, nw, TPP, x, emit);
    } else {
        mf_cells<1, 0>(v, l, c0, c1, w, nw, TPP, x, emit);
    }
}
