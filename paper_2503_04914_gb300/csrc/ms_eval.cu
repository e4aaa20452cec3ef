// Evaluation of the multiscale approximant at query points (eq. fapproximation):
//   f_L(q) = sum_l sum_n alpha_n^(l) Phi_{delta_l}(q - x_n^(l)),
// one warp per query (the lanes over each neighbour cell's points, per-lane FP64 sums
// combined by shuffles in a fixed order), every level's neighbours found through that level's
// cell grid.  An FP32 test on the points' cell-relative
// offsets rejects the clear misses (about 2/3 of the candidates) first; the
// kernel values are FP64 (FP64 builds) or double-float (MIXED builds).
#include <algorithm>

#include "ms_ff.cuh"
#include "ms_internal.cuh"

namespace {

// visit(p, r2) for every sorted point p of level j with |x_p - y|^2 < delta_j^2.  Candidates:
// the (2R+1)^d cells around y's cell.  W holds each point's offset from its own cell's corner
// in units of delta (FP32), so the scaled offset to a candidate in the cell displaced by D
// cells is D cod + W_p - fr (fr: y's offset in its cell): candidates with a squared FP32
// distance above 1 + 1e-4 are dropped (FP32 error is far below that band), the rest are
// decided by the FP64 distance.
template <typename F>
__device__ __forceinline__ void eval_neighbours(const HierView& v, const float* __restrict__ W, int j,
                                                const double* y, int lane, F&& visit) {
    const LevelGrid& g = v.grid[j];
    const double d2 = v.delta[j] * v.delta[j];
    int c[3] = {0, 0, 0};
    float fr[3] = {0.f, 0.f, 0.f};
    for (int a = 0; a < v.d; ++a) {
        c[a] = cell_coord(g, a, y[a]);
        fr[a] = (float)((y[a] - (g.lo[a] + (double)c[a] * g.cell)) * v.inv_delta[j]);
    }
    const int R = v.R;
    const int rz = v.d >= 3 ? R : 0, ry = v.d >= 2 ? R : 0;
    for (int dz = -rz; dz <= rz; ++dz) {
        const int cz = c[2] + dz;
        if (cz < 0 || cz >= g.G[2]) continue;
        const float oz = (float)dz * g.cod - fr[2];
        for (int dy = -ry; dy <= ry; ++dy) {
            const int cy = c[1] + dy;
            if (cy < 0 || cy >= g.G[1]) continue;
            const float oy = (float)dy * g.cod - fr[1];
            for (int dx = -R; dx <= R; ++dx) {
                const int cx = c[0] + dx;
                if (cx < 0 || cx >= g.G[0]) continue;
                const float ox = (float)dx * g.cod - fr[0];
                const int64_t gid = g.cell_off + morton(v.d, cx, cy, cz);
                const int32_t s = v.cell_start[gid], e = v.cell_start[gid + 1];
                for (int32_t p = s + lane; p < e; p += 32) {
                    float t = ox + __ldg(W + p);
                    float qq = t * t;
                    if (v.d >= 2) { t = oy + __ldg(W + v.N + p); qq = fmaf(t, t, qq); }
                    if (v.d >= 3) { t = oz + __ldg(W + 2 * v.N + p); qq = fmaf(t, t, qq); }
                    if (qq > 1.0f + 1e-4f) continue;
                    double r2 = 0.0;
                    for (int a = 0; a < v.d; ++a) {
                        const double u = v.X[a * v.N + p] - y[a];
                        r2 = fma(u, u, r2);
                    }
                    if (r2 < d2) visit(p, r2);
                }
            }
        }
    }
}

// phi(r) for the Wendland closed form w in double-float, 0 for r >= 1 (as in the CSR fill).
__device__ __forceinline__ ff eval_ff_wendland(const WendlandPoly& w, const ff* c, ff r) {
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
    ff p = c[w.k];
    for (int i = w.k - 1; i >= 0; --i) p = ff_add(ff_mul(p, r), c[i]);
    return ff_mul(pw, p);
}

// Per-level cell size / delta and the Wendland coefficients as double-floats (converted
// once on the host).
struct EvalLevels {
    ff cod[MS_MAXL];
    ff c[4];
};

// FF (MIXED builds): the kernel values in double-float arithmetic from the points'
// cell-relative offsets W + Wlo and the query's own offset in its cell (about 48 bits,
// ~1e-14 relative; the sums stay FP64).  Otherwise FP64 distances and values.
template <bool FF>
__global__ void k_eval(const __grid_constant__ HierView v, const float* __restrict__ W, const float* __restrict__ Wlo,
                       const __grid_constant__ EvalLevels el, const double* __restrict__ alpha,
                       const double* __restrict__ Q, int64_t nq, double* __restrict__ out, int nrhs, int col) {
    __shared__ int32_t eq[8][64], eqd[8][64];  // per-warp queues (blocks of 256 threads)
    const int64_t i = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (i >= nq) return;  // warp-uniform
    double y[3] = {0, 0, 0};
    for (int a = 0; a < v.d; ++a) y[a] = Q[i * v.d + a];
    double s = 0.0;
    for (int l = 0; l < v.L; ++l) {
        const double sc = v.dscale[l];
        double sl = 0.0;
        if (!FF) {
            const double inv = 1.0 / v.delta[l];
            eval_neighbours(v, W, l, y, lane, [&](int32_t p, double r2) {
                sl = fma(wendland_eval<double>(v.w, sqrt(r2) * inv), alpha[p], sl);
            });
        } else {
            const LevelGrid& g = v.grid[l];
            int c[3] = {0, 0, 0};
            float fr[3] = {0.f, 0.f, 0.f}, frlo[3] = {0.f, 0.f, 0.f};
            for (int a = 0; a < v.d; ++a) {
                c[a] = cell_coord(g, a, y[a]);
                const double t = (y[a] - (g.lo[a] + (double)c[a] * g.cell)) * v.inv_delta[l];
                fr[a] = (float)t;
                frlo[a] = (float)(t - (double)fr[a]);
            }
            // the candidates passing the FP32 test are queued (point, cell displacement) and their
            // double-float values computed 32 at a time, so that arithmetic runs on full warps
            int32_t* q = eq[threadIdx.x >> 5];
            int32_t* qd = eqd[threadIdx.x >> 5];
            int qn = 0;
            auto entry = [&](int32_t pp, int32_t cd) {
                const int dcs[3] = {(cd & 15) - 4, ((cd >> 4) & 15) - 4, ((cd >> 8) & 15) - 4};
                ff r2 = {0.0f, 0.0f};
                for (int a = 0; a < v.d; ++a) {
                    const ff o = ff_add(ff_mul(el.cod[l], {(float)dcs[a], 0.0f}), ff_neg({fr[a], frlo[a]}));
                    r2 = ff_add(r2, ff_sqr(ff_add(o, {__ldg(W + a * v.N + pp), __ldg(Wlo + a * v.N + pp)})));
                }
                const ff phi = eval_ff_wendland(v.w, el.c, ff_sqrt(r2));
                if (phi.hi != 0.0f) sl = fma(ff_to_double(phi), alpha[pp], sl);
            };
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
                        const int dc[3] = {dx, dy, dz};
                        const int32_t code = (dx + 4) | ((dy + 4) << 4) | ((dz + 4) << 8);
                        float of[3];
                        for (int a = 0; a < 3; ++a)
                            of[a] = ff_add(ff_mul(el.cod[l], {(float)dc[a], 0.0f}), ff_neg({fr[a], frlo[a]})).hi;
                        const int64_t gid = g.cell_off + morton(v.d, cx, cy, cz);
                        const int32_t ps = v.cell_start[gid], pe = v.cell_start[gid + 1];
                        for (int32_t p0 = ps; p0 < pe; p0 += 32) {
                            const int32_t p = p0 + lane;
                            bool pass = false;
                            if (p < pe) {  // FP32 prefilter
                                float t = of[0] + __ldg(W + p);
                                float qq = t * t;
                                if (v.d >= 2) { t = of[1] + __ldg(W + v.N + p); qq = fmaf(t, t, qq); }
                                if (v.d >= 3) { t = of[2] + __ldg(W + 2 * v.N + p); qq = fmaf(t, t, qq); }
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
                                entry(q[lane], qd[lane]);
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
            if (lane < qn) entry(q[lane], qd[lane]);
            __syncwarp();
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) sl += __shfl_xor_sync(0xffffffffu, sl, o);
        s = fma(sc, sl, s);
    }
    if (lane == 0) out[i * nrhs + col] = s;
}

}  // namespace

ms_status ms_evaluate_impl(ms_hierarchy* h, const double* alpha_dev, int nrhs, const double* q_dev, int64_t nq,
                           double* out_dev, cudaStream_t st) {
    if (nq == 0) return MS_OK;
    if (!h->tmp64) {
        void* p = nullptr;
        MS_TRY(ms_alloc(h, &p, sizeof(double) * h->N));
        h->tmp64 = (double*)p;
    }
    EvalLevels el{};
    for (int l = 0; l < h->L; ++l) el.cod[l] = ff_from_double(h->view.grid[l].cell / h->view.delta[l]);
    for (int i = 0; i < 4; ++i) el.c[i] = ff_from_double(h->view.w.c[i]);
    for (int c = 0; c < nrhs; ++c) {
        ms_gather_sorted(alpha_dev, h->tmp64, h->perm, h->N, nrhs, c, st);
        const unsigned blocks = (unsigned)std::max<int64_t>(1, (nq * 32 + 255) / 256);  // a warp per query
        if (h->Wlo)
            k_eval<true><<<blocks, 256, 0, st>>>(h->view, h->W, h->Wlo, el, h->tmp64, q_dev, nq, out_dev, nrhs, c);
        else
            k_eval<false><<<blocks, 256, 0, st>>>(h->view, h->W, nullptr, el, h->tmp64, q_dev, nq, out_dev, nrhs, c);
        ms_count_launch();
        MS_CUDA(cudaGetLastError());
    }
    return MS_OK;
}
