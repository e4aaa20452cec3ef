// Evaluation of the multiscale approximant at query points (eq. fapproximation):
//   f_L(q) = sum_l sum_n alpha_n^(l) Phi_{delta_l}(q - x_n^(l)),
// one thread per query, every level's neighbours found through that level's
// cell grid, FP64 distances, kernel values and accumulation.  An FP32 test on the
// points' cell-relative offsets rejects the clear misses (about 2/3 of the
// candidates) before any FP64 work.
#include <algorithm>

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
                                                const double* y, F&& visit) {
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
                for (int32_t p = s; p < e; ++p) {
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

__global__ void k_eval(HierView v, const float* __restrict__ W, const double* __restrict__ alpha,
                       const double* __restrict__ Q, int64_t nq, double* __restrict__ out, int nrhs, int col) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= nq) return;
    double y[3] = {0, 0, 0};
    for (int a = 0; a < v.d; ++a) y[a] = Q[i * v.d + a];
    double s = 0.0;
    for (int l = 0; l < v.L; ++l) {
        const double inv = 1.0 / v.delta[l], sc = v.dscale[l];
        double sl = 0.0;
        eval_neighbours(v, W, l, y, [&](int32_t p, double r2) {
            sl = fma(wendland_eval<double>(v.w, sqrt(r2) * inv), alpha[p], sl);
        });
        s = fma(sc, sl, s);
    }
    out[i * nrhs + col] = s;
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
    for (int c = 0; c < nrhs; ++c) {
        ms_gather_sorted(alpha_dev, h->tmp64, h->perm, h->N, nrhs, c, st);
        const unsigned blocks = (unsigned)std::max<int64_t>(1, (nq + 127) / 128);
        k_eval<<<blocks, 128, 0, st>>>(h->view, h->W, h->tmp64, q_dev, nq, out_dev, nrhs, c); ms_count_launch();
        MS_CUDA(cudaGetLastError());
    }
    return MS_OK;
}
