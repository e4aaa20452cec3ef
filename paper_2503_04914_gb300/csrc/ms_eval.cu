// Evaluation of the multiscale approximant at query points (eq. fapproximation):
//   f_L(q) = sum_l sum_n alpha_n^(l) Phi_{delta_l}(q - x_n^(l)),
// one thread per query, every level's neighbours found through that level's
// cell grid, FP64 distances, kernel values and accumulation.
#include <algorithm>

#include "ms_internal.cuh"

namespace {

__global__ void k_eval(HierView v, const double* __restrict__ alpha, const double* __restrict__ Q, int64_t nq,
                       double* __restrict__ out, int nrhs, int col) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= nq) return;
    double y[3] = {0, 0, 0};
    for (int a = 0; a < v.d; ++a) y[a] = Q[i * v.d + a];
    double s = 0.0;
    for (int l = 0; l < v.L; ++l) {
        const double inv = 1.0 / v.delta[l], sc = v.dscale[l];
        double sl = 0.0;
        for_each_neighbour(v, l, y, [&](int32_t p, double r2) {
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
        k_eval<<<blocks, 128, 0, st>>>(h->view, h->tmp64, q_dev, nq, out_dev, nrhs, c); ms_count_launch();
        MS_CUDA(cudaGetLastError());
    }
    return MS_OK;
}
