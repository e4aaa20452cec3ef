// Learned factorised sparse-approximate-inverse (FSAI) preconditioner of the
// per-level CG solves (Theorem 8).  The paper has no preconditioner; this is
// the library's extension, justified by the exponential decay of A_l^{-1}
// (Lemma 5) and by the scaling of eq. kernelscaling.
//
//   pattern   P_i = {i} + the (up to) 16 nearest same-level points j within delta
//             with input index j < i (nearest first, ties by input index);
//   exact row g_i = A_P^{-1} e_1 / sqrt(e_1^T A_P^{-1} e_1)  (Kolotilina-Yeremin FSAI);
//             M = G^T G is symmetric positive definite for any G with a positive
//             diagonal, so a learned G can never make the preconditioned CG break down;
//   scale-free ghat_i = delta^{-d/2} g_i depends only on the delta-scaled offsets of
//             the pattern (A_P = delta^-d K(offsets/delta)), so a network trained on
//             coarse levels applies to every level;
//   network   32 -> 64 -> 64 -> 17 m (d = 2; input 16 d), ReLU, BF16-valued weights with
//             FP32 accumulation at inference: m candidate rows (standardised per entry);
//             the row is the FSAI-optimal combination of the candidates (the minimiser
//             of g^T A_P g with g_self = 1 within their span, normalised), solved per row;
//             trained with Adam on FP32 master weights (forward/backward on the
//             BF16-rounded copies) to close the gap log (A_P^-1)_11 - log q between the
//             exact row and the combination, on the exact rows of chosen levels.
#include <algorithm>
#include <climits>
#include <cmath>
#include <cstring>
#include <vector>

#include <cuda_bf16.h>

#include "ms_ff.cuh"
#include "ms_internal.cuh"
#include "ms_matfree.cuh"
#include "ms_scan.cuh"
#include "ms_tc.cuh"

namespace {

inline unsigned nblk(int64_t n, int bs) { return (unsigned)std::max<int64_t>(1, (n + bs - 1) / bs); }

__device__ __forceinline__ double dist2_rn(const HierView& v, int64_t i, int64_t j) {
    double s = 0.0;
    for (int a = 0; a < v.d; ++a) {
        const double t = __dsub_rn(v.X[a * v.N + i], v.X[a * v.N + j]);
        s = __dadd_rn(s, __dmul_rn(t, t));
    }
    return s;
}

__device__ __forceinline__ double dist_rn(const HierView& v, int64_t i, int64_t j) { return sqrt(dist2_rn(v, i, j)); }

// (sqrt(d2a), pa) < (sqrt(d2b), pb) lexicographically, where the square roots are the
// correctly rounded FP64 ones.  Non-negative doubles order like their bit patterns, and
// squared distances more than 64 units in the last place apart order their roots the
// same way (sqrt halves relative gaps), so the decision is an integer compare and the
// (FP64-pipe) roots are taken only for near-ties.
__device__ __forceinline__ bool key_less(double d2a, int32_t pa, double d2b, int32_t pb) {
    const long long gap = __double_as_longlong(d2b) - __double_as_longlong(d2a);
    if (gap > 64) return true;
    if (gap < -64) return false;
    const double da = sqrt(d2a), db = sqrt(d2b);
    return da < db || (da == db && pa < pb);
}

// ---------------------------------------------------------------- pattern

// The (up to) 16 nearest points c != s of sorted row s's level with input index below
// `bound` and |x_c - x_s| < delta (candidates: A's row s), nearest first, ties by input
// index.  bound = perm[s] gives the pattern of s; a larger bound an extra training patch.
__device__ void nearest_below(const HierView& v, const int64_t* Arp, const int32_t* Acol, const int32_t* perm,
                              int64_t s, int64_t bound, int32_t* out) {
    // sorted list keyed by (distance, input index), held in registers (every index below is a
    // compile-time constant); empty slots hold the key (+inf, INT_MAX) and column -1.  bd holds
    // squared distances, compared through key_less as their correctly rounded roots.
    double bd[kPcK];
    int32_t bp[kPcK], bc[kPcK];
#pragma unroll
    for (int i = 0; i < kPcK; ++i) {
        bd[i] = __longlong_as_double(0x7FF0000000000000ll);
        bp[i] = INT_MAX;
        bc[i] = -1;
    }
    for (int64_t k = Arp[s]; k < Arp[s + 1]; ++k) {
        const int32_t c = Acol[k];
        const int32_t pc = perm[c];
        if (pc >= bound || c == s) continue;
        const double d = dist2_rn(v, c, s);
        if (!key_less(d, pc, bd[kPcK - 1], bp[kPcK - 1])) continue;  // not among the 16 nearest so far
        bool lt[kPcK];  // the new key goes before slot i (false ... false, true ... true)
#pragma unroll
        for (int i = 0; i < kPcK; ++i) lt[i] = key_less(d, pc, bd[i], bp[i]);
        // slot i takes slot i-1's entry if the new key goes before that, else the new key if it
        // goes before slot i's entry (the insertion point)
#pragma unroll
        for (int i = kPcK - 1; i > 0; --i) {
            if (lt[i - 1]) {
                bd[i] = bd[i - 1];
                bp[i] = bp[i - 1];
                bc[i] = bc[i - 1];
            } else if (lt[i]) {
                bd[i] = d;
                bp[i] = pc;
                bc[i] = c;
            }
        }
        if (lt[0]) {
            bd[0] = d;
            bp[0] = pc;
            bc[0] = c;
        }
    }
#pragma unroll
    for (int i = 0; i < kPcK; ++i) out[i] = bc[i];
}

constexpr int kPL = 8;        // candidates a lane holds (rows of up to 32 kPL entries)
constexpr int kPcCont = 64;   // contenders a warp ranks exactly
constexpr int kPatW = 4;      // warps per block of the pattern kernels

// nearest_below by a whole warp (every lane calls it; lanes write `out`).  The candidates
// are first keyed by an FP32 squared distance in units of delta^2, from the level's cell
// ids and in-cell offsets W (|error| < 4e-6 for |x_c - x_s| < delta): with k16 the 16th
// smallest FP32 key, every point of the exact pattern has a key <= k16 + 1e-5 (its exact
// squared distance is at most the 16th smallest one, and k16 is at least that less the
// error), so only those contenders are ranked, in the order of nearest_below: by their FP32 keys
// where two differ by more than 1e-5, by key_less on the exact FP64 squared distances otherwise.
// A row of more than 32 kPL entries, or with more than kPcCont contenders (ties), is left to
// nearest_below on lane 0.
__device__ void nearest_below_warp(const HierView& v, const float* __restrict__ W,
                                   const int32_t* __restrict__ cellid, const int64_t* Arp, const int32_t* Acol,
                                   const int32_t* perm, int64_t s, int64_t bound, int32_t* out, int lane,
                                   int32_t* cq, float* kq, int* hist) {
    const int64_t b = Arp[s];
    const int n = (int)(Arp[s + 1] - b);
    constexpr uint32_t kNone = 0xFFFFFFFFu;  // not a candidate (above every float key)
    bool serial = n > 32 * kPL;
    uint32_t key[kPL];
    int32_t col[kPL], pcol[kPL];
    if (!serial) {
        const int l = level_of_row(v.off, v.L, s);
        const float cod = v.grid[l].cod;
        int cs[3];
        demorton(v.d, (uint32_t)__ldg(cellid + s), cs);
        float ws[3] = {0.f, 0.f, 0.f};
        for (int a = 0; a < v.d; ++a) ws[a] = __ldg(W + a * v.N + s);
#pragma unroll
        for (int i = 0; i < kPL; ++i) {
            key[i] = kNone;
            col[i] = -1;
            pcol[i] = INT_MAX;
            const int k = lane + 32 * i;
            if (k < n) {
                const int32_t c = __ldg(Acol + b + k);
                const int32_t pc = __ldg(perm + c);
                if (pc < bound && c != s) {
                    int cc[3];
                    demorton(v.d, (uint32_t)__ldg(cellid + c), cc);
                    float q = 0.f;
                    for (int a = 0; a < v.d; ++a) {
                        const float t = __fadd_rn(__fmul_rn(small_int_to_float(cc[a] - cs[a]), cod),
                                                  __fsub_rn(__ldg(W + a * v.N + c), ws[a]));
                        q = fmaf(t, t, q);
                    }
                    key[i] = __float_as_uint(q);
                    col[i] = c;
                    pcol[i] = pc;
                }
            }
        }
        // a bound on k16 from a histogram of the keys over 256 bins of the float's exponent and
        // top three fraction bits (monotone in the key; a bin spans 1/8 of an octave): B = the
        // first bin at which the count reaches 16, t = B's upper edge + 1e-5 >= k16 + 1e-5
        for (int i = lane; i < 256; i += 32) hist[i] = 0;
        __syncwarp();
#pragma unroll
        for (int i = 0; i < kPL; ++i)
            if (key[i] != kNone) atomicAdd(&hist[min(max((int)(key[i] >> 20) - (103 << 3), 0), 255)], 1);
        __syncwarp();
        int cnt8[8], own = 0;
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            cnt8[j] = hist[lane * 8 + j];
            own += cnt8[j];
        }
        int incl = own;  // inclusive scan of the lanes' bin counts
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += y;
        }
        const unsigned reach = __ballot_sync(0xffffffffu, incl >= kPcK);
        float t = INFINITY;  // fewer than 16 candidates: every candidate contends
        if (reach) {
            const int src = __ffs(reach) - 1;
            int bin = 0;
            if (lane == src) {
                int c = incl - own;
                bin = lane * 8 + 7;
#pragma unroll
                for (int j = 0; j < 8; ++j) {
                    c += cnt8[j];
                    if (c >= kPcK) { bin = lane * 8 + j; break; }
                }
            }
            bin = __shfl_sync(0xffffffffu, bin, src);
            // upper edge of the bin: the smallest float of the next bin
            const float edge = bin >= 255 ? INFINITY : __uint_as_float((uint32_t)(bin + 1 + (103 << 3)) << 20);
            t = __fadd_ru(edge, 1e-5f);
        }
        // contenders to the warp's queue
        int nc = 0;
#pragma unroll
        for (int i = 0; i < kPL; ++i) {
            const bool pass = key[i] != kNone && __uint_as_float(key[i]) <= t;
            const unsigned mask = __ballot_sync(0xffffffffu, pass);
            const int pos = nc + __popc(mask & ((1u << lane) - 1u));
            if (pass && pos < kPcCont) {
                cq[2 * pos] = col[i];
                cq[2 * pos + 1] = pcol[i];
                kq[pos] = __uint_as_float(key[i]);
            }
            nc += __popc(mask);
        }
        serial = nc > kPcCont;
        if (!serial) {
            __syncwarp();
            // rank of each contender: by the FP32 keys where they are more than 1e-5 apart (then
            // the exact keys order the same way: each FP32 key is within 4e-6 of its exact value),
            // else by key_less on the exact FP64 squared distances (near ties only)
            for (int j = lane; j < nc; j += 32) {
                const float qj = kq[j];
                const int32_t cj = cq[2 * j], pj = cq[2 * j + 1];
                double dj = -1.0;
                int rank = 0;
                for (int o = 0; o < nc; ++o) {
                    if (o == j) continue;
                    const float qo = kq[o];
                    if (fabsf(qo - qj) > 1e-5f) {
                        rank += qo < qj ? 1 : 0;
                    } else {
                        if (dj < 0.0) dj = dist2_rn(v, cj, s);
                        rank += key_less(dist2_rn(v, cq[2 * o], s), cq[2 * o + 1], dj, pj) ? 1 : 0;
                    }
                }
                if (rank < kPcK) out[rank] = cj;
            }
            if (lane < kPcK && lane >= nc) out[lane] = -1;
        }
    }
    if (serial && lane == 0) nearest_below(v, Arp, Acol, perm, s, bound, out);
    __syncwarp();
}

__global__ void __launch_bounds__(kPatW * 32, 5) k_pc_pattern(HierView v, const float* W, const int32_t* cellid,
                                                          const int64_t* Arp, const int32_t* Acol,
                                                          const int32_t* perm, int32_t* nbr) {
    __shared__ int32_t cq[kPatW][2 * kPcCont];
    __shared__ float kq[kPatW][kPcCont];
    __shared__ int hist[kPatW][256];
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t s = blockIdx.x * (int64_t)kPatW + w;
    if (s >= v.N) return;  // warp-uniform
    nearest_below_warp(v, W, cellid, Arp, Acol, perm, s, __ldg(perm + s), nbr + s * kPcK, lane, cq[w], kq[w], hist[w]);
}

// Neighbours of training patch i: centre rows[i], input-index bound bounds[i]; out [n][16].
__global__ void __launch_bounds__(kPatW * 32, 5) k_pc_patches(HierView v, const float* W, const int32_t* cellid,
                                                          const int64_t* Arp, const int32_t* Acol,
                                                          const int32_t* perm, const int64_t* rows,
                                                          const int64_t* bounds, int64_t n, int32_t* out) {
    __shared__ int32_t cq[kPatW][2 * kPcCont];
    __shared__ float kq[kPatW][kPcCont];
    __shared__ int hist[kPatW][256];
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t i = blockIdx.x * (int64_t)kPatW + w;
    if (i >= n) return;  // warp-uniform
    nearest_below_warp(v, W, cellid, Arp, Acol, perm, rows[i], bounds[i], out + i * kPcK, lane, cq[w], kq[w], hist[w]);
}

// ---------------------------------------------------------------- exact rows (FP64)

// Scale-free FSAI row of the patch centred on sorted row s with neighbours nb[0..15]
// (self first, zeros past the patch): K = phi(|x_a - x_b| / delta) on the patch, K z = e_1
// by Cholesky, ghat = z / sqrt(z_0).
__device__ void pc_exact_row(const HierView& v, const int32_t* nb, int64_t s, double* ghat) {
    const int l = level_of_row(v.off, v.L, s);
    const double inv = 1.0 / v.delta[l];
    int64_t P[kPcOut];
    int m = 1;
    P[0] = s;
    for (int i = 0; i < kPcK; ++i) {
        const int32_t c = nb[i];
        if (c >= 0) P[m++] = c;
    }
    double L[kPcOut * kPcOut];
    for (int a = 0; a < m; ++a)
        for (int b = 0; b <= a; ++b) L[a * kPcOut + b] = wendland_eval<double>(v.w, dist_rn(v, P[a], P[b]) * inv);
    bool ok = true;
    for (int j = 0; j < m && ok; ++j) {
        double dsum = L[j * kPcOut + j];
        for (int k = 0; k < j; ++k) dsum -= L[j * kPcOut + k] * L[j * kPcOut + k];
        if (!(dsum > 0.0)) { ok = false; break; }
        const double ljj = sqrt(dsum);
        L[j * kPcOut + j] = ljj;
        for (int i = j + 1; i < m; ++i) {
            double t = L[i * kPcOut + j];
            for (int k = 0; k < j; ++k) t -= L[i * kPcOut + k] * L[j * kPcOut + k];
            L[i * kPcOut + j] = t / ljj;
        }
    }
    for (int a = 0; a < kPcOut; ++a) ghat[a] = 0.0;
    if (!ok) {  // numerically singular patch: keep the diagonal scaling only
        ghat[0] = 1.0 / sqrt(wendland_eval<double>(v.w, 0.0));
        return;
    }
    double y[kPcOut], z[kPcOut];
    for (int i = 0; i < m; ++i) {  // L y = e_1
        double t = (i == 0) ? 1.0 : 0.0;
        for (int k = 0; k < i; ++k) t -= L[i * kPcOut + k] * y[k];
        y[i] = t / L[i * kPcOut + i];
    }
    for (int i = m - 1; i >= 0; --i) {  // L^T z = y
        double t = y[i];
        for (int k = i + 1; k < m; ++k) t -= L[k * kPcOut + i] * z[k];
        z[i] = t / L[i * kPcOut + i];
    }
    const double sc = 1.0 / sqrt(z[0]);
    for (int a = 0; a < m; ++a) ghat[a] = z[a] * sc;
}

// Patch i -> ghat[i][17]; optional G values.  rows == nullptr: patch i is the pattern of
// sorted row i (nbr [N][16]); else it is centred on rows[i] with neighbours nbr[i][16].
__global__ void k_pc_exact(HierView v, const int32_t* nbr, const int64_t* rows, int64_t n, double* ghat_out,
                           __half* gval, int32_t* gcol) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int64_t s = rows ? rows[i] : i;
    double g[kPcOut];
    pc_exact_row(v, nbr + i * kPcK, s, g);
    if (ghat_out)
        for (int a = 0; a < kPcOut; ++a) ghat_out[i * kPcOut + a] = g[a];
    if (gval) {  // the scale-free row in FP16; the solve applies delta^d to G^T G
        gcol[s] = (int32_t)s;
        gval[s] = __float2half_rn((float)g[0]);
        for (int k = 0; k < kPcK; ++k) {
            const int32_t c = nbr[s * kPcK + k];
            gcol[(1 + k) * v.N + s] = c;
            gval[(1 + k) * v.N + s] = __float2half_rn(c >= 0 ? (float)g[1 + k] : 0.f);
        }
    }
}

// ---------------------------------------------------------------- features

// Network input of row s: the delta-scaled offsets o_k = (x_{n_k} - x_s)/delta of its
// pattern neighbours (nearest first, zero-padded) in the patch's canonical frame: e_1 along
// o_1; e_2 the perpendicular of e_1 (d = 2) or o_2's component orthogonal to e_1 (d = 3, the
// coordinate axis least aligned with e_1 when o_2 is missing or parallel); e_3 = e_1 x e_2;
// the last axis flipped so that o_d has a non-negative coordinate on it (d = 1: o_1 > 0).
// The kernel is radial, so the exact row does not depend on the frame.  FP64 arithmetic, so
// the frame's sign decisions are those of the FP64 oracle.
// z[k D + a]: coordinate a of neighbour k (D = the point dimension, a compile-time constant
// so that z can live in registers).
template <int D>
__device__ __forceinline__ int pc_features(const HierView& v, const int32_t* nb, int64_t s, float* z) {
    const int l = level_of_row(v.off, v.L, s);
    const double inv = 1.0 / v.delta[l];
    constexpr int d = D;
    auto offset = [&](int k, double* o) {
        const int32_t c = nb[k];
        for (int a = 0; a < 3; ++a) o[a] = (a < d && c >= 0) ? (v.X[a * v.N + c] - v.X[a * v.N + s]) * inv : 0.0;
        return c >= 0;
    };
    int cnt = 0;
    for (int k = 0; k < kPcK; ++k) cnt += nb[k] >= 0;
    double e[3][3] = {{1, 0, 0}, {0, 1, 0}, {0, 0, 1}};
    double o1[3], o2[3], o3[3];
    offset(0, o1);
    offset(1, o2);
    offset(2, o3);
    const double n1 = sqrt(o1[0] * o1[0] + o1[1] * o1[1] + o1[2] * o1[2]);
    if (cnt >= 1 && n1 > 0.0) {
        if (d == 1) {
            e[0][0] = o1[0] >= 0.0 ? 1.0 : -1.0;
        } else if (d == 2) {
            const double a0 = o1[0] / n1, a1 = o1[1] / n1;
            double b0 = -a1, b1 = a0;
            if (cnt >= 2 && o2[0] * b0 + o2[1] * b1 < 0.0) { b0 = -b0; b1 = -b1; }
            e[0][0] = a0; e[0][1] = a1;
            e[1][0] = b0; e[1][1] = b1;
        } else {
            const double a[3] = {o1[0] / n1, o1[1] / n1, o1[2] / n1};
            double w[3] = {0, 0, 0};
            double nw = 0.0, n2 = 0.0;
            if (cnt >= 2) {
                const double p = o2[0] * a[0] + o2[1] * a[1] + o2[2] * a[2];
                for (int i = 0; i < 3; ++i) w[i] = o2[i] - p * a[i];
                nw = sqrt(w[0] * w[0] + w[1] * w[1] + w[2] * w[2]);
                n2 = sqrt(o2[0] * o2[0] + o2[1] * o2[1] + o2[2] * o2[2]);
            }
            double b[3];
            if (cnt >= 2 && nw > 1e-9 * n2) {
                for (int i = 0; i < 3; ++i) b[i] = w[i] / nw;
            } else {
                int ax = 0;  // the coordinate axis least aligned with e_1 (first on ties)
                for (int i = 1; i < 3; ++i)
                    if (fabs(a[i]) < fabs(a[ax])) ax = i;
                double u[3] = {0, 0, 0};
                u[ax] = 1.0;
                const double p = a[ax];
                for (int i = 0; i < 3; ++i) b[i] = u[i] - p * a[i];
                const double nb = sqrt(b[0] * b[0] + b[1] * b[1] + b[2] * b[2]);
                for (int i = 0; i < 3; ++i) b[i] /= nb;
            }
            double c[3] = {a[1] * b[2] - a[2] * b[1], a[2] * b[0] - a[0] * b[2], a[0] * b[1] - a[1] * b[0]};
            if (cnt >= 3 && o3[0] * c[0] + o3[1] * c[1] + o3[2] * c[2] < 0.0)
                for (int i = 0; i < 3; ++i) c[i] = -c[i];
            for (int i = 0; i < 3; ++i) {
                e[0][i] = a[i];
                e[1][i] = b[i];
                e[2][i] = c[i];
            }
        }
    }
#pragma unroll
    for (int k = 0; k < kPcK; ++k) {
        double o[3];
        const bool ok = offset(k, o);
#pragma unroll
        for (int a = 0; a < d; ++a)
            z[k * d + a] = ok ? (float)(e[a][0] * o[0] + e[a][1] * o[1] + e[a][2] * o[2]) : 0.f;
    }
    return cnt;
}

// Features of sample i: centre rows[i], neighbours nbr[i][16].
__global__ void k_pc_features(HierView v, const int32_t* nbr, const int64_t* rows, int64_t n, float* Z, int32_t* cnt) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    float z[kPcK * 3];
    const int64_t s = rows ? rows[i] : i;  // no rows: the pattern of sorted row i
    const int c = v.d == 1 ? pc_features<1>(v, nbr + i * kPcK, s, z)
                : v.d == 2 ? pc_features<2>(v, nbr + i * kPcK, s, z)
                           : pc_features<3>(v, nbr + i * kPcK, s, z);
    const int nin = kPcK * v.d;
    for (int k = 0; k < nin; ++k) Z[i * nin + k] = z[k];
    cnt[i] = c;
}

// Scaled patch matrix K = phi(|x_a - x_b| / delta) of sample i (centre rows[i] first, then its
// neighbours nbr[i][16]; zero-padded to 17x17): the metric of the training loss.
__global__ void k_pc_patchK(HierView v, const int32_t* nbr, const int64_t* rows, int64_t n, float* K) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int64_t s = rows[i];
    const int l = level_of_row(v.off, v.L, s);
    const double inv = 1.0 / v.delta[l];
    int64_t P[kPcOut];
    int m = 1;
    P[0] = s;
    for (int k = 0; k < kPcK; ++k) {
        const int32_t c = nbr[i * kPcK + k];
        if (c >= 0) P[m++] = c;
    }
    float* Ki = K + i * kPcOut * kPcOut;
    for (int a = 0; a < kPcOut; ++a)
        for (int b = 0; b < kPcOut; ++b)
            Ki[a * kPcOut + b] = (a < m && b < m) ? (float)wendland_eval<double>(v.w, dist_rn(v, P[a], P[b]) * inv) : 0.f;
}

// per-entry mean and standard deviation of the exact scale-free rows (the standardisation of
// the network's candidate rows)
__global__ void k_pc_moments(const double* ghat, const int32_t* cnt, int64_t n, float* musig) {
    const int m = blockIdx.x;  // one block per output
    __shared__ double sh[3][256];
    double s0 = 0, s1 = 0, s2 = 0;
    for (int64_t i = threadIdx.x; i < n; i += blockDim.x) {
        if (m <= cnt[i]) {
            const double g = ghat[i * kPcOut + m];
            s0 += 1.0;
            s1 += g;
            s2 += g * g;
        }
    }
    sh[0][threadIdx.x] = s0;
    sh[1][threadIdx.x] = s1;
    sh[2][threadIdx.x] = s2;
    __syncthreads();
    if (threadIdx.x == 0) {
        double a = 0, b = 0, c = 0;
        for (int t = 0; t < (int)blockDim.x; ++t) { a += sh[0][t]; b += sh[1][t]; c += sh[2][t]; }
        const double mu = a > 0 ? b / a : 0.0;
        const double var = a > 0 ? fmax(c / a - mu * mu, 0.0) : 1.0;
        musig[m] = (float)mu;
        musig[kPcOut + m] = (float)sqrt(fmax(var, 1e-30));
    }
}

// q* = (K^-1)_11 of every training patch: the exact scale-free row has unit energy, so
// q* = ghat_self^2 (the value the loss compares the network's combination with)
__global__ void k_pc_qstar(const double* ghat, int64_t n, double* qstar) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < n) qstar[i] = ghat[i * kPcOut] * ghat[i * kPcOut];
}

// ---------------------------------------------------------------- network

// parameter offsets: W1 [64][nin], b1 [64], W2 [64][64], b2 [64], W3 [17 m][64], b3 [17 m]
// (output 17 k + a = entry a of candidate row k)
struct NetLayout {
    int nin, m, nout, oW1, ob1, oW2, ob2, oW3, ob3, P;
};
__host__ __device__ inline NetLayout net_layout(int nin, int m) {
    NetLayout L;
    L.nin = nin;
    L.m = m;
    L.nout = kPcOut * m;
    L.oW1 = 0;
    L.ob1 = L.oW1 + kPcHidden * nin;
    L.oW2 = L.ob1 + kPcHidden;
    L.ob2 = L.oW2 + kPcHidden * kPcHidden;
    L.oW3 = L.ob2 + kPcHidden;
    L.ob3 = L.oW3 + L.nout * kPcHidden;
    L.P = L.ob3 + L.nout;
    return L;
}

// The candidate span is combined with a ridge of 1e-6 of the mean diagonal of S = U^T K U.
constexpr float kPcRidge = 1e-6f;

// Inference copy of the weights in shared memory, laid out for 128-bit broadcast loads:
// W1^T [nin][64], b1 [64], W2 [64][64], b2 [64], W3^T [64][R], b3 [17 m].  R = 68 ceil(m / 4):
// the candidates are computed four at a time (68 outputs), so every row of W3^T holds whole
// groups of four, zero past output 17 m (no read past the row, or past the array).
struct InferLayout {
    int oW1t, ob1, oW2, ob2, oW3t, R, ob3, P;
};
__host__ __device__ inline InferLayout infer_layout(int nin, int m) {
    InferLayout I;
    I.oW1t = 0;
    I.ob1 = kPcHidden * nin;
    I.oW2 = I.ob1 + kPcHidden;
    I.ob2 = I.oW2 + kPcHidden * kPcHidden;
    I.oW3t = I.ob2 + kPcHidden;
    I.R = 4 * kPcOut * ((m + 3) / 4);
    I.ob3 = I.oW3t + kPcHidden * I.R;
    I.P = (I.ob3 + kPcOut * m + 3) & ~3;
    return I;
}

constexpr int kCandBS = 128;  // threads per block of k_pc_cand

inline size_t cand_smem(int nin, int m) { return sizeof(float) * (size_t)infer_layout(nin, m).P; }

// The network's rows are made in two kernels.
// k_pc_cand, one thread per point: the features z of its pattern (canonical frame), the MLP,
// and the m candidate rows u_1 = mu + sigma o_1, u_k = sigma o_k (k > 1), zero past the patch,
// written row-contiguous: Uc[s][17 k + a]; also the features Zc[s][16 d] and the patch size
// cnt[s] (pattern neighbours).  The candidates are computed four at a time with register
// accumulators (the second hidden layer's units streamed, each W3 weight loaded once per four
// candidates from a transposed copy in shared memory, 128-bit broadcast loads).
__global__ void __launch_bounds__(kCandBS) k_pc_cand(HierView v, const int32_t* nbr, const float* theta, int m,
                                                     const float* musig, float* Uc, float* Zc, int32_t* cntc) {
    extern __shared__ __align__(16) float smi[];
    const int nin = kPcK * v.d;
    const NetLayout N = net_layout(nin, m);
    const InferLayout I = infer_layout(nin, m);
    float* W = smi;
    __shared__ float ms[2 * kPcOut];
    for (int i = threadIdx.x; i < kPcHidden * nin; i += blockDim.x) {
        const int k = i / kPcHidden, j = i % kPcHidden;
        W[I.oW1t + i] = theta[N.oW1 + j * nin + k];
    }
    for (int i = threadIdx.x; i < kPcHidden + kPcHidden * kPcHidden + kPcHidden; i += blockDim.x)
        W[I.ob1 + i] = theta[N.ob1 + i];  // b1, W2, b2 are contiguous in both layouts
    for (int i = threadIdx.x; i < kPcHidden * I.R; i += blockDim.x) {
        const int j = i / I.R, r = i % I.R;
        W[I.oW3t + i] = r < N.nout ? theta[N.oW3 + r * kPcHidden + j] : 0.f;
    }
    for (int i = threadIdx.x; i < N.nout; i += blockDim.x) W[I.ob3 + i] = theta[N.ob3 + i];
    if (threadIdx.x < 2 * kPcOut) ms[threadIdx.x] = musig[threadIdx.x];
    __syncthreads();
    const int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (s >= v.N) return;
    float z[kPcK * 3];
    const int cnt = v.d == 1 ? pc_features<1>(v, nbr + s * kPcK, s, z)
                  : v.d == 2 ? pc_features<2>(v, nbr + s * kPcK, s, z)
                             : pc_features<3>(v, nbr + s * kPcK, s, z);
    for (int k = 0; k < nin; ++k) Zc[s * nin + k] = z[k];
    cntc[s] = cnt;
    // layer 1 (inputs streamed, 64 accumulators)
    float h1[kPcHidden];
#pragma unroll
    for (int j = 0; j < kPcHidden; ++j) h1[j] = W[I.ob1 + j];
    for (int k = 0; k < nin; ++k) {
        const float zk = z[k];
        const float4* w4 = reinterpret_cast<const float4*>(W + I.oW1t + k * kPcHidden);
#pragma unroll
        for (int j4 = 0; j4 < kPcHidden / 4; ++j4) {
            const float4 w = w4[j4];
            h1[4 * j4] = fmaf(w.x, zk, h1[4 * j4]);
            h1[4 * j4 + 1] = fmaf(w.y, zk, h1[4 * j4 + 1]);
            h1[4 * j4 + 2] = fmaf(w.z, zk, h1[4 * j4 + 2]);
            h1[4 * j4 + 3] = fmaf(w.w, zk, h1[4 * j4 + 3]);
        }
    }
#pragma unroll
    for (int j = 0; j < kPcHidden; ++j) h1[j] = fmaxf(h1[j], 0.f);
    float* Us = Uc + s * (int64_t)N.nout;
    // layers 2 and 3, four candidates per pass
    for (int k0 = 0; k0 < m; k0 += 4) {
        float acc[4 * kPcOut];
#pragma unroll
        for (int r = 0; r < 4 * kPcOut; ++r) acc[r] = k0 * kPcOut + r < N.nout ? W[I.ob3 + k0 * kPcOut + r] : 0.f;
        for (int j = 0; j < kPcHidden; ++j) {
            float a2 = W[I.ob2 + j];
            const float4* w4 = reinterpret_cast<const float4*>(W + I.oW2 + j * kPcHidden);
#pragma unroll
            for (int k4 = 0; k4 < kPcHidden / 4; ++k4) {
                const float4 w = w4[k4];
                a2 = fmaf(w.x, h1[4 * k4], a2);
                a2 = fmaf(w.y, h1[4 * k4 + 1], a2);
                a2 = fmaf(w.z, h1[4 * k4 + 2], a2);
                a2 = fmaf(w.w, h1[4 * k4 + 3], a2);
            }
            a2 = fmaxf(a2, 0.f);
            // rows 17 k0 .. 17 k0 + 67 of W3^T's row j: 16-byte aligned (17 k0 is a multiple of 4)
            const float4* u4 = reinterpret_cast<const float4*>(W + I.oW3t + j * I.R + k0 * kPcOut);
#pragma unroll
            for (int r4 = 0; r4 < kPcOut; ++r4) {
                const float4 w = u4[r4];
                acc[4 * r4] = fmaf(w.x, a2, acc[4 * r4]);
                acc[4 * r4 + 1] = fmaf(w.y, a2, acc[4 * r4 + 1]);
                acc[4 * r4 + 2] = fmaf(w.z, a2, acc[4 * r4 + 2]);
                acc[4 * r4 + 3] = fmaf(w.w, a2, acc[4 * r4 + 3]);
            }
        }
#pragma unroll
        for (int r = 0; r < 4 * kPcOut; ++r) {
            const int k = k0 + r / kPcOut, a = r % kPcOut;
            // u_1 = mu + sigma o_1, u_k = sigma o_k (k > 1); zero past the patch
            if (k < m) Us[k * kPcOut + a] = a <= cnt ? fmaf(ms[kPcOut + a], acc[r], k == 0 ? ms[a] : 0.f) : 0.f;
        }
    }
}

// ---------------------------------------------------------------- network on the tensor cores
//
// k_pc_mlp: the network's candidate rows for tiles of 128 points on the fifth-generation tensor
// cores.  The three layers are MMAs with M = 128 points (one tensor-memory lane each), BF16
// operands and FP32 accumulators in tensor memory: [128 x nin] x W1^T -> 64 columns, then
// [128 x 64] x W2^T -> 64, then [128 x 64] x W3^T -> 17 m (at most 256 columns per MMA).  The
// weights are BF16-valued (the inference copy), so they are exact operands; each layer's input
// is split into hi + lo BF16 parts (16 significant bits) and both parts are multiplied, so the
// products carry the FP32 activations to about 2^-17.  Biases, ReLU and the output scaling
// u_1 = mu + sigma o_1, u_k = sigma o_k run in the epilogues, one thread per point, which read
// the accumulators with tcgen05.ld and write the next layer's operand to shared memory.  A CTA
// holds the weights for its whole life and walks tiles; two CTAs share an SM (256 tensor-memory
// columns each), so one's MMAs overlap the other's epilogues.
constexpr int kMlpRows = 128;            // points per tile (the MMA's M)
constexpr uint32_t kMlpCols = 256;       // tensor-memory columns per CTA
constexpr int kMlpSmemMin = 100 * 1024;  // at least this much shared memory: <= 2 CTAs per SM
constexpr unsigned long long kMlpWaitNs = 2000000000ull;  // bound on one wait for the MMAs

struct MlpSmem {  // byte offsets into dynamic shared memory
    int n3p, w1, w2, w3, act, b1, b2, b3, ms, mbar, slot, total;
};
__host__ __device__ inline MlpSmem mlp_smem(int nin, int m) {
    MlpSmem S;
    S.n3p = (kPcOut * m + 15) & ~15;  // W3 rows, a multiple of 16 (the MMA's N step)
    S.w1 = 0;
    S.w2 = S.w1 + kPcHidden * nin * 2;
    S.w3 = S.w2 + kPcHidden * kPcHidden * 2;
    S.act = S.w3 + S.n3p * kPcHidden * 2;
    S.b1 = S.act + 2 * kMlpRows * kPcHidden * 2;  // hi and lo operands of [128 x 64]
    S.b2 = S.b1 + kPcHidden * 4;
    S.b3 = S.b2 + kPcHidden * 4;
    S.ms = S.b3 + S.n3p * 4;
    S.mbar = (S.ms + 2 * kPcOut * 4 + 15) & ~15;
    S.slot = S.mbar + 8;
    S.total = S.slot + 8;
    if (S.total < kMlpSmemMin) S.total = kMlpSmemMin;
    return S;
}

// hi + lo BF16 parts of eight FP32 values, as two 16-byte words
__device__ __forceinline__ void split8_bf16(const float* x, uint4& hi, uint4& lo) {
    uint32_t h[4], l[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const __nv_bfloat16 a0 = __float2bfloat16_rn(x[2 * i]), a1 = __float2bfloat16_rn(x[2 * i + 1]);
        const __nv_bfloat16 r0 = __float2bfloat16_rn(x[2 * i] - __bfloat162float(a0));
        const __nv_bfloat16 r1 = __float2bfloat16_rn(x[2 * i + 1] - __bfloat162float(a1));
        h[i] = (uint32_t)__bfloat16_as_ushort(a0) | ((uint32_t)__bfloat16_as_ushort(a1) << 16);
        l[i] = (uint32_t)__bfloat16_as_ushort(r0) | ((uint32_t)__bfloat16_as_ushort(r1) << 16);
    }
    hi = make_uint4(h[0], h[1], h[2], h[3]);
    lo = make_uint4(l[0], l[1], l[2], l[3]);
}

// Waits (bounded) for the mbarrier's phase; the result is the same in every thread.
__device__ __forceinline__ bool mlp_wait(uint64_t* mbar, uint32_t parity) {
    const unsigned long long t0 = ms_globaltimer();
    bool ok = true;
    while (!tc_mbar_try_wait(mbar, parity))
        if (ms_globaltimer() - t0 > kMlpWaitNs) {
            ok = false;
            break;
        }
    return __syncthreads_and(ok) != 0;
}

__global__ void __launch_bounds__(kMlpRows) k_pc_mlp(const float* __restrict__ theta, int nin, int m,
                                                     const float* __restrict__ musig, const float* __restrict__ Zc,
                                                     const int32_t* __restrict__ cntc, int64_t N, float* __restrict__ Uc,
                                                     int* status) {
    extern __shared__ __align__(128) unsigned char smb[];
    const MlpSmem S = mlp_smem(nin, m);
    const NetLayout NL = net_layout(nin, m);
    const int tid = threadIdx.x, warp = tid >> 5;
    const int nout = NL.nout, n3p = S.n3p;
    float* b1 = reinterpret_cast<float*>(smb + S.b1);
    float* b2 = reinterpret_cast<float*>(smb + S.b2);
    float* b3 = reinterpret_cast<float*>(smb + S.b3);
    float* ms = reinterpret_cast<float*>(smb + S.ms);
    uint64_t* mbar = reinterpret_cast<uint64_t*>(smb + S.mbar);
    uint32_t* slot = reinterpret_cast<uint32_t*>(smb + S.slot);
    // the weights (BF16-valued FP32, so the BF16 copies are exact) in the K-major operand layout
    for (int i = tid; i < kPcHidden * nin; i += kMlpRows)
        *reinterpret_cast<__nv_bfloat16*>(smb + S.w1 + tc_kmajor_offset(nin, i / nin, i % nin)) =
            __float2bfloat16_rn(theta[NL.oW1 + i]);
    for (int i = tid; i < kPcHidden * kPcHidden; i += kMlpRows)
        *reinterpret_cast<__nv_bfloat16*>(smb + S.w2 + tc_kmajor_offset(kPcHidden, i / kPcHidden, i % kPcHidden)) =
            __float2bfloat16_rn(theta[NL.oW2 + i]);
    for (int i = tid; i < n3p * kPcHidden; i += kMlpRows) {
        const int r = i / kPcHidden;
        *reinterpret_cast<__nv_bfloat16*>(smb + S.w3 + tc_kmajor_offset(kPcHidden, r, i % kPcHidden)) =
            __float2bfloat16_rn(r < nout ? theta[NL.oW3 + i] : 0.f);
    }
    for (int i = tid; i < kPcHidden; i += kMlpRows) {
        b1[i] = theta[NL.ob1 + i];
        b2[i] = theta[NL.ob2 + i];
    }
    for (int i = tid; i < n3p; i += kMlpRows) b3[i] = i < nout ? theta[NL.ob3 + i] : 0.f;
    for (int i = tid; i < 2 * kPcOut; i += kMlpRows) ms[i] = musig[i];
    if (tid == 0) tc_mbar_init(mbar, 1);
    if (warp == 0) tc_alloc(slot, kMlpCols);
    tc_fence_proxy();
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tbase = *slot;
    const uint32_t tq = tbase + ((uint32_t)(warp * 32) << 16);  // this warp's quarter of the lanes
    const uint32_t a_hi = tc_smem_addr(smb + S.act), a_lo = a_hi + kMlpRows * kPcHidden * 2;
    const uint32_t w1 = tc_smem_addr(smb + S.w1), w2 = tc_smem_addr(smb + S.w2), w3 = tc_smem_addr(smb + S.w3);
    // K-direction core stride 128 bytes; row-group strides 16 Kd (Kd = 64, or nin for W1)
    constexpr uint32_t lbo = 128, sboH = 16 * kPcHidden;
    const uint32_t sbo1 = 16u * (uint32_t)nin;
    const int nA = n3p < 256 ? n3p : 256;  // layer 3 in at most two MMA widths
    uint32_t phase = 0;
    bool ok = true;
    const int64_t ntiles = (N + kMlpRows - 1) / kMlpRows;
    // one layer's MMAs: D[cols] = [a_hi + a_lo] x B^T over K = kd (16 per instruction)
    auto issue = [&](uint32_t dcol, uint32_t b0, uint32_t sboB, int kd, int n) {
        if (tid == 0) {
            tc_fence_after();
            const uint32_t id = tc_idesc_bf16(kMlpRows, n);
            for (int ks = 0; ks < kd / 16; ++ks) {  // K = 16 a step: two core matrices
                const uint64_t bd = tc_sdesc(b0 + ks * 2 * lbo, lbo, sboB);
                tc_mma_bf16(tbase + dcol, tc_sdesc(a_hi + ks * 2 * lbo, lbo, sboH), bd, id, ks > 0 ? 1u : 0u);
                tc_mma_bf16(tbase + dcol, tc_sdesc(a_lo + ks * 2 * lbo, lbo, sboH), bd, id, 1u);
            }
            tc_commit(mbar);
        }
        ok = mlp_wait(mbar, phase);
        phase ^= 1u;
        tc_fence_after();
    };
    // hidden-layer epilogue: relu(D + b) split into the next operand (64 columns)
    auto hidden = [&](uint32_t dcol, const float* bias) {
#pragma unroll 1
        for (int c = 0; c < kPcHidden; c += 16) {
            uint32_t r[16];
            tc_ld16(tq + dcol + c, r);
            tc_wait_ld();
            float x[16];
#pragma unroll
            for (int j = 0; j < 16; ++j) x[j] = fmaxf(__uint_as_float(r[j]) + bias[c + j], 0.f);
            uint4 hi, lo;
            split8_bf16(x, hi, lo);
            *reinterpret_cast<uint4*>(smb + S.act + tc_kmajor_offset(kPcHidden, tid, c)) = hi;
            *reinterpret_cast<uint4*>(smb + S.act + kMlpRows * kPcHidden * 2 + tc_kmajor_offset(kPcHidden, tid, c)) = lo;
            split8_bf16(x + 8, hi, lo);
            *reinterpret_cast<uint4*>(smb + S.act + tc_kmajor_offset(kPcHidden, tid, c + 8)) = hi;
            *reinterpret_cast<uint4*>(smb + S.act + kMlpRows * kPcHidden * 2 + tc_kmajor_offset(kPcHidden, tid, c + 8)) =
                lo;
        }
        tc_fence_proxy();
        tc_fence_before();
        __syncthreads();
    };
    for (int64_t tile = blockIdx.x; tile < ntiles && ok; tile += gridDim.x) {
        const int64_t s = tile * kMlpRows + tid;
        const bool live = s < N;
        // layer-1 operand: the point's features, hi and lo parts
        for (int c = 0; c < nin; c += 8) {
            float x[8];
            if (live) {
                const float4 p = __ldg(reinterpret_cast<const float4*>(Zc + s * nin + c));
                const float4 q = __ldg(reinterpret_cast<const float4*>(Zc + s * nin + c + 4));
                x[0] = p.x; x[1] = p.y; x[2] = p.z; x[3] = p.w; x[4] = q.x; x[5] = q.y; x[6] = q.z; x[7] = q.w;
            } else {
#pragma unroll
                for (int j = 0; j < 8; ++j) x[j] = 0.f;
            }
            uint4 hi, lo;
            split8_bf16(x, hi, lo);
            *reinterpret_cast<uint4*>(smb + S.act + tc_kmajor_offset(kPcHidden, tid, c)) = hi;
            *reinterpret_cast<uint4*>(smb + S.act + kMlpRows * kPcHidden * 2 + tc_kmajor_offset(kPcHidden, tid, c)) = lo;
        }
        const int cnt = live ? __ldg(cntc + s) : 0;
        tc_fence_proxy();
        tc_fence_before();
        __syncthreads();
        issue(0, w1, sbo1, nin, kPcHidden);
        if (!ok) break;
        hidden(0, b1);
        issue(kPcHidden, w2, sboH, kPcHidden, kPcHidden);
        if (!ok) break;
        hidden(kPcHidden, b2);
        // layer 3: columns [0, nA), then (17 m > 256) [256, n3p) into the same tensor memory
        for (int r0 = 0; r0 < n3p; r0 += nA) {
            const int n = n3p - r0 < nA ? n3p - r0 : nA;
            if (r0 > 0) {  // every thread has read the previous columns
                tc_fence_before();
                __syncthreads();
            }
            issue(0, w3 + (uint32_t)(r0 / 8) * sboH, sboH, kPcHidden, n);
            if (!ok) break;
#pragma unroll 1
            for (int c = 0; c < n; c += 16) {
                uint32_t r[16];
                tc_ld16(tq + c, r);
                tc_wait_ld();
                if (live) {
                    float u[16];
#pragma unroll
                    for (int j = 0; j < 16; ++j) {
                        const int o = r0 + c + j;  // output 17 k + a
                        const int k = o / kPcOut, a = o - kPcOut * k;
                        const float acc = __uint_as_float(r[j]) + b3[min(o, n3p - 1)];
                        u[j] = a <= cnt ? fmaf(ms[kPcOut + a], acc, k == 0 ? ms[a] : 0.f) : 0.f;
                    }
                    float* dst = Uc + s * nout + r0 + c;
                    if (r0 + c + 16 <= nout && (nout & 3) == 0) {  // 16-byte aligned: four 128-bit stores
#pragma unroll
                        for (int j = 0; j < 16; j += 4)
                            *reinterpret_cast<float4*>(dst + j) = make_float4(u[j], u[j + 1], u[j + 2], u[j + 3]);
                    } else {
#pragma unroll
                        for (int j = 0; j < 16; ++j)
                            if (r0 + c + j < nout) dst[j] = u[j];
                    }
                }
            }
        }
        tc_fence_before();
        __syncthreads();
    }
    if (!ok && tid == 0) atomicExch(status, (int)MS_ERR_TIMEOUT);
    if (!ok) mlp_wait(mbar, phase ^ 1u);  // one more bounded wait for the MMAs still in flight
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == 0) tc_dealloc(tbase, kMlpCols);
}

// k_pc_combine, one half-warp per point: the factorised-sparse-approximate-inverse row in the
// span of the point's candidates,
//   g = U y / sqrt(q),  y = (S + 1e-6 diag(S))^-1 U^T e_1,  S = U^T K U,  q = e_1^T U y,
// K = phi(|z_a - z_b|) on the patch (self at the origin), or, for a patch of n = cnt + 1 <= m
// points, the exact row (S = K, U = I, no ridge); g^T K g = 1 less the ridge's shift and
// g_self = sqrt(q) > 0.  (A failed factorisation, or q <= 0: the diagonal row e_1 / sqrt(phi(0)).)
// Lane l of the half owns column l of S in registers: t = K u_l from the patch matrix in
// shared memory (rows read as broadcast float4s), S_kl = u_k . t, then S is Jacobi-scaled to
// unit diagonal (the ridge becomes 1e-6 I) and factorised by a right-looking Cholesky over
// the lanes' columns: at step k every lane takes its multiplier L_jk from its own column
// (S is kept symmetric, so S_kj = S_jk), the multipliers are broadcast by shuffles, and the
// forward substitution L w = b runs alongside; q = |w|^2, and L^T y = w by half-warp sums.
// Columns l >= m (or >= n) are identity columns.  Writes the scale-free row (FP16) and its
// pattern, or ghat itself for inspection.
constexpr int kCombPts = 8;  // points per block of k_pc_combine

struct CombBuf {
    float K[kPcOut][20];           // patch matrix, rows padded to 20 floats (16-byte aligned)
    float U[kPcMaxBasis][20];      // candidate k's entries a = 0..16, zero-padded
    float z[kPcK * 3];
};
// 2832 bytes = 16 (mod 128): the two points of a warp broadcast from different banks
static_assert(sizeof(CombBuf) % 128 == 16, "CombBuf bank offset");

__global__ void __launch_bounds__(kCombPts * 16) k_pc_combine(HierView v, float4 wc, const int32_t* nbr, int m,
                                                              const float* Uc, const float* Zc, const int32_t* cntc,
                                                              __half* gval, int32_t* gcol, float* ghat_out) {
    __shared__ __align__(16) CombBuf cb[kCombPts];
    __shared__ uint16_t pairs[kPcOut * kPcK / 2];  // the 136 pairs a < b of 17 points: a | b << 8
    for (int i = threadIdx.x; i < kPcOut * kPcK / 2; i += blockDim.x) {
        int a = 0, rem = i;
        while (rem >= kPcK - a) { rem -= kPcK - a; ++a; }
        pairs[i] = (uint16_t)(a | ((a + 1 + rem) << 8));
    }
    __syncthreads();
    const int hp = threadIdx.x >> 4, l = threadIdx.x & 15;
    const unsigned hmask = 0xFFFFu << (threadIdx.x & 16);  // this half-warp's lanes
    CombBuf& B = cb[hp];
    const int64_t s = blockIdx.x * (int64_t)kCombPts + hp;
    if (s >= v.N) return;  // the whole half-warp (its lanes synchronise among themselves only)
    const int d = v.d, nin = kPcK * d, nout = kPcOut * m;
    const int cnt = cntc[s];
    const int np = cnt + 1;
    const bool exact = np <= m;
    const float wcf[4] = {wc.x, wc.y, wc.z, wc.w};  // Wendland coefficients in FP32 (converted on the host)
    const float phi0 = wcf[0];
    {
        float4* K4 = reinterpret_cast<float4*>(&B.K[0][0]);
        for (int i = l; i < kPcOut * 5; i += 16) K4[i] = make_float4(0.f, 0.f, 0.f, 0.f);
        if (!exact) {
            float4* U4 = reinterpret_cast<float4*>(&B.U[0][0]);
            for (int i = l; i < kPcMaxBasis * 5; i += 16) U4[i] = make_float4(0.f, 0.f, 0.f, 0.f);
        }
    }
    __syncwarp(hmask);
    if (!exact)
        for (int i = l; i < nout; i += 16) B.U[i / kPcOut][i % kPcOut] = __ldg(Uc + s * (int64_t)nout + i);
    for (int i = l; i < nin; i += 16) B.z[i] = __ldg(Zc + s * (int64_t)nin + i);
    __syncwarp(hmask);
    for (int i = l; i < kPcOut * kPcK / 2; i += 16) {
        const int a = pairs[i] & 0xFF, b = pairs[i] >> 8;
        if (b < np) {
            float r2 = 0.f;
            for (int ax = 0; ax < d; ++ax) {
                const float u = (a > 0 ? B.z[(a - 1) * d + ax] : 0.f) - B.z[(b - 1) * d + ax];
                r2 = fmaf(u, u, r2);
            }
            // FP32 entries need no correctly rounded sqrt: r = r2 / sqrt(r2)
            const float kab = wendland_eval_f(v.w, wcf, r2 * rsqrtf(fmaxf(r2, 1e-30f)));
            B.K[a][b] = kab;
            B.K[b][a] = kab;
        }
    }
    if (l < np) B.K[l][l] = phi0;
    if (l == 0 && np == kPcOut) B.K[kPcK][kPcK] = phi0;
    __syncwarp(hmask);

    // column l of S (identity past m, or past n for the exact row) and b_l
    float sc[kPcMaxBasis];
    float diag, bl;
    if (!exact) {
        float u[20];
        {
            const float4* ur = reinterpret_cast<const float4*>(B.U[l]);
#pragma unroll
            for (int j = 0; j < 5; ++j) {
                const float4 q = ur[j];
                u[4 * j] = q.x; u[4 * j + 1] = q.y; u[4 * j + 2] = q.z; u[4 * j + 3] = q.w;
            }
        }
        float t[20];
#pragma unroll
        for (int a = 0; a < 20; ++a) t[a] = 0.f;
#pragma unroll
        for (int a = 0; a < kPcOut; ++a) {
            const float4* kr = reinterpret_cast<const float4*>(B.K[a]);
            float acc = 0.f;
#pragma unroll
            for (int j = 0; j < 5; ++j) {
                const float4 q = kr[j];
                acc = fmaf(q.x, u[4 * j], acc);
                acc = fmaf(q.y, u[4 * j + 1], acc);
                acc = fmaf(q.z, u[4 * j + 2], acc);
                acc = fmaf(q.w, u[4 * j + 3], acc);
            }
            t[a] = acc;
        }
        diag = 0.f;
#pragma unroll
        for (int a = 0; a < kPcOut; ++a) diag = fmaf(u[a], t[a], diag);
#pragma unroll
        for (int k = 0; k < kPcMaxBasis; ++k) {
            const float4* ur = reinterpret_cast<const float4*>(B.U[k]);
            float acc = 0.f;
#pragma unroll
            for (int j = 0; j < 5; ++j) {
                const float4 q = ur[j];
                acc = fmaf(q.x, t[4 * j], acc);
                acc = fmaf(q.y, t[4 * j + 1], acc);
                acc = fmaf(q.z, t[4 * j + 2], acc);
                acc = fmaf(q.w, t[4 * j + 3], acc);
            }
            sc[k] = (k < m && l < m) ? acc : (k == l ? 1.f : 0.f);
        }
        if (l >= m) diag = 1.f;
        bl = l < m ? u[0] : 0.f;
    } else {
#pragma unroll
        for (int k = 0; k < kPcMaxBasis; ++k) sc[k] = (k < np && l < np) ? B.K[k][l] : (k == l ? 1.f : 0.f);
        diag = l < np ? phi0 : 1.f;
        bl = l == 0 ? 1.f : 0.f;
    }
    // Jacobi scaling D = diag(S)^-1/2 (ridge on the scaled diagonal), b' = D b
    const float ridge = exact ? 0.f : kPcRidge;
    const float dl = rsqrtf(fmaxf(diag, 1e-30f));
    bool ok = (__ballot_sync(hmask, !(diag > 0.f)) & hmask) == 0u;
    float dk[kPcMaxBasis], w[kPcMaxBasis];
#pragma unroll
    for (int k = 0; k < kPcMaxBasis; ++k) {
        dk[k] = __shfl_sync(hmask, dl, k, 16);
        w[k] = __shfl_sync(hmask, bl * dl, k, 16);
        sc[k] = sc[k] * dk[k] * dl + (k == l ? ridge : 0.f);
    }
    // Cholesky with the forward substitution L w = b'
    float lkk[kPcMaxBasis], lrow[kPcMaxBasis];
#pragma unroll
    for (int k = 0; k < kPcMaxBasis; ++k) {
        const float piv = __shfl_sync(hmask, sc[k], k, 16);
        ok = ok && piv > 0.f;
        const float dkk = sqrtf(fmaxf(piv, 1e-30f)), inv = 1.f / dkk;
        lkk[k] = dkk;
        const float c = sc[k] * inv;  // lane j > k: L_jk
        lrow[k] = c;
        w[k] *= inv;
#pragma unroll
        for (int i = k + 1; i < kPcMaxBasis; ++i) {
            const float Li = __shfl_sync(hmask, c, i, 16);
            sc[i] = fmaf(-Li, c, sc[i]);
            w[i] = fmaf(-Li, w[k], w[i]);
        }
    }
    float q = 0.f;
#pragma unroll
    for (int k = 0; k < kPcMaxBasis; ++k) q = fmaf(w[k], w[k], q);  // q = b'^T S'^-1 b' = |w|^2
    ok = ok && q > 0.f && isfinite(q);
    // L^T y' = w, then y = D y' (yv); lane l keeps y'_l
    float yown = 0.f, yv[kPcMaxBasis];
#pragma unroll
    for (int k = kPcMaxBasis - 1; k >= 0; --k) {
        float part = l > k ? lrow[k] * yown : 0.f;
#pragma unroll
        for (int o = 8; o > 0; o >>= 1) part += __shfl_xor_sync(hmask, part, o, 16);
        const float yk = (w[k] - part) / lkk[k];
        if (l == k) yown = yk;
        yv[k] = yk * dk[k];
    }
    // g_a = (U y)_a / sqrt(q): lane l entry a = l, lane 0 also entry 16 (exact: y_a / sqrt(q))
    float ga = 0.f, g16 = 0.f;
    if (exact) {
        ga = l < np ? yown * dl : 0.f;
    } else {
#pragma unroll
        for (int k = 0; k < kPcMaxBasis; ++k)
            if (k < m) ga = fmaf(B.U[k][l], yv[k], ga);
        if (l == 0)
#pragma unroll
            for (int k = 0; k < kPcMaxBasis; ++k)
                if (k < m) g16 = fmaf(B.U[k][kPcK], yv[k], g16);
        if (l > cnt) ga = 0.f;
        if (cnt < kPcK) g16 = 0.f;
    }
    const float sq = ok ? rsqrtf(q) : 0.f;
    ga *= sq;
    g16 *= sq;
    if (!ok) {
        ga = l == 0 ? rsqrtf(phi0) : 0.f;
        g16 = 0.f;
    }
    // lane l writes pattern slot l, whose entry is 1 + (present slots before it)
    const int32_t c = nbr[s * kPcK + l];
    const unsigned present = (__ballot_sync(hmask, c >= 0) >> (threadIdx.x & 16)) & 0xFFFFu;
    const int e = 1 + __popc(present & ((1u << l) - 1u));
    const float ge = __shfl_sync(hmask, ga, e & 15, 16);
    const float gl = __shfl_sync(hmask, g16, 0, 16);
    const float gslot = c >= 0 ? (e == kPcK ? gl : ge) : 0.f;
    if (ghat_out) {
        if (l == 0) ghat_out[s * kPcOut] = ga;
        ghat_out[s * kPcOut + 1 + l] = gslot;
        return;
    }
    if (l == 0) {
        gcol[s] = (int32_t)s;
        gval[s] = __float2half_rn(ga);
    }
    gcol[(int64_t)(1 + l) * v.N + s] = c;
    gval[(int64_t)(1 + l) * v.N + s] = __float2half_rn(gslot);
}

// SplitMix64 output function (Steele, Lea and Flood 2014) of counter x: per-element noise.
__device__ __forceinline__ uint64_t sm64_dev(uint64_t x) {
    x += 0x9E3779B97F4A7C15ull;
    x = (x ^ (x >> 30)) * 0xBF58476D1CE4E5B9ull;
    x = (x ^ (x >> 27)) * 0x94D049BB133111EBull;
    return x ^ (x >> 31);
}

// Training samples per block: the per-sample buffers grow with the candidate count m.
__host__ __device__ inline int train_tb(int m) { return m <= 2 ? 64 : (m <= 8 ? 32 : 16); }

// Shared-memory layout of k_pc_train (floats).
struct TrainLayout {
    int W, X, A1, A2, U, KU, Sm, Y, Q, YY, GT, Rr, D2, D1, total;
};
__host__ __device__ inline TrainLayout train_layout(int nin, int m, int tb) {
    const NetLayout N = net_layout(nin, m);
    TrainLayout T;
    int o = 0;
    T.W = o; o += N.P;
    T.X = o; o += tb * nin;
    T.A1 = o; o += tb * kPcHidden;
    T.A2 = o; o += tb * kPcHidden;
    T.U = o; o += tb * N.nout;
    T.KU = o; o += tb * N.nout;
    T.Sm = o; o += tb * m * m;
    T.Y = o; o += tb * m;
    T.Q = o; o += tb;
    T.YY = o; o += tb;
    T.GT = o; o += tb * kPcOut;
    T.Rr = o; o += tb * kPcOut;
    T.D2 = o; o += tb * kPcHidden;
    T.D1 = o; o += tb * kPcHidden;
    T.total = o;
    return T;
}

// One block = tb samples of a step: forward, the combination of the candidates, backward,
// per-block gradient partial.  Sample j of the step is training sample
// (a_mul * ((step * batch + j) mod S) + a_add) mod S; samples with (step * batch + j) >= limit
// are skipped (full-batch inspection).
// Loss of a sample: log q* - log q (q* = (K^-1)_11 of the exact row, q = e_1^T U y of the
// candidates' combination, y = (S + 1e-6 diag(S))^-1 U^T e_1, S = U^T K U, see k_pc_infer).
// With r = e_1 - K U y and the ridge's own dependence on U,
// dq/dU = 2 r y^T - 2e-6 (K U) diag(y)^2, and the error signal of output 17 k + a is
// escale * sigma_a * (-(dq/dU)_ak / q) on the patch's entries (escale = 1 / samples of the
// step).  The m x m system is factorised in FP64 (training only); a sample whose
// factorisation fails, or a patch of n <= m points (its row is the exact one), contributes
// nothing.
// noise > 0: every present input coordinate of a training sample is jittered by
// noise * U[-1, 1) (counter = (noise_key, sample slot, coordinate); targets unchanged).
__global__ void k_pc_train(const float* Z, const double* qstar, const int32_t* cnt, const float* Kp,
                           const float* musig, int64_t S, int nin, int m, const float* theta, int batch, int64_t step,
                           uint64_t a_mul, uint64_t a_add, int64_t limit, float escale, float* grad_part,
                           double* loss_part, float noise, uint64_t noise_key) {
    extern __shared__ float sm[];
    const int tb = train_tb(m);
    const NetLayout N = net_layout(nin, m);
    const TrainLayout L = train_layout(nin, m, tb);
    const int NO = N.nout;
    float* W = sm + L.W;
    float* X = sm + L.X;
    float* A1 = sm + L.A1;
    float* A2 = sm + L.A2;
    float* U = sm + L.U;
    float* KU = sm + L.KU;  // K U, then the error signal of the outputs
    float* Sm = sm + L.Sm;
    float* Y = sm + L.Y;
    float* Q = sm + L.Q;
    float* YY = sm + L.YY;
    float* GT = sm + L.GT;
    float* Rr = sm + L.Rr;
    float* D2 = sm + L.D2;
    float* D1 = sm + L.D1;
    __shared__ double lsum[64];
    __shared__ int64_t sidx[64];
    __shared__ int scnt[64];
    const int t = threadIdx.x, nt = blockDim.x;
    for (int i = t; i < N.P; i += nt) W[i] = theta[i];
    if (t < tb) {
        const int64_t g = step * batch + (int64_t)blockIdx.x * tb + t;
        sidx[t] = g < limit ? (int64_t)((a_mul * (uint64_t)(g % S) + a_add) % (uint64_t)S) : -1;
        scnt[t] = sidx[t] >= 0 ? cnt[sidx[t]] : -1;
    }
    __syncthreads();
    for (int i = t; i < tb * nin; i += nt) {
        const int s = i / nin, k = i % nin;
        float x = sidx[s] >= 0 ? Z[sidx[s] * nin + k] : 0.f;
        if (noise > 0.f && x != 0.f) {
            const uint64_t c = noise_key ^ ((uint64_t)(step * batch + (int64_t)blockIdx.x * tb + s) * 64u + (uint64_t)k);
            x += noise * ((float)(sm64_dev(c) >> 40) * 0x1p-23f - 1.0f);
        }
        X[i] = x;
    }
    __syncthreads();
    // layer 1
    for (int i = t; i < tb * kPcHidden; i += nt) {
        const int s = i / kPcHidden, j = i % kPcHidden;
        float a = W[N.ob1 + j];
        for (int k = 0; k < nin; ++k) a = fmaf(W[N.oW1 + j * nin + k], X[s * nin + k], a);
        A1[i] = a;
    }
    __syncthreads();
    // layer 2
    for (int i = t; i < tb * kPcHidden; i += nt) {
        const int s = i / kPcHidden, j = i % kPcHidden;
        float a = W[N.ob2 + j];
        for (int k = 0; k < kPcHidden; ++k) a = fmaf(W[N.oW2 + j * kPcHidden + k], fmaxf(A1[s * kPcHidden + k], 0.f), a);
        A2[i] = a;
    }
    __syncthreads();
    // candidate rows U[s][17 k + a]: u_1 = mu + sigma o_1, u_k = sigma o_k (zero past the patch)
    for (int i = t; i < tb * NO; i += nt) {
        const int s = i / NO, j = i % NO, a = j % kPcOut;
        float u = 0.f;
        if (a <= scnt[s]) {
            float o = W[N.ob3 + j];
            for (int jj = 0; jj < kPcHidden; ++jj) o = fmaf(W[N.oW3 + j * kPcHidden + jj], fmaxf(A2[s * kPcHidden + jj], 0.f), o);
            u = fmaf(musig[kPcOut + a], o, j < kPcOut ? musig[a] : 0.f);  // the mean on u_1 only
        }
        U[i] = u;
    }
    __syncthreads();
    // K U
    for (int i = t; i < tb * NO; i += nt) {
        const int s = i / NO, j = i % NO, k = j / kPcOut, a = j % kPcOut;
        float v = 0.f;
        if (a <= scnt[s]) {
            const float* Ka = Kp + (sidx[s] * kPcOut + a) * kPcOut;
            for (int b = 0; b <= scnt[s]; ++b) v = fmaf(Ka[b], U[s * NO + k * kPcOut + b], v);
        }
        KU[i] = v;
    }
    __syncthreads();
    // S = U^T K U
    for (int i = t; i < tb * m * m; i += nt) {
        const int s = i / (m * m), k = (i / m) % m, l = i % m;
        float v = 0.f;
        for (int a = 0; a <= scnt[s]; ++a) v = fmaf(U[s * NO + k * kPcOut + a], KU[s * NO + l * kPcOut + a], v);
        Sm[i] = v;
    }
    __syncthreads();
    // per sample: ridge, Cholesky (FP64), y, q
    double lacc = 0.0;
    if (t < tb) {
        const int s = t;
        float q = 0.f, yy = 0.f;
        // patches of n <= m points take the exact row: no dependence on the network
        if (sidx[s] >= 0 && scnt[s] + 1 > m) {
            double R[kPcMaxBasis * kPcMaxBasis];
            bool ok = true;
            for (int k = 0; k < m && ok; ++k) {
                double dkk = (double)Sm[s * m * m + k * m + k] * (1.0 + (double)kPcRidge);
                for (int i = 0; i < k; ++i) dkk -= R[i * m + k] * R[i * m + k];
                if (!(dkk > 0.0)) { ok = false; break; }
                const double rkk = sqrt(dkk);
                R[k * m + k] = rkk;
                for (int l = k + 1; l < m; ++l) {
                    double v = (double)Sm[s * m * m + k * m + l];
                    for (int i = 0; i < k; ++i) v -= R[i * m + k] * R[i * m + l];
                    R[k * m + l] = v / rkk;
                }
            }
            if (ok) {
                double yv[kPcMaxBasis];
                for (int k = 0; k < m; ++k) {
                    double w = (double)U[s * NO + k * kPcOut];
                    for (int i = 0; i < k; ++i) w -= R[i * m + k] * yv[i];
                    yv[k] = w / R[k * m + k];
                }
                for (int k = m - 1; k >= 0; --k) {
                    double w = yv[k];
                    for (int l = k + 1; l < m; ++l) w -= R[k * m + l] * yv[l];
                    yv[k] = w / R[k * m + k];
                }
                double qd = 0.0, yyd = 0.0;
                for (int k = 0; k < m; ++k) {
                    qd += (double)U[s * NO + k * kPcOut] * yv[k];
                    yyd += yv[k] * yv[k];
                }
                if (qd > 0.0 && isfinite(qd)) {
                    q = (float)qd;
                    yy = (float)yyd;
                    for (int k = 0; k < m; ++k) Y[s * m + k] = (float)yv[k];
                    lacc = log(qstar[sidx[s]]) - log(qd);
                }
            }
        }
        if (!(q > 0.f))
            for (int k = 0; k < m; ++k) Y[s * m + k] = 0.f;
        Q[s] = q;
        YY[s] = yy;
    }
    if (t < 64) lsum[t] = lacc;
    __syncthreads();
    // U y, then r = e_1 - K U y
    for (int i = t; i < tb * kPcOut; i += nt) {
        const int s = i / kPcOut, a = i % kPcOut;
        float v = 0.f;
        for (int k = 0; k < m; ++k) v = fmaf(U[s * NO + k * kPcOut + a], Y[s * m + k], v);
        GT[i] = v;
    }
    __syncthreads();
    for (int i = t; i < tb * kPcOut; i += nt) {
        const int s = i / kPcOut, a = i % kPcOut;
        float v = 0.f;
        if (sidx[s] >= 0 && a <= scnt[s]) {
            const float* Ka = Kp + (sidx[s] * kPcOut + a) * kPcOut;
            v = a == 0 ? 1.f : 0.f;
            for (int b = 0; b <= scnt[s]; ++b) v = fmaf(-Ka[b], GT[s * kPcOut + b], v);
        }
        Rr[i] = v;
    }
    __syncthreads();
    // error signal of the outputs (in place of K U)
    for (int i = t; i < tb * NO; i += nt) {
        const int s = i / NO, j = i % NO, k = j / kPcOut, a = j % kPcOut;
        float e = 0.f;
        if (Q[s] > 0.f && a <= scnt[s]) {
            const float yk = Y[s * m + k];
            const float dq = 2.f * Rr[s * kPcOut + a] * yk - 2.f * kPcRidge * yk * yk * KU[i];
            e = -escale * musig[kPcOut + a] * dq / Q[s];
        }
        KU[i] = e;
    }
    __syncthreads();
    const float* E = KU;
    // backward through layers 3 and 2
    for (int i = t; i < tb * kPcHidden; i += nt) {
        const int s = i / kPcHidden, j = i % kPcHidden;
        float a = 0.f;
        for (int o = 0; o < NO; ++o) a = fmaf(E[s * NO + o], W[N.oW3 + o * kPcHidden + j], a);
        D2[i] = A2[i] > 0.f ? a : 0.f;
    }
    __syncthreads();
    for (int i = t; i < tb * kPcHidden; i += nt) {
        const int s = i / kPcHidden, k = i % kPcHidden;
        float a = 0.f;
        for (int j = 0; j < kPcHidden; ++j) a = fmaf(D2[s * kPcHidden + j], W[N.oW2 + j * kPcHidden + k], a);
        D1[i] = A1[i] > 0.f ? a : 0.f;
    }
    __syncthreads();
    // parameter gradients (sums over the block's samples in sample order)
    float* gp = grad_part + (size_t)blockIdx.x * N.P;
    for (int p = t; p < N.P; p += nt) {
        float g = 0.f;
        if (p < N.ob1) {
            const int j = p / nin, k = p % nin;
            for (int s = 0; s < tb; ++s) g = fmaf(D1[s * kPcHidden + j], X[s * nin + k], g);
        } else if (p < N.oW2) {
            const int j = p - N.ob1;
            for (int s = 0; s < tb; ++s) g += D1[s * kPcHidden + j];
        } else if (p < N.ob2) {
            const int j = (p - N.oW2) / kPcHidden, k = (p - N.oW2) % kPcHidden;
            for (int s = 0; s < tb; ++s) g = fmaf(D2[s * kPcHidden + j], fmaxf(A1[s * kPcHidden + k], 0.f), g);
        } else if (p < N.oW3) {
            const int j = p - N.ob2;
            for (int s = 0; s < tb; ++s) g += D2[s * kPcHidden + j];
        } else if (p < N.ob3) {
            const int o = (p - N.oW3) / kPcHidden, j = (p - N.oW3) % kPcHidden;
            for (int s = 0; s < tb; ++s) g = fmaf(E[s * NO + o], fmaxf(A2[s * kPcHidden + j], 0.f), g);
        } else {
            const int o = p - N.ob3;
            for (int s = 0; s < tb; ++s) g += E[s * NO + o];
        }
        gp[p] = g;
    }
    if (t == 0) {
        double a = 0.0;
        for (int i = 0; i < tb; ++i) a += lsum[i];
        loss_part[blockIdx.x] = a;
    }
}

// Sum the per-block partials (fixed order) and take one Adam step on the FP32 master
// weights; refresh their BF16-rounded copies.  grad_out (optional) receives the gradient.
__global__ void k_pc_adam(float* theta, float* theta_bf, float* m1, float* m2, const float* grad_part, int nb, int P,
                          float lr, float bc1, float bc2, const double* loss_part, double* loss_out, double lscale,
                          float* grad_out) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p == 0 && loss_out) {
        double a = 0.0;
        for (int b = 0; b < nb; ++b) a += loss_part[b];
        *loss_out = a * lscale;
    }
    if (p >= P) return;
    float g = 0.f;
    for (int b = 0; b < nb; ++b) g += grad_part[(size_t)b * P + p];
    if (grad_out) {
        grad_out[p] = g;
        return;
    }
    const float a = 0.9f * m1[p] + 0.1f * g;
    const float b2 = 0.999f * m2[p] + 0.001f * g * g;
    m1[p] = a;
    m2[p] = b2;
    const float th = theta[p] - lr * (a / bc1) / (sqrtf(b2 / bc2) + 1e-8f);
    theta[p] = th;
    theta_bf[p] = __bfloat162float(__float2bfloat16_rn(th));
}

__global__ void k_bf16_round(const float* in, float* out, int n) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] = __bfloat162float(__float2bfloat16_rn(in[i]));
}

// ---------------------------------------------------------------- transpose of G

__global__ void k_gt_count(const int32_t* gcol, int64_t N, int32_t* cnt) {
    const int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (s >= N) return;
    for (int k = 0; k < kPcOut; ++k) {
        const int32_t c = gcol[k * N + s];
        if (c >= 0) atomicAdd(&cnt[c], 1);
    }
}
__global__ void k_gt_fill(const int32_t* gcol, const __half* gval, int64_t N, const int64_t* rp, int32_t* cursor,
                          int32_t* col, __half* val) {
    const int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (s >= N) return;
    for (int k = 0; k < kPcOut; ++k) {
        const int32_t c = gcol[k * N + s];
        if (c < 0) continue;
        const int64_t pos = rp[c] + atomicAdd(&cursor[c], 1);
        col[pos] = (int32_t)s;
        val[pos] = gval[k * N + s];
    }
}
// deterministic order inside each row of G^T: by source row.  One warp per row: for rows of up
// to 32 kGtPL entries (all but pathological ones) lane i holds entries i, i + 32, ... and writes
// each at its rank among the row's source rows (all distinct: a row of G names each column
// once), counted against every entry of the row by shuffles; longer rows are sorted in place by
// one lane.
constexpr int kGtPL = 8;
__global__ void k_gt_sort(const int64_t* rp, int32_t* col, __half* val, int64_t N) {
    const int64_t c = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (c >= N) return;  // warp-uniform
    const int64_t s = rp[c], e = rp[c + 1];
    const int n = (int)(e - s);
    if (n <= 1) return;
    if (n <= 32 * kGtPL) {
        int32_t mc[kGtPL];
        __half mv[kGtPL];
        int rank[kGtPL];
#pragma unroll
        for (int t = 0; t < kGtPL; ++t) {
            const int i = lane + 32 * t;
            mc[t] = i < n ? col[s + i] : INT_MAX;
            mv[t] = i < n ? val[s + i] : __float2half_rn(0.f);
            rank[t] = 0;
        }
#pragma unroll
        for (int u = 0; u < kGtPL; ++u) {
            if (32 * u >= n) break;  // warp-uniform
            for (int j = 0; j < 32; ++j) {
                const int32_t o = __shfl_sync(0xffffffffu, mc[u], j);
#pragma unroll
                for (int t = 0; t < kGtPL; ++t) rank[t] += o < mc[t] ? 1 : 0;
            }
        }
        __syncwarp();  // every lane has read its entries before any lane writes
#pragma unroll
        for (int t = 0; t < kGtPL; ++t)
            if (lane + 32 * t < n) {
                col[s + rank[t]] = mc[t];
                val[s + rank[t]] = mv[t];
            }
        return;
    }
    if (lane != 0) return;
    for (int64_t i = s + 1; i < e; ++i) {
        const int32_t kc = col[i];
        const __half kv = val[i];
        int64_t j = i - 1;
        while (j >= s && col[j] > kc) {
            col[j + 1] = col[j];
            val[j + 1] = val[j];
            --j;
        }
        col[j + 1] = kc;
        val[j + 1] = kv;
    }
}


uint64_t sm64(uint64_t seed, uint64_t i) {
    uint64_t z = seed + (i + 1) * 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}
double u01(uint64_t seed, uint64_t i) { return (double)(sm64(seed, i) >> 11) * (1.0 / 9007199254740992.0); }

uint64_t gcd64(uint64_t a, uint64_t b) {
    while (b) {
        const uint64_t t = a % b;
        a = b;
        b = t;
    }
    return a;
}

// G rows (gval/gcol) or, with ghat_out, the scale-free rows of every point from the network.
// uc_out (optional, device [N][17 m]): also a copy of the candidate rows (sorted order).
ms_status launch_infer(ms_hierarchy* h, __half* gval, int32_t* gcol, float* ghat_out, cudaStream_t st,
                       float* uc_out = nullptr) {
    const Precond& pc = h->pc;
    const int m = pc.nbasis;
    const int64_t N = h->N;
    const float* th = pc.fp32_weights ? pc.theta : pc.theta_bf;
    // candidate rows, features and patch sizes of every point (scratch from the library pool)
    float *Uc = nullptr, *Zc = nullptr;
    int32_t* cnt = nullptr;
    MS_TRY(ms_tmp_alloc((void**)&Uc, sizeof(float) * (size_t)N * kPcOut * m, st));
    ms_status s = ms_tmp_alloc((void**)&Zc, sizeof(float) * (size_t)N * pc.n_in, st);
    if (s == MS_OK) s = ms_tmp_alloc((void**)&cnt, sizeof(int32_t) * (size_t)N, st);
    if (s == MS_OK) {
        cudaError_t e = cudaSuccess;
        if (pc.fp32_weights) {  // FP32 weights: the FP32 network on the CUDA cores
            const size_t smem = cand_smem(pc.n_in, m);
            e = cudaFuncSetAttribute(k_pc_cand, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
            if (e == cudaSuccess) {
                k_pc_cand<<<nblk(N, kCandBS), kCandBS, smem, st>>>(h->view, pc.nbr, th, m, pc.musig, Uc, Zc, cnt);
                ms_count_launch();
            }
        } else {  // BF16-valued weights: features, then the network on the tensor cores
            const MlpSmem S = mlp_smem(pc.n_in, m);
            int sms = 0;
            e = cudaFuncSetAttribute(k_pc_mlp, cudaFuncAttributeMaxDynamicSharedMemorySize, S.total);
            if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, h->device);
            if (e == cudaSuccess) e = cudaMemsetAsync(pc.tcstat, 0, sizeof(int), st);
            if (e == cudaSuccess) {
                k_pc_features<<<nblk(N, 128), 128, 0, st>>>(h->view, pc.nbr, nullptr, N, Zc, cnt);
                const int64_t tiles = (N + kMlpRows - 1) / kMlpRows;
                const unsigned grid = (unsigned)std::max<int64_t>(1, std::min<int64_t>(tiles, 2 * (int64_t)sms));
                k_pc_mlp<<<grid, kMlpRows, S.total, st>>>(th, pc.n_in, m, pc.musig, Zc, cnt, N, Uc, pc.tcstat);
                ms_count_launch(2);
            }
        }
        if (e == cudaSuccess && uc_out)
            e = cudaMemcpyAsync(uc_out, Uc, sizeof(float) * (size_t)N * kPcOut * m, cudaMemcpyDeviceToDevice, st);
        if (e == cudaSuccess && (gval || ghat_out)) {
            const WendlandPoly& wp = h->view.w;
            const float4 wc = make_float4((float)wp.c[0], (float)wp.c[1], (float)wp.c[2], (float)wp.c[3]);
            k_pc_combine<<<nblk(N, kCombPts), kCombPts * 16, 0, st>>>(h->view, wc, pc.nbr, m, Uc, Zc, cnt, gval,
                                                                 gcol, ghat_out);
            ms_count_launch();
            e = cudaGetLastError();
        }
        if (e != cudaSuccess) s = ms_cuda_error(e, "network rows", __FILE__, __LINE__);
    }
    if (Uc) cudaFreeAsync(Uc, st);
    if (Zc) cudaFreeAsync(Zc, st);
    if (cnt) cudaFreeAsync(cnt, st);
    return s;
}

ms_status pc_alloc(ms_hierarchy* h) {
    Precond& pc = h->pc;
    if (pc.nbr) return MS_OK;
    pc.n_in = kPcK * h->d;
    pc.n_params = net_layout(pc.n_in, pc.nbasis).P;
    const int pmax = net_layout(pc.n_in, kPcMaxBasis).P;  // room for any candidate count
    const int64_t N = h->N;
    MS_TRY(ms_alloc(h, (void**)&pc.nbr, sizeof(int32_t) * N * kPcK));
    MS_TRY(ms_alloc(h, (void**)&pc.gcol, sizeof(int32_t) * N * kPcOut));
    MS_TRY(ms_alloc(h, (void**)&pc.gval, sizeof(__half) * N * kPcOut));
    MS_TRY(ms_alloc(h, (void**)&pc.gt_rp, sizeof(int64_t) * (N + 1)));
    MS_TRY(ms_alloc(h, (void**)&pc.gt_col, sizeof(int32_t) * N * kPcOut));
    MS_TRY(ms_alloc(h, (void**)&pc.gt_val, sizeof(__half) * N * kPcOut));
    MS_TRY(ms_alloc(h, (void**)&pc.theta, sizeof(float) * pmax));
    MS_TRY(ms_alloc(h, (void**)&pc.theta_bf, sizeof(float) * pmax));
    MS_TRY(ms_alloc(h, (void**)&pc.adam_m, sizeof(float) * pmax));
    MS_TRY(ms_alloc(h, (void**)&pc.adam_v, sizeof(float) * pmax));
    MS_TRY(ms_alloc(h, (void**)&pc.musig, sizeof(float) * 2 * kPcOut));
    MS_TRY(ms_alloc(h, (void**)&pc.tcstat, sizeof(int)));
    MS_CUDA(cudaMemset(pc.tcstat, 0, sizeof(int)));
    return MS_OK;
}

ms_status pc_pattern(ms_hierarchy* h, cudaStream_t st) {
    MS_TRY(pc_alloc(h));
    k_pc_pattern<<<nblk(h->N, kPatW), kPatW * 32, 0, st>>>(h->view, h->W, h->cellid, h->A.rp, h->A.col, h->perm,
                                                            h->pc.nbr);
    ms_count_launch();
    MS_CUDA(cudaGetLastError());
    return MS_OK;
}

// sorted rows of the given (0-based) levels, in level order
std::vector<int64_t> level_rows(const ms_hierarchy* h, const int* levels, int n) {
    std::vector<int64_t> rows;
    for (int i = 0; i < n; ++i) {
        const int l = levels[i];
        for (int64_t s = h->view.off[l]; s < h->view.off[l + 1]; ++s) rows.push_back(s);
    }
    return rows;
}

ms_status check_levels(const ms_hierarchy* h, const int* levels, int n) {
    if (n < 1 || !levels) {
        ms_set_error(MS_ERR_ARG, "at least one training level is required");
        return MS_ERR_ARG;
    }
    for (int i = 0; i < n; ++i)
        if (levels[i] < 0 || levels[i] >= h->L) {
            ms_set_error(MS_ERR_ARG, "level %d out of range 0..%d", levels[i], h->L - 1);
            return MS_ERR_ARG;
        }
    return MS_OK;
}

// Training samples of the chosen levels: features, counts, exact targets, standardisation.
struct TrainSet {
    int64_t S = 0;
    std::vector<void*> bufs;
    float *Z = nullptr, *K = nullptr;
    int32_t* cnt = nullptr;
    double* ghat = nullptr;
    double* qstar = nullptr;   // [S] (K^-1)_11 of each patch
    int64_t* rows = nullptr;   // centre (sorted row) of each patch
    int32_t* nbr = nullptr;    // [S][16] neighbours of each patch (sorted rows, -1 = none)
    ~TrainSet() {
        for (void* p : bufs) cudaFree(p);
    }
    ms_status alloc(void** p, size_t b) {
        cudaError_t e = cudaMalloc(p, std::max<size_t>(b, 16));
        if (e != cudaSuccess) {
            ms_set_error(MS_ERR_OOM, "device allocation of %zu bytes failed", b);
            return MS_ERR_OOM;
        }
        bufs.push_back(*p);
        return MS_OK;
    }
};

constexpr uint64_t kAugSalt = 0x6175676D656E74ull;

// Training patches of the given levels: the pattern of every point (in input order), then
// `augment` extra patches per point (draw r: the nearest points below a random prefix bound).
// centre[i] / bound[i]: sorted row and input-index bound of patch i (host copies).
ms_status patch_list(ms_hierarchy* h, const int* levels, int n, int augment, uint64_t seed,
                     std::vector<int64_t>& centre, std::vector<int64_t>& bound) {
    centre.clear();
    bound.clear();
    std::vector<int64_t> lvl;  // level of each pattern patch
    for (int a = 0; a < n; ++a) {
        const int l = levels[a];
        const int64_t o = h->view.off[l], nl = h->view.off[l + 1] - o;
        std::vector<int32_t> perm(nl);
        MS_CUDA(cudaMemcpy(perm.data(), h->perm + o, sizeof(int32_t) * nl, cudaMemcpyDeviceToHost));
        std::vector<int64_t> inv(nl);
        for (int64_t k = 0; k < nl; ++k) inv[perm[k] - o] = o + k;  // input index -> sorted row
        for (int64_t k = 0; k < nl; ++k) {
            centre.push_back(inv[k]);
            bound.push_back(o + k);
            lvl.push_back(l);
        }
    }
    const int64_t S0 = (int64_t)centre.size();
    for (int r = 0; r < augment; ++r)
        for (int64_t k = 0; k < S0; ++k) {
            const int l = (int)lvl[k];
            const int64_t o = h->view.off[l], nl = h->view.off[l + 1] - o;
            const int64_t gi = bound[k];  // the centre's input index
            const int64_t i = gi - o, m = nl - i;
            const double u = u01(seed ^ kAugSalt, (uint64_t)r * (uint64_t)h->N + (uint64_t)gi);
            const int64_t p = i + 1 + std::min((int64_t)std::floor(u * (double)m), m - 1);
            centre.push_back(centre[k]);
            bound.push_back(o + p);
        }
    return MS_OK;
}

ms_status make_trainset(ms_hierarchy* h, const int* levels, int n, bool set_moments, int augment, uint64_t seed,
                        TrainSet& ts, cudaStream_t st) {
    MS_TRY(check_levels(h, levels, n));
    MS_TRY(pc_pattern(h, st));
    std::vector<int64_t> rows, bounds;
    MS_TRY(patch_list(h, levels, n, augment, seed, rows, bounds));
    ts.S = (int64_t)rows.size();
    const int nin = h->pc.n_in;
    int64_t* dbound = nullptr;
    MS_TRY(ts.alloc((void**)&ts.rows, sizeof(int64_t) * ts.S));
    MS_TRY(ts.alloc((void**)&dbound, sizeof(int64_t) * ts.S));
    MS_TRY(ts.alloc((void**)&ts.nbr, sizeof(int32_t) * ts.S * kPcK));
    MS_TRY(ts.alloc((void**)&ts.Z, sizeof(float) * ts.S * nin));
    MS_TRY(ts.alloc((void**)&ts.qstar, sizeof(double) * ts.S));
    MS_TRY(ts.alloc((void**)&ts.cnt, sizeof(int32_t) * ts.S));
    MS_TRY(ts.alloc((void**)&ts.ghat, sizeof(double) * ts.S * kPcOut));
    MS_TRY(ts.alloc((void**)&ts.K, sizeof(float) * ts.S * kPcOut * kPcOut));
    MS_CUDA(cudaMemcpyAsync(ts.rows, rows.data(), sizeof(int64_t) * ts.S, cudaMemcpyHostToDevice, st));
    MS_CUDA(cudaMemcpyAsync(dbound, bounds.data(), sizeof(int64_t) * ts.S, cudaMemcpyHostToDevice, st));
    k_pc_patches<<<nblk(ts.S, kPatW), kPatW * 32, 0, st>>>(h->view, h->W, h->cellid, h->A.rp, h->A.col, h->perm,
                                                            ts.rows, dbound, ts.S, ts.nbr);
    k_pc_features<<<nblk(ts.S, 128), 128, 0, st>>>(h->view, ts.nbr, ts.rows, ts.S, ts.Z, ts.cnt);
    k_pc_patchK<<<nblk(ts.S, 128), 128, 0, st>>>(h->view, ts.nbr, ts.rows, ts.S, ts.K);
    ms_count_launch(3);
    k_pc_exact<<<nblk(ts.S, 64), 64, 0, st>>>(h->view, ts.nbr, ts.rows, ts.S, ts.ghat, nullptr, nullptr);
    ms_count_launch();
    if (set_moments) {
        k_pc_moments<<<kPcOut, 256, 0, st>>>(ts.ghat, ts.cnt, ts.S, h->pc.musig);
        ms_count_launch();
    }
    k_pc_qstar<<<nblk(ts.S, 128), 128, 0, st>>>(ts.ghat, ts.S, ts.qstar);
    ms_count_launch();
    MS_CUDA(cudaGetLastError());
    // the host arrays go out of scope: the copies must be complete
    MS_CUDA(cudaStreamSynchronize(st));
    return MS_OK;
}

size_t train_smem(int nin, int m) { return sizeof(float) * (size_t)train_layout(nin, m, train_tb(m)).total; }

ms_status set_train_smem(int nin, int m) {
    MS_CUDA(cudaFuncSetAttribute(k_pc_train, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)train_smem(nin, m)));
    return MS_OK;
}

}  // namespace

// Build G (and its transpose) for the requested kind; cached until the weights change.
ms_status ms_pc_build(ms_hierarchy* h, int kind, cudaStream_t st) {
    if (h->pc.built_kind == kind) return MS_OK;
    if (kind == MS_PRECOND_LEARNED && !h->pc.trained) {
        ms_set_error(MS_ERR_STATE, "precond = LEARNED needs a trained network (ms_train_precond or ms_precond_params)");
        return MS_ERR_STATE;
    }
    MS_TRY(pc_pattern(h, st));
    Precond& pc = h->pc;
    const int64_t N = h->N;
    if (kind == MS_PRECOND_EXACT) {
        k_pc_exact<<<nblk(N, 64), 64, 0, st>>>(h->view, pc.nbr, nullptr, N, nullptr, pc.gval, pc.gcol);
        ms_count_launch();
    } else {
        MS_TRY(launch_infer(h, pc.gval, pc.gcol, nullptr, st));
    }
    MS_CUDA(cudaGetLastError());
    // transpose (in-pattern) for z = G^T u
    int32_t* cnt = nullptr;
    int64_t* tiles = nullptr;
    MS_CUDA(cudaMallocAsync((void**)&cnt, sizeof(int32_t) * (N + 1), st));
    MS_CUDA(cudaMallocAsync((void**)&tiles, sizeof(int64_t) * ((N + kScanTile - 1) / kScanTile + 2), st));
    MS_CUDA(cudaMemsetAsync(cnt, 0, sizeof(int32_t) * (N + 1), st));
    k_gt_count<<<nblk(N, 256), 256, 0, st>>>(pc.gcol, N, cnt);
    exclusive_scan<int32_t, int64_t>(cnt, N, pc.gt_rp, tiles, st);
    MS_CUDA(cudaMemsetAsync(cnt, 0, sizeof(int32_t) * (N + 1), st));
    k_gt_fill<<<nblk(N, 256), 256, 0, st>>>(pc.gcol, pc.gval, N, pc.gt_rp, cnt, pc.gt_col, pc.gt_val);
    k_gt_sort<<<nblk(N * 32, 256), 256, 0, st>>>(pc.gt_rp, pc.gt_col, pc.gt_val, N);
    ms_count_launch(3);
    MS_CUDA(cudaFreeAsync(cnt, st));
    MS_CUDA(cudaFreeAsync(tiles, st));
    MS_CUDA(cudaGetLastError());
    pc.built_kind = kind;
    return MS_OK;
}

// ---------------------------------------------------------------- C ABI

extern "C" {

void ms_default_train_opts(ms_train_opts* o) {
    if (!o) return;
    std::memset(o, 0, sizeof(*o));
    o->epochs = 100;
    o->batch = 512;
    o->lr = 3e-3;
    o->lr_final = 1e-4;
    o->seed = 2503049140ull;
    o->input_noise = 0.005f;
    o->augment = 4;
    o->n_basis = kPcBasisDefault;
}

ms_status ms_train_precond(ms_hierarchy* h, const int* levels, int n_levels, const ms_train_opts* opts,
                           ms_train_stats* stats) {
    if (!h) {
        ms_set_error(MS_ERR_ARG, "NULL handle");
        return MS_ERR_ARG;
    }
    ms_train_opts o;
    ms_default_train_opts(&o);
    if (opts) o = *opts;
    if (o.n_basis == 0) o.n_basis = kPcBasisDefault;
    if (o.epochs < 1 || o.batch < 64 || o.batch % 64 != 0 || !(o.lr > 0.0) || o.augment < 0 || o.augment > 16 ||
        o.n_basis < 1 || o.n_basis > kPcMaxBasis) {
        ms_set_error(MS_ERR_ARG, "epochs >= 1, batch a positive multiple of 64, lr > 0, augment in 0..16 and n_basis "
                     "in 1..%d are required", kPcMaxBasis);
        return MS_ERR_ARG;
    }
    cudaStream_t st;
    MS_CUDA(cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking));
    struct StreamGuard {
        cudaStream_t s;
        ~StreamGuard() { cudaStreamSynchronize(s); cudaStreamDestroy(s); }
    } guard{st};
    MS_TRY(pc_alloc(h));
    Precond& pc = h->pc;
    TrainSet ts;
    MS_TRY(make_trainset(h, levels, n_levels, true, o.augment, o.seed, ts, st));
    pc.augment = o.augment;
    pc.seed = o.seed;
    const int m = o.n_basis;
    pc.nbasis = m;
    pc.n_params = net_layout(pc.n_in, m).P;
    // initial weights: U(-1/sqrt(fan_in), 1/sqrt(fan_in)) from SplitMix64(seed), parameter order
    const NetLayout N = net_layout(pc.n_in, m);
    std::vector<float> th(N.P);
    for (int p = 0; p < N.P; ++p) {
        const int fan = p < N.oW2 ? pc.n_in : kPcHidden;
        const double b = 1.0 / std::sqrt((double)fan);
        th[p] = (float)(-b + 2.0 * b * u01(o.seed, (uint64_t)p));
    }
    MS_CUDA(cudaMemcpyAsync(pc.theta, th.data(), sizeof(float) * N.P, cudaMemcpyHostToDevice, st));
    MS_CUDA(cudaMemsetAsync(pc.adam_m, 0, sizeof(float) * N.P, st));
    MS_CUDA(cudaMemsetAsync(pc.adam_v, 0, sizeof(float) * N.P, st));
    k_bf16_round<<<nblk(N.P, 256), 256, 0, st>>>(pc.theta, pc.theta_bf, N.P);
    ms_count_launch();
    pc.fp32_weights = o.fp32_weights;
    MS_TRY(set_train_smem(pc.n_in, m));
    const int nb = o.batch / train_tb(m);
    const int64_t steps_per_epoch = (ts.S + o.batch - 1) / o.batch;
    const int64_t steps = steps_per_epoch * o.epochs;
    float* grad_part = nullptr;
    double *loss_part = nullptr, *loss_hist = nullptr;
    MS_TRY(ts.alloc((void**)&grad_part, sizeof(float) * nb * N.P));
    MS_TRY(ts.alloc((void**)&loss_part, sizeof(double) * nb));
    MS_TRY(ts.alloc((void**)&loss_hist, sizeof(double) * 2));
    cudaEvent_t e0, e1;
    MS_CUDA(cudaEventCreate(&e0));
    MS_CUDA(cudaEventCreate(&e1));
    MS_CUDA(cudaEventRecord(e0, st));
    const size_t smem = train_smem(pc.n_in, m);
    const float escale = 1.0f / (float)o.batch;
    const double lscale = 1.0 / (double)o.batch;
    const double lr_final = o.lr_final > 0 ? o.lr_final : o.lr / 30.0;
    uint64_t a_mul = 1, a_add = 0;
    for (int64_t step = 0; step < steps; ++step) {
        const int64_t epoch = step / steps_per_epoch;
        if (step % steps_per_epoch == 0) {  // new affine shuffle of the samples for this epoch
            a_mul = (sm64(o.seed ^ 0x5DEECE66Dull, 2 * epoch) % (uint64_t)ts.S) | 1ull;
            while (gcd64(a_mul, (uint64_t)ts.S) != 1) a_mul += 2;
            a_add = sm64(o.seed ^ 0x5DEECE66Dull, 2 * epoch + 1) % (uint64_t)ts.S;
        }
        const double frac = (double)step / (double)std::max<int64_t>(steps - 1, 1);
        const float lr = (float)(lr_final + 0.5 * (o.lr - lr_final) * (1.0 + std::cos(M_PI * frac)));
        const int64_t local = step % steps_per_epoch;
        k_pc_train<<<nb, 256, smem, st>>>(ts.Z, ts.qstar, ts.cnt, ts.K, pc.musig, ts.S, pc.n_in, m,
                                          o.fp32_weights ? pc.theta : pc.theta_bf, o.batch, local, a_mul, a_add,
                                          INT64_MAX, escale, grad_part, loss_part, o.input_noise,
                                          sm64(o.seed ^ 0x6E6F697365ull, (uint64_t)epoch));
        const float bc1 = 1.0f - std::pow(0.9f, (float)(step + 1)), bc2 = 1.0f - std::pow(0.999f, (float)(step + 1));
        double* lo = step == 0 ? loss_hist : (step == steps - 1 ? loss_hist + 1 : nullptr);
        k_pc_adam<<<nblk(N.P, 256), 256, 0, st>>>(pc.theta, pc.theta_bf, pc.adam_m, pc.adam_v, grad_part, nb, N.P, lr,
                                                  bc1, bc2, loss_part, lo, lscale, nullptr);
        ms_count_launch(2);
    }
    MS_CUDA(cudaGetLastError());
    MS_CUDA(cudaEventRecord(e1, st));
    double lh[2] = {0, 0};
    MS_CUDA(cudaMemcpyAsync(lh, loss_hist, sizeof(lh), cudaMemcpyDeviceToHost, st));
    MS_CUDA(cudaStreamSynchronize(st));
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    pc.trained = true;
    pc.built_kind = 0;
    if (stats) {
        std::memset(stats, 0, sizeof(*stats));
        stats->samples = ts.S;
        stats->steps = steps;
        stats->loss_first = lh[0];
        stats->loss_last = steps > 1 ? lh[1] : lh[0];
        stats->train_ms = ms;
        stats->n_params = N.P;
    }
    return MS_OK;
}

ms_status ms_precond_params(ms_hierarchy* h, float* params, int64_t n, int set) {
    if (!h || !params) {
        ms_set_error(MS_ERR_ARG, "NULL argument");
        return MS_ERR_ARG;
    }
    MS_TRY(pc_alloc(h));
    Precond& pc = h->pc;
    if (set) {
        // the candidate count m follows from the number of values (17 m outputs of width 64)
        int m = 0;
        for (int k = 1; k <= kPcMaxBasis; ++k)
            if (n == (int64_t)net_layout(pc.n_in, k).P + 2 * kPcOut) m = k;
        if (m == 0) {
            ms_set_error(MS_ERR_ARG, "%lld values match no network of %d inputs with 1..%d candidate rows "
                         "(%d + 1105 m weights + %d standardisation)", (long long)n, pc.n_in, kPcMaxBasis,
                         net_layout(pc.n_in, 0).P, 2 * kPcOut);
            return MS_ERR_ARG;
        }
        pc.nbasis = m;
        pc.n_params = net_layout(pc.n_in, m).P;
    } else if (n != (int64_t)pc.n_params + 2 * kPcOut) {
        ms_set_error(MS_ERR_ARG, "expected %lld values (%d weights + %d standardisation)",
                     (long long)(pc.n_params + 2 * kPcOut), pc.n_params, 2 * kPcOut);
        return MS_ERR_ARG;
    }
    if (set) {
        MS_CUDA(cudaMemcpy(pc.theta, params, sizeof(float) * pc.n_params, cudaMemcpyHostToDevice));
        MS_CUDA(cudaMemcpy(pc.musig, params + pc.n_params, sizeof(float) * 2 * kPcOut, cudaMemcpyHostToDevice));
        k_bf16_round<<<nblk(pc.n_params, 256), 256>>>(pc.theta, pc.theta_bf, pc.n_params);
        ms_count_launch();
        MS_CUDA(cudaDeviceSynchronize());
        pc.trained = true;
        pc.built_kind = 0;
    } else {
        if (!pc.trained) {
            ms_set_error(MS_ERR_STATE, "no trained network");
            return MS_ERR_STATE;
        }
        MS_CUDA(cudaMemcpy(params, pc.theta, sizeof(float) * pc.n_params, cudaMemcpyDeviceToHost));
        MS_CUDA(cudaMemcpy(params + pc.n_params, pc.musig, sizeof(float) * 2 * kPcOut, cudaMemcpyDeviceToHost));
    }
    return MS_OK;
}

ms_status ms_precond_inspect(ms_hierarchy* h, int what, const int* levels, int n_levels, void* out, int64_t n_out) {
    if (!h || !out) {
        ms_set_error(MS_ERR_ARG, "NULL argument");
        return MS_ERR_ARG;
    }
    cudaStream_t st = 0;
    const int64_t N = h->N;
    std::vector<int32_t> perm(N);
    MS_CUDA(cudaMemcpy(perm.data(), h->perm, sizeof(int32_t) * N, cudaMemcpyDeviceToHost));
    MS_TRY(pc_pattern(h, st));
    Precond& pc = h->pc;
    if (what == MS_INSPECT_CANDIDATES) {
        const int64_t w = (int64_t)kPcOut * pc.nbasis;
        if (n_out != N * w) {
            ms_set_error(MS_ERR_ARG, "expected %lld output values", (long long)(N * w));
            return MS_ERR_ARG;
        }
        if (!pc.trained) {
            ms_set_error(MS_ERR_STATE, "no trained network");
            return MS_ERR_STATE;
        }
        float* d = nullptr;
        MS_CUDA(cudaMalloc((void**)&d, sizeof(float) * N * w));
        const ms_status ls = launch_infer(h, nullptr, nullptr, nullptr, 0, d);
        std::vector<float> hd(N * w);
        cudaError_t e = ls == MS_OK ? cudaMemcpy(hd.data(), d, sizeof(float) * N * w, cudaMemcpyDeviceToHost)
                                    : cudaSuccess;
        cudaFree(d);
        if (ls != MS_OK) return ls;
        MS_CUDA(e);
        float* o = static_cast<float*>(out);
        for (int64_t s = 0; s < N; ++s) std::memcpy(o + (int64_t)perm[s] * w, hd.data() + s * w, sizeof(float) * w);
        return MS_OK;
    }
    if (what == MS_INSPECT_PATTERN || what == MS_INSPECT_TARGETS || what == MS_INSPECT_PREDICT) {
        const int width = what == MS_INSPECT_PATTERN ? kPcK : kPcOut;
        if (n_out != N * width) {
            ms_set_error(MS_ERR_ARG, "expected %lld output values", (long long)(N * width));
            return MS_ERR_ARG;
        }
        std::vector<int32_t> nb(N * kPcK);
        MS_CUDA(cudaMemcpy(nb.data(), pc.nbr, sizeof(int32_t) * N * kPcK, cudaMemcpyDeviceToHost));
        if (what == MS_INSPECT_PATTERN) {
            int32_t* o = static_cast<int32_t*>(out);
            for (int64_t s = 0; s < N; ++s)
                for (int k = 0; k < kPcK; ++k) {
                    const int32_t c = nb[s * kPcK + k];
                    o[(int64_t)perm[s] * kPcK + k] = c >= 0 ? perm[c] : -1;
                }
            return MS_OK;
        }
        if (what == MS_INSPECT_TARGETS) {
            double* d = nullptr;
            MS_CUDA(cudaMalloc((void**)&d, sizeof(double) * N * kPcOut));
            k_pc_exact<<<nblk(N, 64), 64>>>(h->view, pc.nbr, nullptr, N, d, nullptr, nullptr);
            ms_count_launch();
            std::vector<double> hd(N * kPcOut);
            cudaError_t e = cudaMemcpy(hd.data(), d, sizeof(double) * N * kPcOut, cudaMemcpyDeviceToHost);
            cudaFree(d);
            MS_CUDA(e);
            double* o = static_cast<double*>(out);
            for (int64_t s = 0; s < N; ++s)
                std::memcpy(o + (int64_t)perm[s] * kPcOut, hd.data() + s * kPcOut, sizeof(double) * kPcOut);
            return MS_OK;
        }
        if (!pc.trained) {
            ms_set_error(MS_ERR_STATE, "no trained network");
            return MS_ERR_STATE;
        }
        float* d = nullptr;
        MS_CUDA(cudaMalloc((void**)&d, sizeof(float) * N * kPcOut));
        {
            const ms_status ls = launch_infer(h, nullptr, nullptr, d, 0);
            if (ls != MS_OK) {
                cudaFree(d);
                return ls;
            }
        }
        std::vector<float> hd(N * kPcOut);
        cudaError_t e = cudaMemcpy(hd.data(), d, sizeof(float) * N * kPcOut, cudaMemcpyDeviceToHost);
        cudaFree(d);
        MS_CUDA(e);
        float* o = static_cast<float*>(out);
        for (int64_t s = 0; s < N; ++s)
            std::memcpy(o + (int64_t)perm[s] * kPcOut, hd.data() + s * kPcOut, sizeof(float) * kPcOut);
        return MS_OK;
    }
    if (what == MS_INSPECT_GRAD) {
        // full-batch loss and gradient over the given levels with the FP32 master weights,
        // using the current standardisation (out: n_params gradient values, then the loss)
        if (!pc.trained) {
            ms_set_error(MS_ERR_STATE, "no network weights");
            return MS_ERR_STATE;
        }
        if (n_out != pc.n_params + 1) {
            ms_set_error(MS_ERR_ARG, "expected %d output values", pc.n_params + 1);
            return MS_ERR_ARG;
        }
        TrainSet ts;
        MS_TRY(make_trainset(h, levels, n_levels, false, 0, pc.seed, ts, st));
        const int tb = train_tb(pc.nbasis);
        const int nb = (int)((ts.S + tb - 1) / tb);
        const NetLayout Nl = net_layout(pc.n_in, pc.nbasis);
        float *gp = nullptr, *gout = nullptr;
        double *lp = nullptr, *lo = nullptr;
        MS_TRY(ts.alloc((void**)&gp, sizeof(float) * nb * Nl.P));
        MS_TRY(ts.alloc((void**)&gout, sizeof(float) * Nl.P));
        MS_TRY(ts.alloc((void**)&lp, sizeof(double) * nb));
        MS_TRY(ts.alloc((void**)&lo, sizeof(double)));
        MS_TRY(set_train_smem(pc.n_in, pc.nbasis));
        k_pc_train<<<nb, 256, train_smem(pc.n_in, pc.nbasis), st>>>(ts.Z, ts.qstar, ts.cnt, ts.K, pc.musig, ts.S,
                                                                    pc.n_in, pc.nbasis, pc.theta, nb * tb, 0, 1, 0,
                                                                    ts.S, 1.0f / (float)ts.S, gp, lp, 0.f, 0ull);
        k_pc_adam<<<nblk(Nl.P, 256), 256, 0, st>>>(nullptr, nullptr, nullptr, nullptr, gp, nb, Nl.P, 0.f, 1.f, 1.f, lp,
                                                   lo, 1.0 / (double)ts.S, gout);
        ms_count_launch(2);
        MS_CUDA(cudaGetLastError());
        float* o = static_cast<float*>(out);
        MS_CUDA(cudaMemcpy(o, gout, sizeof(float) * Nl.P, cudaMemcpyDeviceToHost));
        double l = 0;
        MS_CUDA(cudaMemcpy(&l, lo, sizeof(double), cudaMemcpyDeviceToHost));
        o[Nl.P] = (float)l;
        return MS_OK;
    }
    if (what == MS_INSPECT_PATCHES) {
        MS_TRY(check_levels(h, levels, n_levels));
        std::vector<int64_t> rows, bounds;
        MS_TRY(patch_list(h, levels, n_levels, pc.augment, pc.seed, rows, bounds));
        const int64_t S = (int64_t)rows.size();
        if (n_out != S * 18) {
            ms_set_error(MS_ERR_ARG, "expected %lld output values", (long long)(S * 18));
            return MS_ERR_ARG;
        }
        TrainSet ts;
        int64_t* dbound = nullptr;
        MS_TRY(ts.alloc((void**)&ts.rows, sizeof(int64_t) * S));
        MS_TRY(ts.alloc((void**)&dbound, sizeof(int64_t) * S));
        MS_TRY(ts.alloc((void**)&ts.nbr, sizeof(int32_t) * S * kPcK));
        MS_CUDA(cudaMemcpy(ts.rows, rows.data(), sizeof(int64_t) * S, cudaMemcpyHostToDevice));
        MS_CUDA(cudaMemcpy(dbound, bounds.data(), sizeof(int64_t) * S, cudaMemcpyHostToDevice));
        k_pc_patches<<<nblk(S, kPatW), kPatW * 32>>>(h->view, h->W, h->cellid, h->A.rp, h->A.col, h->perm, ts.rows,
                                                      dbound, S, ts.nbr);
        ms_count_launch();
        MS_CUDA(cudaGetLastError());
        std::vector<int32_t> nb(S * kPcK);
        MS_CUDA(cudaMemcpy(nb.data(), ts.nbr, sizeof(int32_t) * S * kPcK, cudaMemcpyDeviceToHost));
        int32_t* o = static_cast<int32_t*>(out);
        for (int64_t i = 0; i < S; ++i) {
            const int64_t s = rows[i];
            int l = 0;
            while (l + 1 < h->L && s >= h->view.off[l + 1]) ++l;
            o[i * 18] = perm[s];
            o[i * 18 + 1] = (int32_t)(bounds[i] - h->view.off[l]);
            for (int k = 0; k < kPcK; ++k) {
                const int32_t c = nb[i * kPcK + k];
                o[i * 18 + 2 + k] = c >= 0 ? perm[c] : -1;
            }
        }
        return MS_OK;
    }
    ms_set_error(MS_ERR_ARG, "unknown inspection %d", what);
    return MS_ERR_ARG;
}

}  // extern "C"
