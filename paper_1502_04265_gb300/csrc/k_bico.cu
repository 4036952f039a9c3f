// k_bico.cu -- batched weighted nearest-reference query against a snapshot of BICO-style
// clustering features (Section 2.1: a feature (N, S, Q) of a point set gives its size, the sum of
// its points and the sum of their squared lengths; Section 2.3.1: a weighted point (x, w) stands for
// w copies of x, its nearest reference is found once, and the feature takes
//   w' = w                                            if s ||x - mu||^2 - T + c <= 0,
//   w' = min(w, (s T - s c) / (s ||x - mu||^2 - T + c)) otherwise,
// copies, s, mu and c being the feature's size, centroid and error, T the threshold).
//
// The nearest reference is the assignment step against the reference points (kmeans_assign: the
// tensor-core distance GEMM with its certified near-tie recheck).  Then one prep kernel turns every
// feature into (mu_j, c_j) in FP64 and one kernel per point evaluates ||x - mu_j||^2 and w' in FP64,
// with every rounding step of the rule written out (no contraction into FMAs), so that the integer
// count is decided by the same FP64 operations the formula states.
#include "internal.cuh"

namespace gbkm {
namespace {

// one warp per feature: mu_j = S_j / N_j, c_j = Q_j - (S_j . S_j) / N_j (0 and mu = 0 for N_j <= 0)
__global__ void __launch_bounds__(256) k_bico_prep(const double *__restrict__ N, const double *__restrict__ S,
                                                   const double *__restrict__ Q, int64_t m, int64_t d,
                                                   double *__restrict__ mu, double *__restrict__ cerr) {
    const int64_t j = (int64_t)blockIdx.x * 8 + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    if (j >= m) return;
    const double s = N[j];
    const double *Sj = S + j * d;
    double *mj = mu + j * d;
    double ss = 0.0;
    if (s > 0.0) {
        for (int64_t t = lane; t < d; t += 32) {
            const double v = Sj[t];
            mj[t] = __ddiv_rn(v, s);
            ss = __fma_rn(v, v, ss);
        }
    } else {
        for (int64_t t = lane; t < d; t += 32) mj[t] = 0.0;
    }
    ss = warp_sum_d(ss);
    if (lane == 0) cerr[j] = s > 0.0 ? __dsub_rn(Q[j], __ddiv_rn(ss, s)) : 0.0;
}

// 32 points per warp: each point's d2 = ||x_i - mu_j||^2 (FP64, j = ref[i]) is summed by the whole warp
// (lane l takes columns l, l + 32, ...), the 32 partial sums of every lane are then reduced in one
// transposing butterfly (31 exchanges; lane p ends with point p's sum, in a fixed order), and every
// lane evaluates the insertion rule for its own point
__global__ void __launch_bounds__(256) k_bico_take(const float *__restrict__ X, int64_t n, int64_t d,
                                                   const float *__restrict__ w, const int32_t *__restrict__ ref,
                                                   const double *__restrict__ N, const double *__restrict__ mu,
                                                   const double *__restrict__ cerr, int64_t m, double T,
                                                   double *__restrict__ d2_out, double *__restrict__ take_out,
                                                   int *status) {
    const int lane = threadIdx.x & 31;
    const int64_t base = ((int64_t)blockIdx.x * 8 + (threadIdx.x >> 5)) * 32;
    if (base >= n) return;
    double part[32];
#pragma unroll
    for (int p = 0; p < 32; ++p) {
        const int64_t i = base + p;
        double acc = 0.0;
        if (i < n) {
            const int32_t j = ref[i];
            if (j >= 0 && (int64_t)j < m) {
                const float *xi = X + i * d;
                const double *mj = mu + (int64_t)j * d;
                for (int64_t t = lane; t < d; t += 32) {
                    const double df = __dsub_rn((double)xi[t], mj[t]);
                    acc = __fma_rn(df, df, acc);
                }
            }
        }
        part[p] = acc;
    }
    // after the step of width o, element q of lane l holds the sum of point q + (the bits of l at o and
    // above) over the lanes that agree with l below o
#pragma unroll
    for (int o = 16; o >= 1; o >>= 1) {
        const bool upper = (lane & o) != 0;
#pragma unroll
        for (int q = 0; q < o; ++q) {
            const double send = upper ? part[q] : part[q + o];
            const double keep = upper ? part[q + o] : part[q];
            part[q] = __dadd_rn(keep, __shfl_xor_sync(0xffffffffu, send, o));
        }
    }
    const int64_t i = base + lane;
    if (i >= n) return;
    const int32_t j = ref[i];
    if (j < 0 || (int64_t)j >= m) {
        // a label outside the references cannot come from the assignment; skip the row
        status_raise(status, ST_BOUNDS);
        return;
    }
    double acc = part[0];
    const double s = N[j], c = cerr[j];
    const double wi = w ? (double)w[i] : 1.0;
    double take;
    if (!(s > 0.0)) {
        // an empty feature has no error and gains none: the whole point fits
        acc = 0.0;
        take = wi;
    } else {
        const double den = __dadd_rn(__dsub_rn(__dmul_rn(s, acc), T), c);
        if (den <= 0.0) {
            take = wi;
        } else {
            const double q = floor(__ddiv_rn(__dsub_rn(__dmul_rn(s, T), __dmul_rn(s, c)), den));
            take = fmax(0.0, fmin(wi, q));
        }
    }
    if (d2_out) d2_out[i] = acc;
    take_out[i] = take;
}

}  // namespace
}  // namespace gbkm

extern "C" int kmeans_bico_query(gbkm_ctx *c, const void *Xop, const float *Xop_scales, const float *X,
                                 const float *xnorm, int64_t n, int64_t d, const float *w, const float *R,
                                 int64_t m, const double *N, const double *S, const double *Q, double T,
                                 const gbkm_assign_opts *opts, int32_t *ref_out, double *d2_out,
                                 double *take_out) {
    if (!c) return GBKM_EINVAL;
    if (n < 1 || d < 1 || m < 1 || m > 65536 || !X || !R || !N || !S || !Q || !ref_out || !take_out)
        return set_error(c, GBKM_EINVAL, "bico_query: bad arguments");
    if (!(T >= 0.0)) return set_error(c, GBKM_EINVAL, "bico_query: the threshold T must be >= 0");
    if ((uint64_t)m > (uint64_t)INT64_MAX / 8 / (uint64_t)d) return set_error(c, GBKM_EINVAL, "bico_query: m x d overflows");
    // the nearest reference of every point: the exact assignment step against the references
    int rc = kmeans_assign(c, Xop, Xop_scales, X, xnorm, n, d, R, m, opts, ref_out, nullptr, nullptr);
    if (rc != GBKM_OK) return rc;
    struct DeviceGuard {
        int prev = -1;
        explicit DeviceGuard(int dev) {
            cudaGetDevice(&prev);
            if (prev != dev) cudaSetDevice(dev);
        }
        ~DeviceGuard() {
            int cur = -1;
            cudaGetDevice(&cur);
            if (prev >= 0 && cur != prev) cudaSetDevice(prev);
        }
    } g(c->device);
    WsPlan p;
    const size_t o_mu = p.take<double>((size_t)m * d), o_c = p.take<double>(m);
    // (the assignment's workspace is no longer needed: ws_reserve waits for it before any regrowth)
    void *ws = ws_reserve(c, p.off, &rc);
    if (!ws) return rc;
    double *mu = ws_at<double>(ws, o_mu), *cerr = ws_at<double>(ws, o_c);
    prof_begin(c, "bico_take");
    gbkm::k_bico_prep<<<(unsigned)ceil_div(m, 8), 256, 0, c->stream>>>(N, S, Q, m, d, mu, cerr);
    GBKM_LAUNCHED(c);
    gbkm::k_bico_take<<<(unsigned)ceil_div(n, 256), 256, 0, c->stream>>>(X, n, d, w, ref_out, N, mu, cerr, m, T,
                                                                          d2_out, take_out, c->status);
    GBKM_LAUNCHED(c);
    prof_end(c);
    return cuda_check(c, cudaGetLastError(), "bico_query launch");
}
