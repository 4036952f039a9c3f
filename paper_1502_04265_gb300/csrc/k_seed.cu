// k_seed.cu -- A3 k-means++ D^2 seeding (Section 1): for each round, a fused D^2 update
// with per-block FP64 sums, then a one-CTA two-level prefix-sum sampler that writes the chosen
// row into the centers on the device.  2 launches per round, no host synchronisation.
#include "internal.cuh"

namespace gbkm {

namespace {
constexpr int SB = 128;    // rows per sampling block (one CTA of 8 warps, 16 rows per warp)
constexpr int PICK_T = 1024;
}  // namespace

// p_i = w_i * D2_i (or w_i when mode_w) summed per block of SB rows; D2 refreshed against the
// newest center c (init: D2 = distance to c).  One warp per row, rows interleaved across the
// 8 warps; the block sum runs over warps in order, each warp over its rows in order.
template <int VW>
__global__ void __launch_bounds__(256) k_d2_update(const float *__restrict__ X, int64_t n, int64_t d,
                                                   const float *__restrict__ w,
                                                   const float *__restrict__ c, int init,
                                                   double *__restrict__ D2, double *__restrict__ bsum,
                                                   const int *__restrict__ stop) {
    if (*stop) return;
    __shared__ double wsum[8];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int64_t r0 = (int64_t)blockIdx.x * SB, r1 = min(n, r0 + SB);
    double run = 0.0;
    for (int64_t i = r0 + wid; i < r1; i += 8) {
        const float *x = X + i * d;
        DF acc;
        if constexpr (VW == 4) {
            const float4 *x4 = reinterpret_cast<const float4 *>(x);
            const float4 *c4 = reinterpret_cast<const float4 *>(c);
#pragma unroll 4
            for (int64_t t = lane; t < d / 4; t += 32) {
                float4 a = __ldg(x4 + t), b = __ldg(c4 + t);
                acc.add_sqdiff(a.x, b.x);
                acc.add_sqdiff(a.y, b.y);
                acc.add_sqdiff(a.z, b.z);
                acc.add_sqdiff(a.w, b.w);
            }
        } else {
            for (int64_t t = lane; t < d; t += 32) acc.add_sqdiff(x[t], c[t]);
        }
        const double dist = warp_sum_df(acc);
        double nd = dist;
        if (!init) nd = fmin(D2[i], dist);
        if (lane == 0) D2[i] = nd;
        run += (w ? (double)w[i] : 1.0) * nd;
    }
    if (lane == 0) wsum[wid] = run;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int q = 0; q < 8; ++q) s += wsum[q];
        bsum[blockIdx.x] = s;
    }
}

// block sums of w (first center of a weighted run)
__global__ void __launch_bounds__(256) k_wsum(const float *__restrict__ w, int64_t n,
                                              double *__restrict__ bsum) {
    __shared__ double sh[256];
    const int64_t r0 = (int64_t)blockIdx.x * SB, r1 = min(n, r0 + SB);
    double s = 0.0;
    for (int64_t i = r0 + threadIdx.x; i < r1; i += 256) s += (double)w[i];
    sh[threadIdx.x] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int q = 0; q < 256; ++q) t += sh[q];
        bsum[blockIdx.x] = t;
    }
}

__device__ double block_incl_scan_d(double v, double *sh) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    double x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        double y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) sh[wid] = x;
    __syncthreads();
    if (wid == 0) {
        double s = lane < nw ? sh[lane] : 0.0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            double y = __shfl_up_sync(0xffffffffu, s, o);
            if (lane >= o) s += y;
        }
        sh[lane] = s;
    }
    __syncthreads();
    double r = x + (wid > 0 ? sh[wid - 1] : 0.0);
    __syncthreads();
    return r;
}

// One CTA: choose the row for round j.  mode_w: p_i = w_i (weighted first center), else
// p_i = w_i * D2_i.  Blocks: prefix of the block sums; within the block: inclusive prefix in
// row order.  Chosen = smallest i whose global inclusive prefix exceeds t = u_j * total; if
// rounding leaves none, the last i with p_i > 0.  Writes idx_out[j], the center row, D2_i = 0.
__global__ void __launch_bounds__(PICK_T) k_pick(const float *__restrict__ X, int64_t n, int64_t d,
                                                 const float *__restrict__ w,
                                                 double *__restrict__ D2, const double *__restrict__ bsum,
                                                 int64_t nb, const double *__restrict__ u, int64_t j,
                                                 int mode_w, int64_t *__restrict__ idx_out,
                                                 float *__restrict__ C_out, int *stop, int *status) {
    __shared__ double sh[32];
    __shared__ int64_t s_block, s_idx;
    __shared__ double s_base, s_t;
    if (*stop) return;
    const int tid = threadIdx.x;
    // 1. prefix over block sums, per thread over a contiguous range of blocks
    const int64_t per = (nb + PICK_T - 1) / PICK_T;
    const int64_t b0 = (int64_t)tid * per, b1 = min(nb, b0 + per);
    double v = 0.0;
    for (int64_t b = b0; b < b1; ++b) v += bsum[b];
    const double incl = block_incl_scan_d(v, sh);
    const double excl = incl - v;
    if (tid == PICK_T - 1) s_t = incl;  // total
    if (tid == 0) {
        s_block = INT64_MAX;
        s_idx = INT64_MAX;
    }
    __syncthreads();
    const double total = s_t;
    if (!(total > 0.0)) {
        if (tid == 0) {
            *stop = 1;
            status_raise(status, ST_DEGENERATE);
        }
        return;
    }
    const double t = u[j] * total;
    // 2. first block whose inclusive prefix exceeds t (recomputed with the same per-thread order)
    {
        double run = excl;
        for (int64_t b = b0; b < b1; ++b) {
            run += bsum[b];
            if (run > t) {
                atomicMin((unsigned long long *)&s_block, (unsigned long long)b);
                break;
            }
        }
    }
    __syncthreads();
    int64_t blk = s_block;
    bool fallback = (blk == INT64_MAX);
    if (!fallback) {
        // base = inclusive prefix before block blk, in the same order as above
        if (blk >= b0 && blk < b1) {
            double run = excl;
            for (int64_t b = b0; b < blk; ++b) run += bsum[b];
            s_base = run;
        }
        __syncthreads();
        const double base = s_base;
        const int64_t i = blk * SB + tid;
        const bool in_blk = tid < SB && i < n;
        double p = 0.0;
        if (in_blk) p = (w ? (double)w[i] : 1.0) * (mode_w ? 1.0 : D2[i]);
        const double pin = block_incl_scan_d(p, sh);
        if (in_blk && base + pin > t) atomicMin((unsigned long long *)&s_idx, (unsigned long long)i);
        __syncthreads();
        if (s_idx == INT64_MAX) fallback = true;
        __syncthreads();
    }
    if (fallback) {
        // last i with p_i > 0: last block with a positive sum, then its last positive row
        if (tid == 0) {
            int64_t lb = -1;
            for (int64_t b = nb - 1; b >= 0; --b)
                if (bsum[b] > 0.0) {
                    lb = b;
                    break;
                }
            int64_t li = -1;
            if (lb >= 0)
                for (int64_t i = min(n, (lb + 1) * SB) - 1; i >= lb * SB; --i) {
                    double p = (w ? (double)w[i] : 1.0) * (mode_w ? 1.0 : D2[i]);
                    if (p > 0.0) {
                        li = i;
                        break;
                    }
                }
            s_idx = li;
        }
        __syncthreads();
    }
    const int64_t pick = s_idx;
    if (pick < 0 || pick >= n) {
        if (tid == 0) {
            *stop = 1;
            status_raise(status, ST_DEGENERATE);
        }
        return;
    }
    if (tid == 0) {
        idx_out[j] = pick;
        D2[pick] = 0.0;
    }
    for (int64_t q = tid; q < d; q += PICK_T) C_out[j * d + q] = X[pick * d + q];
}

// first center of an unweighted run: row floor(u0 * n)
__global__ void k_pick_uniform(const float *__restrict__ X, int64_t n, int64_t d,
                               const double *__restrict__ u, int64_t *__restrict__ idx_out,
                               float *__restrict__ C_out) {
    int64_t i0 = (int64_t)floor(u[0] * (double)n);
    if (i0 >= n) i0 = n - 1;
    if (i0 < 0) i0 = 0;
    if (threadIdx.x == 0) idx_out[0] = i0;
    for (int64_t q = threadIdx.x; q < d; q += blockDim.x) C_out[q] = X[i0 * d + q];
}

int seed_impl(gbkm_ctx *c, const float *X, int64_t n, int64_t d, const float *w, int64_t k,
              const double *u, int64_t *idx_out, float *C_out) {
    const int64_t nb = ceil_div(n, SB);
    WsPlan p;
    size_t o_d2 = p.take<double>(n), o_b = p.take<double>(nb), o_stop = p.take<int>(1);
    int rc = GBKM_OK;
    void *ws = ws_reserve(c, p.off, &rc);
    if (!ws) return rc;
    double *D2 = ws_at<double>(ws, o_d2), *bsum = ws_at<double>(ws, o_b);
    int *stop = ws_at<int>(ws, o_stop);
    cudaError_t e = cudaMemsetAsync(stop, 0, sizeof(int), c->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(idx_out, 0xff, sizeof(int64_t) * k, c->stream);
    if (e != cudaSuccess) return cuda_check(c, e, "seed memset");
    const bool vec = ((d & 3) == 0) && ((reinterpret_cast<uintptr_t>(X) & 15) == 0) &&
                     ((reinterpret_cast<uintptr_t>(C_out) & 15) == 0);
    if (!w) {
        k_pick_uniform<<<1, 256, 0, c->stream>>>(X, n, d, u, idx_out, C_out);
    } else {
        k_wsum<<<(unsigned)nb, 256, 0, c->stream>>>(w, n, bsum);
        k_pick<<<1, PICK_T, 0, c->stream>>>(X, n, d, w, D2, bsum, nb, u, 0, 1, idx_out, C_out, stop,
                                            c->status);
        c->launches += 1;
    }
    c->launches += 1;
    for (int64_t j = 1; j <= k; ++j) {
        const float *cprev = C_out + (j - 1) * d;
        if (j == k) break;  // D2 against the last center is not needed
        if (vec)
            k_d2_update<4><<<(unsigned)nb, 256, 0, c->stream>>>(X, n, d, w, cprev, j == 1, D2, bsum, stop);
        else
            k_d2_update<1><<<(unsigned)nb, 256, 0, c->stream>>>(X, n, d, w, cprev, j == 1, D2, bsum, stop);
        k_pick<<<1, PICK_T, 0, c->stream>>>(X, n, d, w, D2, bsum, nb, u, j, 0, idx_out, C_out, stop,
                                            c->status);
        c->launches += 2;
    }
    return cuda_check(c, cudaGetLastError(), "seed launch");
}

}  // namespace gbkm
