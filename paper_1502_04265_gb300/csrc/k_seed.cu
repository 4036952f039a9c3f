// k_seed.cu -- A3 k-means++ D^2 seeding (Section 1): two launches per round.  The first refreshes
// D^2 against the newest center and writes per-block FP64 sums; then one CTA samples the next center
// by a two-level prefix search, writes its row into the centers and measures it against the earlier
// centers for the next round's skip test.  No host synchronisation.
//
// The D^2 update skips, exactly, every point the new center cannot reach: with a the point's
// nearest chosen center and D its distance, ||x - c_new|| >= ||c_new - c_a|| - D, so when
// ||c_new - c_a||^2 > 4 D^2 (with a margin far above the rounding of both double-float values) the
// new distance exceeds D and min(D^2, ||x - c_new||^2) = D^2: the point's row is not read and D^2
// keeps its bits.  For the rows it does read, a plain FP32 distance with its error bound comes first;
// only where that cannot show the new center to be farther is the double-float distance taken.
#include "internal.cuh"
#include "seed_util.cuh"

namespace gbkm {

namespace {
constexpr int SB = 128;    // rows per sampling block (one CTA of 8 warps, 16 rows per warp)
constexpr int PICK_T = 256;   // threads of a pick CTA: the FP64 scans cost in proportion
}  // namespace

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
// rounding leaves none, the last i with p_i > 0.  CTA 0 writes idx_out[j] and the center row.
struct PickShared {
    double sh[32];
    int64_t s_block, s_idx;
    double s_base, s_t;
};

// the pick by the whole CTA (blockDim.x threads, a multiple of 32 and at least SB); returns the
// chosen row to every thread, or -1 when the run stops (fewer than k points with positive p_i)
__device__ int64_t pick_center(const float *__restrict__ X, int64_t n, int64_t d, const float *__restrict__ w,
                               double *__restrict__ D2, const double *__restrict__ bsum, int64_t nb,
                               const double *__restrict__ u, int64_t j, int mode_w, int64_t *__restrict__ idx_out,
                               float *__restrict__ C_out, int *stop, int *status, PickShared &ps) {
    double *sh = ps.sh;
    int64_t &s_block = ps.s_block, &s_idx = ps.s_idx;
    double &s_base = ps.s_base, &s_t = ps.s_t;
    const int tid = threadIdx.x, nt = blockDim.x;
    // 1. prefix over block sums, per thread over a contiguous range of blocks
    const int64_t per = (nb + nt - 1) / nt;
    const int64_t b0 = (int64_t)tid * per, b1 = min(nb, b0 + per);
    // the block sums are loaded eight at a time and added in range order (the same sum as one by one)
    double v = 0.0;
    for (int64_t b = b0; b < b1; b += 8) {
        double t8[8];
#pragma unroll
        for (int q = 0; q < 8; ++q) t8[q] = b + q < b1 ? bsum[b + q] : 0.0;
#pragma unroll
        for (int q = 0; q < 8; ++q)
            if (b + q < b1) v += t8[q];
    }
    const double incl = block_incl_scan_d(v, sh);
    const double excl = incl - v;
    if (tid == nt - 1) s_t = incl;  // total
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
        return -1;
    }
    const double t = u[j] * total;
    // 2. first block whose inclusive prefix exceeds t (recomputed with the same per-thread order)
    // a thread whose range ends clearly below t cannot hold the first block over t (the running sum
    // rises monotonically and ends within rounding of incl); one whose range starts clearly above t
    // holds it at its first block; only the thread(s) in between walk their range
    if (b0 < b1 && incl < t * (1.0 - 1e-12)) {
        // nothing in this range
    } else if (b0 < b1 && excl > t * (1.0 + 1e-12)) {
        atomicMin((unsigned long long *)&s_block, (unsigned long long)b0);
    } else {
        double run = excl;
        bool found = false;
        for (int64_t b = b0; b < b1 && !found; b += 8) {
            double t8[8];
#pragma unroll
            for (int q = 0; q < 8; ++q) t8[q] = b + q < b1 ? bsum[b + q] : 0.0;
#pragma unroll
            for (int q = 0; q < 8; ++q) {
                if (!found && b + q < b1) {
                    run += t8[q];
                    if (run > t) {
                        atomicMin((unsigned long long *)&s_block, (unsigned long long)(b + q));
                        found = true;
                    }
                }
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
        return -1;
    }
    // (D2 of the pick is left as it is: other CTAs making the same pick may still read it, and the next
    // round's update sets it to 0, the exact distance of the row to itself)
    if (blockIdx.x == 0) {
        if (tid == 0) idx_out[j] = pick;
        for (int64_t q = tid; q < d; q += nt) C_out[j * d + q] = X[pick * d + q];
    }
    return pick;
}

// One CTA of PICK_T threads: the pick of round j as a kernel of its own (the weighted first center)
__global__ void __launch_bounds__(PICK_T) k_pick(const float *__restrict__ X, int64_t n, int64_t d,
                                                 const float *__restrict__ w,
                                                 double *__restrict__ D2, const double *__restrict__ bsum,
                                                 int64_t nb, const double *__restrict__ u, int64_t j,
                                                 int mode_w, int64_t *__restrict__ idx_out,
                                                 float *__restrict__ C_out, int *stop, int *status) {
    __shared__ PickShared ps;
    if (*stop) return;
    pick_center(X, n, d, w, D2, bsum, nb, u, j, mode_w, idx_out, C_out, stop, status, ps);
}

// D2 refreshed against the newest center c (round j = index of c; round 0: D2 = distance to c), A =
// the index of the nearest center so far.  Every test that only decides whether a row can change is
// made in FP32 on shadow copies with margins that make it certified: D2f = D2 rounded up, ccf[a] =
// ||c - c_a||^2 rounded down (skip test above), the FP32 (or BF16-copy) distance with its error bound.
// FP64 work is left to the rows that may change (their double-float distance, compared with D2) and to
// the blocks where a row did change: such a block recomputes p_i = w_i D2_i summed by a fixed tree,
// the others keep their sum, whose bits a recomputation would give again.
template <int VW>
__global__ void __launch_bounds__(256, 4) k_d2_update(const float *__restrict__ X, int64_t n, int64_t d,
                                                      const float *__restrict__ w,
                                                      const float *__restrict__ c, int64_t j,
                                                      double *__restrict__ D2, float *__restrict__ D2f,
                                                      int32_t *__restrict__ A, const float *__restrict__ ccf,
                                                      double *__restrict__ bsum, const int *__restrict__ stop,
                                                      const __nv_bfloat16 *__restrict__ Xq,
                                                      const float *__restrict__ xresid) {
    if (*stop) return;
    __shared__ double sh[256];
    __shared__ int list[SB];
    __shared__ int nlist, changed;
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    const int64_t r0 = (int64_t)blockIdx.x * SB, r1 = min(n, r0 + SB);
    if (tid == 0) {
        nlist = 0;
        changed = j == 0;
    }
    __syncthreads();
    if (tid < SB) {
        const int64_t i = r0 + tid;
        if (i < r1) {
            // ccf <= cc and D2f >= D2, so this implies cc > 4 D2 (1 + 1e-6)
            const bool skip = j > 0 && ccf[A[i]] > 4.f * D2f[i] * (1.f + 4e-6f);
            if (!skip) list[atomicAdd(&nlist, 1)] = tid;
        }
    }
    __syncthreads();
    const int m = nlist;
    // lpr lanes per listed row (32 / lpr rows per warp at a time)
    const int lpr = lanes_per_row_d2(d, VW), rpw = 32 / lpr, sub = lane / lpr, sl = lane % lpr;
    // relative error bound of the FP32 distances below (each difference rounded once, each
    // fma-accumulated square once, at most d terms per lane, five butterfly additions), with room for
    // the rounding of the product that applies it
    const float g32 = (float)(d + 40) * 5.9604645e-8f;
    // two listed rows per lane group at a time: both rows' loads are issued before either is summed,
    // so a warp keeps twice the bytes in flight (the distance passes wait on DRAM, not on arithmetic)
    constexpr int NR = 2;
    for (int e0 = wid * rpw * NR; e0 < m; e0 += 8 * rpw * NR) {
        int64_t ii[NR];
        bool hh[NR], need[NR];
        float dold[NR];
#pragma unroll
        for (int r = 0; r < NR; ++r) {
            const int e = e0 + r * rpw + sub;
            hh[r] = e < m;
            ii[r] = r0 + (hh[r] ? list[e] : 0);
            need[r] = hh[r];
            // above D2 whatever the rounding of the product
            dold[r] = (j > 0 && hh[r]) ? D2f[ii[r]] * (1.f + 2e-6f) : 0.f;
        }
        if (j > 0) {
            if (Xq) {
                // ||x - c|| >= ||x~ - c|| - ||x~ - x|| with x~ the BF16 copy (d % 8 == 0) and ||x~ - x|| <= the
                // row's residual: when that bound exceeds D the FP32 row is not read
                float a16[NR];
#pragma unroll
                for (int r = 0; r < NR; ++r) a16[r] = 0.f;
                const uint4 *q8[NR];
#pragma unroll
                for (int r = 0; r < NR; ++r) q8[r] = reinterpret_cast<const uint4 *>(Xq + ii[r] * d);
                const float4 *c4 = reinterpret_cast<const float4 *>(c);
#pragma unroll 4
                for (int64_t q = sl; q < d / 8; q += lpr) {
                    uint4 v[NR];
#pragma unroll
                    for (int r = 0; r < NR; ++r) v[r] = hh[r] ? __ldg(q8[r] + q) : make_uint4(0u, 0u, 0u, 0u);
                    const float4 b0 = __ldg(c4 + 2 * q), b1 = __ldg(c4 + 2 * q + 1);
#pragma unroll
                    for (int r = 0; r < NR; ++r) {
                        const float f0 = __uint_as_float(v[r].x << 16) - b0.x, f1 = __uint_as_float(v[r].x & 0xffff0000u) - b0.y;
                        const float f2 = __uint_as_float(v[r].y << 16) - b0.z, f3 = __uint_as_float(v[r].y & 0xffff0000u) - b0.w;
                        const float f4 = __uint_as_float(v[r].z << 16) - b1.x, f5 = __uint_as_float(v[r].z & 0xffff0000u) - b1.y;
                        const float f6 = __uint_as_float(v[r].w << 16) - b1.z, f7 = __uint_as_float(v[r].w & 0xffff0000u) - b1.w;
                        float a = a16[r];
                        a = fmaf(f0, f0, a);
                        a = fmaf(f1, f1, a);
                        a = fmaf(f2, f2, a);
                        a = fmaf(f3, f3, a);
                        a = fmaf(f4, f4, a);
                        a = fmaf(f5, f5, a);
                        a = fmaf(f6, f6, a);
                        a = fmaf(f7, f7, a);
                        a16[r] = a;
                    }
                }
#pragma unroll
                for (int r = 0; r < NR; ++r) {
                    for (int o = lpr >> 1; o > 0; o >>= 1) a16[r] += __shfl_xor_sync(0xffffffffu, a16[r], o);
                    if (hh[r]) {
                        // a lower bound of ||x~ - c|| (sqrtf is correctly rounded; the factor covers it and the
                        // product), then of ||x - c||^2
                        const float lo = sqrtf(fmaxf(a16[r] * (1.f - g32), 0.f)) * (1.f - 2.4e-7f) - xresid[ii[r]];
                        const float L = lo > 0.f ? lo * lo * (1.f - 1e-6f) : 0.f;
                        need[r] = !(L > dold[r]);
                    }
                }
                if (!__any_sync(0xffffffffu, need[0] || need[1])) continue;
            }
            // the FP32 distance: when its lower bound exceeds D, D^2 keeps its bits
            float a32[NR];
#pragma unroll
            for (int r = 0; r < NR; ++r) a32[r] = 0.f;
            if constexpr (VW == 4) {
                const float4 *x4[NR];
#pragma unroll
                for (int r = 0; r < NR; ++r) x4[r] = reinterpret_cast<const float4 *>(X + ii[r] * d);
                const float4 *c4 = reinterpret_cast<const float4 *>(c);
#pragma unroll 4
                for (int64_t q = sl; q < d / 4; q += lpr) {
                    float4 a[NR];
#pragma unroll
                    for (int r = 0; r < NR; ++r) a[r] = need[r] ? __ldg(x4[r] + q) : make_float4(0.f, 0.f, 0.f, 0.f);
                    const float4 b = __ldg(c4 + q);
#pragma unroll
                    for (int r = 0; r < NR; ++r) {
                        const float e0_ = a[r].x - b.x, e1 = a[r].y - b.y, e2 = a[r].z - b.z, e3 = a[r].w - b.w;
                        float s = a32[r];
                        s = fmaf(e0_, e0_, s);
                        s = fmaf(e1, e1, s);
                        s = fmaf(e2, e2, s);
                        s = fmaf(e3, e3, s);
                        a32[r] = s;
                    }
                }
            } else {
#pragma unroll
                for (int r = 0; r < NR; ++r)
                    if (need[r]) {
                        const float *x = X + ii[r] * d;
                        for (int64_t q = sl; q < d; q += lpr) {
                            const float df = x[q] - c[q];
                            a32[r] = fmaf(df, df, a32[r]);
                        }
                    }
            }
#pragma unroll
            for (int r = 0; r < NR; ++r) {
                for (int o = lpr >> 1; o > 0; o >>= 1) a32[r] += __shfl_xor_sync(0xffffffffu, a32[r], o);
                need[r] = need[r] && !(a32[r] * (1.f - g32) > dold[r]);
            }
        }
#pragma unroll
        for (int r = 0; r < NR; ++r) {
            if (!__any_sync(0xffffffffu, need[r])) continue;
            const int64_t i = ii[r];
            DF acc;
            if (need[r]) {
                const float *x = X + i * d;
                if constexpr (VW == 4) {
                    const float4 *x4 = reinterpret_cast<const float4 *>(x);
                    const float4 *c4 = reinterpret_cast<const float4 *>(c);
#pragma unroll 2
                    for (int64_t q = sl; q < d / 4; q += lpr) {
                        float4 a = __ldg(x4 + q), b = __ldg(c4 + q);
                        acc.add_sqdiff(a.x, b.x);
                        acc.add_sqdiff(a.y, b.y);
                        acc.add_sqdiff(a.z, b.z);
                        acc.add_sqdiff(a.w, b.w);
                    }
                } else {
                    for (int64_t q = sl; q < d; q += lpr) acc.add_sqdiff(x[q], c[q]);
                }
            }
            const double dist = group_sum_df(acc, lpr);
            if (need[r] && sl == 0 && (j == 0 || dist < D2[i])) {
                D2[i] = dist;
                D2f[i] = __double2float_ru(dist);
                A[i] = (int32_t)j;
                changed = 1;
            }
        }
    }
    __syncthreads();
    if (!changed) return;
    double p = 0.0;
    if (tid < SB && r0 + tid < r1) p = (w ? (double)w[r0 + tid] : 1.0) * D2[r0 + tid];
    const double s = block_tree_sum_d(p, sh);
    if (tid == 0) bsum[blockIdx.x] = s;
}

// One CTA of PICK_T threads after each round's D^2 update: picks center j and measures it against the
// earlier centers (ccf, rounded down, for the next round's skip test; double-float, lpr lanes per center)
__global__ void __launch_bounds__(PICK_T) k_pick_cc(const float *__restrict__ X, int64_t n, int64_t d,
                                                    const float *__restrict__ w, double *__restrict__ D2,
                                                    const double *__restrict__ bsum, int64_t nb,
                                                    const double *__restrict__ u, int64_t j, int64_t k,
                                                    int64_t *__restrict__ idx_out, float *__restrict__ C_out,
                                                    float *__restrict__ ccf, int *stop, int *status) {
    __shared__ PickShared ps;
    if (*stop) return;
    const int64_t pick = pick_center(X, n, d, w, D2, bsum, nb, u, j, 0, idx_out, C_out, stop, status, ps);
    if (pick < 0 || j + 1 >= k) return;
    // this CTA's share of the earlier centers, against the new one's row of X
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const int lpr = lanes_per_row(d, 1), cpw = 32 / lpr, sl = lane % lpr;
    const float *cj = X + pick * d;
    for (int64_t a0 = ((int64_t)blockIdx.x * nw + wid) * cpw; a0 < j; a0 += (int64_t)gridDim.x * nw * cpw) {
        const int64_t a = a0 + lane / lpr;
        const bool has = a < j;
        DF acc;
        if (has)
            for (int64_t t = sl; t < d; t += lpr) acc.add_sqdiff(cj[t], C_out[a * d + t]);
        const double v = group_sum_df(acc, lpr);
        if (has && sl == 0) ccf[a] = __double2float_rd(v);
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
              const double *u, int64_t *idx_out, float *C_out, const void *Xq, const float *xresid) {
    const int64_t nb = ceil_div(n, SB);
    WsPlan p;
    size_t o_d2 = p.take<double>(n), o_d2f = p.take<float>(n), o_a = p.take<int32_t>(n), o_cc = p.take<float>(k),
           o_b = p.take<double>(nb), o_stop = p.take<int>(2);
    int rc = GBKM_OK;
    void *ws = ws_reserve(c, p.off, &rc);
    if (!ws) return rc;
    double *D2 = ws_at<double>(ws, o_d2), *bsum = ws_at<double>(ws, o_b);
    float *D2f = ws_at<float>(ws, o_d2f), *ccf = ws_at<float>(ws, o_cc);
    int32_t *A = ws_at<int32_t>(ws, o_a);
    int *stop = ws_at<int>(ws, o_stop);
    cudaError_t e = cudaMemsetAsync(stop, 0, 2 * sizeof(int), c->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(idx_out, 0xff, sizeof(int64_t) * k, c->stream);
    if (e != cudaSuccess) return cuda_check(c, e, "seed memset");
    const bool vec = ((d & 3) == 0) && ((reinterpret_cast<uintptr_t>(X) & 15) == 0) &&
                     ((reinterpret_cast<uintptr_t>(C_out) & 15) == 0);
    // the BF16 filter pass reads 16-byte groups of 8 elements of the copy
    const __nv_bfloat16 *xq = (Xq && xresid && vec && (d & 7) == 0 && (reinterpret_cast<uintptr_t>(Xq) & 15) == 0)
                                  ? static_cast<const __nv_bfloat16 *>(Xq) : nullptr;
    if (!w) {
        k_pick_uniform<<<1, 256, 0, c->stream>>>(X, n, d, u, idx_out, C_out);
    } else {
        k_wsum<<<(unsigned)nb, 256, 0, c->stream>>>(w, n, bsum);
        k_pick<<<1, PICK_T, 0, c->stream>>>(X, n, d, w, D2, bsum, nb, u, 0, 1, idx_out, C_out, stop,
                                            c->status);
        c->launches += 1;
    }
    c->launches += 1;
    for (int64_t j = 1; j < k; ++j) {
        // refresh D2 against center j - 1 (chosen in the previous round), then pick center j and
        // measure it against the earlier ones
        const int64_t jc = j - 1;
        const float *cprev = C_out + jc * d;
        prof_begin(c, "seed_d2");
        if (vec)
            k_d2_update<4><<<(unsigned)nb, 256, 0, c->stream>>>(X, n, d, w, cprev, jc, D2, D2f, A, ccf, bsum, stop,
                                                                xq, xresid);
        else
            k_d2_update<1><<<(unsigned)nb, 256, 0, c->stream>>>(X, n, d, w, cprev, jc, D2, D2f, A, ccf, bsum, stop,
                                                                nullptr, nullptr);
        prof_end(c);
        prof_begin(c, "seed_pick");
        // every CTA makes the same pick (the same data, the same operations) and measures its share
        // of the earlier centers against it; CTA 0 records it
        const int lpr = lanes_per_row(d, 1), per_cta = (PICK_T / 32) * (32 / lpr);
        const unsigned g = j + 1 < k ? (unsigned)std::min<int64_t>(ceil_div(j, (int64_t)per_cta), 64) : 1u;
        k_pick_cc<<<g, PICK_T, 0, c->stream>>>(X, n, d, w, D2, bsum, nb, u, j, k, idx_out, C_out, ccf, stop,
                                               c->status);
        prof_end(c);
        c->launches += 2;
    }
    return cuda_check(c, cudaGetLastError(), "seed launch");
}

}  // namespace gbkm
