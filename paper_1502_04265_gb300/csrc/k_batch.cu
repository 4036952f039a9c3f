// k_batch.cu -- A8: many independent k-means problems (uneven n, d, k) x several k-means++ seeds in
// one run.  Every phase is a single launch over all (problem, seed) pairs:
//   preparation   row norms (+ BF16 copy) over a table of 128-row blocks of all problems
//   seeding       per round r: D^2 update of all pairs still seeding (one read of X per problem
//                 serves all its seeds), then one sampler CTA per pair
//   assignment    k_tcb (k_tc.cu): persistent tcgen05 kernel over (problem, row tile) items, the
//                 seeds' centers concatenated along N, per-seed top-2 epilogue
//   recheck       one warp per flagged (problem, seed, point)
//   update        the counting-sort / segmented-sum pipeline of the single-problem update, over a
//                 pair table: the label table of every pair is one device-wide scan
// The run is recorded into one CUDA graph (when asked) and launched.
#include <cuda.h>
#include <math.h>
#include <string.h>

#include <algorithm>
#include <vector>

#include "internal.cuh"
#include "seed_util.cuh"

namespace gbkm {

namespace {
constexpr int RB = 128;             // rows per preparation / sampling block
constexpr int SEGR = 256;           // rows per label segment (one warp)
constexpr int64_t BIG = 2048;       // rows per segmented-sum item
constexpr int PICKB_T = 256;

struct PairInfo {                   // one (problem, seed) pair of the update pipeline
    int32_t p, s, S, nseg_pad;      // problem, seed, label segments of the pair
    int64_t hbase, gbase, seg0;     // first entry of its label table / first global cluster / first segment
};

__device__ __forceinline__ unsigned lanemask_lt_b() {
    unsigned m;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
    return m;
}

// largest i with arr[i] <= key (arr sorted, arr[0] <= key)
__device__ __forceinline__ int64_t upper_index(const int64_t *arr, int64_t n, int64_t key) {
    int64_t lo = 0, hi = n - 1;
    while (lo < hi) {
        const int64_t mid = (lo + hi + 1) >> 1;
        if (arr[mid] <= key) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}
__device__ __forceinline__ int64_t upper_index32(const int32_t *arr, int64_t n, int64_t key) {
    int64_t lo = 0, hi = n - 1;
    while (lo < hi) {
        const int64_t mid = (lo + hi + 1) >> 1;
        if (arr[mid] <= key) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}
}  // namespace

// ---------------------------------------------------------------- preparation
// blocks: (problem, first row) of every 128-row block of every problem
__global__ void __launch_bounds__(256) k_b_prep(const BProb *__restrict__ probs, const int2 *__restrict__ blocks,
                                                int bf16) {
    const int2 b = blocks[blockIdx.x];
    const BProb &P = probs[b.x];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    for (int64_t i = b.y + w; i < min(P.n, (int64_t)b.y + RB); i += 8) {
        const float *x = P.X + i * P.d;
        float s = 0.f;
        for (int64_t t = lane; t < P.d; t += 32) {
            const float v = x[t];
            s = fmaf(v, v, s);
            if (bf16) const_cast<__nv_bfloat16 *>(static_cast<const __nv_bfloat16 *>(P.Xop))[i * P.d + t] = __float2bfloat16_rn(v);
        }
        s = warp_sum_f(s);
        if (lane == 0) P.xnorm[i] = s;
    }
}

// ---------------------------------------------------------------- k-means++ (Section 1), batched
__global__ void k_b_seed_first(const BProb *__restrict__ probs, const int2 *__restrict__ pairs) {
    const int2 ps = pairs[blockIdx.x];
    const BProb &P = probs[ps.x];
    int64_t i0 = (int64_t)floor(P.u[(int64_t)ps.y * P.k] * (double)P.n);
    if (i0 >= P.n) i0 = P.n - 1;
    if (i0 < 0) i0 = 0;
    float *c = P.C[0] + (int64_t)ps.y * P.k * P.d;
    for (int64_t t = threadIdx.x; t < P.d; t += blockDim.x) c[t] = P.X[i0 * P.d + t];
    if (threadIdx.x == 0) {
        P.stop[ps.y] = 0;
        P.dirty[ps.y] = -1;
    }
}

// round r >= 1: D^2 of every seed of the block's problem against that seed's center r-1, and the
// block sum of D^2 per seed (a fixed tree over the rows).  As in the single-problem update, every test
// that only decides whether a row can change is certified in FP32 on shadow copies (D2f = D2 rounded
// up, ccf = the center distances rounded down): the skip test (a row whose nearest center a satisfies
// ||c_{r-1} - c_a||^2 > 4 D^2 keeps D^2: the new center cannot come closer), then a plain FP32 distance
// with its error bound.  Only rows that may change take the double-float distance, and only blocks
// where a row changed (or the last pick's block) recompute their sum; the others keep the same bits.
__global__ void __launch_bounds__(256) k_b_d2(const BProb *__restrict__ probs, const int2 *__restrict__ blocks,
                                              int r) {
    const int2 b = blocks[blockIdx.x];
    const BProb &P = probs[b.x];
    if (r >= P.k) return;
    __shared__ double nd_s[256];
    __shared__ int list[RB];
    __shared__ int nlist, changed;
    const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
    const int64_t blk = b.y / RB;
    const int64_t jc = r - 1;
    const int64_t r0 = b.y, r1 = min(P.n, (int64_t)b.y + RB);
    const float g32 = (float)(P.d + 40) * 5.9604645e-8f;
    for (int s = 0; s < P.seeds; ++s) {
        if (P.stop[s]) continue;  // uniform over the block
        const float *c = P.C[0] + ((int64_t)s * P.k + jc) * P.d;
        double *D2 = P.D2 + (int64_t)s * P.n;
        float *D2f = P.D2f + (int64_t)s * P.n;
        int32_t *A = P.A + (int64_t)s * P.n;
        const float *ccf = P.ccf + (int64_t)s * P.k;
        if (tid == 0) {
            nlist = 0;
            changed = jc == 0 || P.dirty[s] == blk;
        }
        __syncthreads();
        if (tid < RB) {
            const int64_t i = r0 + tid;
            if (i < r1) {
                const bool skip = jc > 0 && ccf[A[i]] > 4.f * D2f[i] * (1.f + 4e-6f);
                if (!skip) list[atomicAdd(&nlist, 1)] = tid;
            }
        }
        __syncthreads();
        const int m = nlist;
        const bool v4 = (P.d % 4) == 0 && ((reinterpret_cast<uintptr_t>(P.X) & 15) == 0) &&
                        ((reinterpret_cast<uintptr_t>(c) & 15) == 0);
        const int lpr = lanes_per_row_d2(P.d, v4 ? 4 : 1), rpw = 32 / lpr, sub = lane / lpr, sl = lane % lpr;
        for (int e0 = w * rpw; e0 < m; e0 += 8 * rpw) {
            const int e = e0 + sub;
            const bool has = e < m;
            const int t = has ? list[e] : 0;
            const int64_t i = r0 + t;
            const float *x = P.X + i * P.d;
            bool need = has;
            if (jc > 0) {
                float a32 = 0.f;
                if (has) {
                    if (v4) {
                        for (int64_t q = sl; q < P.d / 4; q += lpr) {
                            const float4 a4 = __ldg(reinterpret_cast<const float4 *>(x) + q);
                            const float4 b4 = __ldg(reinterpret_cast<const float4 *>(c) + q);
                            const float f0 = a4.x - b4.x, f1 = a4.y - b4.y, f2 = a4.z - b4.z, f3 = a4.w - b4.w;
                            a32 = fmaf(f0, f0, a32);
                            a32 = fmaf(f1, f1, a32);
                            a32 = fmaf(f2, f2, a32);
                            a32 = fmaf(f3, f3, a32);
                        }
                    } else {
                        for (int64_t q = sl; q < P.d; q += lpr) {
                            const float f = x[q] - c[q];
                            a32 = fmaf(f, f, a32);
                        }
                    }
                }
                for (int o = lpr >> 1; o > 0; o >>= 1) a32 += __shfl_xor_sync(0xffffffffu, a32, o);
                need = has && !(a32 * (1.f - g32) > D2f[i] * (1.f + 2e-6f));
            }
            if (!__any_sync(0xffffffffu, need)) continue;
            DF acc;
            if (need) {
                if (v4) {
                    for (int64_t q = sl; q < P.d / 4; q += lpr) {
                        const float4 a4 = __ldg(reinterpret_cast<const float4 *>(x) + q);
                        const float4 b4 = __ldg(reinterpret_cast<const float4 *>(c) + q);
                        acc.add_sqdiff(a4.x, b4.x);
                        acc.add_sqdiff(a4.y, b4.y);
                        acc.add_sqdiff(a4.z, b4.z);
                        acc.add_sqdiff(a4.w, b4.w);
                    }
                } else {
                    for (int64_t q = sl; q < P.d; q += lpr) acc.add_sqdiff(x[q], c[q]);
                }
            }
            const double dist = group_sum_df(acc, lpr);
            if (need && sl == 0 && (jc == 0 || dist < D2[i])) {
                D2[i] = dist;
                D2f[i] = __double2float_ru(dist);
                A[i] = (int32_t)jc;
                changed = 1;
            }
        }
        __syncthreads();
        if (changed) {
            const double v = (tid < RB && r0 + tid < r1) ? D2[r0 + tid] : 0.0;
            const double tot = block_tree_sum_d(v, nd_s);
            if (tid == 0) P.bsum[(int64_t)s * P.nb + blk] = tot;
        }
        __syncthreads();
    }
}

// round r >= 2: ccf[s][a] = ||c_{r-1} - c_a||^2 (double-float, rounded down to FP32) for a < r - 1, one
// warp per (pair, earlier center); grid.y = pair
__global__ void __launch_bounds__(256) k_b_cc(const BProb *__restrict__ probs, const int2 *__restrict__ pairs, int r) {
    const int2 ps = pairs[blockIdx.y];
    const BProb &P = probs[ps.x];
    if (r >= P.k || P.stop[ps.y]) return;
    // lpr lanes per earlier center (the grid provides 32; the rest of a warp's lanes take further
    // centers): short rows keep the lanes busy
    const int lpr = lanes_per_row(P.d, 1), sl = (threadIdx.x & 31) % lpr;
    const int64_t jc = r - 1;
    const int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const int64_t a = g / lpr;
    if ((g & ~(int64_t)31) / lpr >= jc) return;  // the whole warp is past the last center
    const bool has = a < jc;
    const float *C = P.C[0] + (int64_t)ps.y * P.k * P.d;
    DF acc;
    if (has)
        for (int64_t t = sl; t < P.d; t += lpr) acc.add_sqdiff(C[jc * P.d + t], C[a * P.d + t]);
    const double v = group_sum_df(acc, lpr);
    if (has && sl == 0) P.ccf[(int64_t)ps.y * P.k + a] = __double2float_rd(v);
}

__device__ double block_incl_scan_db(double v, double *sh) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    double x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const double y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) sh[wid] = x;
    __syncthreads();
    if (wid == 0) {
        double t = lane < nw ? sh[lane] : 0.0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const double y = __shfl_up_sync(0xffffffffu, t, o);
            if (lane >= o) t += y;
        }
        sh[lane] = t;
    }
    __syncthreads();
    const double res = x + (wid > 0 ? sh[wid - 1] : 0.0);
    __syncthreads();
    return res;
}

// round r >= 1: one CTA per pair picks the smallest i whose inclusive prefix of D^2 exceeds
// u[r] * sum D^2 (two levels: block sums, then rows of the block), or the last positive row
__global__ void __launch_bounds__(PICKB_T) k_b_pick(const BProb *__restrict__ probs, const int2 *__restrict__ pairs,
                                                    int r, int *status) {
    __shared__ double sh[32];
    __shared__ long long s_blk, s_idx;
    __shared__ double s_base, s_tot;
    const int2 ps = pairs[blockIdx.x];
    const BProb &P = probs[ps.x];
    if (r >= P.k || P.stop[ps.y]) return;
    const int tid = threadIdx.x;
    const double *bs = P.bsum + (int64_t)ps.y * P.nb;
    const double *D2 = P.D2 + (int64_t)ps.y * P.n;
    const int64_t per = (P.nb + PICKB_T - 1) / PICKB_T;
    const int64_t b0 = (int64_t)tid * per, b1 = min((int64_t)P.nb, b0 + per);
    double v = 0.0;
    for (int64_t b = b0; b < b1; ++b) v += bs[b];
    const double incl = block_incl_scan_db(v, sh);
    const double excl = incl - v;
    if (tid == PICKB_T - 1) s_tot = incl;
    if (tid == 0) {
        s_blk = LLONG_MAX;
        s_idx = LLONG_MAX;
    }
    __syncthreads();
    const double total = s_tot;
    if (!(total > 0.0)) {
        if (tid == 0) {
            P.stop[ps.y] = 1;
            status_raise(status, ST_DEGENERATE);
        }
        return;
    }
    const double t = P.u[(int64_t)ps.y * P.k + r] * total;
    {
        double run = excl;
        for (int64_t b = b0; b < b1; ++b) {
            run += bs[b];
            if (run > t) {
                atomicMin(&s_blk, (long long)b);
                break;
            }
        }
    }
    __syncthreads();
    const long long blk = s_blk;
    bool fallback = blk == LLONG_MAX;
    if (!fallback) {
        if (blk >= b0 && blk < b1) {
            double run = excl;
            for (int64_t b = b0; b < blk; ++b) run += bs[b];
            s_base = run;
        }
        __syncthreads();
        const int64_t i = blk * RB + tid;
        const bool in = tid < RB && i < P.n;
        const double pin = block_incl_scan_db(in ? D2[i] : 0.0, sh);
        if (in && s_base + pin > t) atomicMin(&s_idx, (long long)i);
        __syncthreads();
        if (s_idx == LLONG_MAX) fallback = true;
        __syncthreads();
    }
    if (fallback) {
        if (tid == 0) {
            long long li = -1;
            for (int64_t i = P.n - 1; i >= 0; --i)
                if (D2[i] > 0.0) {
                    li = i;
                    break;
                }
            s_idx = li;
        }
        __syncthreads();
    }
    const long long pick = s_idx;
    if (pick < 0 || pick >= P.n) {
        if (tid == 0) {
            P.stop[ps.y] = 1;
            status_raise(status, ST_DEGENERATE);
        }
        return;
    }
    float *c = P.C[0] + ((int64_t)ps.y * P.k + r) * P.d;
    for (int64_t q = tid; q < P.d; q += PICKB_T) c[q] = P.X[pick * P.d + q];
    if (tid == 0) {
        const_cast<double *>(D2)[pick] = 0.0;
        P.D2f[(int64_t)ps.y * P.n + pick] = 0.f;
        P.dirty[ps.y] = pick / RB;  // that block's sum is refreshed in the next round
    }
}

// ---------------------------------------------------------------- per-iteration center preparation
// one CTA per operand row (problem p, seed s, local center j < kps): ||c||^2, max ||c|| per problem,
// operand copy (BF16, or TF32 hi / lo); padding rows j >= k are zero with ||c||^2 = +inf
__global__ void __launch_bounds__(128) k_b_cprep(const BProb *__restrict__ probs, const int64_t *__restrict__ crow0,
                                                 int64_t nprob, int par, int bf16) {
    __shared__ double red[4];
    const int64_t row = blockIdx.x;
    const int64_t p = upper_index(crow0, nprob, row);
    const BProb &P = probs[p];
    const int64_t lr = row - P.crow0;
    const int64_t s = lr / P.kps, j = lr % P.kps;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    if (j >= P.k) {
        for (int64_t t = threadIdx.x; t < P.d; t += blockDim.x) {
            if (bf16) static_cast<__nv_bfloat16 *>(P.cop)[lr * P.d + t] = __float2bfloat16_rn(0.f);
            else {
                static_cast<float *>(P.cop)[lr * P.d + t] = 0.f;
                static_cast<float *>(P.cop_lo)[lr * P.d + t] = 0.f;
            }
        }
        if (threadIdx.x == 0) P.cnorm[lr] = __int_as_float(0x7f800000);
        return;
    }
    const float *c = P.C[par] + (s * P.k + j) * P.d;
    DF acc;
    for (int64_t t = threadIdx.x; t < P.d; t += blockDim.x) {
        const float v = c[t];
        acc.add_prod(v, v);
        if (bf16) {
            static_cast<__nv_bfloat16 *>(P.cop)[lr * P.d + t] = __float2bfloat16_rn(v);
        } else {
            const float hi = __uint_as_float(__float_as_uint(v) & 0xffffe000u);
            static_cast<float *>(P.cop)[lr * P.d + t] = hi;
            static_cast<float *>(P.cop_lo)[lr * P.d + t] = __uint_as_float(__float_as_uint(__fsub_rn(v, hi)) & 0xffffe000u);
        }
    }
    const double sw = warp_sum_df(acc);
    if (lane == 0) red[w] = sw;
    __syncthreads();
    if (threadIdx.x == 0) {
        const double tot = (red[0] + red[1]) + (red[2] + red[3]);
        P.cnorm[lr] = (float)tot;
        atomicMax(P.cmax, __float_as_uint((float)sqrt(tot) * (1.f + 1.0e-6f)));
    }
}

// ---------------------------------------------------------------- exact recheck of flagged points
// squared distance from direct differences in FP32, 4 accumulators per lane + butterfly: relative
// error <= (ceil(d/128) + 10) 2^-24, inside the 1e-5 near-tie band
__device__ __forceinline__ float warp_dd2(const float *__restrict__ x, const float *__restrict__ c, int64_t d) {
    const int lane = threadIdx.x & 31;
    float a0 = 0.f, a1 = 0.f, a2 = 0.f, a3 = 0.f;
    const float4 *x4 = reinterpret_cast<const float4 *>(x);
    const float4 *c4 = reinterpret_cast<const float4 *>(c);
#pragma unroll 4
    for (int64_t t = lane; t < d / 4; t += 32) {
        const float4 a = __ldg(x4 + t), b = __ldg(c4 + t);
        const float e0 = a.x - b.x, e1 = a.y - b.y, e2 = a.z - b.z, e3 = a.w - b.w;
        a0 = fmaf(e0, e0, a0);
        a1 = fmaf(e1, e1, a1);
        a2 = fmaf(e2, e2, a2);
        a3 = fmaf(e3, e3, a3);
    }
    float v = (a0 + a1) + (a2 + a3);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

__global__ void __launch_bounds__(256) k_b_recheck(const BProb *__restrict__ probs, const int32_t *__restrict__ flags,
                                                   const int32_t *__restrict__ count, int par) {
    const int lane = threadIdx.x & 31;
    const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = (gridDim.x * (int64_t)blockDim.x) >> 5;
    const int cnt = *count;
    for (int64_t f = warp; f < cnt; f += nwarps) {
        const int32_t *e = flags + f * BFLAG_STRIDE;
        const BProb &P = probs[e[0]];
        const int s = e[1];
        const int64_t row = e[2];
        const float *x = P.X + row * P.d;
        const float *C = P.C[par] + (int64_t)s * P.k * P.d;
        float best = 0.f;
        int arg = -1;
        if (e[3] > 0 && e[3] <= BCAND_MAX) {
            for (int q = 0; q < e[3]; ++q) {
                const int j = e[4 + q];
                const float v = warp_dd2(x, C + (int64_t)j * P.d, P.d);
                if (arg < 0 || v < best || (v == best && j < arg)) {
                    best = v;
                    arg = j;
                }
            }
        } else {
            for (int64_t j = 0; j < P.k; ++j) {
                const float v = warp_dd2(x, C + j * P.d, P.d);
                if (arg < 0 || v < best) {
                    best = v;
                    arg = (int)j;
                }
            }
        }
        if (lane == 0) P.labels[(int64_t)s * P.n + row] = arg;
    }
}

// ---------------------------------------------------------------- update over the pair table
// segments: (pair, first row) of every 256-row label segment; per-warp histograms in shared memory
__global__ void __launch_bounds__(256) k_b_hist(const BProb *__restrict__ probs, const PairInfo *__restrict__ pinfo,
                                                const int2 *__restrict__ segs, int64_t nseg, int64_t kmax,
                                                int32_t *__restrict__ hist) {
    extern __shared__ int32_t hsm[];
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    const int64_t sg = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    if (sg >= nseg) return;
    const int2 sd = segs[sg];
    const PairInfo &Q = pinfo[sd.x];
    const BProb &P = probs[Q.p];
    volatile int32_t *mine = hsm + (int64_t)wib * kmax;
    for (int64_t j = lane; j < P.k; j += 32) mine[j] = 0;
    __syncwarp();
    const int32_t *lab = P.labels + (int64_t)Q.s * P.n;
    const int64_t r1 = min(P.n, (int64_t)sd.y + SEGR);
    for (int64_t base = sd.y; base < r1; base += 32) {
        const int64_t i = base + lane;
        const int32_t l = i < r1 ? lab[i] : -1;
        const bool ok = l >= 0 && l < P.k;
        const unsigned act = __ballot_sync(0xffffffffu, ok);
        if (ok) {
            const unsigned grp = __match_any_sync(act, l);
            if (lane == __ffs(grp) - 1) mine[l] = mine[l] + __popc(grp);
        }
        __syncwarp();
    }
    const int64_t sl = sg - Q.seg0;
    for (int64_t j = lane; j < P.k; j += 32) hist[Q.hbase + j * Q.S + sl] = mine[j];
}

__global__ void __launch_bounds__(256) k_b_scatter(const BProb *__restrict__ probs, const PairInfo *__restrict__ pinfo,
                                                   const int2 *__restrict__ segs, int64_t nseg, int64_t kmax,
                                                   const int32_t *__restrict__ off, int32_t *__restrict__ perm) {
    extern __shared__ int32_t hsm[];
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    const int64_t sg = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    if (sg >= nseg) return;
    const int2 sd = segs[sg];
    const PairInfo &Q = pinfo[sd.x];
    const BProb &P = probs[Q.p];
    volatile int32_t *mine = hsm + (int64_t)wib * kmax;
    const int64_t sl = sg - Q.seg0;
    for (int64_t j = lane; j < P.k; j += 32) mine[j] = off[Q.hbase + j * Q.S + sl];
    __syncwarp();
    const int32_t *lab = P.labels + (int64_t)Q.s * P.n;
    const int64_t r1 = min(P.n, (int64_t)sd.y + SEGR);
    for (int64_t base = sd.y; base < r1; base += 32) {
        const int64_t i = base + lane;
        const int32_t l = i < r1 ? lab[i] : -1;
        const bool ok = l >= 0 && l < P.k;
        const unsigned act = __ballot_sync(0xffffffffu, ok);
        if (ok) {
            const unsigned grp = __match_any_sync(act, l);
            perm[mine[l] + __popc(grp & lanemask_lt_b())] = (int32_t)i;
            __syncwarp(act);
            if (lane == __ffs(grp) - 1) mine[l] = mine[l] + __popc(grp);
        }
        __syncwarp();
    }
}

// per global cluster g (pair q, local cluster j): first slot in the concatenated permutation
__global__ void k_b_starts(const PairInfo *__restrict__ pinfo, const int32_t *__restrict__ cpair,
                           const int32_t *__restrict__ off, int64_t G, int64_t total_rows, int32_t *__restrict__ start) {
    const int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (g < G) {
        const PairInfo &Q = pinfo[cpair[g]];
        start[g] = off[Q.hbase + (g - Q.gbase) * Q.S];
    }
    if (g == 0) start[G] = (int32_t)total_rows;
}

// items of BIG rows per cluster and the float2 offset of every cluster's partials (one CTA)
__global__ void __launch_bounds__(1024) k_b_items(const int32_t *__restrict__ start, const int32_t *__restrict__ cd,
                                                  int64_t G, int32_t *__restrict__ item_start,
                                                  int64_t *__restrict__ pbase) {
    __shared__ int32_t sh[32];
    __shared__ long long shl[1024];
    const int64_t per = (G + 1023) / 1024;
    const int64_t g0 = (int64_t)threadIdx.x * per, g1 = min(G, g0 + per);
    int32_t vi = 0;
    long long ve = 0;
    for (int64_t g = g0; g < g1; ++g) {
        const int32_t ni = (int32_t)((start[g + 1] - start[g] + BIG - 1) / BIG);
        vi += ni;
        ve += (long long)ni * cd[g];
    }
    int32_t total;
    int32_t run = block_excl_scan(vi, sh, total);
    // exclusive scan of the 64-bit element counts (Hillis-Steele over 1024 threads in shared memory)
    shl[threadIdx.x] = ve;
    __syncthreads();
    for (int o = 1; o < 1024; o <<= 1) {
        const long long add = (int)threadIdx.x >= o ? shl[threadIdx.x - o] : 0;
        __syncthreads();
        shl[threadIdx.x] += add;
        __syncthreads();
    }
    long long ebase = shl[threadIdx.x] - ve;
    for (int64_t g = g0; g < g1; ++g) {
        const int32_t ni = (int32_t)((start[g + 1] - start[g] + BIG - 1) / BIG);
        item_start[g] = run;
        pbase[g] = ebase;
        run += ni;
        ebase += (long long)ni * cd[g];
    }
    if (threadIdx.x == 0) item_start[G] = total;
}

__device__ __forceinline__ DF df_add_b(DF a, DF b) {
    float s, e;
    two_sum(a.hi, b.hi, s, e);
    a.hi = s;
    a.lo = __fadd_rn(__fadd_rn(a.lo, b.lo), e);
    return a;
}

// one CTA per item (<= BIG rows of one cluster): sums of the rows shifted by the cluster's first
// row (as the single-problem k_segsum).  The 256 threads form rp row slots of dp columns (dp = d
// rounded up to a power of two in [32, 256], rp = 256 / dp): thread (slot, column) sums its column
// over the rows slot, slot + rp, ... four at a time (loads in flight together) into double-float
// accumulators; the slots are then combined in a fixed order.  Wider rows take several 256-column
// passes.
__global__ void __launch_bounds__(256) k_b_segsum(const BProb *__restrict__ probs, const PairInfo *__restrict__ pinfo,
                                                  const int32_t *__restrict__ cpair, const int32_t *__restrict__ perm,
                                                  const int32_t *__restrict__ start,
                                                  const int32_t *__restrict__ item_start,
                                                  const int64_t *__restrict__ pbase, int64_t G,
                                                  float2 *__restrict__ part_s, double *__restrict__ part_nq) {
    __shared__ float2 red2[256];
    __shared__ double qred[256];
    const int64_t item = blockIdx.x;
    if (item >= item_start[G]) return;
    const int64_t g = upper_index32(item_start, G, item);
    const PairInfo &Q = pinfo[cpair[g]];
    const BProb &P = probs[Q.p];
    const int64_t d = P.d;
    const int64_t it = item - item_start[g];
    const int64_t r0 = start[g] + it * BIG;
    const int rows = (int)min((int64_t)start[g + 1] - r0, BIG);
    const float *ref = P.X + (int64_t)perm[start[g]] * d;
    float2 *out = part_s + pbase[g] + it * d;
    const int tid = threadIdx.x;
    int dp = 32;
    while (dp < d && dp < 256) dp <<= 1;
    const int rp = 256 / dp, slot = tid / dp, cl = tid % dp;
    const int32_t *pr = perm + r0;
    DF qacc;
    for (int64_t cb = 0; cb < d; cb += dp) {
        const int64_t col = cb + cl;
        const bool act = col < d;
        const float c = act ? ref[col] : 0.f;
        DF sacc;
        int r = slot;
        for (; r + 3 * rp < rows; r += 4 * rp) {
            float v[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) v[u] = act ? __ldg(P.X + (int64_t)pr[r + u * rp] * d + col) : c;
            float sb = 0.f, qb = 0.f;
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const float t = __fsub_rn(v[u], c);
                sb = __fadd_rn(sb, t);
                qb = __fmaf_rn(t, t, qb);
            }
            sacc.add(sb);
            qacc.add(qb);
        }
        for (; r < rows; r += rp) {
            const float t = act ? __fsub_rn(__ldg(P.X + (int64_t)pr[r] * d + col), c) : 0.f;
            sacc.add(t);
            qacc.add(__fmul_rn(t, t));
        }
        // combine the row slots of each column in slot order
        red2[tid] = make_float2(sacc.hi, sacc.lo);
        __syncthreads();
        if (slot == 0 && act) {
            DF tot;
            tot.hi = red2[cl].x, tot.lo = red2[cl].y;
            for (int q = 1; q < rp; ++q) {
                const float2 o = red2[q * dp + cl];
                float hs, he;
                two_sum(tot.hi, o.x, hs, he);
                tot.hi = hs;
                tot.lo = __fadd_rn(__fadd_rn(tot.lo, o.y), he);
            }
            out[col] = make_float2(tot.hi, tot.lo);
        }
        __syncthreads();
    }
    const double q = block_tree_sum_d(qacc.value(), qred);
    if (tid == 0) {
        part_nq[item * 2] = (double)rows;
        part_nq[item * 2 + 1] = q;
    }
}

// one CTA per (global cluster, 256 columns): centroid into the other center buffer and CF cost terms
__global__ void __launch_bounds__(256) k_b_finalize(const BProb *__restrict__ probs, const PairInfo *__restrict__ pinfo,
                                                    const int32_t *__restrict__ cpair, const int32_t *__restrict__ perm,
                                                    const int32_t *__restrict__ start,
                                                    const int32_t *__restrict__ item_start,
                                                    const int64_t *__restrict__ pbase, const float2 *__restrict__ part_s,
                                                    const double *__restrict__ part_nq, int par, int64_t maxcb,
                                                    double *__restrict__ nq, double *__restrict__ blk) {
    __shared__ double sh[256];
    const int64_t g = blockIdx.x, cb = blockIdx.y;
    const PairInfo &Q = pinfo[cpair[g]];
    const BProb &P = probs[Q.p];
    const int64_t d = P.d, j = g - Q.gbase;
    if (cb * 256 >= d) {
        if (threadIdx.x == 0) blk[(g * maxcb + cb) * 2] = blk[(g * maxcb + cb) * 2 + 1] = 0.0;
        return;
    }
    const int32_t i0 = item_start[g], i1 = item_start[g + 1];
    double n_part = 0.0, q_part = 0.0;
    for (int32_t it = i0 + (int32_t)threadIdx.x; it < i1; it += (int32_t)blockDim.x) {
        n_part += part_nq[(int64_t)it * 2];
        q_part += part_nq[(int64_t)it * 2 + 1];
    }
    const double N = block_tree_sum_d(n_part, sh);
    const double Qt = block_tree_sum_d(q_part, sh);
    double a_old = 0.0, b_sq = 0.0;
    const int64_t t = cb * 256 + threadIdx.x;
    const float *co_row = P.C[par] + ((int64_t)Q.s * P.k + j) * d;
    float *cn_row = P.C[par ^ 1] + ((int64_t)Q.s * P.k + j) * d;
    if (t < d) {
        DF acc;
        for (int32_t it = i0; it < i1; ++it) {
            const float2 pv = part_s[pbase[g] + (int64_t)(it - i0) * d + t];
            DF o;
            o.hi = pv.x, o.lo = pv.y;
            acc = df_add_b(acc, o);
        }
        const double Sp = acc.value();
        const float co = co_row[t];
        if (N > 0.0) {
            const double sref = (double)P.X[(int64_t)perm[start[g]] * d + t];
            const double e = sref - (double)co;
            a_old = 2.0 * e * Sp + N * e * e;
            b_sq = Sp * Sp;
            cn_row[t] = (float)(sref + Sp / N);
        } else {
            cn_row[t] = co;
        }
    }
    const double at = block_tree_sum_d(a_old, sh);
    const double bt = block_tree_sum_d(b_sq, sh);
    if (threadIdx.x == 0) {
        if (cb == 0) {
            nq[g * 2] = N;
            nq[g * 2 + 1] = Qt;
        }
        blk[(g * maxcb + cb) * 2] = at;
        blk[(g * maxcb + cb) * 2 + 1] = bt;
    }
}

// empty clusters (no item) keep their center: the finalize grid covers only clusters with items
// through N = 0; one CTA per pair sums its clusters' costs
__global__ void __launch_bounds__(256) k_b_final(const BProb *__restrict__ probs, const PairInfo *__restrict__ pinfo,
                                                 const double *__restrict__ nq, const double *__restrict__ blk,
                                                 int64_t maxcb, double *__restrict__ costs) {
    __shared__ double sh[256];
    const PairInfo &Q = pinfo[blockIdx.x];
    const BProb &P = probs[Q.p];
    double x = 0.0, y = 0.0;
    for (int64_t j = threadIdx.x; j < P.k; j += 256) {
        const int64_t g = Q.gbase + j;
        const double N = nq[g * 2], Qt = nq[g * 2 + 1];
        double a = 0.0, b = 0.0;
        for (int64_t c = 0; c < maxcb; ++c) {
            a += blk[(g * maxcb + c) * 2];
            b += blk[(g * maxcb + c) * 2 + 1];
        }
        if (N > 0.0) {
            x += Qt + a;
            y += Qt - b / N;
        }
    }
    x = block_tree_sum_d(x, sh);
    y = block_tree_sum_d(y, sh);
    if (threadIdx.x == 0) {
        costs[blockIdx.x * 2] = x;
        costs[blockIdx.x * 2 + 1] = y;
    }
}

// results to the caller's buffers
__global__ void __launch_bounds__(256) k_b_out(const BProb *__restrict__ probs, const PairInfo *__restrict__ pinfo,
                                               const gbkm_problem *__restrict__ up, const double *__restrict__ costs,
                                               int par) {
    const PairInfo &Q = pinfo[blockIdx.x];
    const BProb &P = probs[Q.p];
    const gbkm_problem &U = up[Q.p];
    const float *c = P.C[par] + (int64_t)Q.s * P.k * P.d;
    for (int64_t e = threadIdx.x; e < P.k * P.d; e += 256) U.C_out[(int64_t)Q.s * P.k * P.d + e] = c[e];
    if (U.labels_out)
        for (int64_t e = threadIdx.x; e < P.n; e += 256)
            U.labels_out[(int64_t)Q.s * P.n + e] = P.labels[(int64_t)Q.s * P.n + e];
    if (U.cost_out && threadIdx.x == 0) {
        U.cost_out[Q.s * 2] = costs[blockIdx.x * 2];
        U.cost_out[Q.s * 2 + 1] = costs[blockIdx.x * 2 + 1];
    }
}

// ---------------------------------------------------------------- host orchestration
namespace {
template <class T>
T *carve(char *&cur, size_t count, size_t align = 256) {
    uintptr_t a = (reinterpret_cast<uintptr_t>(cur) + align - 1) & ~(uintptr_t)(align - 1);
    T *p = reinterpret_cast<T *>(a);
    cur = reinterpret_cast<char *>(a + count * sizeof(T));
    return p;
}
}  // namespace

int batch_run(gbkm_ctx *c, const gbkm_problem *up, int64_t count, int64_t seeds, int64_t iters, int dtype,
              int flags, const int *bn_caps) {
    const bool bf = dtype == GBKM_BF16;
    const int64_t S = seeds;
    // ---- plan
    std::vector<BProb> P(count);
    int64_t tiles = 0, blocks = 0, crows = 0, nseg = 0, G = 0, hist_total = 0, rows_total = 0, items_max = 0;
    int64_t kmax = 0, dmax = 0, maxcb = 1, pelems = 0;
    size_t wbytes = 0;
    int bn_max = 16;
    for (int64_t p = 0; p < count; ++p) {
        BProb &b = P[p];
        memset(&b, 0, sizeof(b));
        b.X = up[p].X;
        b.n = up[p].n, b.d = up[p].d, b.k = up[p].k;
        b.kps = ceil_div(b.k, 16) * 16;
        b.seeds = (int32_t)S;
        b.m_tiles = (int32_t)ceil_div(b.n, 128);
        const int64_t ncols = S * b.kps;
        const int cap = bn_caps ? bn_caps[p] : 256;
        b.n_chunks = (int32_t)ceil_div(ncols, cap);
        b.bn = (int32_t)(ceil_div(ceil_div(ncols, b.n_chunks), 16) * 16);
        const int64_t es = bf ? 2 : 4;
        b.kb = (int32_t)ceil_div(b.d * es, 128);
        b.nb = (int32_t)ceil_div(b.n, RB);
        const uint32_t ab = bf ? 1u : 2u;
        b.idesc = (1u << 4) | (ab << 7) | (ab << 10) | ((uint32_t)(b.bn >> 3) << 17) | ((uint32_t)(128 >> 4) << 24);
        b.tx_bytes = 128u * 128u + (bf ? 1u : 2u) * (uint32_t)b.bn * 128u;
        score_error_coeffs(dtype, 1, b.d, b.err_rel, b.err_abs);
        b.u = up[p].u;
        b.pair0 = p * S;
        b.crow0 = crows;
        b.tile0 = tiles;
        tiles += b.m_tiles;
        blocks += b.nb;
        crows += S * b.kps;
        const int64_t S_seg = ceil_div(b.n, SEGR);
        nseg += S * S_seg;
        hist_total += S * b.k * S_seg;
        G += S * b.k;
        rows_total += S * b.n;
        items_max += S * (ceil_div(b.n, BIG) + b.k);
        pelems += S * (ceil_div(b.n, BIG) + b.k) * b.d;
        kmax = std::max(kmax, b.k);
        dmax = std::max(dmax, b.d);
        bn_max = std::max(bn_max, b.bn);
        // per-problem device buffers (sizes; carved below)
        wbytes += 256 * 14 + b.n * 4 + (bf ? b.n * b.d * 2 : 0) + 2 * S * b.k * b.d * 4 + S * b.kps * 4 + 4 +
                  S * b.kps * b.d * (bf ? 2 : 8) + S * b.n * 4 + S * b.n * 8 + S * b.n * 4 + S * b.n * 4 +
                  S * b.k * 4 + S * 8 + 2 * 256 + S * b.nb * 8 + S * 4;
    }
    maxcb = std::max<int64_t>(1, ceil_div(dmax, 256));
    const int64_t npairs = count * S;
    const int64_t nbs = ceil_div(hist_total, 4096);
    wbytes += 4096 + count * (sizeof(BProb) + 3 * 128 + sizeof(gbkm_problem) + 8) + tiles * 4 + blocks * 8 +
              npairs * (8 + sizeof(PairInfo)) + nseg * 8 + G * (4 + 4 + 4 + 8 + 16 + 16 * maxcb) + 2 * hist_total * 4 +
              nbs * 4 + rows_total * 4 + items_max * 16 + pelems * 8 + npairs * 16 + (int64_t)count * 4 +
              rows_total * BFLAG_STRIDE * 4 + 64 * 256 + blocks * 8 + npairs * 8 + 2 * 256;
    int rc = GBKM_OK;
    void *ws = ws_reserve(c, wbytes, &rc);
    if (!ws) return rc;
    char *cur = static_cast<char *>(ws);
    // ---- per-problem buffers
    for (int64_t p = 0; p < count; ++p) {
        BProb &b = P[p];
        b.xnorm = carve<float>(cur, b.n);
        b.Xop = bf ? static_cast<const void *>(carve<__nv_bfloat16>(cur, b.n * b.d)) : static_cast<const void *>(b.X);
        b.C[0] = carve<float>(cur, S * b.k * b.d);
        b.C[1] = carve<float>(cur, S * b.k * b.d);
        b.cnorm = carve<float>(cur, S * b.kps);
        b.cop = bf ? static_cast<void *>(carve<__nv_bfloat16>(cur, S * b.kps * b.d)) : static_cast<void *>(carve<float>(cur, S * b.kps * b.d));
        b.cop_lo = bf ? nullptr : static_cast<void *>(carve<float>(cur, S * b.kps * b.d));
        b.labels = carve<int32_t>(cur, S * b.n);
        b.D2 = carve<double>(cur, S * b.n);
        b.D2f = carve<float>(cur, S * b.n);
        b.A = carve<int32_t>(cur, S * b.n);
        b.ccf = carve<float>(cur, S * b.k);
        b.dirty = carve<int64_t>(cur, S);
        b.bsum = carve<double>(cur, S * b.nb);
        b.stop = carve<int32_t>(cur, S);
    }
    unsigned *d_cmax = carve<unsigned>(cur, count);
    for (int64_t p = 0; p < count; ++p) P[p].cmax = d_cmax + p;
    BProb *d_probs = carve<BProb>(cur, count);
    CUtensorMap *d_maps = carve<CUtensorMap>(cur, 3 * count, 128);
    gbkm_problem *d_up = carve<gbkm_problem>(cur, count);
    int32_t *d_tile_prob = carve<int32_t>(cur, tiles);
    int2 *d_blocks = carve<int2>(cur, blocks);
    int2 *d_pairs = carve<int2>(cur, npairs);
    // the same tables with the problems in decreasing k: round r of the seeding launches only the
    // prefix of problems with k > r
    int2 *d_sblocks = carve<int2>(cur, blocks);
    int2 *d_spairs = carve<int2>(cur, npairs);
    PairInfo *d_pinfo = carve<PairInfo>(cur, npairs);
    int2 *d_segs = carve<int2>(cur, nseg);
    int64_t *d_crow0 = carve<int64_t>(cur, count);
    int32_t *d_cpair = carve<int32_t>(cur, G);
    int32_t *d_cd = carve<int32_t>(cur, G);
    int32_t *d_hist = carve<int32_t>(cur, hist_total);
    int32_t *d_off = carve<int32_t>(cur, hist_total);
    int32_t *d_bsum = carve<int32_t>(cur, nbs);
    int32_t *d_start = carve<int32_t>(cur, G + 1);
    int32_t *d_items = carve<int32_t>(cur, G + 1);
    int64_t *d_pbase = carve<int64_t>(cur, G);
    int32_t *d_perm = carve<int32_t>(cur, rows_total);
    float2 *d_part = carve<float2>(cur, pelems);
    double *d_pnq = carve<double>(cur, items_max * 2);
    double *d_nq = carve<double>(cur, G * 2);
    double *d_blk = carve<double>(cur, G * maxcb * 2);
    double *d_costs = carve<double>(cur, npairs * 2);
    int32_t *d_flags = carve<int32_t>(cur, rows_total * BFLAG_STRIDE);
    int32_t *d_fcount = carve<int32_t>(cur, 1);
    if ((size_t)(cur - static_cast<char *>(ws)) > c->ws_bytes)
        return set_error(c, GBKM_ENOMEM, "batched workspace plan overflow");
    // ---- host tables
    std::vector<CUtensorMap> maps(3 * count);
    std::vector<int32_t> tile_prob(tiles);
    std::vector<int2> blk_tab(blocks), pairs(npairs), segs(nseg);
    std::vector<PairInfo> pinfo(npairs);
    std::vector<int64_t> crow0(count);
    std::vector<int32_t> cpair(G), cdv(G);
    int64_t ti = 0, bi = 0, si = 0, hb = 0, gb = 0;
    for (int64_t p = 0; p < count; ++p) {
        const BProb &b = P[p];
        if ((rc = make_batch_tmaps(c, dtype, b, &maps[3 * p])) != GBKM_OK) return rc;
        for (int t = 0; t < b.m_tiles; ++t) tile_prob[ti++] = (int32_t)p;
        for (int64_t r = 0; r < b.n; r += RB) blk_tab[bi++] = make_int2((int)p, (int)r);
        crow0[p] = b.crow0;
        const int64_t S_seg = ceil_div(b.n, SEGR);
        for (int64_t s = 0; s < S; ++s) {
            const int64_t q = p * S + s;
            pairs[q] = make_int2((int)p, (int)s);
            PairInfo &pi = pinfo[q];
            pi.p = (int32_t)p, pi.s = (int32_t)s, pi.S = (int32_t)S_seg, pi.nseg_pad = 0;
            pi.hbase = hb, pi.gbase = gb, pi.seg0 = si;
            for (int64_t r = 0; r < b.n; r += SEGR) segs[si++] = make_int2((int)q, (int)r);
            for (int64_t j = 0; j < b.k; ++j) {
                cpair[gb + j] = (int32_t)q;
                cdv[gb + j] = (int32_t)b.d;
            }
            hb += b.k * S_seg;
            gb += b.k;
        }
    }
    std::vector<int64_t> ord(count);
    for (int64_t p = 0; p < count; ++p) ord[p] = p;
    std::stable_sort(ord.begin(), ord.end(), [&](int64_t x, int64_t y) { return P[x].k > P[y].k; });
    std::vector<int2> sblk_tab, spairs;
    std::vector<int64_t> sblk_pre(count + 1, 0);  // blocks of the first i problems in that order
    sblk_tab.reserve(blocks);
    spairs.reserve(npairs);
    for (int64_t i = 0; i < count; ++i) {
        const int64_t p = ord[i];
        for (int64_t r = 0; r < P[p].n; r += RB) sblk_tab.push_back(make_int2((int)p, (int)r));
        for (int64_t s2 = 0; s2 < S; ++s2) spairs.push_back(make_int2((int)p, (int)s2));
        sblk_pre[i + 1] = (int64_t)sblk_tab.size();
    }
    cudaStream_t st = c->stream;
    cudaError_t e = cudaSuccess;
#define CPY(dst, src, bytes) \
    if (e == cudaSuccess) e = cudaMemcpyAsync(dst, src, bytes, cudaMemcpyHostToDevice, st)
    CPY(d_probs, P.data(), sizeof(BProb) * count);
    CPY(d_maps, maps.data(), sizeof(CUtensorMap) * 3 * count);
    CPY(d_up, up, sizeof(gbkm_problem) * count);
    CPY(d_tile_prob, tile_prob.data(), 4 * tiles);
    CPY(d_blocks, blk_tab.data(), 8 * blocks);
    CPY(d_pairs, pairs.data(), 8 * npairs);
    CPY(d_sblocks, sblk_tab.data(), 8 * blocks);
    CPY(d_spairs, spairs.data(), 8 * npairs);
    CPY(d_pinfo, pinfo.data(), sizeof(PairInfo) * npairs);
    CPY(d_segs, segs.data(), 8 * nseg);
    CPY(d_crow0, crow0.data(), 8 * count);
    CPY(d_cpair, cpair.data(), 4 * G);
    CPY(d_cd, cdv.data(), 4 * G);
#undef CPY
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);  // host tables must outlive their copies
    if (e != cudaSuccess) return cuda_check(c, e, "batched tables");
    // ---- the run (recorded into one graph when asked, on a private stream: the caller's stream may
    // be the legacy default stream, which cannot be captured; the graph is launched on it)
    const bool graph = flags & 1;
    cudaGraph_t g = nullptr;
    const cudaStream_t user_stream = c->stream;
    const int64_t launches0 = c->launches;  // the kernels recorded below are counted as they are queued
    if (graph) {
        if (!c->cap_stream) {
            e = cudaStreamCreateWithFlags(&c->cap_stream, cudaStreamNonBlocking);
            if (e != cudaSuccess) return cuda_check(c, e, "capture stream");
        }
        c->stream = st = c->cap_stream;
        e = cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal);
        if (e != cudaSuccess) {
            c->stream = user_stream;
            return cuda_check(c, e, "begin capture");
        }
    }
    const size_t hsm = sizeof(int32_t) * 8 * (size_t)kmax;
    if (hsm > 48 * 1024) {
        cudaFuncSetAttribute(k_b_hist, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)hsm);
        cudaFuncSetAttribute(k_b_scatter, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)hsm);
    }
    int64_t kmax_all = 0;
    for (auto &b : P) kmax_all = std::max(kmax_all, b.k);
    // per-kernel timing brackets only outside a capture (a recorded graph is timed as a whole)
    auto pb = [&](const char *name) {
        if (!graph) prof_begin(c, name);
    };
    auto pe = [&]() {
        if (!graph) prof_end(c);
    };
    k_b_prep<<<(unsigned)blocks, 256, 0, st>>>(d_probs, d_blocks, bf ? 1 : 0);
    pb("seed_batched");
    k_b_seed_first<<<(unsigned)npairs, 128, 0, st>>>(d_probs, d_pairs);
    c->launches += 2;
    int64_t na = count;  // problems with k > r: a prefix of the decreasing-k order
    for (int r = 1; r < kmax_all; ++r) {
        while (na > 0 && P[ord[na - 1]].k <= r) --na;
        const unsigned nbl = (unsigned)sblk_pre[na], npr = (unsigned)(na * S);
        if (r >= 2) {
            k_b_cc<<<dim3((unsigned)ceil_div((int64_t)(r - 1) * 32, 256), npr), 256, 0, st>>>(d_probs, d_spairs, r);
            c->launches += 1;
        }
        k_b_d2<<<nbl, 256, 0, st>>>(d_probs, d_sblocks, r);
        k_b_pick<<<npr, PICKB_T, 0, st>>>(d_probs, d_spairs, r, c->status);
        c->launches += 2;
    }
    pe();
    int par = 0;
    for (int64_t it = 0; it < iters; ++it) {
        e = cudaMemsetAsync(d_cmax, 0, 4 * count, st);
        if (e == cudaSuccess) e = cudaMemsetAsync(d_fcount, 0, 4, st);
        if (e != cudaSuccess) break;
        k_b_cprep<<<(unsigned)crows, 128, 0, st>>>(d_probs, d_crow0, count, par, bf ? 1 : 0);
        c->launches += 1;
        pb("assign_batched");
        rc = launch_assign_tc_batched(c, dtype, d_maps, d_probs, count, d_tile_prob, tiles, par, bn_max, d_flags,
                                      d_fcount);
        pe();
        if (rc != GBKM_OK) break;
        pb("recheck_batched");
        k_b_recheck<<<(unsigned)c->sm_count * 4, 256, 0, st>>>(d_probs, d_flags, d_fcount, par);
        pe();
        pb("update_batched");
        k_b_hist<<<(unsigned)ceil_div(nseg, 8), 256, hsm, st>>>(d_probs, d_pinfo, d_segs, nseg, kmax, d_hist);
        scan_excl(st, d_hist, hist_total, d_bsum, d_off);
        k_b_starts<<<(unsigned)ceil_div(G, 256), 256, 0, st>>>(d_pinfo, d_cpair, d_off, G, rows_total, d_start);
        k_b_scatter<<<(unsigned)ceil_div(nseg, 8), 256, hsm, st>>>(d_probs, d_pinfo, d_segs, nseg, kmax, d_off, d_perm);
        k_b_items<<<1, 1024, 0, st>>>(d_start, d_cd, G, d_items, d_pbase);
        k_b_segsum<<<(unsigned)items_max, 256, 0, st>>>(d_probs, d_pinfo, d_cpair, d_perm, d_start, d_items, d_pbase, G,
                                                         d_part, d_pnq);
        k_b_finalize<<<dim3((unsigned)G, (unsigned)maxcb), 256, 0, st>>>(d_probs, d_pinfo, d_cpair, d_perm, d_start,
                                                                          d_items, d_pbase, d_part, d_pnq, par, maxcb,
                                                                          d_nq, d_blk);
        k_b_final<<<(unsigned)npairs, 256, 0, st>>>(d_probs, d_pinfo, d_nq, d_blk, maxcb, d_costs);
        pe();
        c->launches += 11;
        par ^= 1;
    }
    if (rc == GBKM_OK && e == cudaSuccess) {
        k_b_out<<<(unsigned)npairs, 256, 0, st>>>(d_probs, d_pinfo, d_up, d_costs, par);
        c->launches += 1;
    }
    cudaError_t le = cudaGetLastError();
    if (graph) {
        cudaError_t ee = cudaStreamEndCapture(st, &g);
        c->stream = st = user_stream;
        if (rc != GBKM_OK || e != cudaSuccess || le != cudaSuccess || ee != cudaSuccess) {
            if (g) cudaGraphDestroy(g);
            if (rc != GBKM_OK) return rc;
            return cuda_check(c, e != cudaSuccess ? e : (le != cudaSuccess ? le : ee), "batched capture");
        }
        cudaGraphExec_t ex = nullptr;
        e = cudaGraphInstantiate(&ex, g, 0);
        cudaGraphDestroy(g);
        if (e != cudaSuccess) return cuda_check(c, e, "graph instantiate");
        if (c->graph_exec) cudaGraphExecDestroy((cudaGraphExec_t)c->graph_exec);
        c->graph_exec = ex;
        c->graph_epoch = c->ws_epoch;
        c->graph_launches = c->launches - launches0;  // already counted once: this first launch
        e = cudaGraphLaunch(ex, st);
        if (e != cudaSuccess) return cuda_check(c, e, "graph launch");
        return GBKM_OK;
    }
    if (rc != GBKM_OK) return rc;
    if (e != cudaSuccess) return cuda_check(c, e, "batched run");
    return cuda_check(c, le, "batched launches");
}

}  // namespace gbkm
