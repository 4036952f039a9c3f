// k_update.cu -- A6 centroid update through clustering features and A7 cost (CF identity).
//
// Pipeline (all on the context's stream, no host synchronisation, no float atomics):
//   1. k_hist      one warp per label segment: warp-aggregated (match_any) label histogram,
//                  column s of the cluster-major table hist[j * S + s]
//   2. offsets     k <= 2048 (per-warp tables in shared memory): k_row_scan, one CTA per cluster
//                  scanning its row, the last CTA deriving the cluster starts and the work items;
//                  otherwise a device-wide exclusive scan of the table, k_starts and k_items
//   3. k_scatter   one warp per segment: stable rank inside the warp + running slot -> perm
//                  (work items: chunks of R rows per cluster, item_start = their exclusive scan)
//   4. k_segsum    one CTA per chunk of 128 rows: sums of w (x - s), w, w ||x - s||^2 with s the
//                  cluster's first row -> FP64 partials
//   5. k_fold      one CTA per (run of 32 work items, 256 columns): double-float sums of each
//                  cluster's partials inside the run, so no cluster's sum is one long chain
//   6. k_finalize  one CTA per (cluster, 256 columns): the cluster's folded sums in run order,
//                  centroid and CF cost terms
//   7. k_final     one CTA: FP64 totals in cluster order
#include <mutex>

#include "internal.cuh"

namespace gbkm {

namespace {
constexpr int SCAN_T = 1024, SCAN_E = 4;           // scan block: 1024 threads x 4 elements
constexpr int64_t CHUNK_R = 128;                    // rows per segmented-sum work item
constexpr int32_t FOLD_I = 32;                      // work items per k_fold run
constexpr int64_t SMEM_HIST_MAX_K = 2048;           // per-warp histograms in shared memory up to here
constexpr int HIST_PF = 8;                          // label steps a warp loads ahead

__device__ __forceinline__ unsigned lanemask_lt_u() {
    unsigned m;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
    return m;
}
}  // namespace

__global__ void __launch_bounds__(256) k_hist(const int32_t *__restrict__ labels, int64_t n, int64_t k,
                                              int64_t R, int64_t S, int32_t *__restrict__ hist,
                                              int *status) {
    const int lane = threadIdx.x & 31;
    const int64_t s = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    if (s >= S) return;
    const int64_t r0 = s * R, r1 = min(n, r0 + R);
    for (int64_t base = r0; base < r1; base += 32) {
        const int64_t i = base + lane;
        int32_t l = (i < r1) ? labels[i] : -1;
        bool ok = (i < r1) && l >= 0 && l < k;
        if (i < r1 && !ok) status_raise(status, ST_BADLABEL);
        const unsigned act = __ballot_sync(0xffffffffu, ok);
        if (ok) {
            const unsigned grp = __match_any_sync(act, l);
            volatile int32_t *slot = hist + (int64_t)l * S + s;  // column s belongs to this warp only
            if (lane == __ffs(grp) - 1) *slot = *slot + __popc(grp);
        }
        __syncwarp();
    }
}

__global__ void __launch_bounds__(256) k_scatter(const int32_t *__restrict__ labels, int64_t n, int64_t k,
                                                 int64_t R, int64_t S, int32_t *__restrict__ off,
                                                 int32_t *__restrict__ perm) {
    const int lane = threadIdx.x & 31;
    const int64_t s = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    if (s >= S) return;
    const int64_t r0 = s * R, r1 = min(n, r0 + R);
    for (int64_t base = r0; base < r1; base += 32) {
        const int64_t i = base + lane;
        int32_t l = (i < r1) ? labels[i] : -1;
        bool ok = (i < r1) && l >= 0 && l < k;
        const unsigned act = __ballot_sync(0xffffffffu, ok);
        if (ok) {
            const unsigned grp = __match_any_sync(act, l);
            volatile int32_t *slot = off + (int64_t)l * S + s;  // column s belongs to this warp only
            const int32_t pos = *slot + __popc(grp & lanemask_lt_u());
            perm[pos] = (int32_t)i;
            __syncwarp(act);
            if (lane == __ffs(grp) - 1) *slot = *slot + __popc(grp);
        }
        __syncwarp();
    }
}

// Shared-memory forms of the two label walks (k <= SMEM_HIST_MAX_K): each warp keeps its
// segment's counts (k_hist_sm) or running output slots (k_scatter_sm) in its own slice of shared
// memory, so the per-step read-modify-write never leaves the SM; every table entry is written
// (no clearing pass needed).
__global__ void __launch_bounds__(256) k_hist_sm(const int32_t *__restrict__ labels, int64_t n, int64_t k,
                                                 int64_t R, int64_t S, int32_t *__restrict__ hist,
                                                 int *status, int32_t *__restrict__ ticket) {
    extern __shared__ int32_t hsm[];
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    if (blockIdx.x == 0 && threadIdx.x == 0) *ticket = 0;  // for k_row_scan, which runs next
    const int64_t s = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    if (s >= S) return;
    volatile int32_t *mine = hsm + (int64_t)wib * k;
    for (int64_t j = lane; j < k; j += 32) mine[j] = 0;
    __syncwarp();
    const int64_t r0 = s * R, r1 = min(n, r0 + R);
    for (int64_t base = r0; base < r1; base += 32 * HIST_PF) {
        int32_t lab[HIST_PF];  // the next 32 * HIST_PF labels, loaded together
#pragma unroll
        for (int q = 0; q < HIST_PF; ++q) {
            const int64_t i = base + q * 32 + lane;
            lab[q] = (i < r1) ? labels[i] : INT32_MIN;
        }
#pragma unroll
        for (int q = 0; q < HIST_PF; ++q) {
            const int32_t l = lab[q];
            const bool ok = l >= 0 && l < k;
            if (l != INT32_MIN && !ok) status_raise(status, ST_BADLABEL);
            const unsigned act = __ballot_sync(0xffffffffu, ok);
            if (ok) {
                const unsigned grp = __match_any_sync(act, l);
                if (lane == __ffs(grp) - 1) mine[l] = mine[l] + __popc(grp);
            }
            __syncwarp();
        }
    }
    for (int64_t j = lane; j < k; j += 32) hist[j * S + s] = mine[j];
}

__global__ void __launch_bounds__(256) k_scatter_sm(const int32_t *__restrict__ labels, int64_t n, int64_t k,
                                                    int64_t R, int64_t S, const int32_t *__restrict__ off,
                                                    const int32_t *__restrict__ start, int32_t *__restrict__ perm) {
    extern __shared__ int32_t hsm[];
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    const int64_t s = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    if (s >= S) return;
    volatile int32_t *mine = hsm + (int64_t)wib * k;
    for (int64_t j = lane; j < k; j += 32) mine[j] = start[j] + off[j * S + s];
    __syncwarp();
    const int64_t r0 = s * R, r1 = min(n, r0 + R);
    for (int64_t base = r0; base < r1; base += 32 * HIST_PF) {
        int32_t lab[HIST_PF];
#pragma unroll
        for (int q = 0; q < HIST_PF; ++q) {
            const int64_t i = base + q * 32 + lane;
            lab[q] = (i < r1) ? labels[i] : INT32_MIN;
        }
#pragma unroll
        for (int q = 0; q < HIST_PF; ++q) {
            const int32_t l = lab[q];
            const bool ok = l >= 0 && l < k;
            const unsigned act = __ballot_sync(0xffffffffu, ok);
            if (ok) {
                const unsigned grp = __match_any_sync(act, l);
                const int32_t pos = mine[l] + __popc(grp & lanemask_lt_u());
                perm[pos] = (int32_t)(base + q * 32 + lane);
                __syncwarp(act);
                if (lane == __ffs(grp) - 1) mine[l] = mine[l] + __popc(grp);
            }
            __syncwarp();
        }
    }
}

// ---------------------------------------------------------------- device-wide exclusive scan
// (int32; totals < 2^31 because they count rows)
__global__ void __launch_bounds__(SCAN_T) k_scan_partial(const int32_t *__restrict__ in, int64_t L,
                                                         int32_t *__restrict__ bsum) {
    __shared__ int32_t sh[32];
    const int64_t base = (int64_t)blockIdx.x * SCAN_T * SCAN_E + (int64_t)threadIdx.x * SCAN_E;
    int32_t v = 0;
#pragma unroll
    for (int q = 0; q < SCAN_E; ++q)
        if (base + q < L) v += in[base + q];
    int32_t total;
    block_excl_scan(v, sh, total);
    if (threadIdx.x == 0) bsum[blockIdx.x] = total;
}

// single CTA: exclusive scan of nb block sums (sequential per thread over a contiguous range)
__global__ void __launch_bounds__(SCAN_T) k_scan_bsum(int32_t *__restrict__ bsum, int64_t nb) {
    __shared__ int32_t sh[32];
    const int64_t per = (nb + SCAN_T - 1) / SCAN_T;
    const int64_t b0 = (int64_t)threadIdx.x * per, b1 = min(nb, b0 + per);
    int32_t v = 0;
    for (int64_t b = b0; b < b1; ++b) v += bsum[b];
    int32_t total;
    int32_t run = block_excl_scan(v, sh, total);
    for (int64_t b = b0; b < b1; ++b) {
        int32_t t = bsum[b];
        bsum[b] = run;
        run += t;
    }
}

__global__ void __launch_bounds__(SCAN_T) k_scan_final(const int32_t *__restrict__ in, int64_t L,
                                                       const int32_t *__restrict__ bsum,
                                                       int32_t *__restrict__ out) {
    __shared__ int32_t sh[32];
    const int64_t base = (int64_t)blockIdx.x * SCAN_T * SCAN_E + (int64_t)threadIdx.x * SCAN_E;
    int32_t v[SCAN_E];
    int32_t tsum = 0;
#pragma unroll
    for (int q = 0; q < SCAN_E; ++q) {
        v[q] = (base + q < L) ? in[base + q] : 0;
        tsum += v[q];
    }
    int32_t total;
    int32_t run = block_excl_scan(tsum, sh, total) + bsum[blockIdx.x];
#pragma unroll
    for (int q = 0; q < SCAN_E; ++q) {
        if (base + q < L) out[base + q] = run;
        run += v[q];
    }
}

void scan_excl(cudaStream_t st, const int32_t *in, int64_t L, int32_t *bsum, int32_t *out) {
    const int64_t nb = ceil_div(L, (int64_t)SCAN_T * SCAN_E);
    k_scan_partial<<<(unsigned)nb, SCAN_T, 0, st>>>(in, L, bsum);
    k_scan_bsum<<<1, SCAN_T, 0, st>>>(bsum, nb);
    k_scan_final<<<(unsigned)nb, SCAN_T, 0, st>>>(in, L, bsum, out);
}

// start[j] = first sorted slot of cluster j, start[k] = number of valid rows
__global__ void k_starts(const int32_t *__restrict__ off, const int32_t *__restrict__ hist, int64_t k,
                         int64_t S, int32_t *__restrict__ start) {
    const int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (j < k) start[j] = off[j * S];
    if (j == k - 1) start[k] = off[(k - 1) * S + S - 1] + hist[(k - 1) * S + S - 1];
}

// work items: item_start[j] = sum_{j' < j} ceil(cnt_j' / R); item_start[k] = total
__global__ void __launch_bounds__(SCAN_T) k_items(const int32_t *__restrict__ start, int64_t k, int64_t R,
                                                  int32_t *__restrict__ item_start) {
    __shared__ int32_t sh[32];
    const int64_t per = (k + SCAN_T - 1) / SCAN_T;
    const int64_t j0 = (int64_t)threadIdx.x * per, j1 = min(k, j0 + per);
    int32_t v = 0;
    for (int64_t j = j0; j < j1; ++j) v += (int32_t)((start[j + 1] - start[j] + R - 1) / R);
    int32_t total;
    int32_t run = block_excl_scan(v, sh, total);
    for (int64_t j = j0; j < j1; ++j) {
        item_start[j] = run;
        run += (int32_t)((start[j + 1] - start[j] + R - 1) / R);
    }
    if (threadIdx.x == 0) item_start[k] = total;
}

// Offsets of the shared-memory path in one launch: one CTA per cluster j scans its row of the
// table, off[j, s] = sum_{s' < s} hist[j, s'] (relative to the cluster's first slot), and stores
// the row total cnt[j]; the last CTA to finish (atomic ticket, zeroed by k_hist_sm) turns the
// totals into start[] (exclusive scan over clusters, start[k] = valid rows) and item_start[]
// (work items of R rows per cluster, item_start[k] = total).  No CTA waits for another.
__global__ void __launch_bounds__(256) k_row_scan(const int32_t *__restrict__ hist, int64_t k, int64_t S,
                                                  int64_t R, int32_t *__restrict__ off, int32_t *cnt,
                                                  int32_t *__restrict__ start, int32_t *__restrict__ item_start,
                                                  int32_t *ticket) {
    __shared__ int32_t sh[32];
    __shared__ int last;
    // cluster j = blockIdx.x: every thread scans a contiguous range of the row, one block scan
    // places the ranges
    {
        const int64_t j = blockIdx.x;
        const int32_t *h = hist + j * S;
        int32_t *o = off + j * S;
        const int64_t per = (S + blockDim.x - 1) / blockDim.x;
        const int64_t s0 = min(S, (int64_t)threadIdx.x * per), s1 = min(S, s0 + per);
        int32_t v = 0;
        for (int64_t sx = s0; sx < s1; ++sx) v += h[sx];
        int32_t total;
        int32_t run = block_excl_scan(v, sh, total);
        for (int64_t sx = s0; sx < s1; ++sx) {
            const int32_t c = h[sx];
            o[sx] = run;
            run += c;
        }
        if (threadIdx.x == 0) cnt[j] = total;
    }
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) last = atomicAdd(ticket, 1) == (int)gridDim.x - 1;
    __syncthreads();
    if (!last) return;
    __threadfence();
    const volatile int32_t *vc = cnt;
    const int64_t per = (k + blockDim.x - 1) / blockDim.x;
    const int64_t j0 = (int64_t)threadIdx.x * per, j1 = min(k, j0 + per);
    int32_t rows = 0, items = 0;
    for (int64_t q = j0; q < j1; ++q) {
        const int32_t c = vc[q];
        rows += c;
        items += (int32_t)((c + R - 1) / R);
    }
    int32_t total_rows, total_items;
    int32_t r0 = block_excl_scan(rows, sh, total_rows);
    int32_t i0 = block_excl_scan(items, sh, total_items);
    for (int64_t q = j0; q < j1; ++q) {
        const int32_t c = vc[q];
        start[q] = r0;
        item_start[q] = i0;
        r0 += c;
        i0 += (int32_t)((c + R - 1) / R);
    }
    if (threadIdx.x == 0) {
        start[k] = total_rows;
        item_start[k] = total_items;
    }
}

// ---------------------------------------------------------------- segmented CF sums
// One CTA (256 threads) per work item = up to R rows of one cluster j in sorted order.  Sums are
// taken of the rows shifted by the cluster's reference row s_j (its first row in sorted order, a
// point of the same cluster, so the shifted values are of the size of the cluster's spread):
// S'_c = sum w (x - s_j), Q'_c = sum w ||x - s_j||^2, N_c = sum w.  Every FP32 cancellation is
// therefore bounded by the cluster's own scatter; k_finalize moves the cluster's sums to other
// references exactly.  Each thread keeps UNR row loads in flight (16 when the G row groups times 16
// rows do not exceed an item, else 8; row offsets staged in shared memory, the tail padded with the
// reference row at weight 0), sums S over UNR-row blocks and Q over 4-row blocks in FP32 and adds
// every block into a double-float accumulator (error-free
// TwoSum); the G = 256 / tpr row groups are combined in double-float in group order.  The item's
// S' is stored as (hi, lo) float pairs, its N and Q' in FP64.  Small items (R = 128 rows) keep
// every SM busy to the end.

__device__ __forceinline__ DF df_add(DF a, DF b) {
    float s, e;
    two_sum(a.hi, b.hi, s, e);
    a.hi = s;
    a.lo = __fadd_rn(__fadd_rn(a.lo, b.lo), e);
    return a;
}

template <int VW, bool WEIGHTED, int SEG_UNROLL>
__global__ void __launch_bounds__(256) k_segsum(const float *__restrict__ X, int64_t d,
                                                const float *__restrict__ w,
                                                const int32_t *__restrict__ perm,
                                                const int32_t *__restrict__ start,
                                                const int32_t *__restrict__ item_start, int64_t k,
                                                int64_t R, float2 *__restrict__ part_s,
                                                double *__restrict__ part_nq) {
    __shared__ int64_t roff_s[CHUNK_R + SEG_UNROLL * 256];
    __shared__ float w_s[CHUNK_R + SEG_UNROLL * 256];
    __shared__ float2 red[256 * VW];
    __shared__ double qred[256];
    const int64_t item = blockIdx.x;
    const int32_t total = item_start[k];
    if (item >= total) return;
    // cluster of this item: largest j with item_start[j] <= item
    int64_t lo = 0, hi = k - 1;
    while (lo < hi) {
        int64_t mid = (lo + hi + 1) >> 1;
        if (item_start[mid] <= item) lo = mid;
        else hi = mid - 1;
    }
    const int64_t j = lo;
    const int64_t row0 = start[j] + (item - item_start[j]) * R;
    const int rows = (int)min((int64_t)start[j + 1] - row0, R);
    const int tid = threadIdx.x;
    const int64_t ref_off = (int64_t)perm[start[j]] * d;
    const int64_t ncv = d / VW;
    // largest row stride any column pass uses (the last pass is the narrowest): rows are padded
    // up to a multiple of Gmax * SEG_UNROLL, which CHUNK_R + SEG_UNROLL * 256 always covers
    const int last_pass = (int)(ncv - ((ncv - 1) / 256) * 256);
    int tpr0 = 1;
    while (tpr0 < last_pass) tpr0 <<= 1;
    const int Gmax = 256 / tpr0;
    const int rows_pad = ((rows + Gmax * SEG_UNROLL - 1) / (Gmax * SEG_UNROLL)) * (Gmax * SEG_UNROLL);
    for (int r = tid; r < rows_pad; r += 256) {
        const bool real = r < rows;
        const int32_t i = real ? perm[row0 + r] : 0;
        roff_s[r] = real ? (int64_t)i * d : ref_off;
        w_s[r] = real ? (WEIGHTED ? w[i] : 1.f) : 0.f;
    }
    __syncthreads();
    double wpart = 0.0;
    for (int r = tid; r < rows; r += 256) wpart += (double)w_s[r];
    const double wsum_s = block_tree_sum_d(wpart, qred);
    float2 *out_s = part_s + item * d;
    const float *ref = X + ref_off;
    DF qacc;
    for (int64_t cb = 0; cb < ncv; cb += 256) {
        const int pass = (int)min((int64_t)256, ncv - cb);
        int tpr = 1;
        while (tpr < pass) tpr <<= 1;
        const int G = 256 / tpr, g = tid / tpr, cv = tid % tpr;
        const bool active = cv < pass;
        DF sacc[VW];
        if (active) {
            const int64_t col = (cb + cv) * VW;
            float c[VW];
            if constexpr (VW == 4) {
                const float4 c4 = __ldg(reinterpret_cast<const float4 *>(ref + col));
                c[0] = c4.x, c[1] = c4.y, c[2] = c4.z, c[3] = c4.w;
            } else {
                c[0] = __ldg(ref + col);
            }
            for (int r = g; r < rows; r += G * SEG_UNROLL) {
                float v[SEG_UNROLL][VW];
#pragma unroll
                for (int u = 0; u < SEG_UNROLL; ++u) {
                    const float *xr = X + roff_s[r + u * G] + col;
                    if constexpr (VW == 4) {
                        const float4 q4 = __ldg(reinterpret_cast<const float4 *>(xr));
                        v[u][0] = q4.x, v[u][1] = q4.y, v[u][2] = q4.z, v[u][3] = q4.w;
                    } else {
                        v[u][0] = __ldg(xr);
                    }
                }
                float sb[VW];
#pragma unroll
                for (int q = 0; q < VW; ++q) sb[q] = 0.f;
#pragma unroll
                for (int b = 0; b < SEG_UNROLL; b += 4) {
                    float qb[VW];
#pragma unroll
                    for (int q = 0; q < VW; ++q) qb[q] = 0.f;
#pragma unroll
                    for (int u = b; u < b + 4; ++u) {
                        if constexpr (WEIGHTED) {
                            const float wt = w_s[r + u * G];
#pragma unroll
                            for (int q = 0; q < VW; ++q) {
                                const float t = __fsub_rn(v[u][q], c[q]);
                                const float wtt = __fmul_rn(wt, t);
                                sb[q] = __fadd_rn(sb[q], wtt);
                                qb[q] = __fmaf_rn(wtt, t, qb[q]);
                            }
                        } else {
                            // padded rows repeat the reference row, so t = 0 there
#pragma unroll
                            for (int q = 0; q < VW; ++q) {
                                const float t = __fsub_rn(v[u][q], c[q]);
                                sb[q] = __fadd_rn(sb[q], t);
                                qb[q] = __fmaf_rn(t, t, qb[q]);
                            }
                        }
                    }
                    float qs = qb[0];
#pragma unroll
                    for (int q = 1; q < VW; ++q) qs = __fadd_rn(qs, qb[q]);
                    qacc.add(qs);
                }
#pragma unroll
                for (int q = 0; q < VW; ++q) sacc[q].add(sb[q]);
            }
        }
#pragma unroll
        for (int q = 0; q < VW; ++q) red[tid * VW + q] = active ? make_float2(sacc[q].hi, sacc[q].lo) : make_float2(0.f, 0.f);
        __syncthreads();
        for (int e = tid; e < pass * VW; e += 256) {
            const int cvv = e / VW, q = e % VW;
            DF acc;
            for (int gg = 0; gg < G; ++gg) {
                const float2 t2 = red[(gg * tpr + cvv) * VW + q];
                DF o;
                o.hi = t2.x;
                o.lo = t2.y;
                acc = df_add(acc, o);
            }
            out_s[(cb + cvv) * VW + q] = make_float2(acc.hi, acc.lo);
        }
        __syncthreads();
    }
    const double qtot = block_tree_sum_d(qacc.value(), qred);
    if (tid == 0) {
        part_nq[item * 2] = wsum_s;
        part_nq[item * 2 + 1] = qtot;
    }
}

// Work items are ordered by cluster, so the items of run g = [32 g, 32 g + 32) belong to a
// contiguous range of clusters.  One CTA per (run g, block of 256 columns) sums, per column, the
// items of each cluster j it touches and writes that sum to slot g + j: along the item order both
// g and j only grow (and one of them grows between two consecutive (run, cluster) pairs), so no two
// pairs share a slot, and there are fewer than runs + k slots.  Cluster j's slots are then
// g + j for g from its first item's run to its last item's run.
__global__ void __launch_bounds__(256) k_fold(const float2 *__restrict__ part_s,
                                              const int32_t *__restrict__ item_start, int64_t k, int64_t d,
                                              float2 *__restrict__ fold_s) {
    const int32_t total = item_start[k];
    const int32_t a = (int32_t)blockIdx.x * FOLD_I;
    if (a >= total) return;
    const int32_t b = min(a + FOLD_I, total);
    const int64_t t = (int64_t)blockIdx.y * 256 + threadIdx.x;
    if (t >= d) return;
    // cluster of item a: largest j with item_start[j] <= a
    int64_t lo = 0, hi = k - 1;
    while (lo < hi) {
        const int64_t mid = (lo + hi + 1) >> 1;
        if (item_start[mid] <= a) lo = mid;
        else hi = mid - 1;
    }
    for (int64_t j = lo; j < k && item_start[j] < b; ++j) {
        const int32_t s0 = max(item_start[j], a), s1 = min(item_start[j + 1], b);
        if (s0 >= s1) continue;
        DF acc[8];
        int32_t it = s0;
        for (; it + 8 <= s1; it += 8) {
#pragma unroll
            for (int q = 0; q < 8; ++q) {
                const float2 p = part_s[(int64_t)(it + q) * d + t];
                DF o;
                o.hi = p.x, o.lo = p.y;
                acc[q] = df_add(acc[q], o);
            }
        }
        for (int q = 0; it < s1; ++it, ++q) {
            const float2 p = part_s[(int64_t)it * d + t];
            DF o;
            o.hi = p.x, o.lo = p.y;
            acc[q] = df_add(acc[q], o);
        }
#pragma unroll
        for (int q = 1; q < 8; ++q) acc[0] = df_add(acc[0], acc[q]);
        fold_s[((int64_t)blockIdx.x + j) * d + t] = make_float2(acc[0].hi, acc[0].lo);
    }
}

// One CTA per (cluster j, block of 256 columns).  Sums of the cluster's items (N_j, Q'_j in FP64,
// in item order; S'_j in double-float, over the cluster's k_fold slots in run order) are its CF
// shifted by the reference row s_j.  Then, in
// FP64 (Section 2.1's CF identity: sum_x ||x - y||^2 = Q' + 2 (s - y) . S' + N ||s - y||^2):
//   centroid         mu_j = s_j + S'_j / N_j
//   cost of c_old    Q'_j + sum_t [2 (s_t - c_t) S'_t + N (s_t - c_t)^2]
//   cost of mu_j     Q'_j - ||S'_j||^2 / N_j
// The per-column terms are summed per block here and across blocks by k_final.
__global__ void __launch_bounds__(256) k_finalize(const float2 *__restrict__ fold_s,
                                                  const double *__restrict__ part_nq,
                                                  const float *__restrict__ X, const int32_t *__restrict__ perm,
                                                  const int32_t *__restrict__ start, int64_t d, int64_t k,
                                                  const int32_t *__restrict__ item_start,
                                                  const float *__restrict__ C_old, float *__restrict__ C_new,
                                                  double *__restrict__ counts, double *__restrict__ nq,
                                                  double *__restrict__ blk) {
    __shared__ double sh[3 * 256];
    __shared__ double inv_s;
    const int64_t j = blockIdx.x, cb = blockIdx.y;
    const int32_t i0 = item_start[j], i1 = item_start[j + 1];
    double n_part = 0.0, q_part = 0.0;
    for (int32_t it = i0 + (int32_t)threadIdx.x; it < i1; it += (int32_t)blockDim.x) {
        n_part += part_nq[(int64_t)it * 2];
        if (cb == 0) q_part += part_nq[(int64_t)it * 2 + 1];
    }
    const double N = block_tree_sum_d(n_part, sh);
    // one FP64 reciprocal per CTA (FP64 division is a long sequence on the slow FP64 pipe)
    if (threadIdx.x == 0) inv_s = N > 0.0 ? 1.0 / N : 0.0;
    __syncthreads();
    const double invN = inv_s;
    double a_old = 0.0, b_sq = 0.0;
    const int64_t t = cb * 256 + threadIdx.x;
    if (t < d) {
        // the cluster's slots g + j, g = first run .. last run (none for an empty cluster); 8
        // independent double-float accumulators keep 8 loads in flight, combined in order
        DF acc[8];
        if (i1 > i0) {
            const int64_t s0 = i0 / FOLD_I + j, s1 = (i1 - 1) / FOLD_I + j + 1;
            int64_t sl = s0;
            for (; sl + 8 <= s1; sl += 8) {
#pragma unroll
                for (int q = 0; q < 8; ++q) {
                    const float2 p = fold_s[(sl + q) * d + t];
                    DF o;
                    o.hi = p.x, o.lo = p.y;
                    acc[q] = df_add(acc[q], o);
                }
            }
            for (int q = 0; sl < s1; ++sl, ++q) {
                const float2 p = fold_s[sl * d + t];
                DF o;
                o.hi = p.x, o.lo = p.y;
                acc[q] = df_add(acc[q], o);
            }
        }
#pragma unroll
        for (int q = 1; q < 8; ++q) acc[0] = df_add(acc[0], acc[q]);
        const double Sp = acc[0].value();
        const float co = C_old[j * d + t];
        if (N > 0.0) {
            const double sref = (double)X[(int64_t)perm[start[j]] * d + t];
            const double e = sref - (double)co;
            a_old = 2.0 * e * Sp + N * e * e;
            b_sq = Sp * Sp;
            C_new[j * d + t] = (float)(sref + Sp * invN);
        } else {
            C_new[j * d + t] = co;
        }
    }
    // the three block sums in one tree (fixed order)
    sh[threadIdx.x] = a_old;
    sh[256 + threadIdx.x] = b_sq;
    sh[512 + threadIdx.x] = q_part;
    __syncthreads();
    for (int o = 128; o > 0; o >>= 1) {
        if ((int)threadIdx.x < o) {
            sh[threadIdx.x] += sh[threadIdx.x + o];
            sh[256 + threadIdx.x] += sh[256 + threadIdx.x + o];
            if (cb == 0) sh[512 + threadIdx.x] += sh[512 + threadIdx.x + o];
        }
        __syncthreads();
    }
    const double at = sh[0], bt = sh[256];
    if (cb == 0) {
        const double Q = sh[512];
        if (threadIdx.x == 0) {
            if (counts) counts[j] = N;
            nq[j * 2] = N;
            nq[j * 2 + 1] = Q;
        }
    }
    if (threadIdx.x == 0) {
        blk[(j * gridDim.y + cb) * 2] = at;
        blk[(j * gridDim.y + cb) * 2 + 1] = bt;
    }
}

// one CTA: cost(C_old) and cost(C_new) summed over clusters, and the empty-cluster count
__global__ void __launch_bounds__(256) k_final(const double *__restrict__ nq, const double *__restrict__ blk,
                                               int64_t k, int64_t ncb, double *cost_old, double *cost_new,
                                               int64_t *n_empty) {
    __shared__ double sh[256];
    double x = 0.0, y = 0.0, z = 0.0;
    for (int64_t j = threadIdx.x; j < k; j += 256) {
        const double N = nq[j * 2], Q = nq[j * 2 + 1];
        double a = 0.0, b = 0.0;
        for (int64_t c = 0; c < ncb; ++c) {
            a += blk[(j * ncb + c) * 2];
            b += blk[(j * ncb + c) * 2 + 1];
        }
        if (N > 0.0) {
            x += Q + a;
            y += Q - b / N;
        } else {
            z += 1.0;
        }
    }
    x = block_tree_sum_d(x, sh);
    y = block_tree_sum_d(y, sh);
    z = block_tree_sum_d(z, sh);
    if (threadIdx.x == 0) {
        if (cost_old) *cost_old = x;
        if (cost_new) *cost_new = y;
        if (n_empty) *n_empty = (int64_t)z;
    }
}

// sizes and workspace layout of one update
struct UpdatePlan {
    int64_t R, S, L, nbs, items_max, runs_max, ncb;
    bool smem_hist;
    size_t o_hist, o_off, o_bsum, o_start, o_items, o_perm, o_part, o_fold, o_nq, o_terms, o_cnt, o_ticket,
        bytes;
};

static UpdatePlan update_plan(int64_t n, int64_t d, int64_t k) {
    UpdatePlan P;
    // label segments: R rows each (one warp per segment), with the histogram table k * S kept
    // below ~8M entries
    P.smem_hist = k <= SMEM_HIST_MAX_K;
    P.R = P.smem_hist ? 256 : 128;
    while (ceil_div(n, P.R) * k > (int64_t)8 << 20) P.R *= 2;
    P.ncb = ceil_div(d, 256);
    P.S = ceil_div(n, P.R);
    P.L = k * P.S;
    P.nbs = ceil_div(P.L, (int64_t)SCAN_T * SCAN_E);
    P.items_max = ceil_div(n, CHUNK_R) + k;
    P.runs_max = ceil_div(P.items_max, (int64_t)FOLD_I);
    WsPlan p;
    P.o_hist = p.take<int32_t>(P.L);
    P.o_off = p.take<int32_t>(P.L);
    P.o_bsum = p.take<int32_t>(P.nbs);
    P.o_start = p.take<int32_t>(k + 1);
    P.o_items = p.take<int32_t>(k + 1);
    P.o_perm = p.take<int32_t>(n);
    P.o_part = p.take<float2>(P.items_max * d);
    P.o_fold = p.take<float2>((P.runs_max + k) * d);
    P.o_nq = p.take<double>(P.items_max * 2);
    P.o_terms = p.take<double>(k * (2 + 2 * P.ncb));
    P.o_cnt = p.take<int32_t>(k);
    P.o_ticket = p.take<int32_t>(1);
    P.bytes = p.off;
    return P;
}

template <int VW, bool WEIGHTED>
static void launch_segsum(bool u16, unsigned items, cudaStream_t st, const float *X, int64_t d, const float *w,
                          const int32_t *perm, const int32_t *start, const int32_t *item_start, int64_t k,
                          float2 *part, double *part_nq) {
    if (u16)
        k_segsum<VW, WEIGHTED, 16><<<items, 256, 0, st>>>(X, d, w, perm, start, item_start, k, CHUNK_R, part, part_nq);
    else
        k_segsum<VW, WEIGHTED, 8><<<items, 256, 0, st>>>(X, d, w, perm, start, item_start, k, CHUNK_R, part, part_nq);
}

// the update pipeline on a workspace block of P.bytes bytes; returns the number of launches
// (or -1 on a CUDA error, left in cudaGetLastError).  With a context, the segmented sums are
// timed as the part "segsum" of the caller's "update" bracket.
static int update_run(gbkm_ctx *c, cudaStream_t st, int *status, void *ws, const UpdatePlan &P, const float *X,
                      int64_t n, int64_t d, const float *w, const int32_t *labels, int64_t k,
                      const float *C_old, float *C_new, double *counts, double *cost_old,
                      double *cost_new, int64_t *n_empty) {
    int32_t *hist = ws_at<int32_t>(ws, P.o_hist), *off = ws_at<int32_t>(ws, P.o_off),
            *bsum = ws_at<int32_t>(ws, P.o_bsum), *start = ws_at<int32_t>(ws, P.o_start),
            *item_start = ws_at<int32_t>(ws, P.o_items), *perm = ws_at<int32_t>(ws, P.o_perm),
            *cnt = ws_at<int32_t>(ws, P.o_cnt), *ticket = ws_at<int32_t>(ws, P.o_ticket);
    float2 *part = ws_at<float2>(ws, P.o_part), *fold = ws_at<float2>(ws, P.o_fold);
    double *part_nq = ws_at<double>(ws, P.o_nq), *terms = ws_at<double>(ws, P.o_terms);
    const unsigned seg_blocks = (unsigned)ceil_div(P.S, 8);
    const size_t hsm = P.smem_hist ? sizeof(int32_t) * 8 * (size_t)k : 0;
    if (P.smem_hist) {
        if (hsm > 48 * 1024) {
            cudaFuncSetAttribute(k_hist_sm, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)hsm);
            cudaFuncSetAttribute(k_scatter_sm, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)hsm);
        }
        k_hist_sm<<<seg_blocks, 256, hsm, st>>>(labels, n, k, P.R, P.S, hist, status, ticket);
        k_row_scan<<<(unsigned)k, 256, 0, st>>>(hist, k, P.S, CHUNK_R, off, cnt, start, item_start,
                                                            ticket);
        k_scatter_sm<<<seg_blocks, 256, hsm, st>>>(labels, n, k, P.R, P.S, off, start, perm);
    } else {
        if (cudaMemsetAsync(hist, 0, sizeof(int32_t) * P.L, st) != cudaSuccess) return -1;
        k_hist<<<seg_blocks, 256, 0, st>>>(labels, n, k, P.R, P.S, hist, status);
        scan_excl(st, hist, P.L, bsum, off);
        k_starts<<<(unsigned)ceil_div(k, 256), 256, 0, st>>>(off, hist, k, P.S, start);
        k_scatter<<<seg_blocks, 256, 0, st>>>(labels, n, k, P.R, P.S, off, perm);
        k_items<<<1, SCAN_T, 0, st>>>(start, k, CHUNK_R, item_start);
    }
    const bool vec = ((d & 3) == 0) && ((reinterpret_cast<uintptr_t>(X) & 15) == 0);
    const unsigned items = (unsigned)P.items_max;
    // 16 loads in flight per thread unless the row groups of the narrowest column pass would then
    // pad an item beyond its 128 rows
    const int64_t ncv = vec ? d / 4 : d, last_pass = ncv - ((ncv - 1) / 256) * 256;
    int64_t tpr = 1;
    while (tpr < last_pass) tpr <<= 1;
    const bool u16 = (256 / tpr) * 16 <= CHUNK_R;
    if (c) prof_begin(c, "segsum");
    if (vec && w)
        launch_segsum<4, true>(u16, items, st, X, d, w, perm, start, item_start, k, part, part_nq);
    else if (vec)
        launch_segsum<4, false>(u16, items, st, X, d, w, perm, start, item_start, k, part, part_nq);
    else if (w)
        launch_segsum<1, true>(u16, items, st, X, d, w, perm, start, item_start, k, part, part_nq);
    else
        launch_segsum<1, false>(u16, items, st, X, d, w, perm, start, item_start, k, part, part_nq);
    if (c) prof_end(c);
    k_fold<<<dim3((unsigned)P.runs_max, (unsigned)P.ncb), 256, 0, st>>>(part, item_start, k, d, fold);
    k_finalize<<<dim3((unsigned)k, (unsigned)P.ncb), 256, 0, st>>>(fold, part_nq, X, perm, start, d, k,
                                                                  item_start, C_old, C_new, counts, terms,
                                                                  terms + 2 * k);
    k_final<<<1, 256, 0, st>>>(terms, terms + 2 * k, k, P.ncb, cost_old, cost_new, n_empty);
    return cudaPeekAtLastError() == cudaSuccess ? (P.smem_hist ? 7 : 11) : -1;
}

int update_impl(gbkm_ctx *c, const float *X, int64_t n, int64_t d, const float *w,
                const int32_t *labels, int64_t k, const float *C_old, float *C_new, double *counts,
                double *cost_old, double *cost_new, int64_t *n_empty) {
    const UpdatePlan P = update_plan(n, d, k);
    int rc = GBKM_OK;
    void *ws = ws_reserve(c, P.bytes, &rc);
    if (!ws) return rc;
    const int nl = update_run(c, c->stream, c->status, ws, P, X, n, d, w, labels, k, C_old, C_new, counts,
                              cost_old, cost_new, n_empty);
    if (nl < 0) return cuda_check(c, cudaGetLastError(), "update launch");
    c->launches += nl;
    return GBKM_OK;
}

}  // namespace gbkm

// ---------------------------------------------------------------- allocation-free update
// Scratch for kmeans_update_noalloc: a fixed block in the library's own device image.  Every GPU
// that loads this library holds it until the process exits.  The first 256 bytes take the
// label-check word the histogram kernel writes; the update pipeline's workspace follows.
namespace {
static __device__ __align__(256) unsigned char g_noalloc_scratch[GBKM_NOALLOC_SCRATCH_BYTES];
std::mutex g_noalloc_mu;
void *g_noalloc_base[256] = {};  // device address of g_noalloc_scratch, per device ordinal
}  // namespace

extern "C" int64_t kmeans_update_scratch_bytes(int64_t n, int64_t d, int64_t k) {
    if (n < 1 || d < 1 || k < 1 || k > 65536 || n >= ((int64_t)1 << 31)) return -1;
    if ((uint64_t)n > (uint64_t)INT64_MAX / 64 / (uint64_t)d) return -1;
    return (int64_t)gbkm::update_plan(n, d, k).bytes + 256;
}

extern "C" int kmeans_update_noalloc(void *cuda_stream, const float *X, int64_t n, int64_t d,
                                     const float *w, const int32_t *labels, int64_t k,
                                     const float *C_old, float *C_new, double *counts,
                                     double *cost_old, double *cost_new, int64_t *n_empty) {
    if (n < 1 || d < 1 || k < 1 || k > 65536 || !X || !labels || !C_old || !C_new || C_old == C_new)
        return GBKM_EINVAL;
    if (n >= ((int64_t)1 << 31)) return GBKM_EUNSUPPORTED;
    const gbkm::UpdatePlan P = gbkm::update_plan(n, d, k);
    if (P.bytes + 256 > (size_t)GBKM_NOALLOC_SCRATCH_BYTES) return GBKM_ETOOBIG;
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0) {
        cudaGetLastError();
        return GBKM_ECUDA;
    }
    if (dev >= 256) return GBKM_EUNSUPPORTED;
    void *base = nullptr;
    {
        // set-up, once per device, with that device current: in host code the array's name is
        // only a host-side stand-in, so the kernels get the device address from the runtime
        std::lock_guard<std::mutex> lock(g_noalloc_mu);
        if (!g_noalloc_base[dev]) {
            void *p = nullptr;
            cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
            if (e != cudaSuccess || !p) {
                cudaGetLastError();
                return GBKM_ECUDA;
            }
            g_noalloc_base[dev] = p;
        }
        base = g_noalloc_base[dev];
    }
    int *label_check = static_cast<int *>(base);
    void *ws = static_cast<char *>(base) + 256;
    const int nl = gbkm::update_run(nullptr, (cudaStream_t)cuda_stream, label_check, ws, P, X, n, d, w, labels,
                                    k, C_old, C_new, counts, cost_old, cost_new, n_empty);
    if (nl < 0) {
        cudaGetLastError();
        return GBKM_ECUDA;
    }
    return GBKM_OK;
}
