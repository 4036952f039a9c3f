// k_update.cu -- A6 centroid update through clustering features and A7 cost (CF identity).
//
// Pipeline (all on the context's stream, no host synchronisation, no float atomics):
//   1. k_hist      one warp per label segment: warp-aggregated (match_any) label histogram,
//                  column s of the cluster-major table hist[j * S + s]
//   2. scan        exclusive scan of the table -> stable output slot of every (cluster, segment)
//   3. k_starts    first slot of every cluster
//   4. k_scatter   one warp per segment: stable rank inside the warp + running slot -> perm
//   5. k_items     chunks of R rows per cluster, exclusive scan -> work-item table
//   6. k_segsum    one CTA per chunk: error-free FP32 sums of w x, w, w ||x||^2 -> FP64 partials
//   7. k_finalize  one CTA per cluster: FP64 sum of its partials in chunk order, centroid, CF costs
//   8. k_final     one CTA: FP64 totals in cluster order
#include <mutex>

#include "internal.cuh"

namespace gbkm {

namespace {
constexpr int SCAN_T = 1024, SCAN_E = 4;           // scan block: 1024 threads x 4 elements
constexpr int64_t CHUNK_R = 256;                    // rows per segmented-sum work item

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

// ---------------------------------------------------------------- device-wide exclusive scan
// (int32; totals < 2^31 because they count rows)
__device__ int32_t block_excl_scan(int32_t v, int32_t *sh, int32_t &total) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    int32_t x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        int32_t y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) sh[wid] = x;
    __syncthreads();
    if (wid == 0) {
        int32_t w = lane < nw ? sh[lane] : 0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            int32_t y = __shfl_up_sync(0xffffffffu, w, o);
            if (lane >= o) w += y;
        }
        sh[lane] = w;  // inclusive over warps
    }
    __syncthreads();
    const int32_t warp_base = wid > 0 ? sh[wid - 1] : 0;
    total = sh[nw - 1];
    __syncthreads();
    return warp_base + x - v;
}

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

static void scan_excl(cudaStream_t st, const int32_t *in, int64_t L, int32_t *bsum, int32_t *out) {
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

// ---------------------------------------------------------------- segmented CF sums
// One CTA (256 threads) per work item = up to R rows of one cluster in sorted order.
// Columns are processed in passes of 256 vectors (float4 when rows are 16-byte aligned);
// threads form G = 256 / tpr row groups; group partials are combined in FP64 in group order.
template <int VW>
__global__ void __launch_bounds__(256) k_segsum(const float *__restrict__ X, int64_t d,
                                                const float *__restrict__ w,
                                                const int32_t *__restrict__ perm,
                                                const int32_t *__restrict__ start,
                                                const int32_t *__restrict__ item_start, int64_t k,
                                                int64_t R, double *__restrict__ part) {
    __shared__ double red[256 * VW];
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
    const int64_t rows = min((int64_t)start[j + 1] - row0, R);
    double *out = part + item * (d + 2);
    const int tid = threadIdx.x;
    const int64_t ncv = d / VW;
    DF qacc;
    for (int64_t cb = 0; cb < ncv; cb += 256) {
        const int pass = (int)min((int64_t)256, ncv - cb);
        int tpr = 1;
        while (tpr < pass) tpr <<= 1;
        const int G = 256 / tpr, g = tid / tpr, cv = tid % tpr;
        const bool active = cv < pass;
        DF acc[VW];
        if (active) {
            for (int64_t r = g; r < rows; r += G) {
                const int64_t i = perm[row0 + r];
                const float wi = w ? w[i] : 1.f;
                const float *xr = X + i * d + (cb + cv) * VW;
                float v[VW];
                if constexpr (VW == 4) {
                    float4 q = __ldg(reinterpret_cast<const float4 *>(xr));
                    v[0] = q.x, v[1] = q.y, v[2] = q.z, v[3] = q.w;
                } else {
                    v[0] = xr[0];
                }
#pragma unroll
                for (int q = 0; q < VW; ++q) {
                    acc[q].add_prod(wi, v[q]);
                    const float p = __fmul_rn(v[q], v[q]);
                    const float pe = __fmaf_rn(v[q], v[q], -p);
                    qacc.add_prod(wi, p);
                    qacc.lo = __fmaf_rn(wi, pe, qacc.lo);
                }
            }
        }
#pragma unroll
        for (int q = 0; q < VW; ++q) red[tid * VW + q] = active ? acc[q].value() : 0.0;
        __syncthreads();
        for (int e = tid; e < pass * VW; e += 256) {
            const int cvv = e / VW, q = e % VW;
            double s = 0.0;
            for (int gg = 0; gg < G; ++gg) s += red[(gg * tpr + cvv) * VW + q];
            out[(cb + cvv) * VW + q] = s;
        }
        __syncthreads();
    }
    qred[tid] = qacc.value();
    __syncthreads();
    if (tid == 0) {
        double q = 0.0, nsum = 0.0;
        for (int t = 0; t < 256; ++t) q += qred[t];
        for (int64_t r = 0; r < rows; ++r) nsum += w ? (double)w[perm[row0 + r]] : 1.0;
        out[d] = nsum;
        out[d + 1] = q;
    }
}

// one CTA per cluster: FP64 sums of its partials in item order, centroid, CF cost terms
__global__ void __launch_bounds__(256) k_finalize(const double *__restrict__ part, int64_t d, int64_t k,
                                                  const int32_t *__restrict__ item_start,
                                                  const float *__restrict__ C_old, float *__restrict__ C_new,
                                                  double *__restrict__ counts, double *__restrict__ terms) {
    __shared__ double r_old[256], r_new[256];
    __shared__ double NQ[2];
    const int64_t j = blockIdx.x;
    const int32_t i0 = item_start[j], i1 = item_start[j + 1];
    if (threadIdx.x == 0) {
        double N = 0.0, Q = 0.0;
        for (int32_t it = i0; it < i1; ++it) {
            N += part[(int64_t)it * (d + 2) + d];
            Q += part[(int64_t)it * (d + 2) + d + 1];
        }
        NQ[0] = N;
        NQ[1] = Q;
    }
    __syncthreads();
    const double N = NQ[0], Q = NQ[1];
    double t_old = 0.0, t_new = 0.0;
    for (int64_t t = threadIdx.x; t < d; t += blockDim.x) {
        double S = 0.0;
        for (int32_t it = i0; it < i1; ++it) S += part[(int64_t)it * (d + 2) + t];
        const double co = (double)C_old[j * d + t];
        t_old += co * (N * co - 2.0 * S);
        if (N > 0.0) {
            t_new += S * S;
            C_new[j * d + t] = (float)(S / N);
        } else {
            C_new[j * d + t] = C_old[j * d + t];
        }
    }
    r_old[threadIdx.x] = t_old;
    r_new[threadIdx.x] = t_new;
    __syncthreads();
    for (int o = 128; o > 0; o >>= 1) {
        if ((int)threadIdx.x < o) {
            r_old[threadIdx.x] += r_old[threadIdx.x + o];
            r_new[threadIdx.x] += r_new[threadIdx.x + o];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        if (counts) counts[j] = N;
        terms[j * 3 + 0] = Q + r_old[0];                      // Q - 2 c.S + N ||c||^2
        terms[j * 3 + 1] = N > 0.0 ? Q - r_new[0] / N : 0.0;  // Q - ||S||^2 / N
        terms[j * 3 + 2] = N > 0.0 ? 0.0 : 1.0;
    }
}

__global__ void __launch_bounds__(256) k_final(const double *__restrict__ terms, int64_t k,
                                               double *cost_old, double *cost_new, int64_t *n_empty) {
    __shared__ double a[256], b[256], e[256];
    double x = 0.0, y = 0.0, z = 0.0;
    const int64_t per = (k + 255) / 256;
    const int64_t j0 = (int64_t)threadIdx.x * per, j1 = min(k, j0 + per);
    for (int64_t j = j0; j < j1; ++j) {
        x += terms[j * 3];
        y += terms[j * 3 + 1];
        z += terms[j * 3 + 2];
    }
    a[threadIdx.x] = x;
    b[threadIdx.x] = y;
    e[threadIdx.x] = z;
    __syncthreads();
    if (threadIdx.x == 0) {
        double sx = 0.0, sy = 0.0, sz = 0.0;
        for (int t = 0; t < 256; ++t) {
            sx += a[t];
            sy += b[t];
            sz += e[t];
        }
        if (cost_old) *cost_old = sx;
        if (cost_new) *cost_new = sy;
        if (n_empty) *n_empty = (int64_t)sz;
    }
}

// sizes and workspace layout of one update
struct UpdatePlan {
    int64_t R, S, L, nbs, items_max;
    size_t o_hist, o_off, o_bsum, o_start, o_items, o_perm, o_part, o_terms, bytes;
};

static UpdatePlan update_plan(int64_t n, int64_t d, int64_t k) {
    UpdatePlan P;
    // label segments: R rows each, with the histogram table k * S kept below ~8M entries
    P.R = 1024;
    while (ceil_div(n, P.R) * k > (int64_t)8 << 20) P.R *= 2;
    P.S = ceil_div(n, P.R);
    P.L = k * P.S;
    P.nbs = ceil_div(P.L, (int64_t)SCAN_T * SCAN_E);
    P.items_max = ceil_div(n, CHUNK_R) + k;
    WsPlan p;
    P.o_hist = p.take<int32_t>(P.L);
    P.o_off = p.take<int32_t>(P.L);
    P.o_bsum = p.take<int32_t>(P.nbs);
    P.o_start = p.take<int32_t>(k + 1);
    P.o_items = p.take<int32_t>(k + 1);
    P.o_perm = p.take<int32_t>(n);
    P.o_part = p.take<double>(P.items_max * (d + 2));
    P.o_terms = p.take<double>(k * 3);
    P.bytes = p.off;
    return P;
}

// the update pipeline on a workspace block of P.bytes bytes; returns the number of launches
// (or -1 on a CUDA error, left in cudaGetLastError)
static int update_run(cudaStream_t st, int *status, void *ws, const UpdatePlan &P, const float *X,
                      int64_t n, int64_t d, const float *w, const int32_t *labels, int64_t k,
                      const float *C_old, float *C_new, double *counts, double *cost_old,
                      double *cost_new, int64_t *n_empty) {
    int32_t *hist = ws_at<int32_t>(ws, P.o_hist), *off = ws_at<int32_t>(ws, P.o_off),
            *bsum = ws_at<int32_t>(ws, P.o_bsum), *start = ws_at<int32_t>(ws, P.o_start),
            *item_start = ws_at<int32_t>(ws, P.o_items), *perm = ws_at<int32_t>(ws, P.o_perm);
    double *part = ws_at<double>(ws, P.o_part), *terms = ws_at<double>(ws, P.o_terms);
    if (cudaMemsetAsync(hist, 0, sizeof(int32_t) * P.L, st) != cudaSuccess) return -1;
    const unsigned seg_blocks = (unsigned)ceil_div(P.S, 8);
    k_hist<<<seg_blocks, 256, 0, st>>>(labels, n, k, P.R, P.S, hist, status);
    scan_excl(st, hist, P.L, bsum, off);
    k_starts<<<(unsigned)ceil_div(k, 256), 256, 0, st>>>(off, hist, k, P.S, start);
    k_scatter<<<seg_blocks, 256, 0, st>>>(labels, n, k, P.R, P.S, off, perm);
    k_items<<<1, SCAN_T, 0, st>>>(start, k, CHUNK_R, item_start);
    const bool vec = ((d & 3) == 0) && ((reinterpret_cast<uintptr_t>(X) & 15) == 0);
    if (vec)
        k_segsum<4><<<(unsigned)P.items_max, 256, 0, st>>>(X, d, w, perm, start, item_start, k,
                                                           CHUNK_R, part);
    else
        k_segsum<1><<<(unsigned)P.items_max, 256, 0, st>>>(X, d, w, perm, start, item_start, k,
                                                           CHUNK_R, part);
    k_finalize<<<(unsigned)k, 256, 0, st>>>(part, d, k, item_start, C_old, C_new, counts, terms);
    k_final<<<1, 256, 0, st>>>(terms, k, cost_old, cost_new, n_empty);
    return cudaPeekAtLastError() == cudaSuccess ? 10 : -1;
}

int update_impl(gbkm_ctx *c, const float *X, int64_t n, int64_t d, const float *w,
                const int32_t *labels, int64_t k, const float *C_old, float *C_new, double *counts,
                double *cost_old, double *cost_new, int64_t *n_empty) {
    const UpdatePlan P = update_plan(n, d, k);
    int rc = GBKM_OK;
    void *ws = ws_reserve(c, P.bytes, &rc);
    if (!ws) return rc;
    const int nl = update_run(c->stream, c->status, ws, P, X, n, d, w, labels, k, C_old, C_new, counts,
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
    const int nl = gbkm::update_run((cudaStream_t)cuda_stream, label_check, ws, P, X, n, d, w, labels,
                                    k, C_old, C_new, counts, cost_old, cost_new, n_empty);
    if (nl < 0) {
        cudaGetLastError();
        return GBKM_ECUDA;
    }
    return GBKM_OK;
}
