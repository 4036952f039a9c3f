// k_svd.cu -- randomised truncated SVD of a piece (Section 2.2), weighted rows (Section 2.3.2).
//
// The top l right singular vectors of A' = diag(sqrt(w)) A (n x d, one point per row) after the
// randomised scheme of Halko, Martinsson and Tropp that the paper adopts: the columns of A' are
// reduced by a random d x s matrix Omega (s = l + oversampling), the rows by an orthonormal basis
// of the result, and only the s x d matrix left over is decomposed.  All on the context's stream:
//   1. Y = A' Omega (n x s): the tensor cores' 3xTF32 store GEMM (k_tc), or k_gemm_rows on the CUDA
//      cores where the shape does not allow TMA tiles                       first read of A
//   2. CholeskyQR2   k_gram (Y^T Y, FP32 blocks of 8 rows added in double-float), k_chol (double-
//                    float Cholesky with a small diagonal shift, R^-1), Y <- Y R^-1; twice -> Q
//   3. Bt = A'^T Q (d x s): k_tn_tc on the tensor cores (A's tiles transposed in shared memory,
//      3xTF32, split over row ranges, the splits added in fixed order), or k_gemm_tn on the CUDA
//      cores, split over row chunks added in fixed order                   second read of A
//   4. k_gram, k_chol  R_b with R_b^T R_b = Bt^T Bt, so Bt = Q_b R_b
//   5. k_jacobi      one-sided Jacobi on R_b^T (one CTA): R_b^T J = W Sigma, singular values in
//                    decreasing order, T = R_b^-1 J (first l columns of the order)
//   6. k_gemm_rows   V = Bt T (d x l), the right singular vectors of B = Q^T A' = Bt^T
//   7. k_sign        each column's entry of largest magnitude made positive
#include "internal.cuh"

namespace gbkm {

namespace {
constexpr int GR_BM = 128, GR_BK = 16;   // k_gemm_rows tile
constexpr int TN_BJ = 64, TN_RS = 32;    // k_gemm_tn: 64 columns of d per CTA, 32-row stages
constexpr int TN_CHUNKS = 16;            // row chunks of k_gemm_tn (partials added in order)

__device__ __forceinline__ void df_add_f(float &hi, float &lo, float v) {
    const float s = __fadd_rn(hi, v);
    const float bb = __fsub_rn(s, hi);
    const float e = __fadd_rn(__fsub_rn(hi, __fsub_rn(s, bb)), __fsub_rn(v, bb));
    hi = s;
    lo = __fadd_rn(lo, e);
}
}  // namespace

// ---------------------------------------------------------------- Out = diag(scale) In W
// In: M x K row-major, W: K x N row-major (N <= 16 NJ), Out: M x N row-major; scale: M or null.
// One CTA per 128 rows; thread (tx, ty) owns rows ty + 16 i and columns tx + 16 j.  FP32 FFMA.
template <int NJ>
__global__ void __launch_bounds__(256, NJ <= 5 ? 3 : 2) k_gemm_rows(const float *__restrict__ In, const float *__restrict__ W,
                                                   const float *__restrict__ wrow, int64_t M, int64_t K, int64_t N,
                                                   float *__restrict__ Out) {
    constexpr int NC = 16 * NJ;
    __shared__ float As[GR_BK][GR_BM + 4];
    __shared__ float Ws[GR_BK][NC + 4];
    const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
    const int64_t m0 = (int64_t)blockIdx.x * GR_BM;
    const bool vec = (K & 3) == 0 && (reinterpret_cast<uintptr_t>(In) & 15) == 0;
    float acc[8][NJ];
#pragma unroll
    for (int i = 0; i < 8; ++i)
#pragma unroll
        for (int j = 0; j < NJ; ++j) acc[i][j] = 0.f;
    for (int64_t k0 = 0; k0 < K; k0 += GR_BK) {
        if (vec) {
#pragma unroll
            for (int q = 0; q < 2; ++q) {
                const int e = tid + 256 * q, r = e >> 2, kq = (e & 3) * 4;
                const int64_t gr = m0 + r, gk = k0 + kq;
                float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
                if (gr < M && gk < K) v = __ldg(reinterpret_cast<const float4 *>(In + gr * K + gk));
                As[kq][r] = v.x, As[kq + 1][r] = v.y, As[kq + 2][r] = v.z, As[kq + 3][r] = v.w;
            }
        } else {
            for (int e = tid; e < GR_BM * GR_BK; e += 256) {
                const int r = e / GR_BK, q = e % GR_BK;
                const int64_t gr = m0 + r, gk = k0 + q;
                As[q][r] = (gr < M && gk < K) ? In[gr * K + gk] : 0.f;
            }
        }
        for (int e = tid; e < GR_BK * NC; e += 256) {
            const int q = e / NC, cc = e % NC;
            const int64_t gk = k0 + q;
            Ws[q][cc] = (gk < K && cc < N) ? W[gk * N + cc] : 0.f;
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < GR_BK; ++kk) {
            float a[8], b[NJ];
#pragma unroll
            for (int i = 0; i < 8; ++i) a[i] = As[kk][ty + 16 * i];
#pragma unroll
            for (int j = 0; j < NJ; ++j) b[j] = Ws[kk][tx + 16 * j];
#pragma unroll
            for (int i = 0; i < 8; ++i)
#pragma unroll
                for (int j = 0; j < NJ; ++j) acc[i][j] = fmaf(a[i], b[j], acc[i][j]);
        }
        __syncthreads();
    }
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        const int64_t r = m0 + ty + 16 * i;
        if (r >= M) continue;
        const float sc = wrow ? sqrtf(fmaxf(wrow[r], 0.f)) : 1.f;
#pragma unroll
        for (int j = 0; j < NJ; ++j) {
            const int64_t cc = tx + 16 * j;
            if (cc < N) Out[r * N + cc] = acc[i][j] * sc;
        }
    }
}

static int launch_gemm_rows(gbkm_ctx *c, const float *In, const float *W, const float *wrow, int64_t M, int64_t K,
                            int64_t N, float *Out) {
    const dim3 grid((unsigned)ceil_div(M, GR_BM));
    const int nj = (int)ceil_div(N, 16);
    switch (nj) {
        case 1: k_gemm_rows<1><<<grid, 256, 0, c->stream>>>(In, W, wrow, M, K, N, Out); break;
        case 2: k_gemm_rows<2><<<grid, 256, 0, c->stream>>>(In, W, wrow, M, K, N, Out); break;
        case 3: k_gemm_rows<3><<<grid, 256, 0, c->stream>>>(In, W, wrow, M, K, N, Out); break;
        case 4: k_gemm_rows<4><<<grid, 256, 0, c->stream>>>(In, W, wrow, M, K, N, Out); break;
        case 5: k_gemm_rows<5><<<grid, 256, 0, c->stream>>>(In, W, wrow, M, K, N, Out); break;
        case 6: k_gemm_rows<6><<<grid, 256, 0, c->stream>>>(In, W, wrow, M, K, N, Out); break;
        case 7: k_gemm_rows<7><<<grid, 256, 0, c->stream>>>(In, W, wrow, M, K, N, Out); break;
        case 8: k_gemm_rows<8><<<grid, 256, 0, c->stream>>>(In, W, wrow, M, K, N, Out); break;
        default: return set_error(c, GBKM_EUNSUPPORTED, "gemm_rows: N = %lld above 128", (long long)N);
    }
    GBKM_LAUNCHED(c);
    return cuda_check(c, cudaGetLastError(), "gemm_rows launch");
}

// ---------------------------------------------------------------- Gram matrix X^T X
// X: m x s row-major (s % 4 == 0, s <= 128, rows 16-byte aligned).  CTA g sums the rows
// [g * rows, (g + 1) * rows) into the upper triangle of the s x s Gram matrix: the triangle's 4 x 4
// tiles (p, q), p <= q, are dealt to the threads (tile e to thread e mod 256), each row's 16 products
// of a tile summed in FP32 over 8 rows and each 8-row sum added into a double-float accumulator.
// part[(g * s + i) * s + j] = (hi, lo) for i <= j (and for the lower half of a diagonal tile).
constexpr int GM_RS = 32;  // rows per shared-memory stage
template <int TPT>         // tiles per thread: s (s + 4) / 32 <= 256 TPT
__global__ void __launch_bounds__(256) k_gram(const float *__restrict__ X, int64_t m, int64_t s, int64_t rows,
                                              float2 *__restrict__ part) {
    __shared__ __align__(16) float Xs[GM_RS][128];
    const int tid = threadIdx.x, S4 = (int)(s >> 2), ntiles = S4 * (S4 + 1) / 2;
    int tp[TPT], tq[TPT];
    bool own[TPT];
#pragma unroll
    for (int u = 0; u < TPT; ++u) {
        const int e = tid + 256 * u;
        own[u] = e < ntiles;
        int p = 0, rem = own[u] ? e : 0;
        while (rem >= S4 - p) rem -= S4 - p++;  // row-major order of the upper triangle
        tp[u] = p, tq[u] = p + rem;
    }
    float hi[TPT][16], lo[TPT][16];
#pragma unroll
    for (int u = 0; u < TPT; ++u)
#pragma unroll
        for (int e = 0; e < 16; ++e) hi[u][e] = lo[u][e] = 0.f;
    const int64_t r0 = (int64_t)blockIdx.x * rows, r1 = min(m, r0 + rows);
    for (int64_t base = r0; base < r1; base += GM_RS) {
        for (int e = tid; e < GM_RS * S4; e += 256) {
            const int rr = e / S4, c4 = e - rr * S4;
            const int64_t r = base + rr;
            float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
            if (r < r1) v = __ldg(reinterpret_cast<const float4 *>(X + r * s) + c4);
            *reinterpret_cast<float4 *>(&Xs[rr][4 * c4]) = v;
        }
        __syncthreads();
#pragma unroll
        for (int g8 = 0; g8 < GM_RS; g8 += 8) {
            float acc[TPT][16];
#pragma unroll
            for (int u = 0; u < TPT; ++u)
#pragma unroll
                for (int e = 0; e < 16; ++e) acc[u][e] = 0.f;
#pragma unroll
            for (int rr = g8; rr < g8 + 8; ++rr) {
#pragma unroll
                for (int u = 0; u < TPT; ++u) {
                    if (!own[u]) continue;
                    const float4 a = *reinterpret_cast<const float4 *>(&Xs[rr][4 * tp[u]]);
                    const float4 b = *reinterpret_cast<const float4 *>(&Xs[rr][4 * tq[u]]);
                    const float av[4] = {a.x, a.y, a.z, a.w}, bv[4] = {b.x, b.y, b.z, b.w};
#pragma unroll
                    for (int i = 0; i < 4; ++i)
#pragma unroll
                        for (int j = 0; j < 4; ++j) acc[u][4 * i + j] = fmaf(av[i], bv[j], acc[u][4 * i + j]);
                }
            }
#pragma unroll
            for (int u = 0; u < TPT; ++u)
#pragma unroll
                for (int e = 0; e < 16; ++e) df_add_f(hi[u][e], lo[u][e], acc[u][e]);
        }
        __syncthreads();
    }
    float2 *o = part + (int64_t)blockIdx.x * s * s;
#pragma unroll
    for (int u = 0; u < TPT; ++u) {
        if (!own[u]) continue;
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
            for (int j = 0; j < 4; ++j)
                o[(int64_t)(4 * tp[u] + i) * s + 4 * tq[u] + j] = make_float2(hi[u][4 * i + j], lo[u][4 * i + j]);
    }
}

// the chunks' partials added (double-float) into the full symmetric FP64 G: one warp per entry of the
// upper triangle, lane l taking chunks l, l + 32, ..., then a fixed butterfly
__global__ void __launch_bounds__(256) k_gram_reduce(const float2 *__restrict__ part, int64_t s, int chunks,
                                                     double *__restrict__ G) {
    const int e = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31, S = (int)s;
    if (e >= S * S) return;
    const int i = e / S, j = e - i * S;
    if (i > j) return;
    float hi = 0.f, lo = 0.f;
    for (int g = lane; g < chunks; g += 32) {
        const float2 v = part[((int64_t)g * S + i) * S + j];
        df_add_f(hi, lo, v.x);
        df_add_f(hi, lo, v.y);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const float h2 = __shfl_xor_sync(0xffffffffu, hi, o), l2 = __shfl_xor_sync(0xffffffffu, lo, o);
        // lanes l and l ^ o form the same sum in the same operand order (lower lane first)
        float a_hi = hi, a_lo = lo, b_hi = h2, b_lo = l2;
        if (lane & o) a_hi = h2, a_lo = l2, b_hi = hi, b_lo = lo;
        df_add_f(a_hi, a_lo, b_hi);
        a_lo = __fadd_rn(a_lo, b_lo);
        hi = a_hi, lo = a_lo;
    }
    if (lane == 0) {
        const double v = (double)hi + (double)lo;
        G[i * S + j] = v;
        G[j * S + i] = v;
    }
}

// row chunks: about two CTAs per SM, at least 64 rows each
static int gram_chunks(int64_t m, int sm_count) {
    return (int)std::min<int64_t>(2 * (int64_t)sm_count, std::max<int64_t>(1, ceil_div(m, (int64_t)64)));
}

static int launch_gram(gbkm_ctx *c, const float *X, int64_t m, int64_t s, float2 *part, double *G) {
    const int chunks = gram_chunks(m, c->sm_count);
    const int64_t rows = ceil_div(m, (int64_t)chunks);
    const int64_t ntiles = (s / 4) * (s / 4 + 1) / 2;
    if (ntiles <= 256)
        k_gram<1><<<(unsigned)chunks, 256, 0, c->stream>>>(X, m, s, rows, part);
    else if (ntiles <= 512)
        k_gram<2><<<(unsigned)chunks, 256, 0, c->stream>>>(X, m, s, rows, part);
    else
        k_gram<3><<<(unsigned)chunks, 256, 0, c->stream>>>(X, m, s, rows, part);
    k_gram_reduce<<<(unsigned)ceil_div(s * s * 32, (int64_t)256), 256, 0, c->stream>>>(part, s, chunks, G);
    c->launches += 2;
    return cuda_check(c, cudaGetLastError(), "gram launch");
}

// ---------------------------------------------------------------- double-float arithmetic
// A value is the unevaluated sum h + l of two FP32 numbers with |l| <= ulp(h) / 2 (Dekker 1971,
// Knuth's TwoSum): about 48 significant bits on the FP32 pipe, which on this GPU runs 73 times
// the FP64 rate.  Every step uses explicit round-to-nearest intrinsics, so nothing is contracted.
struct F2 {
    float h, l;
};
__device__ __forceinline__ F2 f2_quick(float a, float b) {  // |a| >= |b| or a == 0
    const float s = __fadd_rn(a, b);
    return {s, __fsub_rn(b, __fsub_rn(s, a))};
}
__device__ __forceinline__ F2 f2_add(F2 a, F2 b) {
    float s, e, t, f;
    two_sum(a.h, b.h, s, e);
    two_sum(a.l, b.l, t, f);
    F2 r = f2_quick(s, __fadd_rn(e, t));
    return f2_quick(r.h, __fadd_rn(r.l, f));
}
__device__ __forceinline__ F2 f2_mul(F2 a, F2 b) {
    const float p = __fmul_rn(a.h, b.h);
    float e = __fmaf_rn(a.h, b.h, -p);
    e = __fmaf_rn(a.h, b.l, e);
    e = __fmaf_rn(a.l, b.h, e);
    return f2_quick(p, e);
}
__device__ __forceinline__ F2 f2_neg(F2 a) { return {-a.h, -a.l}; }
// 1 / sqrt(d) for d > 0: rsqrtf's estimate and two Newton steps y <- y + y (1 - d y^2) / 2, the
// residual 1 - d y^2 formed in double-float (its high part 1 - t.h is exact: t.h is near 1)
__device__ __forceinline__ F2 f2_rsqrt(F2 d) {
    F2 y = {rsqrtf(d.h), 0.f};
#pragma unroll
    for (int it = 0; it < 2; ++it) {
        const F2 t = f2_mul(f2_mul(d, y), y);
        const float r = __fsub_rn(__fsub_rn(1.f, t.h), t.l);
        y = f2_add(y, f2_quick(__fmul_rn(__fmul_rn(0.5f, y.h), r), 0.f));
    }
    return y;
}

// ---------------------------------------------------------------- Cholesky of G + shift I, R^-1
// One CTA in double-float.  G (s x s, FP64, symmetric) is first scaled by 2^-2e, a power of two that
// brings its mean diagonal near 1 (so FP32's exponent range holds any FP64 Gram matrix of a piece),
// and shift = shift_rel * trace(G) / s is added to the diagonal; R and R^-1 are scaled back by 2^e
// and 2^-e, exactly.  G = R^T R with R upper triangular, right-looking: at pivot k every thread
// forms y_k = 1 / sqrt(M_kk) itself (the same operations, the same bits), row k becomes R's row
// (M_kj y_k), and the trailing matrix loses R_ki R_kj.  A pivot at or below a tiny floor is
// clamped and flagged in *status.  Then X = R^-1, column by column: X_jj = y_j and
// X_ij = -(sum_{i <= q < j} X_iq R_qj) y_j, the sums accumulated right-looking (when column q is
// final its terms are added to every later column), one barrier per column.  Shared memory: hi and
// lo planes of s rows of stride s + 1; R's strict upper triangle in place, X transposed into the
// strict lower triangle, the diagonals of R and X in four vectors.  Outputs R (FP64, optional) and
// Rinv32 = R^-1 in FP32.
__global__ void __launch_bounds__(256) k_chol(const double *__restrict__ G, int64_t s, double shift_rel,
                                              double *__restrict__ R, float *__restrict__ Rinv32, int *status) {
    extern __shared__ __align__(16) float chol_smem[];
    const int S = (int)s, L = S + 1, tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
    float *H = chol_smem, *Lo = H + S * L;
    float *rdh = Lo + S * L, *rdl = rdh + S, *yh = rdl + S, *yl = yh + S;
    __shared__ double red[256];
    const float tiny = 1e-30f;
    double tr = 0.0;
    for (int i = tid; i < S; i += 256) tr += G[i * S + i];
    red[tid] = tr;
    __syncthreads();
    for (int o = 128; o > 0; o >>= 1) {
        if (tid < o) red[tid] += red[tid + o];
        __syncthreads();
    }
    const double mean = red[0] / (double)s;
    int ex = 0;
    if (mean > 0.0 && isfinite(mean)) frexp(mean, &ex);
    const int e = ex >= 0 ? ex / 2 : -((1 - ex) / 2);  // floor(ex / 2): mean 2^-2e in [0.5, 2)
    // the FP64 pipe is slow here: one exact scaling product, one sum and the splitting per entry of
    // the upper triangle only
    const double down = ldexp(1.0, -2 * e), shift = shift_rel * mean * down;
    for (int i = ty; i < S; i += 16)
        for (int j = i + ((tx - i) & 15); j < S; j += 16) {
            const double g = G[i * S + j] * down + (i == j ? shift : 0.0);
            const float h = __double2float_rn(g);
            H[i * L + j] = h;
            Lo[i * L + j] = __double2float_rn(g - (double)h);
        }
    __syncthreads();
    // row 0 of R, then one barrier per pivot: in step k warp 0 brings row k + 1 up to date, forms its
    // pivot and scales it into R's row (look-ahead), while warps 1-7 update rows k + 2 onwards with
    // row k; nobody reads row k + 1 in step k
    auto pivot = [&](int k, F2 dk, F2 &y) {
        if (!(dk.h > tiny)) {
            dk = {tiny, 0.f};
            if ((tid & 31) == 0) atomicOr(status, 1);
        }
        y = f2_rsqrt(dk);
        return f2_mul(dk, y);
    };
    if (tid < 32) {
        F2 y;
        const F2 r = pivot(0, {H[0], Lo[0]}, y);
        for (int j = 1 + tid; j < S; j += 32) {
            const F2 v = f2_mul({H[j], Lo[j]}, y);
            H[j] = v.h, Lo[j] = v.l;
        }
        if (tid == 0) rdh[0] = r.h, rdl[0] = r.l, yh[0] = y.h, yl[0] = y.l;
    }
    __syncthreads();
    for (int k = 0; k + 1 < S; ++k) {
        const float *rkh = H + k * L, *rkl = Lo + k * L;
        if (tid < 32) {
            const int i = k + 1;
            const F2 a = {rkh[i], rkl[i]};
            for (int j = i + tid; j < S; j += 32) {
                const F2 v = f2_add({H[i * L + j], Lo[i * L + j]}, f2_neg(f2_mul(a, {rkh[j], rkl[j]})));
                H[i * L + j] = v.h, Lo[i * L + j] = v.l;
            }
            __syncwarp();
            F2 y;
            const F2 r = pivot(i, {H[i * L + i], Lo[i * L + i]}, y);
            for (int j = i + 1 + tid; j < S; j += 32) {
                const F2 v = f2_mul({H[i * L + j], Lo[i * L + j]}, y);
                H[i * L + j] = v.h, Lo[i * L + j] = v.l;
            }
            if (tid == 0) rdh[i] = r.h, rdl[i] = r.l, yh[i] = y.h, yl[i] = y.l;
        } else {
            const int u = tid - 32, uy = u >> 4;  // 14 row lanes x 16 column lanes
            for (int i = k + 2 + uy; i < S; i += 14) {
                const F2 a = {rkh[i], rkl[i]};
                for (int j = i + ((tx - i) & 15); j < S; j += 32) {  // j >= i, j = tx (mod 16), two at a time
                    const bool two = j + 16 < S;
                    F2 m0 = {H[i * L + j], Lo[i * L + j]}, b0 = {rkh[j], rkl[j]}, m1 = {0.f, 0.f}, b1 = {0.f, 0.f};
                    if (two) m1 = {H[i * L + j + 16], Lo[i * L + j + 16]}, b1 = {rkh[j + 16], rkl[j + 16]};
                    m0 = f2_add(m0, f2_neg(f2_mul(a, b0)));
                    m1 = f2_add(m1, f2_neg(f2_mul(a, b1)));
                    H[i * L + j] = m0.h, Lo[i * L + j] = m0.l;
                    if (two) H[i * L + j + 16] = m1.h, Lo[i * L + j + 16] = m1.l;
                }
            }
        }
        __syncthreads();
    }
    for (int q = tid; q < S * S; q += 256) {  // the strict lower triangle holds X's sums: start at 0
        const int i = q / S, j = q - i * S;
        if (i > j) H[i * L + j] = Lo[i * L + j] = 0.f;
    }
    __syncthreads();
    for (int q = 0; q + 1 < S; ++q) {
        for (int i = ty; i <= q; i += 16) {
            const F2 xiq = i == q ? F2{yh[q], yl[q]} : F2{H[q * L + i], Lo[q * L + i]};
            for (int j = q + 1 + tx; j < S; j += 32) {  // two at a time
                const bool two = j + 16 < S;
                F2 a0 = {H[j * L + i], Lo[j * L + i]}, b0 = {H[q * L + j], Lo[q * L + j]}, a1 = {0.f, 0.f},
                   b1 = {0.f, 0.f};
                if (two) a1 = {H[(j + 16) * L + i], Lo[(j + 16) * L + i]}, b1 = {H[q * L + j + 16], Lo[q * L + j + 16]};
                a0 = f2_add(a0, f2_mul(xiq, b0));
                a1 = f2_add(a1, f2_mul(xiq, b1));
                if (j == q + 1) a0 = f2_neg(f2_mul(a0, {yh[j], yl[j]}));
                H[j * L + i] = a0.h, Lo[j * L + i] = a0.l;
                if (two) H[(j + 16) * L + i] = a1.h, Lo[(j + 16) * L + i] = a1.l;
            }
        }
        __syncthreads();
    }
    // R in FP64 (scaled back by 2^e, exactly), R^-1 in FP32 (h + l rounded, scaled by 2^-e in FP32: exact
    // unless it leaves FP32's range, where the FP32 copy could not hold it anyway)
    const double up = ldexp(1.0, e);
    const float rinv_scale = __double2float_rn(ldexp(1.0, -e));
    for (int q = tid; q < S * S; q += 256) {
        const int i = q / S, j = q - i * S;
        float x = 0.f;
        if (i < j) {
            if (R) R[q] = ((double)H[i * L + j] + (double)Lo[i * L + j]) * up;
            x = __fadd_rn(H[j * L + i], Lo[j * L + i]);
        } else if (i == j) {
            if (R) R[q] = ((double)rdh[i] + (double)rdl[i]) * up;
            x = __fadd_rn(yh[i], yl[i]);
        } else if (R) {
            R[q] = 0.0;
        }
        Rinv32[q] = x * rinv_scale;
    }
}
// ---------------------------------------------------------------- Bt = A'^T Q
// A: n x d, Q: n x s (s <= 128, s % 16 == 0), w: n or null.  CTA (column block jb, row chunk g):
// columns [64 jb, 64 jb + 64) of d, rows of chunk g; thread (tx, ty) owns columns tx + 16 q and
// singular-space indices ty + 16 p; FP32 sums over 32-row stages added into double-float.
// part[(g * d + j) * s + i] = (hi, lo).
template <int NP>
__global__ void __launch_bounds__(256, 2) k_gemm_tn(const float *__restrict__ A, const float *__restrict__ Q,
                                                 const float *__restrict__ w, int64_t n, int64_t d, int64_t s,
                                                 int64_t rows, float2 *__restrict__ part) {
    __shared__ float As[TN_RS][TN_BJ + 4];
    __shared__ float Qs[TN_RS][16 * NP + 4];
    const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
    const int64_t j0 = (int64_t)blockIdx.x * TN_BJ;
    const int64_t r0 = (int64_t)blockIdx.y * rows, r1 = min(n, r0 + rows);
    const bool vec = (d & 3) == 0 && (reinterpret_cast<uintptr_t>(A) & 15) == 0;
    float hi[4][NP], lo[4][NP];
#pragma unroll
    for (int q = 0; q < 4; ++q)
#pragma unroll
        for (int p = 0; p < NP; ++p) hi[q][p] = lo[q][p] = 0.f;
    for (int64_t base = r0; base < r1; base += TN_RS) {
        if (vec) {
#pragma unroll
            for (int u = 0; u < 2; ++u) {
                const int e = tid + 256 * u, rr = e >> 4, c4 = (e & 15) * 4;
                const int64_t r = base + rr, j = j0 + c4;
                float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
                if (r < r1 && j < d) {
                    v = __ldg(reinterpret_cast<const float4 *>(A + r * d + j));
                    if (w) {
                        const float sc = sqrtf(fmaxf(w[r], 0.f));
                        v.x *= sc, v.y *= sc, v.z *= sc, v.w *= sc;
                    }
                }
                As[rr][c4] = v.x, As[rr][c4 + 1] = v.y, As[rr][c4 + 2] = v.z, As[rr][c4 + 3] = v.w;
            }
        } else {
            for (int e = tid; e < TN_RS * TN_BJ; e += 256) {
                const int rr = e / TN_BJ, cc = e % TN_BJ;
                const int64_t r = base + rr, j = j0 + cc;
                float v = 0.f;
                if (r < r1 && j < d) {
                    v = A[r * d + j];
                    if (w) v *= sqrtf(fmaxf(w[r], 0.f));
                }
                As[rr][cc] = v;
            }
        }
        for (int e = tid; e < TN_RS * 16 * NP; e += 256) {
            const int rr = e / (16 * NP), cc = e % (16 * NP);
            const int64_t r = base + rr;
            Qs[rr][cc] = (r < r1 && cc < s) ? Q[r * s + cc] : 0.f;
        }
        __syncthreads();
        float acc[4][NP];
#pragma unroll
        for (int q = 0; q < 4; ++q)
#pragma unroll
            for (int p = 0; p < NP; ++p) acc[q][p] = 0.f;
#pragma unroll 8
        for (int kk = 0; kk < TN_RS; ++kk) {
            float a[4], b[NP];
#pragma unroll
            for (int q = 0; q < 4; ++q) a[q] = As[kk][tx + 16 * q];
#pragma unroll
            for (int p = 0; p < NP; ++p) b[p] = Qs[kk][ty + 16 * p];
#pragma unroll
            for (int q = 0; q < 4; ++q)
#pragma unroll
                for (int p = 0; p < NP; ++p) acc[q][p] = fmaf(a[q], b[p], acc[q][p]);
        }
#pragma unroll
        for (int q = 0; q < 4; ++q)
#pragma unroll
            for (int p = 0; p < NP; ++p) df_add_f(hi[q][p], lo[q][p], acc[q][p]);
        __syncthreads();
    }
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const int64_t j = j0 + tx + 16 * q;
        if (j >= d) continue;
#pragma unroll
        for (int p = 0; p < NP; ++p) {
            const int64_t i = ty + 16 * p;
            if (i < s) part[((int64_t)blockIdx.y * d + j) * s + i] = make_float2(hi[q][p], lo[q][p]);
        }
    }
}

__global__ void __launch_bounds__(256) k_tn_reduce(const float2 *__restrict__ part, int64_t d, int64_t s,
                                                   int chunks, float *__restrict__ Bt) {
    const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e >= d * s) return;
    float hi = 0.f, lo = 0.f;
    for (int g = 0; g < chunks; ++g) {
        const float2 v = part[(int64_t)g * d * s + e];
        df_add_f(hi, lo, v.x);
        df_add_f(hi, lo, v.y);
    }
    Bt[e] = (float)((double)hi + (double)lo);
}

static int launch_gemm_tn(gbkm_ctx *c, const float *A, const float *Q, const float *w, int64_t n, int64_t d,
                          int64_t s, float2 *part, float *Bt) {
    // as many row chunks as fill one wave of resident CTAs (2 per SM)
    const int64_t cols = ceil_div(d, (int64_t)TN_BJ), per_sm = 2;
    int64_t ch = std::min<int64_t>((int64_t)TN_CHUNKS, ceil_div(n, (int64_t)1024));
    ch = std::min<int64_t>(ch, std::max<int64_t>(1, per_sm * c->sm_count / cols));
    const int chunks = (int)std::max<int64_t>(1, ch);
    const int64_t rows = ceil_div(n, (int64_t)chunks);
    const dim3 grid((unsigned)ceil_div(d, (int64_t)TN_BJ), (unsigned)chunks);
    switch (s / 16) {
        case 1: k_gemm_tn<1><<<grid, 256, 0, c->stream>>>(A, Q, w, n, d, s, rows, part); break;
        case 2: k_gemm_tn<2><<<grid, 256, 0, c->stream>>>(A, Q, w, n, d, s, rows, part); break;
        case 3: k_gemm_tn<3><<<grid, 256, 0, c->stream>>>(A, Q, w, n, d, s, rows, part); break;
        case 4: k_gemm_tn<4><<<grid, 256, 0, c->stream>>>(A, Q, w, n, d, s, rows, part); break;
        case 5: k_gemm_tn<5><<<grid, 256, 0, c->stream>>>(A, Q, w, n, d, s, rows, part); break;
        case 6: k_gemm_tn<6><<<grid, 256, 0, c->stream>>>(A, Q, w, n, d, s, rows, part); break;
        case 7: k_gemm_tn<7><<<grid, 256, 0, c->stream>>>(A, Q, w, n, d, s, rows, part); break;
        case 8: k_gemm_tn<8><<<grid, 256, 0, c->stream>>>(A, Q, w, n, d, s, rows, part); break;
        default: return set_error(c, GBKM_EUNSUPPORTED, "gemm_tn: s = %lld", (long long)s);
    }
    k_tn_reduce<<<(unsigned)ceil_div(d * s, (int64_t)256), 256, 0, c->stream>>>(part, d, s, chunks, Bt);
    c->launches += 2;
    return cuda_check(c, cudaGetLastError(), "gemm_tn launch");
}

// ---------------------------------------------------------------- one-sided Jacobi (one CTA)
// X = R_b^T (s x s, column c of X = row c of R_b) is orthogonalised by plane rotations applied on
// the right, accumulated in J: X J = W Sigma with orthogonal columns whose norms are the singular
// values.  Rounds follow the circle method (s - 1 rounds of s / 2 disjoint pairs per sweep); each
// half-warp rotates one pair of a round (8 s threads: s is a multiple of 16), its lanes holding rows
// gl, gl + 16, ... of both columns in registers for the round.  A pair is rotated when
// |x_p . x_q| > tol ||x_p|| ||x_q||; sweeps stop when no pair is (or after 30, flagged in *status).
// A rotation built as c = 1 / sqrt(1 + t^2), s = c t is orthogonal to rounding whatever the accuracy
// of its angle t, so the angle's quotient and root take the fast forms.  Then the singular values are
// ranked (decreasing, lower index first on ties), sigma[0..l) written, and T = R_b^-1 J[:, order[0..l)]
// (s x l, FP32) from R_b^-1 staged, transposed, in X's place.  Dynamic shared memory: 2 s^2 floats +
// s ints.
constexpr int JAC_ROWS = 8;  // rows per lane of a half-warp: s <= 128
__global__ void __launch_bounds__(1024) k_jacobi(const double *__restrict__ R, const float *__restrict__ Rinv32,
                                                 int64_t s, int64_t ell, float tol, float *__restrict__ sigma,
                                                 float *__restrict__ T, int *status) {
    extern __shared__ float js[];
    const int S = (int)s, nt = (int)blockDim.x;
    float *X = js;      // column-major: X[c * s + r]
    float *J = js + S * S;  // column-major
    int *order = reinterpret_cast<int *>(js + 2 * S * S);
    __shared__ float nrm[128];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int g = tid >> 4, gl = tid & 15;
    for (int e = tid; e < S * S; e += nt) {
        const int cc = e / S, r = e - cc * S;
        X[e] = (float)R[e];
        J[e] = cc == r ? 1.f : 0.f;
    }
    __syncthreads();
    const int half = S / 2, rounds = S - 1;
    const bool act = g < half;
    int sweep = 0;
    for (; sweep < 30; ++sweep) {
        bool any = false;
        for (int t = 0; t < rounds; ++t) {
            int p = S - 1, q = t;
            if (g != 0) {
                p = t + g;
                if (p >= S - 1) p -= S - 1;
                q = t - g;
                if (q < 0) q += S - 1;
            }
            float *xp = X + p * S, *xq = X + q * S;
            float a[JAC_ROWS], b[JAC_ROWS];
            float al = 0.f, be = 0.f, ga = 0.f;
#pragma unroll
            for (int u = 0; u < JAC_ROWS; ++u) {
                const int r = gl + 16 * u;
                const bool in = act && r < S;
                a[u] = in ? xp[r] : 0.f;
                b[u] = in ? xq[r] : 0.f;
            }
#pragma unroll
            for (int u = 0; u < JAC_ROWS; ++u) {
                al = fmaf(a[u], a[u], al);
                be = fmaf(b[u], b[u], be);
                ga = fmaf(a[u], b[u], ga);
            }
#pragma unroll
            for (int o = 8; o > 0; o >>= 1) {  // sums within each half-warp
                al += __shfl_xor_sync(0xffffffffu, al, o);
                be += __shfl_xor_sync(0xffffffffu, be, o);
                ga += __shfl_xor_sync(0xffffffffu, ga, o);
            }
            if (act && fabsf(ga) > tol * sqrtf(al * be) && ga != 0.f) {
                const float zeta = __fdividef(be - al, 2.f * ga);
                const float tt = copysignf(__fdividef(1.f, fabsf(zeta) + sqrtf(fmaf(zeta, zeta, 1.f))), zeta);
                const float cs = rsqrtf(fmaf(tt, tt, 1.f)), sn = cs * tt;
                float *jp = J + p * S, *jq = J + q * S;
#pragma unroll
                for (int u = 0; u < JAC_ROWS; ++u) {
                    const int r = gl + 16 * u;
                    if (r < S) {
                        const float ja = jp[r], jb = jq[r];
                        xp[r] = cs * a[u] - sn * b[u];
                        xq[r] = sn * a[u] + cs * b[u];
                        jp[r] = cs * ja - sn * jb;
                        jq[r] = sn * ja + cs * jb;
                    }
                }
                any = true;
            }
            __syncthreads();
        }
        if (!__syncthreads_or(any)) break;  // the same verdict on every thread
    }
    // bits 8-15: sweeps run (the sweep that found no pair to rotate included); bit 1: the cap
    if (tid == 0) atomicOr(status, sweep == 30 ? (2 | (30 << 8)) : ((sweep + 1) << 8));
    for (int cc = warp; cc < S; cc += nt >> 5) {
        float a = 0.f;
        for (int r = lane; r < S; r += 32) a = fmaf(X[cc * S + r], X[cc * S + r], a);
        a = warp_sum_f(a);
        if (lane == 0) nrm[cc] = sqrtf(a);
    }
    __syncthreads();
    for (int cc = tid; cc < S; cc += nt) {
        int rank = 0;
        for (int o = 0; o < S; ++o) rank += (nrm[o] > nrm[cc]) || (nrm[o] == nrm[cc] && o < cc);
        order[rank] = cc;
    }
    for (int e = tid; e < S * S; e += nt) {  // X <- (R_b^-1)^T: Xt[k * s + r] = R_b^-1[r][k]
        const int k = e / S, r = e - k * S;
        X[e] = Rinv32[r * S + k];
    }
    __syncthreads();
    for (int64_t m = tid; m < ell; m += nt) sigma[m] = nrm[order[m]];
    // T[r][m] = sum_k R_b^-1[r][k] J[k][order[m]] (R_b^-1 is upper triangular: the zeros add nothing)
    for (int e = tid; e < S * (int)ell; e += nt) {
        const int m = e / S, r = e - m * S;
        const float *jc = J + order[m] * S;
        float acc = 0.f;
        for (int k = 0; k < S; ++k) acc = fmaf(X[k * S + r], jc[k], acc);
        T[(int64_t)r * ell + m] = acc;
    }
}

// ---------------------------------------------------------------- column signs of V (d x l)
__global__ void __launch_bounds__(256) k_sign(float *__restrict__ V, int64_t d, int64_t ell) {
    __shared__ float bv[256];
    __shared__ int64_t bi[256];
    const int64_t m = blockIdx.x;
    float best = -1.f;
    int64_t arg = 0;
    for (int64_t r = threadIdx.x; r < d; r += 256) {
        const float a = fabsf(V[r * ell + m]);
        if (a > best) best = a, arg = r;
    }
    bv[threadIdx.x] = best;
    bi[threadIdx.x] = arg;
    __syncthreads();
    for (int o = 128; o > 0; o >>= 1) {
        if ((int)threadIdx.x < o) {
            const float b2 = bv[threadIdx.x + o];
            const int64_t i2 = bi[threadIdx.x + o];
            if (b2 > bv[threadIdx.x] || (b2 == bv[threadIdx.x] && i2 < bi[threadIdx.x]))
                bv[threadIdx.x] = b2, bi[threadIdx.x] = i2;
        }
        __syncthreads();
    }
    const bool flip = V[bi[0] * ell + m] < 0.f;
    if (flip)
        for (int64_t r = threadIdx.x; r < d; r += 256) V[r * ell + m] = -V[r * ell + m];
}

// ---------------------------------------------------------------- orchestration
struct SvdPlan {
    size_t o_y, o_q, o_gpart, o_g, o_r, o_rinv32, o_tpart, o_bt, o_t, o_sig, o_status, o_omt, o_qt, o_rpart,
        bytes;
    bool tc;  // the two passes over the piece on the tensor cores
};

static SvdPlan svd_plan(int64_t n, int64_t d, int64_t s, int64_t ell, int sm_count, bool tc) {
    SvdPlan P;
    WsPlan p;
    P.tc = tc;
    const int64_t gchunks = std::max<int64_t>(gram_chunks(n, sm_count), gram_chunks(d, sm_count));
    P.o_y = p.take<float>(n * s);
    P.o_q = p.take<float>(n * s);
    P.o_gpart = p.take<float2>(gchunks * s * s);
    P.o_g = p.take<double>(s * s);
    P.o_r = p.take<double>(s * s);
    P.o_rinv32 = p.take<float>(s * s);
    P.o_tpart = p.take<float2>((int64_t)TN_CHUNKS * d * s);
    P.o_bt = p.take<float>(d * s);
    P.o_t = p.take<float>(s * ell);
    P.o_sig = p.take<float>(ell);
    P.o_status = p.take<int>(1);
    int splits = 1, kbs = 1;
    if (tc) tc_rows_shape(n, d, sm_count, &splits, &kbs);
    P.o_omt = p.take<float>(tc ? 2 * s * d : 0);
    P.o_qt = p.take<float>(tc ? 2 * s * (ceil_div(n, (int64_t)4) * 4) : 0);
    P.o_rpart = p.take<float>(tc ? (int64_t)splits * d * s : 0);
    P.bytes = p.off;
    return P;
}

int rsvd_impl(gbkm_ctx *c, const float *A, int64_t n, int64_t d, const float *w, const float *Omega, int64_t s,
              int64_t ell, float *V, float *sigma, int32_t *info) {
    // the passes over the piece run on the tensor cores (3xTF32) when the shapes allow TMA tiles
    const bool tc = tc_rows_supported(d, s) && (reinterpret_cast<uintptr_t>(A) & 15) == 0;
    const SvdPlan P = svd_plan(n, d, s, ell, c->sm_count, tc);
    int rc = GBKM_OK;
    void *ws = ws_reserve(c, P.bytes, &rc);
    if (!ws) return rc;
    float *Y = ws_at<float>(ws, P.o_y), *Q = ws_at<float>(ws, P.o_q);
    float2 *gpart = ws_at<float2>(ws, P.o_gpart), *tpart = ws_at<float2>(ws, P.o_tpart);
    double *G = ws_at<double>(ws, P.o_g), *R = ws_at<double>(ws, P.o_r);
    float *Rinv32 = ws_at<float>(ws, P.o_rinv32), *Bt = ws_at<float>(ws, P.o_bt), *T = ws_at<float>(ws, P.o_t);
    int *st = info ? reinterpret_cast<int *>(info) : ws_at<int>(ws, P.o_status);
    if (!sigma) sigma = ws_at<float>(ws, P.o_sig);
    if (cudaMemsetAsync(st, 0, sizeof(int), c->stream) != cudaSuccess) return cuda_check(c, cudaGetLastError(), "rsvd info");
    const size_t jsm = sizeof(float) * 2 * (size_t)s * (size_t)s + sizeof(int) * (size_t)s;
    if (jsm > 48 * 1024) cudaFuncSetAttribute(k_jacobi, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)jsm);
    const size_t csm = sizeof(float) * (2 * (size_t)s * (size_t)(s + 1) + 4 * (size_t)s);
    if (csm > 48 * 1024) cudaFuncSetAttribute(k_chol, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)csm);

    // 1. Y = A' Omega
    prof_begin(c, "rsvd_sketch");
    rc = tc ? launch_sketch_tc(c, A, w, n, d, Omega, s, ws_at<float>(ws, P.o_omt), Y)
            : launch_gemm_rows(c, A, Omega, w, n, d, s, Y);
    prof_end(c);
    if (rc != GBKM_OK) return rc;
    // 2. CholeskyQR2: Y -> Q (via Q) -> Y
    prof_begin(c, "rsvd_qr");
    if ((rc = launch_gram(c, Y, n, s, gpart, G)) != GBKM_OK) return rc;
    k_chol<<<1, 256, csm, c->stream>>>(G, s, 1e-6, R, Rinv32, st);
    GBKM_LAUNCHED(c);
    if ((rc = launch_gemm_rows(c, Y, Rinv32, nullptr, n, s, s, Q)) != GBKM_OK) return rc;
    if ((rc = launch_gram(c, Q, n, s, gpart, G)) != GBKM_OK) return rc;
    k_chol<<<1, 256, csm, c->stream>>>(G, s, 1e-9, R, Rinv32, st);
    GBKM_LAUNCHED(c);
    if ((rc = launch_gemm_rows(c, Q, Rinv32, nullptr, n, s, s, Y)) != GBKM_OK) return rc;
    prof_end(c);
    // 3. Bt = A'^T Q
    prof_begin(c, "rsvd_rows");
    rc = tc ? launch_rows_tc(c, A, w, n, d, Y, s, ws_at<float>(ws, P.o_qt), ws_at<float>(ws, P.o_rpart), Bt)
            : launch_gemm_tn(c, A, Y, w, n, d, s, tpart, Bt);
    prof_end(c);
    if (rc != GBKM_OK) return rc;
    // 4. R_b from the Gram of Bt
    prof_begin(c, "rsvd_small");
    if ((rc = launch_gram(c, Bt, d, s, gpart, G)) != GBKM_OK) return rc;
    k_chol<<<1, 256, csm, c->stream>>>(G, s, 1e-9, R, Rinv32, st);
    GBKM_LAUNCHED(c);
    // 5. singular values and T
    const float tol = (float)s * 1.2e-7f;
    k_jacobi<<<1, (unsigned)(8 * s), jsm, c->stream>>>(R, Rinv32, s, ell, tol, sigma, T, st);
    GBKM_LAUNCHED(c);
    prof_end(c);
    // 6. V = Bt T, 7. signs
    if ((rc = launch_gemm_rows(c, Bt, T, nullptr, d, s, ell, V)) != GBKM_OK) return rc;
    k_sign<<<(unsigned)ell, 256, 0, c->stream>>>(V, d, ell);
    GBKM_LAUNCHED(c);
    return cuda_check(c, cudaGetLastError(), "rsvd launch");
}

}  // namespace gbkm
