// k_svd.cu -- randomised truncated SVD of a piece (Section 2.2), weighted rows (Section 2.3.2).
//
// The top l right singular vectors of A' = diag(sqrt(w)) A (n x d, one point per row) after the
// randomised scheme of Halko, Martinsson and Tropp that the paper adopts: the columns of A' are
// reduced by a random d x s matrix Omega (s = l + oversampling), the rows by an orthonormal basis
// of the result, and only the s x d matrix left over is decomposed.  All on the context's stream:
//   1. Y = A' Omega (n x s): the tensor cores' 3xTF32 store GEMM (k_tc), or k_gemm_rows on the CUDA
//      cores where the shape does not allow TMA tiles                       first read of A
//   2. CholeskyQR2   k_gram (Y^T Y, FP32 blocks of 8 rows added in double-float), k_chol (FP64
//                    Cholesky with a small diagonal shift, R^-1), Y <- Y R^-1; twice -> Q
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
constexpr int GM_B = 64, GM_RS = 32;     // k_gram: 64 x 64 output blocks, 32-row stages
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
// X: m x s row-major.  CTA (block pair p, row chunk g) sums rows [g * rows, (g + 1) * rows) into
// the 64 x 64 block (bi, bj), bi <= bj, of the Gram matrix: FP32 products summed over 8 rows, each
// 8-row sum added into a double-float accumulator.  part[(g * npairs + p) * 4096 + local] = (hi, lo).
__global__ void __launch_bounds__(256) k_gram(const float *__restrict__ X, int64_t m, int64_t s, int64_t rows,
                                              float2 *__restrict__ part) {
    __shared__ float Xi[GM_RS][GM_B + 1];
    __shared__ float Xj[GM_RS][GM_B + 1];
    const int nb = (int)((s + GM_B - 1) / GM_B);
    int p = blockIdx.x, bi = 0;
    while (p >= nb - bi) {  // pair index -> (bi, bj), bi <= bj
        p -= nb - bi;
        ++bi;
    }
    const int bj = bi + p;
    const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
    const int64_t r0 = (int64_t)blockIdx.y * rows, r1 = min(m, r0 + rows);
    float hi[4][4], lo[4][4];
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) hi[a][b] = lo[a][b] = 0.f;
    for (int64_t base = r0; base < r1; base += GM_RS) {
        for (int e = tid; e < GM_RS * GM_B; e += 256) {
            const int rr = e / GM_B, cc = e % GM_B;
            const int64_t r = base + rr, ci = (int64_t)bi * GM_B + cc, cj = (int64_t)bj * GM_B + cc;
            Xi[rr][cc] = (r < r1 && ci < s) ? X[r * s + ci] : 0.f;
            Xj[rr][cc] = (r < r1 && cj < s) ? X[r * s + cj] : 0.f;
        }
        __syncthreads();
#pragma unroll
        for (int g8 = 0; g8 < GM_RS; g8 += 8) {
            float acc[4][4];
#pragma unroll
            for (int a = 0; a < 4; ++a)
#pragma unroll
                for (int b = 0; b < 4; ++b) acc[a][b] = 0.f;
#pragma unroll
            for (int rr = g8; rr < g8 + 8; ++rr) {
                float x[4], y[4];
#pragma unroll
                for (int a = 0; a < 4; ++a) x[a] = Xi[rr][ty + 16 * a];
#pragma unroll
                for (int b = 0; b < 4; ++b) y[b] = Xj[rr][tx + 16 * b];
#pragma unroll
                for (int a = 0; a < 4; ++a)
#pragma unroll
                    for (int b = 0; b < 4; ++b) acc[a][b] = fmaf(x[a], y[b], acc[a][b]);
            }
#pragma unroll
            for (int a = 0; a < 4; ++a)
#pragma unroll
                for (int b = 0; b < 4; ++b) df_add_f(hi[a][b], lo[a][b], acc[a][b]);
        }
        __syncthreads();
    }
    const int npairs = nb * (nb + 1) / 2;
    float2 *o = part + ((int64_t)blockIdx.y * npairs + blockIdx.x) * (GM_B * GM_B);
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) o[(ty + 16 * a) * GM_B + tx + 16 * b] = make_float2(hi[a][b], lo[a][b]);
}

// the chunks' partial blocks added (double-float) into the full symmetric FP64 G: one warp per
// entry of the upper triangle, lane l taking chunks l, l + 32, ..., then a fixed butterfly
__global__ void __launch_bounds__(256) k_gram_reduce(const float2 *__restrict__ part, int64_t s, int chunks,
                                                     double *__restrict__ G) {
    const int e = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31, S = (int)s;
    if (e >= S * S) return;
    const int i = e / S, j = e - i * S;
    if (i > j) return;
    const int nb = (S + GM_B - 1) / GM_B;
    const int bi = i / GM_B, bj = j / GM_B;
    int pidx = 0;
    for (int q = 0; q < bi; ++q) pidx += nb - q;
    pidx += bj - bi;
    const int npairs = nb * (nb + 1) / 2;
    const int loc = (i % GM_B) * GM_B + (j % GM_B);
    float hi = 0.f, lo = 0.f;
    for (int g = lane; g < chunks; g += 32) {
        const float2 v = part[((int64_t)g * npairs + pidx) * (GM_B * GM_B) + loc];
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

static int gram_chunks(int64_t m) { return (int)std::min<int64_t>(96, std::max<int64_t>(1, ceil_div(m, 256))); }

static int launch_gram(gbkm_ctx *c, const float *X, int64_t m, int64_t s, float2 *part, double *G) {
    const int chunks = gram_chunks(m);
    const int64_t rows = ceil_div(m, (int64_t)chunks);
    const int nb = (int)ceil_div(s, (int64_t)GM_B);
    k_gram<<<dim3((unsigned)(nb * (nb + 1) / 2), (unsigned)chunks), 256, 0, c->stream>>>(X, m, s, rows, part);
    k_gram_reduce<<<(unsigned)ceil_div(s * s * 32, (int64_t)256), 256, 0, c->stream>>>(part, s, chunks, G);
    c->launches += 2;
    return cuda_check(c, cudaGetLastError(), "gram launch");
}

// ---------------------------------------------------------------- Cholesky of G + shift I, R^-1
// One CTA, the factor in shared memory (s rows of s + 1 values of type W; FP64 here: an FP32
// factor with the shift FP32 needs leaves Q's columns short by that shift, which lowers every
// singular value by about 3e-4 relative).  G = R^T R, R upper triangular;
// shift = shift_rel * trace(G) / s is added to the diagonal, and a pivot that still falls to or
// below a tiny floor is clamped and flagged in *status.  R^-1 overwrites R in place, one column at
// a time: X R = I gives X[i][j] = -(sum_{i <= q < j} X[i][q] R[q][j]) / R[j][j], which reads the
// finished columns of X and the column j of R that is replaced next.  Outputs R and Rinv (FP64,
// each optional) and Rinv32.
template <typename W>
__global__ void __launch_bounds__(256) k_chol(const double *__restrict__ G, int64_t s, double shift_rel,
                                              double *__restrict__ R, double *__restrict__ Rinv,
                                              float *__restrict__ Rinv32, int *status) {
    extern __shared__ __align__(8) unsigned char chol_smem[];
    W *Rs = reinterpret_cast<W *>(chol_smem);
    __shared__ double red[256];
    __shared__ W inv_s;
    const W tiny = sizeof(W) == 4 ? (W)1e-30 : (W)1e-300;
    const int tid = threadIdx.x, S = (int)s, L = S + 1;  // row stride S + 1: a column walk spreads over banks
    double tr = 0.0;
    for (int i = tid; i < S; i += 256) tr += G[i * S + i];
    red[tid] = tr;
    __syncthreads();
    for (int o = 128; o > 0; o >>= 1) {
        if (tid < o) red[tid] += red[tid + o];
        __syncthreads();
    }
    const double shift = shift_rel * red[0] / (double)s;
    for (int e = tid; e < S * S; e += 256) {
        const int i = e / S, j = e - i * S;
        Rs[i * L + j] = (W)(i <= j ? G[e] + (i == j ? shift : 0.0) : 0.0);
    }
    __syncthreads();
    for (int k = 0; k < S; ++k) {
        if (tid == 0) {
            W dk = Rs[k * L + k];
            if (!(dk > tiny)) {
                dk = tiny;
                atomicOr(status, 1);
            }
            const W rkk = sqrt(dk);
            Rs[k * L + k] = rkk;
            inv_s = (W)1 / rkk;  // division and square root are long sequences: once per step
        }
        __syncthreads();
        const W inv = inv_s;
        for (int j = k + 1 + tid; j < S; j += 256) Rs[k * L + j] *= inv;
        __syncthreads();
        // trailing update of the upper triangle: row i = k + 1 + tid / 2 ... (threads stride rows)
        for (int i = k + 1 + (tid >> 3); i < S; i += 32) {
            const W rki = Rs[k * L + i];
            for (int j = i + (tid & 7); j < S; j += 8) Rs[i * L + j] -= rki * Rs[k * L + j];
        }
        __syncthreads();
    }
    if (R)
        for (int e = tid; e < S * S; e += 256) R[e] = (double)Rs[(e / S) * L + e % S];
    __syncthreads();
    for (int j = 0; j < S; ++j) {
        if (tid == 0) inv_s = (W)1 / Rs[j * L + j];
        __syncthreads();
        const W inv_jj = inv_s;
        W t = 0;
        const int i = tid;
        if (i < j)
            for (int q = i; q < j; ++q) t += Rs[i * L + q] * Rs[q * L + j];
        __syncthreads();
        if (i < j) Rs[i * L + j] = -t * inv_jj;
        if (i == j) Rs[j * L + j] = inv_jj;
        __syncthreads();
    }
    for (int e = tid; e < S * S; e += 256) {
        const W v = Rs[(e / S) * L + e % S];
        if (Rinv) Rinv[e] = (double)v;
        Rinv32[e] = (float)v;
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
// half-warp rotates one pair of a round (1,024 threads: 64 half-warps >= s / 2).  Sweeps stop
// when no pair has |x_p . x_q| > tol ||x_p|| ||x_q|| (or after 30, flagged in *status).  Then the
// singular values are ranked (decreasing, lower index first on ties), sigma[0..l) written, and
// T = R_b^-1 J[:, order[0..l)] (s x l, FP32).  Dynamic shared memory: 2 s^2 floats + s ints.
__global__ void __launch_bounds__(1024) k_jacobi(const double *__restrict__ R, const float *__restrict__ Rinv32,
                                                 int64_t s, int64_t ell, float tol, float *__restrict__ sigma,
                                                 float *__restrict__ T, int *status) {
    extern __shared__ float js[];
    float *X = js;               // column-major: X[c * s + r]
    float *J = js + s * s;       // column-major
    int *order = reinterpret_cast<int *>(js + 2 * s * s);
    __shared__ int rotated;
    __shared__ float nrm[128];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int g = tid >> 4, gl = tid & 15, S = (int)s;
    for (int e = tid; e < S * S; e += 1024) {
        const int cc = e / S, r = e - cc * S;
        X[e] = (float)R[e];
        J[e] = cc == r ? 1.f : 0.f;
    }
    __syncthreads();
    const int half = S / 2, rounds = S - 1;
    int sweep = 0;
    for (; sweep < 30; ++sweep) {
        if (tid == 0) rotated = 0;
        __syncthreads();
        for (int t = 0; t < rounds; ++t) {
            const bool act = g < half;
            const int m = act ? g : 0;
            int p = S - 1, q = t;
            if (m != 0) {
                p = t + m;
                if (p >= S - 1) p -= S - 1;
                q = t - m;
                if (q < 0) q += S - 1;
            }
            float *xp = X + p * S, *xq = X + q * S;
            float al = 0.f, be = 0.f, ga = 0.f;
            if (act)
                for (int r = gl; r < S; r += 16) {
                    const float a = xp[r], b = xq[r];
                    al = fmaf(a, a, al);
                    be = fmaf(b, b, be);
                    ga = fmaf(a, b, ga);
                }
#pragma unroll
            for (int o = 8; o > 0; o >>= 1) {  // sums within each half-warp
                al += __shfl_xor_sync(0xffffffffu, al, o);
                be += __shfl_xor_sync(0xffffffffu, be, o);
                ga += __shfl_xor_sync(0xffffffffu, ga, o);
            }
            if (act && fabsf(ga) > tol * sqrtf(al * be) && ga != 0.f) {
                const float zeta = (be - al) / (2.f * ga);
                const float tt = copysignf(1.f, zeta) / (fabsf(zeta) + sqrtf(1.f + zeta * zeta));
                const float cs = 1.f / sqrtf(1.f + tt * tt), sn = cs * tt;
                float *jp = J + p * S, *jq = J + q * S;
                for (int r = gl; r < S; r += 16) {
                    const float a = xp[r], b = xq[r];
                    xp[r] = cs * a - sn * b;
                    xq[r] = sn * a + cs * b;
                    const float ja = jp[r], jb = jq[r];
                    jp[r] = cs * ja - sn * jb;
                    jq[r] = sn * ja + cs * jb;
                }
                if (gl == 0) rotated = 1;
            }
            __syncthreads();
        }
        if (!rotated) break;
        __syncthreads();
    }
    // bits 8-15: sweeps run (the sweep that found no pair to rotate included); bit 1: the cap
    if (tid == 0) atomicOr(status, sweep == 30 ? (2 | (30 << 8)) : ((sweep + 1) << 8));
    for (int64_t cc = warp; cc < s; cc += 32) {
        float a = 0.f;
        for (int64_t r = lane; r < s; r += 32) a = fmaf(X[cc * s + r], X[cc * s + r], a);
        a = warp_sum_f(a);
        if (lane == 0) nrm[cc] = sqrtf(a);
    }
    __syncthreads();
    for (int64_t cc = tid; cc < s; cc += 1024) {
        int rank = 0;
        for (int64_t o = 0; o < s; ++o) rank += (nrm[o] > nrm[cc]) || (nrm[o] == nrm[cc] && o < cc);
        order[rank] = (int)cc;
    }
    __syncthreads();
    for (int64_t m = tid; m < ell; m += 1024) sigma[m] = nrm[order[m]];
    // T = R_b^-1 J[:, order[m]]
    for (int64_t e = tid; e < s * ell; e += 1024) {
        const int64_t r = e / ell, m = e % ell;
        const float *jc = J + (int64_t)order[m] * s;
        float acc = 0.f;
        for (int64_t k = r; k < s; ++k) acc = fmaf(Rinv32[r * s + k], jc[k], acc);
        T[r * ell + m] = acc;
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
    size_t o_y, o_q, o_gpart, o_g, o_r, o_rinv, o_rinv32, o_tpart, o_bt, o_t, o_sig, o_status, o_omt, o_qt, o_rpart,
        bytes;
    bool tc;  // the two passes over the piece on the tensor cores
};

static SvdPlan svd_plan(int64_t n, int64_t d, int64_t s, int64_t ell, int sm_count, bool tc) {
    SvdPlan P;
    WsPlan p;
    P.tc = tc;
    const int nb = (int)ceil_div(s, (int64_t)GM_B);
    const int64_t gchunks = std::max<int64_t>(gram_chunks(n), gram_chunks(d));
    P.o_y = p.take<float>(n * s);
    P.o_q = p.take<float>(n * s);
    P.o_gpart = p.take<float2>(gchunks * (nb * (nb + 1) / 2) * GM_B * GM_B);
    P.o_g = p.take<double>(s * s);
    P.o_r = p.take<double>(s * s);
    P.o_rinv = p.take<double>(s * s);
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
    double *G = ws_at<double>(ws, P.o_g), *R = ws_at<double>(ws, P.o_r), *Rinv = ws_at<double>(ws, P.o_rinv);
    float *Rinv32 = ws_at<float>(ws, P.o_rinv32), *Bt = ws_at<float>(ws, P.o_bt), *T = ws_at<float>(ws, P.o_t);
    int *st = info ? reinterpret_cast<int *>(info) : ws_at<int>(ws, P.o_status);
    if (!sigma) sigma = ws_at<float>(ws, P.o_sig);
    if (cudaMemsetAsync(st, 0, sizeof(int), c->stream) != cudaSuccess) return cuda_check(c, cudaGetLastError(), "rsvd info");
    const size_t jsm = sizeof(float) * 2 * (size_t)s * (size_t)s + sizeof(int) * (size_t)s;
    if (jsm > 48 * 1024) cudaFuncSetAttribute(k_jacobi, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)jsm);
    const size_t csm = sizeof(double) * (size_t)s * (size_t)(s + 1);
    if (csm > 48 * 1024) cudaFuncSetAttribute(k_chol<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)csm);

    // 1. Y = A' Omega
    prof_begin(c, "rsvd_sketch");
    rc = tc ? launch_sketch_tc(c, A, w, n, d, Omega, s, ws_at<float>(ws, P.o_omt), Y)
            : launch_gemm_rows(c, A, Omega, w, n, d, s, Y);
    prof_end(c);
    if (rc != GBKM_OK) return rc;
    // 2. CholeskyQR2: Y -> Q (via Q) -> Y
    prof_begin(c, "rsvd_qr");
    if ((rc = launch_gram(c, Y, n, s, gpart, G)) != GBKM_OK) return rc;
    k_chol<double><<<1, 256, csm, c->stream>>>(G, s, 1e-6, R, Rinv, Rinv32, st);
    GBKM_LAUNCHED(c);
    if ((rc = launch_gemm_rows(c, Y, Rinv32, nullptr, n, s, s, Q)) != GBKM_OK) return rc;
    if ((rc = launch_gram(c, Q, n, s, gpart, G)) != GBKM_OK) return rc;
    k_chol<double><<<1, 256, csm, c->stream>>>(G, s, 1e-9, R, Rinv, Rinv32, st);
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
    k_chol<double><<<1, 256, csm, c->stream>>>(G, s, 1e-9, R, Rinv, Rinv32, st);
    GBKM_LAUNCHED(c);
    // 5. singular values and T
    const float tol = (float)s * 1.2e-7f;
    k_jacobi<<<1, 1024, jsm, c->stream>>>(R, Rinv32, s, ell, tol, sigma, T, st);
    GBKM_LAUNCHED(c);
    prof_end(c);
    // 6. V = Bt T, 7. signs
    if ((rc = launch_gemm_rows(c, Bt, T, nullptr, d, s, ell, V)) != GBKM_OK) return rc;
    k_sign<<<(unsigned)ell, 256, 0, c->stream>>>(V, d, ell);
    GBKM_LAUNCHED(c);
    return cuda_check(c, cudaGetLastError(), "rsvd launch");
}

}  // namespace gbkm
