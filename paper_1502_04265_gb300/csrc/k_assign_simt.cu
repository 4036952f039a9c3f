// k_assign_simt.cu -- CUDA-core (FFMA) distance tiles with the fused top-2 epilogue,
// a plain SIMT GEMM (projection fallback), and the exact near-tie recheck (A5).
#include <float.h>

#include "internal.cuh"

namespace gbkm {

namespace {
constexpr int BM = 128, BN = 64, BK = 16;

__device__ __forceinline__ void top2_push(float s, int j, float &b1, int &a1, float &b2) {
    if (s < b1) {
        b2 = b1;
        b1 = s;
        a1 = j;
    } else if (s < b2) {
        b2 = s;
    }
}

// merge (c1, j1, c2) into (b1, a1, b2); ties on the best value go to the lower index
__device__ __forceinline__ void top2_merge(float &b1, int &a1, float &b2, float c1, int j1, float c2) {
    if (c1 < b1 || (c1 == b1 && j1 < a1)) {
        b2 = fminf(b1, c2);
        b1 = c1;
        a1 = j1;
    } else {
        b2 = fminf(b2, c1);
    }
}

__device__ __forceinline__ unsigned lanemask_lt() {
    unsigned m;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
    return m;
}
}  // namespace

// certified near-tie bound of a row: E(x) = err_rel ||x|| cmax + err_abs cmax^2; the argmin
// is certain when second - best > 2 E(x)
__device__ __forceinline__ bool near_tie(float b1, float b2, float xn, float cm, float err_rel,
                                         float err_abs) {
    float xr = sqrtf(fmaxf(xn, 0.f)) * (1.f + 1.0e-6f);
    float E = err_rel * xr * cm + err_abs * cm * cm;
    return !((b2 - b1) > 2.f * E);
}

__device__ __forceinline__ void emit_row(int64_t row, float b1, int a1, float b2, float xn, float cm,
                                         float err_rel, float err_abs, bool valid,
                                         const AssignOut &o) {
    const int lane = threadIdx.x & 31;
    bool flag = valid && near_tie(b1, b2, xn, cm, err_rel, err_abs);
    if (valid) {
        o.labels[row] = a1;
        if (o.min_d2) o.min_d2[row] = fmaxf(0.f, xn + b1);
    }
    if (o.flag_list) {
        unsigned m = __ballot_sync(0xffffffffu, flag);
        if (m) {
            int leader = __ffs(m) - 1;
            int base = 0;
            if (lane == leader) base = atomicAdd(o.flag_count, __popc(m));
            base = __shfl_sync(0xffffffffu, base, leader);
            if (flag) {
                const int slot = base + __popc(m & lanemask_lt());
                o.flag_list[slot] = (int32_t)row;
                o.cand[(int64_t)slot * CAND_STRIDE] = -1;
            }
        }
    }
}

// ---------------------------------------------------------------- FFMA distance tiles
// CTA: 128 rows x all k centers in chunks of 64, K in steps of 16.  Thread (ty, tx) owns rows
// ty + 16 i and columns tx + 16 j of each chunk; per-row top-2 is merged across the 16 tx
// lanes with shuffles at the end.
__global__ void __launch_bounds__(256) k_assign_simt(const float *__restrict__ X,
                                                     const float *__restrict__ xnorm, int64_t n,
                                                     int64_t d, const float *__restrict__ C,
                                                     const float *__restrict__ cnorm,
                                                     const unsigned *__restrict__ cmax, int64_t k,
                                                     float err_rel, float err_abs, AssignOut o) {
    __shared__ float As[BK][BM + 4];
    __shared__ float Bs[BK][BN + 4];
    const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
    const int64_t m0 = (int64_t)blockIdx.x * BM;
    const bool vec = ((d & 3) == 0) && ((reinterpret_cast<uintptr_t>(X) & 15) == 0) &&
                     ((reinterpret_cast<uintptr_t>(C) & 15) == 0);
    float b1[8], b2[8];
    int a1[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        b1[i] = FLT_MAX * 2.f;
        b2[i] = FLT_MAX * 2.f;
        a1[i] = 0;
    }
    const int lr = tid >> 2, lc = (tid & 3) * 4;
    for (int64_t n0 = 0; n0 < k; n0 += BN) {
        float acc[8][4];
#pragma unroll
        for (int i = 0; i < 8; ++i)
#pragma unroll
            for (int j = 0; j < 4; ++j) acc[i][j] = 0.f;
        for (int64_t k0 = 0; k0 < d; k0 += BK) {
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int r = lr + 64 * h;
                const int64_t gr = m0 + r;
                float v[4] = {0.f, 0.f, 0.f, 0.f};
                if (gr < n) {
                    if (vec && k0 + lc + 3 < d) {
                        float4 q = __ldg(reinterpret_cast<const float4 *>(X + gr * d + k0 + lc));
                        v[0] = q.x, v[1] = q.y, v[2] = q.z, v[3] = q.w;
                    } else {
#pragma unroll
                        for (int q = 0; q < 4; ++q)
                            if (k0 + lc + q < d) v[q] = X[gr * d + k0 + lc + q];
                    }
                }
#pragma unroll
                for (int q = 0; q < 4; ++q) As[lc + q][r] = v[q];
            }
            {
                const int64_t gc = n0 + lr;
                float v[4] = {0.f, 0.f, 0.f, 0.f};
                if (gc < k) {
                    if (vec && k0 + lc + 3 < d) {
                        float4 q = __ldg(reinterpret_cast<const float4 *>(C + gc * d + k0 + lc));
                        v[0] = q.x, v[1] = q.y, v[2] = q.z, v[3] = q.w;
                    } else {
#pragma unroll
                        for (int q = 0; q < 4; ++q)
                            if (k0 + lc + q < d) v[q] = C[gc * d + k0 + lc + q];
                    }
                }
#pragma unroll
                for (int q = 0; q < 4; ++q) Bs[lc + q][lr] = v[q];
            }
            __syncthreads();
#pragma unroll
            for (int kk = 0; kk < BK; ++kk) {
                float a[8], b[4];
#pragma unroll
                for (int i = 0; i < 8; ++i) a[i] = As[kk][ty + 16 * i];
#pragma unroll
                for (int j = 0; j < 4; ++j) b[j] = Bs[kk][tx + 16 * j];
#pragma unroll
                for (int i = 0; i < 8; ++i)
#pragma unroll
                    for (int j = 0; j < 4; ++j) acc[i][j] = fmaf(a[i], b[j], acc[i][j]);
            }
            __syncthreads();
        }
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int64_t col = n0 + tx + 16 * j;
            if (col < k) {
                const float cn = __ldg(cnorm + col);
#pragma unroll
                for (int i = 0; i < 8; ++i) top2_push(fmaf(-2.f, acc[i][j], cn), (int)col, b1[i], a1[i], b2[i]);
            }
        }
    }
    const float cm = __uint_as_float(*cmax);
#pragma unroll
    for (int i = 0; i < 8; ++i) {
#pragma unroll
        for (int o2 = 1; o2 < 16; o2 <<= 1) {
            float c1 = __shfl_xor_sync(0xffffffffu, b1[i], o2);
            int j1 = __shfl_xor_sync(0xffffffffu, a1[i], o2);
            float c2 = __shfl_xor_sync(0xffffffffu, b2[i], o2);
            top2_merge(b1[i], a1[i], b2[i], c1, j1, c2);
        }
        const int64_t row = m0 + ty + 16 * i;
        const bool valid = (tx == 0) && (row < n);
        const float xn = valid ? xnorm[row] : 0.f;
        emit_row(row, b1[i], a1[i], b2[i], xn, cm, err_rel, err_abs, valid, o);
    }
}

int launch_assign_simt(gbkm_ctx *c, const float *X, const float *xnorm, int64_t n, int64_t d,
                       const float *C, const float *cnorm, const unsigned *cmax, int64_t k,
                       float err_rel, float err_abs, const AssignOut &o) {
    if (n == 0) return GBKM_OK;
    k_assign_simt<<<(unsigned)ceil_div(n, BM), 256, 0, c->stream>>>(X, xnorm, n, d, C, cnorm, cmax, k,
                                                                   err_rel, err_abs, o);
    GBKM_LAUNCHED(c);
    return cuda_check(c, cudaGetLastError(), "assign_simt launch");
}

// ---------------------------------------------------------------- plain SIMT GEMM
// Out[M x N] = A[M x K] * B^T with B addressed as B[nn * sbn + kk * sbk] (so both a K-major
// N x K matrix and a row-major K x N matrix can be passed).  FP32 FFMA, row-major Out.
__global__ void __launch_bounds__(256) k_gemm_simt(const float *__restrict__ A, const float *__restrict__ B,
                                                   int64_t M, int64_t N, int64_t K, int64_t sbn,
                                                   int64_t sbk, float *__restrict__ Out) {
    __shared__ float As[BK][BM + 4];
    __shared__ float Bs[BK][BN + 4];
    const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
    const int64_t m0 = (int64_t)blockIdx.x * BM, n0 = (int64_t)blockIdx.y * BN;
    float acc[8][4];
#pragma unroll
    for (int i = 0; i < 8; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = 0.f;
    for (int64_t k0 = 0; k0 < K; k0 += BK) {
        for (int e = tid; e < BM * BK; e += 256) {
            int r = e / BK, q = e % BK;
            int64_t gr = m0 + r, gk = k0 + q;
            As[q][r] = (gr < M && gk < K) ? A[gr * K + gk] : 0.f;
        }
        for (int e = tid; e < BN * BK; e += 256) {
            int r = e % BN, q = e / BN;
            int64_t gc = n0 + r, gk = k0 + q;
            Bs[q][r] = (gc < N && gk < K) ? B[gc * sbn + gk * sbk] : 0.f;
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < BK; ++kk) {
            float a[8], b[4];
#pragma unroll
            for (int i = 0; i < 8; ++i) a[i] = As[kk][ty + 16 * i];
#pragma unroll
            for (int j = 0; j < 4; ++j) b[j] = Bs[kk][tx + 16 * j];
#pragma unroll
            for (int i = 0; i < 8; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) acc[i][j] = fmaf(a[i], b[j], acc[i][j]);
        }
        __syncthreads();
    }
#pragma unroll
    for (int i = 0; i < 8; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            int64_t r = m0 + ty + 16 * i, cc = n0 + tx + 16 * j;
            if (r < M && cc < N) Out[r * N + cc] = acc[i][j];
        }
}

int launch_gemm_simt_strided(gbkm_ctx *c, const float *A, const float *B, int64_t M, int64_t N,
                             int64_t K, int64_t sbn, int64_t sbk, float *Out) {
    if (M == 0) return GBKM_OK;
    dim3 grid((unsigned)ceil_div(M, BM), (unsigned)ceil_div(N, BN));
    k_gemm_simt<<<grid, 256, 0, c->stream>>>(A, B, M, N, K, sbn, sbk, Out);
    GBKM_LAUNCHED(c);
    return cuda_check(c, cudaGetLastError(), "gemm_simt launch");
}

// ---------------------------------------------------------------- A5: exact recheck
// Squared distance of row x to center c from direct differences in FP32, summed by the whole warp
// (same value on every lane).  Each lane keeps 4 interleaved accumulators (<= ceil(d/128)
// terms each), combined pairwise, then a 5-level butterfly: the relative error is at most
// (ceil(d/128) + 10) * 2^-24 (about 1e-6 for d = 1024), far inside the 1e-5 near-tie band, so
// the order of two centers is resolved exactly whenever their gap exceeds that band.
__device__ __forceinline__ float warp_direct_d2(const float *__restrict__ x, const float *__restrict__ c,
                                                int64_t d, bool vec) {
    const int lane = threadIdx.x & 31;
    float a0 = 0.f, a1 = 0.f, a2 = 0.f, a3 = 0.f;
    if (vec) {
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
    } else {
        for (int64_t t = lane; t < d; t += 32) {
            const float e = x[t] - c[t];
            a0 = fmaf(e, e, a0);
        }
    }
    float v = (a0 + a1) + (a2 + a3);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// the same distance with the row x already held in registers (d <= 1024, d % 4 == 0, aligned):
// lane l owns float4 columns l, l + 32, ..., and the 8 center loads are issued together
__device__ __forceinline__ float warp_direct_d2_rx(const float4 (&xr)[8], const float *__restrict__ c,
                                                   int64_t nv) {
    const int lane = threadIdx.x & 31;
    const float4 *c4 = reinterpret_cast<const float4 *>(c);
    float4 cv[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) cv[q] = (lane + 32 * q < nv) ? __ldg(c4 + lane + 32 * q) : xr[q];
    float a0 = 0.f, a1 = 0.f, a2 = 0.f, a3 = 0.f;
#pragma unroll
    for (int q = 0; q < 8; ++q) {
        const float e0 = xr[q].x - cv[q].x, e1 = xr[q].y - cv[q].y, e2 = xr[q].z - cv[q].z, e3 = xr[q].w - cv[q].w;
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

// (3 CTAs per SM: 24 warps, each with one flagged row's loads in flight)
__global__ void __launch_bounds__(256, 3) k_recheck(const float *__restrict__ X, int64_t d,
                                                 const float *__restrict__ C, int64_t k,
                                                 const int32_t *__restrict__ list,
                                                 const int32_t *__restrict__ cand,
                                                 const int32_t *__restrict__ count, int64_t n,
                                                 int32_t *__restrict__ labels, float *__restrict__ min_d2,
                                                 int64_t *n_rechecked, int *status, Escalation esc,
                                                 const int32_t *__restrict__ row_map) {
    const int lane = threadIdx.x & 31;
    const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = (gridDim.x * (int64_t)blockDim.x) >> 5;
    const int cnt = *count;
    if (warp == 0 && lane == 0 && n_rechecked) *n_rechecked = cnt;
    for (int64_t f = warp; f < cnt; f += nwarps) {
        const int64_t row = list[f];
        if (row < 0 || row >= n) {
            if (lane == 0) status_raise(status, ST_BOUNDS);
            continue;
        }
        const float *x = X + row * d;
        const bool vec = ((d & 3) == 0) && ((reinterpret_cast<uintptr_t>(X) & 15) == 0) &&
                         ((reinterpret_cast<uintptr_t>(C) & 15) == 0);
        float best = 0.f;
        int arg = -1;
        const int32_t *cf = cand + f * CAND_STRIDE;
        const int nc = cf[0];
        if (esc.list && !(nc > 0 && nc <= CAND_MAX)) {
            // the band is not listed: the row goes to the next precision's pass
            int slot = 0;
            if (lane == 0) slot = atomicAdd(esc.count, 1);
            slot = __shfl_sync(0xffffffffu, slot, 0);
            if (lane == 0) {
                esc.list[slot] = (int32_t)row;
                esc.xne[slot] = esc.xnorm[row];
            }
            float *y = esc.Xe + (int64_t)slot * d;
            for (int64_t t = lane; t < d; t += 32) y[t] = x[t];
            continue;
        }
        const bool cached = vec && d <= 1024;
        float4 xr[8];
        if (cached) {
            const float4 *x4 = reinterpret_cast<const float4 *>(x);
#pragma unroll
            for (int q = 0; q < 8; ++q)
                xr[q] = (lane + 32 * q < d / 4) ? __ldg(x4 + lane + 32 * q) : make_float4(0.f, 0.f, 0.f, 0.f);
        }
        auto dist = [&](int64_t j) -> float {
            return cached ? warp_direct_d2_rx(xr, C + j * d, d / 4) : warp_direct_d2(x, C + j * d, d, vec);
        };
        if (nc > 0 && nc <= CAND_MAX) {
            // the certified band holds these centers (increasing index): compare by (distance, index)
            for (int q = 0; q < nc; ++q) {
                const int j = cf[1 + q];
                if (j < 0 || j >= k) {
                    if (lane == 0) status_raise(status, ST_BOUNDS);
                    continue;
                }
                const float v = dist(j);
                if (arg < 0 || v < best || (v == best && j < arg)) {
                    best = v;
                    arg = j;
                }
            }
        } else {
            for (int64_t j = 0; j < k; ++j) {
                const float v = dist(j);
                if (arg < 0 || v < best) {
                    best = v;
                    arg = (int)j;
                }
            }
        }
        if (lane == 0) {
            const int64_t dst = row_map ? (int64_t)row_map[row] : row;
            labels[dst] = arg;
            if (min_d2) min_d2[dst] = best;
        }
    }
}

int launch_recheck(gbkm_ctx *c, const float *X, int64_t n, int64_t d, const float *C, int64_t k,
                   const AssignOut &o, int64_t *n_rechecked, const Escalation *esc, const int32_t *row_map) {
    unsigned blocks = (unsigned)c->sm_count * 3;
    Escalation e{};
    if (esc) e = *esc;
    k_recheck<<<blocks, 256, 0, c->stream>>>(X, d, C, k, o.flag_list, o.cand, o.flag_count, n, o.labels,
                                             o.min_d2, n_rechecked, c->status, e, row_map);
    GBKM_LAUNCHED(c);
    return cuda_check(c, cudaGetLastError(), "recheck launch");
}

}  // namespace gbkm
