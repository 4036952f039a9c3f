// k_prep.cu -- A1 row norms, A0 operand quantisation, per-call center preparation.
#include "internal.cuh"

namespace gbkm {

// ---------------------------------------------------------------- A1: ||x_i||^2
// One warp per row (grid-stride), 128-bit loads when rows are 16-byte aligned.
__global__ void __launch_bounds__(256) k_row_norms(const float *__restrict__ X, int64_t n,
                                                   int64_t d, float *__restrict__ out) {
    const int lane = threadIdx.x & 31;
    const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = (gridDim.x * (int64_t)blockDim.x) >> 5;
    const bool vec = ((d & 3) == 0) && ((reinterpret_cast<uintptr_t>(X) & 15) == 0);
    for (int64_t i = warp; i < n; i += nwarps) {
        const float *x = X + i * d;
        float s = 0.f;
        if (vec) {
            const float4 *x4 = reinterpret_cast<const float4 *>(x);
            for (int64_t t = lane; t < d / 4; t += 32) {
                float4 v = __ldg(x4 + t);
                s = fmaf(v.x, v.x, s);
                s = fmaf(v.y, v.y, s);
                s = fmaf(v.z, v.z, s);
                s = fmaf(v.w, v.w, s);
            }
        } else {
            for (int64_t t = lane; t < d; t += 32) s = fmaf(x[t], x[t], s);
        }
        s = warp_sum_f(s);
        if (lane == 0) out[i] = s;
    }
}

int launch_row_norms(gbkm_ctx *c, const float *X, int64_t n, int64_t d, float *xnorm) {
    if (n == 0) return GBKM_OK;
    int64_t blocks = ceil_div(n, 8);
    int64_t cap = (int64_t)c->sm_count * 8;
    if (blocks > cap) blocks = cap;
    k_row_norms<<<(unsigned)blocks, 256, 0, c->stream>>>(X, n, d, xnorm);
    GBKM_LAUNCHED(c);
    return cuda_check(c, cudaGetLastError(), "row_norms launch");
}

// ---------------------------------------------------------------- A0: bf16 copy
__global__ void __launch_bounds__(256) k_to_bf16(const float *__restrict__ X, int64_t m,
                                                 __nv_bfloat16 *__restrict__ out) {
    const int64_t tid = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const int64_t nth = gridDim.x * (int64_t)blockDim.x;
    const bool vec = ((reinterpret_cast<uintptr_t>(X) & 15) == 0) &&
                     ((reinterpret_cast<uintptr_t>(out) & 15) == 0);
    int64_t m8 = vec ? m / 8 : 0;
    for (int64_t g = tid; g < m8; g += nth) {
        const float4 *src = reinterpret_cast<const float4 *>(X) + 2 * g;
        float4 a = __ldg(src), b = __ldg(src + 1);
        __nv_bfloat162 p0 = __floats2bfloat162_rn(a.x, a.y);
        __nv_bfloat162 p1 = __floats2bfloat162_rn(a.z, a.w);
        __nv_bfloat162 p2 = __floats2bfloat162_rn(b.x, b.y);
        __nv_bfloat162 p3 = __floats2bfloat162_rn(b.z, b.w);
        uint4 o;
        o.x = *reinterpret_cast<uint32_t *>(&p0);
        o.y = *reinterpret_cast<uint32_t *>(&p1);
        o.z = *reinterpret_cast<uint32_t *>(&p2);
        o.w = *reinterpret_cast<uint32_t *>(&p3);
        reinterpret_cast<uint4 *>(out)[g] = o;
    }
    for (int64_t e = m8 * 8 + tid; e < m; e += nth) out[e] = __float2bfloat16_rn(X[e]);
}

// The same copy, one warp per row, with the row's rounding residual ||x - bf16(x)||: the residual
// of each element is exact in FP32 (x and its rounding are within a factor of two), its square and
// the row sum round up to (d + 4) 2^-23 relative at most, which the stored bound covers.
__global__ void __launch_bounds__(256) k_to_bf16_rows(const float *__restrict__ X, int64_t n, int64_t d,
                                                      __nv_bfloat16 *__restrict__ out, float *__restrict__ resid) {
    const int lane = threadIdx.x & 31;
    const int64_t row = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    if (row >= n) return;
    const float *x = X + row * d;
    __nv_bfloat16 *o = out + row * d;
    float s = 0.f;
    const bool vec = (d % 4) == 0 && ((reinterpret_cast<uintptr_t>(X) & 15) == 0) &&
                     ((reinterpret_cast<uintptr_t>(out) & 7) == 0);
    if (vec) {
        for (int64_t t = lane; t < d / 4; t += 32) {
            const float4 v = __ldg(reinterpret_cast<const float4 *>(x) + t);
            const __nv_bfloat162 h0 = __floats2bfloat162_rn(v.x, v.y), h1 = __floats2bfloat162_rn(v.z, v.w);
            uint2 w;
            w.x = *reinterpret_cast<const uint32_t *>(&h0);
            w.y = *reinterpret_cast<const uint32_t *>(&h1);
            reinterpret_cast<uint2 *>(o)[t] = w;
            const float2 f0 = __bfloat1622float2(h0), f1 = __bfloat1622float2(h1);
            const float e0 = v.x - f0.x, e1 = v.y - f0.y, e2 = v.z - f1.x, e3 = v.w - f1.y;
            s = fmaf(e0, e0, s);
            s = fmaf(e1, e1, s);
            s = fmaf(e2, e2, s);
            s = fmaf(e3, e3, s);
        }
    } else {
        for (int64_t t = lane; t < d; t += 32) {
            const float v = x[t];
            const __nv_bfloat16 h = __float2bfloat16_rn(v);
            o[t] = h;
            const float e = v - __bfloat162float(h);
            s = fmaf(e, e, s);
        }
    }
#pragma unroll
    for (int w = 16; w > 0; w >>= 1) s += __shfl_xor_sync(0xffffffffu, s, w);
    if (lane == 0) resid[row] = sqrtf(s * (1.f + (float)(d + 4) * 1.1920929e-7f)) * (1.f + 2.4e-7f);
}

// ---------------------------------------------------------------- A0 + A1 in one pass
// One warp per row of a source that may sit in page-locked host memory mapped into the device's
// address space: the row is copied to HBM and its squared norm, BF16 copy and BF16 rounding
// residual are formed from the same registers, so the source is read once.  Each lane issues up
// to 8 four-float loads before it uses any, keeping a row's bytes in flight together across the
// long-latency CPU-GPU link.  With d % 4 == 0 lane l takes the element groups 4t..4t+3 for
// t = l, l + 32, ... (as k_row_norms and k_to_bf16_rows do on aligned rows), otherwise the
// elements t = l, l + 32, ...: the sums are formed in the same order as those kernels', so the
// results are bitwise theirs.
__device__ __forceinline__ float4 ld_row4(const float *x, int64_t t, bool vload) {
    if (vload) return __ldg(reinterpret_cast<const float4 *>(x) + t);
    return make_float4(__ldg(x + 4 * t), __ldg(x + 4 * t + 1), __ldg(x + 4 * t + 2), __ldg(x + 4 * t + 3));
}

__global__ void __launch_bounds__(256) k_ingest(const float *__restrict__ src, int64_t n, int64_t d,
                                                float *__restrict__ xdev, float *__restrict__ xnorm,
                                                __nv_bfloat16 *__restrict__ xq, float *__restrict__ resid) {
    const int lane = threadIdx.x & 31;
    const int64_t row = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    if (row >= n) return;
    const float *x = src + row * d;
    float s = 0.f, r = 0.f;
    if ((d & 3) == 0) {
        const bool vload = (reinterpret_cast<uintptr_t>(src) & 15) == 0;
        const bool vstore = (reinterpret_cast<uintptr_t>(xdev) & 15) == 0;
        const int64_t q = d / 4;
        float *xo = xdev ? xdev + row * d : nullptr;
        __nv_bfloat16 *qo = xq ? xq + row * d : nullptr;
        for (int64_t base = 0; base < q; base += 256) {
            float4 v[8];
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                const int64_t t = base + u * 32 + lane;
                if (t < q) v[u] = ld_row4(x, t, vload);
            }
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                const int64_t t = base + u * 32 + lane;
                if (t >= q) break;
                if (xo) {
                    if (vstore) {
                        reinterpret_cast<float4 *>(xo)[t] = v[u];
                    } else {
                        xo[4 * t] = v[u].x, xo[4 * t + 1] = v[u].y, xo[4 * t + 2] = v[u].z, xo[4 * t + 3] = v[u].w;
                    }
                }
                s = fmaf(v[u].x, v[u].x, s);
                s = fmaf(v[u].y, v[u].y, s);
                s = fmaf(v[u].z, v[u].z, s);
                s = fmaf(v[u].w, v[u].w, s);
                if (qo) {
                    const __nv_bfloat162 h0 = __floats2bfloat162_rn(v[u].x, v[u].y);
                    const __nv_bfloat162 h1 = __floats2bfloat162_rn(v[u].z, v[u].w);
                    uint2 w;
                    w.x = *reinterpret_cast<const uint32_t *>(&h0);
                    w.y = *reinterpret_cast<const uint32_t *>(&h1);
                    reinterpret_cast<uint2 *>(qo)[t] = w;
                    const float2 f0 = __bfloat1622float2(h0), f1 = __bfloat1622float2(h1);
                    const float e0 = v[u].x - f0.x, e1 = v[u].y - f0.y, e2 = v[u].z - f1.x, e3 = v[u].w - f1.y;
                    r = fmaf(e0, e0, r);
                    r = fmaf(e1, e1, r);
                    r = fmaf(e2, e2, r);
                    r = fmaf(e3, e3, r);
                }
            }
        }
    } else {
        for (int64_t t = lane; t < d; t += 32) {
            const float v = __ldg(x + t);
            if (xdev) xdev[row * d + t] = v;
            s = fmaf(v, v, s);
            if (xq) {
                const __nv_bfloat16 h = __float2bfloat16_rn(v);
                xq[row * d + t] = h;
                const float e = v - __bfloat162float(h);
                r = fmaf(e, e, r);
            }
        }
    }
    s = warp_sum_f(s);
    r = warp_sum_f(r);
    if (lane == 0) {
        if (xnorm) xnorm[row] = s;
        if (resid) resid[row] = sqrtf(r * (1.f + (float)(d + 4) * 1.1920929e-7f)) * (1.f + 2.4e-7f);
    }
}

int launch_ingest(gbkm_ctx *c, const float *src, int64_t n, int64_t d, float *xdev, float *xnorm, void *xq,
                  float *resid) {
    if (n == 0) return GBKM_OK;
    k_ingest<<<(unsigned)ceil_div(n, 8), 256, 0, c->stream>>>(src, n, d, xdev, xnorm, (__nv_bfloat16 *)xq,
                                                              resid);
    GBKM_LAUNCHED(c);
    return cuda_check(c, cudaGetLastError(), "ingest launch");
}

// smallest e with amax * 2^-e <= 448 (e = 0 when amax == 0)
__device__ __forceinline__ int e4m3_scale_exp(float amax) {
    if (!(amax > 0.f)) return 0;
    int e = ilogbf(amax) - 9;
    while (!(ldexpf(amax, -e) <= 448.f)) ++e;
    return e;
}

// ---------------------------------------------------------------- A0: E4M3 copy, one scale per
// 128-element row block.  One warp per (row, block).
__global__ void __launch_bounds__(256) k_to_e4m3(const float *__restrict__ X, int64_t n, int64_t d,
                                                 uint8_t *__restrict__ out, float *__restrict__ scales) {
    const int lane = threadIdx.x & 31;
    const int64_t nb = (d + 127) / 128;
    const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = (gridDim.x * (int64_t)blockDim.x) >> 5;
    for (int64_t wb = warp; wb < n * nb; wb += nwarps) {
        const int64_t i = wb / nb, b = wb % nb;
        const int64_t t0 = b * 128;
        float v[4];
        float amax = 0.f;
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            int64_t t = t0 + lane * 4 + q;
            v[q] = (t < d) ? X[i * d + t] : 0.f;
            amax = fmaxf(amax, fabsf(v[q]));
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) amax = fmaxf(amax, __shfl_xor_sync(0xffffffffu, amax, o));
        const int e = e4m3_scale_exp(amax);
        if (lane == 0) scales[i * nb + b] = ldexpf(1.f, e);
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            int64_t t = t0 + lane * 4 + q;
            if (t < d)
                out[i * d + t] = (uint8_t)__nv_cvt_float_to_fp8(ldexpf(v[q], -e), __NV_SATFINITE, __NV_E4M3);
        }
    }
}

int launch_quantize(gbkm_ctx *c, const float *X, int64_t n, int64_t d, int dtype, void *Xq,
                    float *scales) {
    if (n == 0) return GBKM_OK;
    int64_t cap = (int64_t)c->sm_count * 8;
    if (dtype == GBKM_BF16 && scales) {
        // with the per-row rounding residuals (the assignment's tighter certified band)
        k_to_bf16_rows<<<(unsigned)ceil_div(n, 8), 256, 0, c->stream>>>(X, n, d, (__nv_bfloat16 *)Xq, scales);
    } else if (dtype == GBKM_BF16) {
        int64_t blocks = ceil_div(n * d, 256 * 8);
        if (blocks > cap) blocks = cap;
        k_to_bf16<<<(unsigned)blocks, 256, 0, c->stream>>>(X, n * d, (__nv_bfloat16 *)Xq);
    } else {
        int64_t blocks = ceil_div(n * ceil_div(d, 128), 8);
        if (blocks > cap) blocks = cap;
        k_to_e4m3<<<(unsigned)blocks, 256, 0, c->stream>>>(X, n, d, (uint8_t *)Xq, scales);
    }
    GBKM_LAUNCHED(c);
    return cuda_check(c, cudaGetLastError(), "quantize launch");
}

// ---------------------------------------------------------------- center preparation
// One CTA per (padded) center row: ||c_j||^2 from error-free FP32 sums (stored FP32),
// max_j ||c_j|| (rounded up) as float bits, and the operand copy of the row in the
// GEMM's format.  Rows k..k_pad-1 are zero operands with ||c||^2 = +inf so they never win.
__global__ void __launch_bounds__(256) k_center_prep(const float *__restrict__ C, int64_t k,
                                                     int64_t d, int dtype, CenterPrep cp) {
    const int64_t j = blockIdx.x;
    __shared__ double red[8];
    __shared__ float amax_s[8];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (j >= k) {
        for (int64_t t = threadIdx.x; t < d; t += blockDim.x) {
            if (dtype == GBKM_BF16 && cp.cop) ((__nv_bfloat16 *)cp.cop)[j * d + t] = __float2bfloat16_rn(0.f);
            if (dtype == GBKM_BF16 && cp.cop_lo) ((__nv_bfloat16 *)cp.cop_lo)[j * d + t] = __float2bfloat16_rn(0.f);
            if (dtype == GBKM_FP8E4M3 && cp.cop) ((uint8_t *)cp.cop)[j * d + t] = 0;
            if (dtype == GBKM_F32 && cp.cop) {
                ((float *)cp.cop)[j * d + t] = 0.f;
                ((float *)cp.cop_lo)[j * d + t] = 0.f;
            }
            if (cp.esc_hi) {
                cp.esc_hi[j * d + t] = 0.f;
                cp.esc_lo[j * d + t] = 0.f;
            }
        }
        if (threadIdx.x == 0) {
            cp.cnorm[j] = __int_as_float(0x7f800000);
            if (cp.cscale) cp.cscale[j] = 1.f;
        }
        return;
    }
    const float *c = C + j * d;
    DF acc;
    float amax = 0.f, res = 0.f;  // res: sum of the squared BF16 rounding residuals (one-term BF16)
    for (int64_t t = threadIdx.x; t < d; t += blockDim.x) {
        float v = c[t];
        acc.add_prod(v, v);
        amax = fmaxf(amax, fabsf(v));
        if (cp.emax) {
            const float e = v - __bfloat162float(__float2bfloat16_rn(v));
            res = fmaf(e, e, res);
        }
    }
    double s = warp_sum_d(acc.value());
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        amax = fmaxf(amax, __shfl_xor_sync(0xffffffffu, amax, o));
        res += __shfl_xor_sync(0xffffffffu, res, o);
    }
    __shared__ float res_s[8];
    if (lane == 0) {
        red[wid] = s;
        amax_s[wid] = amax;
        res_s[wid] = res;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double tot = 0.0;
        float am = 0.f, rs = 0.f;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
            tot += red[w];
            am = fmaxf(am, amax_s[w]);
            rs += res_s[w];
        }
        cp.cnorm[j] = (float)tot;
        float nrm = (float)sqrt(tot) * (1.f + 1.0e-6f);
        atomicMax(cp.cmax, __float_as_uint(nrm));
        // ||c_j - bf16(c_j)|| rounded up: each residual is exact, its square and the sums round to
        // (d + 4) 2^-23 relative at most
        if (cp.emax)
            atomicMax(cp.emax, __float_as_uint(sqrtf(rs * (1.f + (float)(d + 4) * 1.1920929e-7f)) * (1.f + 2.4e-7f)));
        amax_s[0] = am;
    }
    __syncthreads();
    if (cp.esc_hi) {
        // the 3xTF32 split as well, for rows escalated from a low-precision form
        for (int64_t t = threadIdx.x; t < d; t += blockDim.x) {
            const float v = c[t];
            const float hi = __uint_as_float(__float_as_uint(v) & 0xffffe000u);
            cp.esc_hi[j * d + t] = hi;
            cp.esc_lo[j * d + t] = __uint_as_float(__float_as_uint(__fsub_rn(v, hi)) & 0xffffe000u);
        }
    }
    if (!cp.cop) return;
    if (dtype == GBKM_BF16) {
        // with a low part: c = hi + lo + O(2^-16 |c|), hi = bf16(c), lo = bf16(c - hi)
        for (int64_t t = threadIdx.x; t < d; t += blockDim.x) {
            const __nv_bfloat16 hi = __float2bfloat16_rn(c[t]);
            ((__nv_bfloat16 *)cp.cop)[j * d + t] = hi;
            if (cp.cop_lo)
                ((__nv_bfloat16 *)cp.cop_lo)[j * d + t] = __float2bfloat16_rn(__fsub_rn(c[t], __bfloat162float(hi)));
        }
    } else if (dtype == GBKM_FP8E4M3) {
        const int e = e4m3_scale_exp(amax_s[0]);
        if (threadIdx.x == 0) cp.cscale[j] = ldexpf(1.f, e);
        for (int64_t t = threadIdx.x; t < d; t += blockDim.x)
            ((uint8_t *)cp.cop)[j * d + t] =
                (uint8_t)__nv_cvt_float_to_fp8(ldexpf(c[t], -e), __NV_SATFINITE, __NV_E4M3);
    } else {
        // 3xTF32 split: hi = c truncated to TF32 (19 bits), lo = (c - hi) truncated to TF32
        for (int64_t t = threadIdx.x; t < d; t += blockDim.x) {
            float v = c[t];
            float hi = __uint_as_float(__float_as_uint(v) & 0xffffe000u);
            float lo = __uint_as_float(__float_as_uint(__fsub_rn(v, hi)) & 0xffffe000u);
            ((float *)cp.cop)[j * d + t] = hi;
            ((float *)cp.cop_lo)[j * d + t] = lo;
        }
    }
}

int launch_center_prep(gbkm_ctx *c, const float *C, int64_t k, int64_t d, int dtype,
                       int64_t k_pad, const CenterPrep &cp) {
    k_center_prep<<<(unsigned)k_pad, 256, 0, c->stream>>>(C, k, d, dtype, cp);
    GBKM_LAUNCHED(c);
    return cuda_check(c, cudaGetLastError(), "center_prep launch");
}

}  // namespace gbkm
