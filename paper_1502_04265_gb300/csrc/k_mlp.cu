// k_mlp.cu -- A9: learned candidate proposal (no paper counterpart).
//
// An MLP d -> h -> h -> k (GELU) maps a point to logits over the k centers; its top-m logits are
// the candidates.  Exact FP32 distances to the candidates give the best candidate b, which is
// accepted when ||x - c_b|| < s(c_b) = half the distance from c_b to its nearest other center
// (then every other center is strictly farther: ||x - c'|| >= ||c_b - c'|| - ||x - c_b|| >
// 2 s - s = s > ||x - c_b||); other points fall back to the full distance scan.  Labels are
// therefore those of the exact method; the network only decides how much work is skipped.
// Training runs on the GPU: tcgen05 GEMMs (k_tc.cu) for every matrix product of the forward and
// backward passes, and the small kernels below (softmax cross-entropy gradient, GELU backward,
// bias gradients, transposes, AdamW).
#include <math.h>

#include "internal.cuh"

namespace gbkm {

namespace {
// d/dx of 0.5 x (1 + erf(x / sqrt 2)) = Phi(x) + x phi(x)
__device__ __forceinline__ float gelu_grad(float x) {
    const float Phi = 0.5f * (1.f + erff(x * 0.70710678118654752f));
    const float phi = 0.39894228040143268f * expf(-0.5f * x * x);
    return Phi + x * phi;
}
}  // namespace

// out[c][r] = in[r][c] for an R x C BF16 matrix (32 x 32 tiles through shared memory)
__global__ void __launch_bounds__(256) k_transpose_bf16(const __nv_bfloat16 *__restrict__ in, int64_t R, int64_t C,
                                                        __nv_bfloat16 *__restrict__ out) {
    __shared__ __nv_bfloat16 tile[32][34];
    const int64_t r0 = (int64_t)blockIdx.y * 32, c0 = (int64_t)blockIdx.x * 32;
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
    for (int i = ty; i < 32; i += 8) {
        const int64_t r = r0 + i, c = c0 + tx;
        tile[i][tx] = (r < R && c < C) ? in[r * C + c] : __float2bfloat16_rn(0.f);
    }
    __syncthreads();
    for (int i = ty; i < 32; i += 8) {
        const int64_t c = c0 + i, r = r0 + tx;
        if (c < C && r < R) out[c * R + r] = tile[tx][i];
    }
}

__global__ void k_cast_bf16(const float *__restrict__ in, int64_t m, __nv_bfloat16 *__restrict__ out) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < m) out[i] = __float2bfloat16_rn(in[i]);
}

// one CTA per row of B x K logits: loss_i = log sum exp - logit[label]; grad = (softmax - onehot) / B
// written in BF16 (the backward GEMM operand)
__global__ void __launch_bounds__(256) k_softmax_xent(const float *__restrict__ logits, const int32_t *__restrict__ labels,
                                                      int64_t K, float inv_b, __nv_bfloat16 *__restrict__ grad,
                                                      float *__restrict__ loss) {
    __shared__ float red[8];
    const int64_t i = blockIdx.x;
    const float *z = logits + i * K;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    float mx = -__int_as_float(0x7f800000);
    for (int64_t j = threadIdx.x; j < K; j += 256) mx = fmaxf(mx, z[j]);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    if (lane == 0) red[w] = mx;
    __syncthreads();
    mx = red[0];
    for (int q = 1; q < 8; ++q) mx = fmaxf(mx, red[q]);
    __syncthreads();
    float se = 0.f;
    for (int64_t j = threadIdx.x; j < K; j += 256) se += expf(z[j] - mx);
    se = warp_sum_f(se);
    if (lane == 0) red[w] = se;
    __syncthreads();
    se = 0.f;
    for (int q = 0; q < 8; ++q) se += red[q];
    const int32_t y = labels[i];
    const float inv = 1.f / se;
    for (int64_t j = threadIdx.x; j < K; j += 256) {
        const float p = expf(z[j] - mx) * inv;
        grad[i * K + j] = __float2bfloat16_rn((p - (j == y ? 1.f : 0.f)) * inv_b);
    }
    if (threadIdx.x == 0) loss[i] = logf(se) + mx - z[y];
}

// dpre = dh * GELU'(pre), BF16 out
__global__ void k_gelu_bwd(const float *__restrict__ dh, const float *__restrict__ pre, int64_t m,
                           __nv_bfloat16 *__restrict__ out) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < m) out[i] = __float2bfloat16_rn(dh[i] * gelu_grad(pre[i]));
}

// bias gradient: column sums of an R x C BF16 matrix, FP32, one thread per column (rows in order)
__global__ void k_colsum_bf16(const __nv_bfloat16 *__restrict__ g, int64_t R, int64_t C, float *__restrict__ out) {
    const int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (c >= C) return;
    float s = 0.f;
    for (int64_t r = 0; r < R; ++r) s += __bfloat162float(g[r * C + c]);
    out[c] = s;
}

// AdamW on FP32 master parameters; decoupled weight decay where wdmask is 1 (weights, not biases);
// refreshes the BF16 copy used by the GEMMs
__global__ void k_adamw(float *__restrict__ p, const float *__restrict__ g, float *__restrict__ m, float *__restrict__ v,
                        const uint8_t *__restrict__ wdmask, int64_t n, float lr, float b1, float b2, float eps,
                        float wd, float c1, float c2, __nv_bfloat16 *__restrict__ ph) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.f - b1) * gi;
    const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    float pi = p[i];
    if (wdmask[i]) pi -= lr * wd * pi;
    pi -= lr * (mi * c1) / (sqrtf(vi * c2) + eps);
    p[i] = pi;
    ph[i] = __float2bfloat16_rn(pi);
}

// s2[j] = (1/4) min_{i != j} ||c_j - c_i||^2 (direct FP32 differences), one warp per center;
// the square of the acceptance radius of the certificate
__global__ void __launch_bounds__(256) k_center_sep(const float *__restrict__ C, int64_t k, int64_t d,
                                                    float *__restrict__ s2) {
    const int lane = threadIdx.x & 31;
    const int64_t j = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    if (j >= k) return;
    const float *cj = C + j * d;
    float best = __int_as_float(0x7f800000);
    for (int64_t i = 0; i < k; ++i) {
        if (i == j) continue;
        const float *ci = C + i * d;
        float a = 0.f;
        for (int64_t t = lane; t < d; t += 32) {
            const float e = cj[t] - ci[t];
            a = fmaf(e, e, a);
        }
        a = warp_sum_f(a);
        best = fminf(best, a);
    }
    if (lane == 0) s2[j] = 0.25f * best;
}

// one warp per point (four candidates at a time, the row held in registers, when d is a multiple of
// 128 up to 1,024): exact FP32 distances to its candidates in rank order until one, b, satisfies
// d(x, c_b) < s2[b] = min_c ||c_b - c||^2 / 4 certifiably (relative margins of 1e-5 cover the FP32
// rounding of both sides): then c_b is the unique nearest center of all k (Elkan's bound), so the
// first such candidate is the label and the rest need no distance; a point without one goes to the
// fallback list
__global__ void __launch_bounds__(256) k_cand_check(const float *__restrict__ X, int64_t n, int64_t d,
                                                    const float *__restrict__ C, int64_t k,
                                                    const int32_t *__restrict__ cand, int m,
                                                    const float *__restrict__ s2, int32_t *__restrict__ labels,
                                                    int32_t *__restrict__ fb_list, int32_t *__restrict__ fb_count) {
    const int lane = threadIdx.x & 31;
    const int64_t i = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    if (i >= n) return;
    const float *x = X + i * d;
    int arg = -1;
    const bool v4 = (d % 128) == 0 && d <= 1024 && ((reinterpret_cast<uintptr_t>(X) & 15) == 0) &&
                    ((reinterpret_cast<uintptr_t>(C) & 15) == 0);
    if (v4) {
        // the row in registers (d / 128 float4 per lane) and four candidates' rows in flight at a
        // time; the first of them in rank order that certifies is taken
        const int nv = (int)(d / 128);
        float4 xr[8];
#pragma unroll
        for (int v = 0; v < 8; ++v)
            xr[v] = v < nv ? __ldg(reinterpret_cast<const float4 *>(x) + v * 32 + lane) : make_float4(0.f, 0.f, 0.f, 0.f);
        for (int q0 = 0; q0 < m && arg < 0; q0 += 4) {
            int js[4];
            float acc[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const int j = q0 + u < m ? cand[i * m + q0 + u] : -1;
                js[u] = (j >= 0 && j < k) ? j : -1;
                acc[u] = 0.f;
            }
#pragma unroll
            for (int v = 0; v < 8; ++v) {
                if (v >= nv) break;
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    if (js[u] < 0) continue;
                    const float4 c4 = __ldg(reinterpret_cast<const float4 *>(C + (int64_t)js[u] * d) + v * 32 + lane);
                    const float e0 = xr[v].x - c4.x, e1 = xr[v].y - c4.y, e2 = xr[v].z - c4.z, e3 = xr[v].w - c4.w;
                    acc[u] = fmaf(e0, e0, fmaf(e1, e1, fmaf(e2, e2, fmaf(e3, e3, acc[u]))));
                }
            }
#pragma unroll
            for (int u = 0; u < 4; ++u) acc[u] = warp_sum_f(acc[u]);
#pragma unroll
            for (int u = 0; u < 4; ++u)
                if (arg < 0 && js[u] >= 0 && acc[u] * (1.f + 1e-5f) < s2[js[u]] * (1.f - 1e-5f)) arg = js[u];
        }
    } else {
        for (int q = 0; q < m && arg < 0; ++q) {
            const int j = cand[i * m + q];
            if (j < 0 || j >= k) continue;
            const float *c = C + (int64_t)j * d;
            float a = 0.f;
            for (int64_t t = lane; t < d; t += 32) {
                const float e = x[t] - c[t];
                a = fmaf(e, e, a);
            }
            a = warp_sum_f(a);
            if (a * (1.f + 1e-5f) < s2[j] * (1.f - 1e-5f)) arg = j;
        }
    }
    if (lane == 0) {
        if (arg >= 0) {
            labels[i] = arg;
        } else {
            const int slot = atomicAdd(fb_count, 1);
            fb_list[slot] = (int32_t)i;
        }
    }
}

// gather the fallback rows (list, count on the device) into a contiguous block; rows past the
// count are left untouched
// gathers the listed rows of X (FP32) and of its BF16 copy Xh into compact row-major blocks, with
// each row's rounding residual ||x - xh|| rounded up (the assignment's narrower certified band;
// the residuals are exact in FP32, their squares and sums round to (d + 4) 2^-23 relative at most)
__global__ void __launch_bounds__(128) k_gather_rows(const float *__restrict__ X, const __nv_bfloat16 *__restrict__ Xh,
                                                     int64_t d, const int32_t *__restrict__ list,
                                                     const int32_t *__restrict__ count, float *__restrict__ out,
                                                     __nv_bfloat16 *__restrict__ outh, float *__restrict__ resid) {
    __shared__ float part[4];
    const int64_t r = blockIdx.x;
    if (r >= *count) return;
    const int64_t src = list[r];
    float s = 0.f;
    for (int64_t t = threadIdx.x; t < d; t += blockDim.x) {
        const float v = X[src * d + t];
        const __nv_bfloat16 h = Xh[src * d + t];
        out[r * d + t] = v;
        outh[r * d + t] = h;
        const float e = v - __bfloat162float(h);
        s = fmaf(e, e, s);
    }
#pragma unroll
    for (int w = 16; w > 0; w >>= 1) s += __shfl_xor_sync(0xffffffffu, s, w);
    if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0)
        resid[r] = sqrtf((part[0] + part[1] + part[2] + part[3]) * (1.f + (float)(d + 4) * 1.1920929e-7f)) *
                   (1.f + 2.4e-7f);
}

__global__ void k_scatter_labels(const int32_t *__restrict__ sub, const int32_t *__restrict__ list,
                                 const int32_t *__restrict__ count, int32_t *__restrict__ labels) {
    const int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (r < *count) labels[list[r]] = sub[r];
}

// ---------------------------------------------------------------- host side
namespace {
struct MlpLayout {
    int64_t oW1, ob1, oW2, ob2, oW3, ob3, total;
};
MlpLayout mlp_layout(const gbkm_mlp &m) {
    MlpLayout L;
    L.oW1 = 0;
    L.ob1 = L.oW1 + m.hidden * m.d_in;
    L.oW2 = L.ob1 + m.hidden;
    L.ob2 = L.oW2 + m.hidden * m.hidden;
    L.oW3 = L.ob2 + m.hidden;
    L.ob3 = L.oW3 + m.k * m.hidden;
    L.total = L.ob3 + m.k;
    return L;
}
bool mlp_ok(const gbkm_mlp *m) {
    return m && m->params && m->params_bf16 && m->d_in >= 8 && m->d_in % 16 == 0 && m->hidden >= 16 &&
           m->hidden % 16 == 0 && m->k >= 16 && m->k % 16 == 0;
}
}  // namespace

int64_t mlp_param_count(const gbkm_mlp *m) { return mlp_layout(*m).total; }

// forward through the two hidden layers; returns H2 (BF16, n x h) in ws
static int mlp_hidden(gbkm_ctx *c, const gbkm_mlp *m, const void *Xh, int64_t n, __nv_bfloat16 *H1, __nv_bfloat16 *H2,
                      float *H1pre, float *H2pre) {
    const MlpLayout L = mlp_layout(*m);
    const __nv_bfloat16 *Wh = static_cast<const __nv_bfloat16 *>(m->params_bf16);
    int rc = launch_gemm_bf16_tc(c, Xh, Wh + L.oW1, n, m->hidden, m->d_in, m->params + L.ob1, 1, 1, H1, m->hidden,
                                 H1pre, m->hidden, nullptr, nullptr, 0);
    if (rc != GBKM_OK) return rc;
    return launch_gemm_bf16_tc(c, H1, Wh + L.oW2, n, m->hidden, m->hidden, m->params + L.ob2, 1, 1, H2, m->hidden,
                               H2pre, m->hidden, nullptr, nullptr, 0);
}

int mlp_forward(gbkm_ctx *c, const gbkm_mlp *m, const void *Xh, int64_t n, float *logits, int32_t *top_idx, int topm,
                int group) {
    if (!mlp_ok(m) || n < 1 || !Xh || (!logits && !top_idx)) return set_error(c, GBKM_EINVAL, "mlp_forward: bad arguments");
    const MlpLayout L = mlp_layout(*m);
    WsPlan p;
    const size_t oH1 = p.take<__nv_bfloat16>(n * m->hidden), oH2 = p.take<__nv_bfloat16>(n * m->hidden);
    int rc = GBKM_OK;
    void *ws = ws_reserve(c, p.off, &rc);
    if (!ws) return rc;
    __nv_bfloat16 *H1 = ws_at<__nv_bfloat16>(ws, oH1), *H2 = ws_at<__nv_bfloat16>(ws, oH2);
    prof_begin(c, "mlp_hidden");
    rc = mlp_hidden(c, m, Xh, n, H1, H2, nullptr, nullptr);
    prof_end(c);
    if (rc != GBKM_OK) return rc;
    const __nv_bfloat16 *Wh = static_cast<const __nv_bfloat16 *>(m->params_bf16);
    if (logits) {
        prof_begin(c, "mlp_logits");
        rc = launch_gemm_bf16_tc(c, H2, Wh + L.oW3, n, m->k, m->hidden, m->params + L.ob3, 0, 0, logits, m->k, nullptr,
                                 0, nullptr, nullptr, 0);
        prof_end(c);
        if (rc != GBKM_OK) return rc;
    }
    if (top_idx) {
        prof_begin(c, "mlp_topm");
        rc = launch_gemm_bf16_tc(c, H2, Wh + L.oW3, n, m->k, m->hidden, m->params + L.ob3, 0, 0, nullptr, 0, nullptr, 0,
                                 top_idx, nullptr, topm, group);
        prof_end(c);
    }
    return rc;
}

static void transpose(gbkm_ctx *c, const __nv_bfloat16 *in, int64_t R, int64_t C, __nv_bfloat16 *out) {
    dim3 grid((unsigned)ceil_div(C, 32), (unsigned)ceil_div(R, 32));
    k_transpose_bf16<<<grid, 256, 0, c->stream>>>(in, R, C, out);
    GBKM_LAUNCHED(c);
}

int mlp_train_step(gbkm_ctx *c, gbkm_mlp *m, const void *Xh, const int32_t *labels, int64_t B, float lr, float wd,
                   float *loss_rows, float *grad_out) {
    if (!mlp_ok(m) || !m->adam_m || !m->adam_v || !m->wd_mask || B < 1 || B % 8 || !Xh || !labels)
        return set_error(c, GBKM_EINVAL, "mlp_train_step: bad arguments (B must be a multiple of 8)");
    const MlpLayout L = mlp_layout(*m);
    const int64_t d = m->d_in, h = m->hidden, K = m->k;
    WsPlan p;
    const size_t oH1 = p.take<__nv_bfloat16>(B * h), oH2 = p.take<__nv_bfloat16>(B * h), oH1p = p.take<float>(B * h),
                 oH2p = p.take<float>(B * h), oZ = p.take<float>(B * K), oG = p.take<__nv_bfloat16>(B * K),
                 oGT = p.take<__nv_bfloat16>(K * B), oH2T = p.take<__nv_bfloat16>(h * B),
                 oW3T = p.take<__nv_bfloat16>(h * K), odH2 = p.take<float>(B * h),
                 odH2p = p.take<__nv_bfloat16>(B * h), odH2pT = p.take<__nv_bfloat16>(h * B),
                 oH1T = p.take<__nv_bfloat16>(h * B), oW2T = p.take<__nv_bfloat16>(h * h), odH1 = p.take<float>(B * h),
                 odH1p = p.take<__nv_bfloat16>(B * h), odH1pT = p.take<__nv_bfloat16>(h * B),
                 oXT = p.take<__nv_bfloat16>(d * B), oGrad = p.take<float>(L.total), oLoss = p.take<float>(B);
    int rc = GBKM_OK;
    void *ws = ws_reserve(c, p.off, &rc);
    if (!ws) return rc;
    auto bf = [&](size_t o) { return ws_at<__nv_bfloat16>(ws, o); };
    auto f32 = [&](size_t o) { return ws_at<float>(ws, o); };
    const __nv_bfloat16 *Wh = static_cast<const __nv_bfloat16 *>(m->params_bf16);
    float *grad = f32(oGrad);
    // forward, keeping the pre-activations
    if ((rc = mlp_hidden(c, m, Xh, B, bf(oH1), bf(oH2), f32(oH1p), f32(oH2p))) != GBKM_OK) return rc;
    if ((rc = launch_gemm_bf16_tc(c, bf(oH2), Wh + L.oW3, B, K, h, m->params + L.ob3, 0, 0, f32(oZ), K, nullptr, 0,
                                  nullptr, nullptr, 0)) != GBKM_OK)
        return rc;
    float *loss = loss_rows ? loss_rows : f32(oLoss);
    k_softmax_xent<<<(unsigned)B, 256, 0, c->stream>>>(f32(oZ), labels, K, 1.f / (float)B, bf(oG), loss);
    GBKM_LAUNCHED(c);
    // layer 3: dW3 = G^T H2, db3 = colsum G, dH2 = G W3
    transpose(c, bf(oG), B, K, bf(oGT));
    transpose(c, bf(oH2), B, h, bf(oH2T));
    transpose(c, Wh + L.oW3, K, h, bf(oW3T));
    if ((rc = launch_gemm_bf16_tc(c, bf(oGT), bf(oH2T), K, h, B, nullptr, 0, 0, grad + L.oW3, h, nullptr, 0, nullptr,
                                  nullptr, 0)) != GBKM_OK)
        return rc;
    k_colsum_bf16<<<(unsigned)ceil_div(K, 256), 256, 0, c->stream>>>(bf(oG), B, K, grad + L.ob3);
    GBKM_LAUNCHED(c);
    if ((rc = launch_gemm_bf16_tc(c, bf(oG), bf(oW3T), B, h, K, nullptr, 0, 0, f32(odH2), h, nullptr, 0, nullptr,
                                  nullptr, 0)) != GBKM_OK)
        return rc;
    // layer 2
    k_gelu_bwd<<<(unsigned)ceil_div(B * h, 256), 256, 0, c->stream>>>(f32(odH2), f32(oH2p), B * h, bf(odH2p));
    GBKM_LAUNCHED(c);
    transpose(c, bf(odH2p), B, h, bf(odH2pT));
    transpose(c, bf(oH1), B, h, bf(oH1T));
    transpose(c, Wh + L.oW2, h, h, bf(oW2T));
    if ((rc = launch_gemm_bf16_tc(c, bf(odH2pT), bf(oH1T), h, h, B, nullptr, 0, 0, grad + L.oW2, h, nullptr, 0, nullptr,
                                  nullptr, 0)) != GBKM_OK)
        return rc;
    k_colsum_bf16<<<(unsigned)ceil_div(h, 256), 256, 0, c->stream>>>(bf(odH2p), B, h, grad + L.ob2);
    GBKM_LAUNCHED(c);
    if ((rc = launch_gemm_bf16_tc(c, bf(odH2p), bf(oW2T), B, h, h, nullptr, 0, 0, f32(odH1), h, nullptr, 0, nullptr,
                                  nullptr, 0)) != GBKM_OK)
        return rc;
    // layer 1
    k_gelu_bwd<<<(unsigned)ceil_div(B * h, 256), 256, 0, c->stream>>>(f32(odH1), f32(oH1p), B * h, bf(odH1p));
    GBKM_LAUNCHED(c);
    transpose(c, bf(odH1p), B, h, bf(odH1pT));
    transpose(c, static_cast<const __nv_bfloat16 *>(Xh), B, d, bf(oXT));
    if ((rc = launch_gemm_bf16_tc(c, bf(odH1pT), bf(oXT), h, d, B, nullptr, 0, 0, grad + L.oW1, d, nullptr, 0, nullptr,
                                  nullptr, 0)) != GBKM_OK)
        return rc;
    k_colsum_bf16<<<(unsigned)ceil_div(h, 256), 256, 0, c->stream>>>(bf(odH1p), B, h, grad + L.ob1);
    GBKM_LAUNCHED(c);
    if (grad_out) {
        cudaError_t e = cudaMemcpyAsync(grad_out, grad, sizeof(float) * L.total, cudaMemcpyDeviceToDevice, c->stream);
        if (e != cudaSuccess) return cuda_check(c, e, "gradient copy");
    }
    // AdamW (beta1 0.9, beta2 0.999, eps 1e-8)
    m->step += 1;
    const float b1 = 0.9f, b2 = 0.999f;
    const float c1 = 1.f / (1.f - powf(b1, (float)m->step)), c2 = 1.f / (1.f - powf(b2, (float)m->step));
    k_adamw<<<(unsigned)ceil_div(L.total, 256), 256, 0, c->stream>>>(m->params, grad, m->adam_m, m->adam_v,
                                                                      m->wd_mask, L.total, lr, b1, b2, 1e-8f, wd, c1, c2,
                                                                      static_cast<__nv_bfloat16 *>(m->params_bf16));
    GBKM_LAUNCHED(c);
    return cuda_check(c, cudaGetLastError(), "mlp train step");
}

int center_separation(gbkm_ctx *c, const float *C, int64_t k, int64_t d, float *s2) {
    k_center_sep<<<(unsigned)ceil_div(k * 32, 256), 256, 0, c->stream>>>(C, k, d, s2);
    GBKM_LAUNCHED(c);
    return cuda_check(c, cudaGetLastError(), "center separation");
}

int learned_assign(gbkm_ctx *c, const gbkm_mlp *m, const float *X, const void *Xh, int64_t n, int64_t d,
                   const float *C, int64_t k, const float *s2, int topm, int32_t *labels, int64_t *n_fallback,
                   int32_t *cand_out) {
    if (!mlp_ok(m) || m->d_in != d || m->k != k || topm < 1 || topm > 32)
        return set_error(c, GBKM_EINVAL, "learned_assign: network shape does not match the problem");
    // private buffers of this call (the forward pass and the fallback scan use the workspace)
    int32_t *cand = cand_out, *fl = nullptr, *fc = nullptr;
    cudaError_t e = cudaSuccess;
    if (!cand) e = cudaMallocAsync(&cand, sizeof(int32_t) * n * topm, c->stream);
    if (e == cudaSuccess) e = cudaMallocAsync(&fl, sizeof(int32_t) * n + 64, c->stream);
    if (e == cudaSuccess) e = cudaMallocAsync(&fc, 64, c->stream);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return set_error(c, GBKM_ENOMEM, "learned_assign: buffer allocation failed");
    }
    int rc = mlp_forward(c, m, Xh, n, nullptr, cand, topm, 16);
    if (rc == GBKM_OK) {
        e = cudaMemsetAsync(fc, 0, 8, c->stream);
        prof_begin(c, "cand_check");
        k_cand_check<<<(unsigned)ceil_div(n * 32, 256), 256, 0, c->stream>>>(X, n, d, C, k, cand, topm, s2, labels, fl, fc);
        prof_end(c);
        GBKM_LAUNCHED(c);
        // the rejected points get the full scan: their count is read back once
        int32_t nf = 0;
        if (e == cudaSuccess) e = cudaMemcpyAsync(&nf, fc, 4, cudaMemcpyDeviceToHost, c->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
        if (e != cudaSuccess) rc = cuda_check(c, e, "fallback count");
        if (rc == GBKM_OK && n_fallback) {
            const int64_t nf64 = nf;
            e = cudaMemcpyAsync(n_fallback, &nf64, 8, cudaMemcpyHostToDevice, c->stream);
            if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
            if (e != cudaSuccess) rc = cuda_check(c, e, "fallback count out");
        }
        if (rc == GBKM_OK && nf > 0) {
            float *sub = nullptr, *subr = nullptr;
            __nv_bfloat16 *subh = nullptr;
            int32_t *subl = nullptr;
            e = cudaMallocAsync(&sub, sizeof(float) * (size_t)nf * d, c->stream);
            if (e == cudaSuccess) e = cudaMallocAsync(&subr, sizeof(float) * (size_t)nf, c->stream);
            if (e == cudaSuccess) e = cudaMallocAsync(&subh, sizeof(__nv_bfloat16) * (size_t)nf * d, c->stream);
            if (e == cudaSuccess) e = cudaMallocAsync(&subl, sizeof(int32_t) * (size_t)nf, c->stream);
            if (e != cudaSuccess) {
                cudaGetLastError();
                rc = set_error(c, GBKM_ENOMEM, "learned_assign: fallback allocation failed");
            } else {
                prof_begin(c, "fallback");
                k_gather_rows<<<(unsigned)nf, 128, 0, c->stream>>>(X, static_cast<const __nv_bfloat16 *>(Xh), d, fl,
                                                                   fc, sub, subh, subr);
                GBKM_LAUNCHED(c);
                // BF16 distance GEMM with the certified near-tie recheck: the same exact labels as the
                // FP32 scan at a fraction of its tensor time
                gbkm_assign_opts o = {GBKM_BF16, GBKM_ENGINE_AUTO, 1, 0};
                rc = kmeans_assign(c, subh, subr, sub, nullptr, nf, d, C, k, &o, subl, nullptr, nullptr);
                if (rc == GBKM_OK) {
                    k_scatter_labels<<<(unsigned)ceil_div(nf, 256), 256, 0, c->stream>>>(subl, fl, fc, labels);
                    GBKM_LAUNCHED(c);
                }
                prof_end(c);
            }
            if (sub) cudaFreeAsync(sub, c->stream);
            if (subr) cudaFreeAsync(subr, c->stream);
            if (subh) cudaFreeAsync(subh, c->stream);
            if (subl) cudaFreeAsync(subl, c->stream);
        }
    }
    if (!cand_out && cand) cudaFreeAsync(cand, c->stream);
    if (fl) cudaFreeAsync(fl, c->stream);
    if (fc) cudaFreeAsync(fc, c->stream);
    if (rc != GBKM_OK) return rc;
    return cuda_check(c, cudaGetLastError(), "learned assign");
}

}  // namespace gbkm
