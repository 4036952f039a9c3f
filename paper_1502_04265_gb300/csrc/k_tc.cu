// k_tc.cu -- tcgen05 engines: the distance GEMM with the fused top-2 argmin epilogue (A4) and the
// block projection GEMM (A2).
//
// One persistent CTA per SM walks a list of units (row tile of 128 points x chunk of <= 256
// centers).  Warp roles:
//   warp 0      TMA producer: X tile (128 rows x 128 B) and center tile (BN rows x 128 B) per
//               K block into a ring of shared-memory stages, 128-byte swizzle
//   warp 1      MMA issuer (one thread): tcgen05.mma into one of two TMEM accumulators
//               (M=128, N=BN, FP32), commits free the stage / publish the accumulator
//   warp 2      allocates / frees TMEM
//   warps 4-7   epilogue: tcgen05.ld of the accumulator (one TMEM lane = one point),
//               score = ||c||^2 - 2 x.c, running top-3 values and top-2 indices per point,
//               certified near-tie flag, or a plain FP32 store for the projection
//   warps 8-11  (3xTF32 only) split the staged FP32 X tile into TF32 hi and lo parts in place
// The two TMEM accumulators let the epilogue of one unit overlap the MMAs of the next.
// Every wait is bounded (%globaltimer); a timeout raises ST_TIMEOUT and the CTA drains and exits.
#include <cuda.h>

#include <algorithm>

#include "internal.cuh"

namespace gbkm {
namespace tc {

constexpr int BM = 128;
constexpr int MAX_STAGES = 8;
constexpr uint64_t WAIT_LIMIT_NS = 2000000000ull;  // 2 s per wait
constexpr int SMEM_BUDGET = 200 * 1024;

enum Form : int { F_BF16 = 0, F_TF32X3 = 1, F_FP8 = 2, F_TF32 = 3 };
enum Epi : int { E_ARGMIN = 0, E_STORE = 1, E_TOPM = 2 };
constexpr int TOPBUF = 64;  // per-row candidate buffer of the top-m epilogue (shared memory)

struct Args {
    int64_t n, d, k, k_pad;
    int n_chunks, bn, kb, stages, tmem_cols, m_tiles;
    uint32_t a_bytes, b_bytes, stage_bytes, tx_bytes;
    uint32_t idesc;
    // argmin epilogue
    const float *cnorm, *cscale, *xscale, *xnorm;
    const unsigned *cmax;
    float err_rel, err_abs;
    int32_t *labels;
    float *min_d2;
    int32_t *flag_list;
    int32_t *cand;
    int32_t *flag_count;
    // store epilogue: Y[row, col] = act(acc + bias[col]) in FP32 or BF16; Ypre = acc + bias (FP32)
    float *Y;
    int64_t ldy;
    const float *bias;
    int act;       // 0: none, 1: GELU (erf form)
    int out_bf16;
    float *Ypre;
    int64_t ldpre;
    // top-m epilogue: the m largest (acc + bias) of every row, over all N chunks
    int32_t *top_idx;
    float *top_val;
    int topm;
    int *status;
};

__device__ __forceinline__ float gelu_erf(float x) { return 0.5f * x * (1.f + erff(x * 0.70710678118654752f)); }

// order-preserving map of floats to unsigned keys
__device__ __forceinline__ uint32_t fkey(float f) {
    const uint32_t u = __float_as_uint(f);
    return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}
__device__ __forceinline__ float fkey_inv(uint32_t k) {
    return __uint_as_float((k & 0x80000000u) ? (k & 0x7fffffffu) : ~k);
}

// the m-th largest key among a thread's cnt buffered candidates (stride 128 in shared memory):
// the largest T with #{key >= T} >= m, found bit by bit from the top
__device__ __forceinline__ uint32_t topm_threshold(const float *bv, int t, int cnt, int m) {
    uint32_t T = 0;
    for (int b = 31; b >= 0; --b) {
        const uint32_t cand = T | (1u << b);
        int c = 0;
        for (int i = 0; i < cnt; ++i) c += fkey(bv[i * 128 + t]) >= cand;
        if (c >= m) T = cand;
    }
    return T;
}

// ---------------------------------------------------------------- PTX helpers
__device__ __forceinline__ uint32_t smem_u32(const void *p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint64_t *bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}
// Bounded wait for the phase of `parity`.  Gives up when the CTA's abort flag is raised, or after
// WAIT_LIMIT_NS, in which case it raises the flag itself.  Returns false when it gave up.
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity, volatile int *abort_flag) {
    if (mbar_try_wait(bar, parity)) return true;
    const uint64_t t0 = globaltimer_ns();
    for (uint32_t it = 1;; ++it) {
        if (mbar_try_wait(bar, parity)) return true;
        if ((it & 63) == 0) {
            if (*abort_flag) return false;
            if (globaltimer_ns() - t0 > WAIT_LIMIT_NS) {
                *abort_flag = 1;
                return false;
            }
        }
    }
}
// drain wait used on the abort path only: bounded, ignores the abort flag
__device__ __forceinline__ void mbar_drain(uint64_t *bar, uint32_t parity, uint64_t limit_ns) {
    const uint64_t t0 = globaltimer_ns();
    while (!mbar_try_wait(bar, parity))
        if (globaltimer_ns() - t0 > limit_ns) return;
}
__device__ __forceinline__ void tma_load_2d(void *dst, const CUtensorMap *tm, uint64_t *bar, int32_t c0,
                                            int32_t c1) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(
            smem_u32(dst)),
        "l"(reinterpret_cast<uint64_t>(tm)), "r"(c0), "r"(c1), "r"(smem_u32(bar))
        : "memory");
}
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_commit(uint64_t *bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
                 : "memory");
}
template <int FORM>
__device__ __forceinline__ void tc_mma(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                       uint32_t accumulate) {
    if constexpr (FORM == F_BF16) {
        asm volatile(
            "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
            "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
            "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
            : "memory");
    } else if constexpr (FORM == F_FP8) {
        asm volatile(
            "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
            "tcgen05.mma.cta_group::1.kind::f8f6f4 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
            "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
            : "memory");
    } else {
        asm volatile(
            "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
            "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
            "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
            : "memory");
    }
}
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, uint32_t (&r)[16]) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, "
        "%14, %15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr)
        : "memory");
}
__device__ __forceinline__ void tmem_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }
// wait for the thread's TMEM loads, with the loaded registers as operands so that no use of them
// can be scheduled before the wait
__device__ __forceinline__ void tmem_wait_ld(uint32_t (&r)[16]) {
    asm volatile("tcgen05.wait::ld.sync.aligned;"
                 : "+r"(r[0]), "+r"(r[1]), "+r"(r[2]), "+r"(r[3]), "+r"(r[4]), "+r"(r[5]), "+r"(r[6]), "+r"(r[7]),
                   "+r"(r[8]), "+r"(r[9]), "+r"(r[10]), "+r"(r[11]), "+r"(r[12]), "+r"(r[13]), "+r"(r[14]),
                   "+r"(r[15])
                 :
                 : "memory");
}

// Shared-memory matrix descriptor of a K-major tile with 128-byte swizzle: rows of 128 B, 8-row
// atoms of 1024 B (stride byte offset 1024), tile base 1024-byte aligned, descriptor version 1.
__device__ __forceinline__ uint64_t sw128_desc(const void *tile) {
    const uint32_t a = smem_u32(tile);
    uint64_t desc = (uint64_t)((a & 0x3FFFFu) >> 4);
    desc |= (uint64_t)(1024u >> 4) << 32;
    desc |= (uint64_t)1 << 46;
    desc |= (uint64_t)2 << 61;
    return desc;
}

__device__ __forceinline__ unsigned lanemask_lt() {
    unsigned m;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
    return m;
}

// ---------------------------------------------------------------- the kernel
template <int FORM, int EPI>
__global__ void __launch_bounds__(FORM == F_TF32X3 ? 384 : 256, 1)
    k_tc(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB,
         const __grid_constant__ CUtensorMap tmB2, const Args a) {
    constexpr bool X3 = (FORM == F_TF32X3);
    extern __shared__ uint8_t smem_raw[];
    // 1024-byte aligned stage base, derived by pointer arithmetic on the shared array so that
    // accesses through it stay shared-memory accesses
    uint8_t *base = smem_raw + ((1024u - (smem_u32(smem_raw) & 1023u)) & 1023u);
    uint64_t *bars = reinterpret_cast<uint64_t *>(base + (size_t)a.stages * a.stage_bytes);
    uint64_t *full = bars, *tfull = bars + MAX_STAGES, *empty = bars + 2 * MAX_STAGES;
    uint64_t *accf = bars + 3 * MAX_STAGES, *acce = accf + 2;
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(acce + 2);
    volatile int *abort_flag = reinterpret_cast<volatile int *>(tmem_slot + 1);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (threadIdx.x == 0) {
        for (int s = 0; s < a.stages; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&tfull[s], 4);
            mbar_init(&empty[s], 1);
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(&accf[b], 1);
            mbar_init(&acce[b], 4);
        }
        *abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 2) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                     "r"((uint32_t)a.tmem_cols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem_base = *tmem_slot;
    const int bn_alloc = a.tmem_cols / 2;
    const int units_per_tile = a.n_chunks;

    if (warp == 0) {
        // ------------------------------------------------ TMA producer
        if (lane == 0) {
            int s = 0;
            uint32_t ph = 0;
            uint32_t issued = 0, last_par = 0;  // per-stage: issued bit, parity of the last issue
            for (int tile = blockIdx.x; tile < a.m_tiles && !*abort_flag; tile += gridDim.x) {
                for (int nc = 0; nc < units_per_tile; ++nc) {
                    for (int kb = 0; kb < a.kb; ++kb) {
                        if (!mbar_wait(&empty[s], ph ^ 1, abort_flag)) goto producer_done;
                        uint8_t *st = base + (size_t)s * a.stage_bytes;
                        mbar_expect_tx(&full[s], a.tx_bytes);
                        const int32_t kx = kb * (int32_t)(128 / (FORM == F_BF16 ? 2 : (FORM == F_FP8 ? 1 : 4)));
                        tma_load_2d(st, &tmA, &full[s], kx, tile * BM);
                        uint8_t *bdst = st + (X3 ? 2 : 1) * a.a_bytes;
                        tma_load_2d(bdst, &tmB, &full[s], kx, nc * a.bn);
                        if constexpr (X3) tma_load_2d(bdst + a.b_bytes, &tmB2, &full[s], kx, nc * a.bn);
                        issued |= 1u << s;
                        last_par = (last_par & ~(1u << s)) | (ph << s);
                        if (++s == a.stages) {
                            s = 0;
                            ph ^= 1;
                        }
                    }
                }
            }
        producer_done:
            if (*abort_flag) {
                // let every bulk copy still in flight land before the CTA exits
                for (int q = 0; q < a.stages; ++q)
                    if (issued & (1u << q)) mbar_drain(&full[q], (last_par >> q) & 1, 500000000ull);
            }
        }
    } else if (warp == 1) {
        // ------------------------------------------------ MMA issuer
        if (lane == 0) {
            int s = 0, ab = 0;
            uint32_t ph = 0, aph = 0;
            bool committed = false;
            uint64_t *last_bar = nullptr;
            uint32_t last_parity = 0;
            for (int tile = blockIdx.x; tile < a.m_tiles && !*abort_flag; tile += gridDim.x) {
                for (int nc = 0; nc < units_per_tile; ++nc) {
                    if (!mbar_wait(&acce[ab], aph ^ 1, abort_flag)) goto mma_done;
                    tc_fence_after();
                    const uint32_t d_tmem = tmem_base + (uint32_t)(ab * bn_alloc);
                    for (int kb = 0; kb < a.kb; ++kb) {
                        if (!mbar_wait(X3 ? &tfull[s] : &full[s], ph, abort_flag)) goto mma_done;
                        tc_fence_after();
                        uint8_t *st = base + (size_t)s * a.stage_bytes;
                        const uint64_t adesc = sw128_desc(st);
                        const uint64_t bdesc = sw128_desc(st + (X3 ? 2 : 1) * a.a_bytes);
#pragma unroll
                        for (int kk = 0; kk < 4; ++kk) {
                            const uint32_t acc = (kb > 0 || kk > 0) ? 1u : 0u;
                            const uint64_t off = (uint64_t)(kk * 2);  // 32 bytes per MMA step
                            if constexpr (X3) {
                                const uint64_t alo = sw128_desc(st + a.a_bytes);
                                const uint64_t blo = sw128_desc(st + 2 * a.a_bytes + a.b_bytes);
                                tc_mma<FORM>(d_tmem, alo + off, bdesc + off, a.idesc, acc);
                                tc_mma<FORM>(d_tmem, adesc + off, blo + off, a.idesc, 1u);
                                tc_mma<FORM>(d_tmem, adesc + off, bdesc + off, a.idesc, 1u);
                            } else {
                                tc_mma<FORM>(d_tmem, adesc + off, bdesc + off, a.idesc, acc);
                            }
                        }
                        tc_commit(&empty[s]);
                        committed = true;
                        last_bar = &empty[s];
                        last_parity = ph;
                        if (++s == a.stages) {
                            s = 0;
                            ph ^= 1;
                        }
                    }
                    tc_commit(&accf[ab]);
                    last_bar = &accf[ab];
                    last_parity = aph;
                    if (++ab == 2) {
                        ab = 0;
                        aph ^= 1;
                    }
                }
            }
        mma_done:
            if (*abort_flag && committed && last_bar) mbar_drain(last_bar, last_parity, 500000000ull);
        }
    } else if (X3 && warp >= 8) {
        // ------------------------------------------------ 3xTF32 split of the staged X tile
        const int t = threadIdx.x - 256;  // 0..127
        int s = 0;
        uint32_t ph = 0;
        for (int tile = blockIdx.x; tile < a.m_tiles && !*abort_flag; tile += gridDim.x) {
            for (int nc = 0; nc < units_per_tile; ++nc) {
                for (int kb = 0; kb < a.kb; ++kb) {
                    if (!mbar_wait(&full[s], ph, abort_flag)) goto split_done;
                    uint8_t *st = base + (size_t)s * a.stage_bytes;
                    uint4 *hi = reinterpret_cast<uint4 *>(st);
                    uint4 *lo = reinterpret_cast<uint4 *>(st + a.a_bytes);
#pragma unroll 4
                    for (int e = t; e < (int)(a.a_bytes / 16); e += 128) {
                        uint4 v = hi[e], h, l;
                        h.x = v.x & 0xffffe000u;
                        h.y = v.y & 0xffffe000u;
                        h.z = v.z & 0xffffe000u;
                        h.w = v.w & 0xffffe000u;
                        l.x = __float_as_uint(__fsub_rn(__uint_as_float(v.x), __uint_as_float(h.x))) & 0xffffe000u;
                        l.y = __float_as_uint(__fsub_rn(__uint_as_float(v.y), __uint_as_float(h.y))) & 0xffffe000u;
                        l.z = __float_as_uint(__fsub_rn(__uint_as_float(v.z), __uint_as_float(h.z))) & 0xffffe000u;
                        l.w = __float_as_uint(__fsub_rn(__uint_as_float(v.w), __uint_as_float(h.w))) & 0xffffe000u;
                        hi[e] = h;
                        lo[e] = l;
                    }
                    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                    __syncwarp();
                    if (lane == 0) mbar_arrive(&tfull[s]);
                    if (++s == a.stages) {
                        s = 0;
                        ph ^= 1;
                    }
                }
            }
        }
    split_done:;
    } else if (warp >= 4 && warp < 8) {
        // ------------------------------------------------ epilogue: one TMEM lane = one point
        const int q = warp - 4;
        int ab = 0;
        uint32_t aph = 0;
        const float cm = (EPI == E_ARGMIN) ? __uint_as_float(*a.cmax) : 0.f;
        for (int tile = blockIdx.x; tile < a.m_tiles && !*abort_flag; tile += gridDim.x) {
            const int64_t row = (int64_t)tile * BM + q * 32 + lane;
            const bool valid = row < a.n;
            float v0 = __int_as_float(0x7f800000), v1 = v0, v2 = v0;
            int i0 = 0, i1 = 0;
            float sx = 1.f;
            if (EPI == E_ARGMIN && FORM == F_FP8 && valid) sx = a.xscale[row];
            // top-m state: threshold and this thread's buffer (slot-major, stride 128)
            float tau = -__int_as_float(0x7f800000);
            int tcnt = 0;
            const int et = q * 32 + lane;
            float *tbv = reinterpret_cast<float *>(base + (size_t)a.stages * a.stage_bytes + 1024);
            int32_t *tbi = reinterpret_cast<int32_t *>(tbv + TOPBUF * 128);
            for (int nc = 0; nc < units_per_tile; ++nc) {
                if (!mbar_wait(&accf[ab], aph, abort_flag)) goto epi_done;
                tc_fence_after();
                const uint32_t tbase = tmem_base + ((uint32_t)(q * 32) << 16) + (uint32_t)(ab * bn_alloc);
                // 16 accumulator columns per tcgen05.ld; the load of the next group is in flight
                // while the current group is processed
                auto process = [&](const uint32_t (&r)[16], int c) {
                    const int64_t j0 = (int64_t)nc * a.bn + c;
                    if constexpr (EPI == E_ARGMIN) {
                        if (j0 >= a.k) return;
                        float cn[16], ms[16];
                        if (j0 + 16 <= a.k_pad) {
#pragma unroll
                            for (int g = 0; g < 4; ++g) {
                                const float4 t4 = __ldg(reinterpret_cast<const float4 *>(a.cnorm + j0) + g);
                                cn[4 * g] = t4.x, cn[4 * g + 1] = t4.y, cn[4 * g + 2] = t4.z, cn[4 * g + 3] = t4.w;
                            }
                        } else {
#pragma unroll
                            for (int g = 0; g < 16; ++g)
                                cn[g] = (j0 + g < a.k_pad) ? a.cnorm[j0 + g] : __int_as_float(0x7f800000);
                        }
#pragma unroll
                        for (int g = 0; g < 16; ++g) {
                            if constexpr (FORM == F_FP8)
                                ms[g] = (j0 + g < a.k) ? -2.f * sx * a.cscale[j0 + g] : -2.f;
                            else
                                ms[g] = -2.f;
                        }
#pragma unroll
                        for (int g = 0; g < 16; ++g) {
                            const int j = (int)(j0 + g);
                            const float s = (j < a.k) ? fmaf(ms[g], __uint_as_float(r[g]), cn[g])
                                                      : __int_as_float(0x7f800000);
                            const bool lt0 = s < v0, lt1 = s < v1;
                            const float m0 = fmaxf(v0, s), m1 = fmaxf(v1, s);
                            v2 = fminf(v2, m1);
                            v1 = fminf(v1, m0);
                            v0 = fminf(v0, s);
                            i1 = lt0 ? i0 : (lt1 ? j : i1);
                            i0 = lt0 ? j : i0;
                        }
                    } else if constexpr (EPI == E_STORE) {
                        const int64_t col0 = (int64_t)nc * a.bn + c;
                        if (valid && col0 < a.k) {
                            float v[16];
#pragma unroll
                            for (int g = 0; g < 16; ++g) v[g] = __uint_as_float(r[g]);
                            if (a.bias) {
#pragma unroll
                                for (int g = 0; g < 4; ++g) {
                                    const float4 b4 = __ldg(reinterpret_cast<const float4 *>(a.bias + col0) + g);
                                    v[4 * g] += b4.x, v[4 * g + 1] += b4.y, v[4 * g + 2] += b4.z, v[4 * g + 3] += b4.w;
                                }
                            }
                            if (a.Ypre) {
                                float4 *pr = reinterpret_cast<float4 *>(a.Ypre + row * a.ldpre + col0);
#pragma unroll
                                for (int g = 0; g < 4; ++g) pr[g] = make_float4(v[4 * g], v[4 * g + 1], v[4 * g + 2], v[4 * g + 3]);
                            }
                            if (a.act == 1) {
#pragma unroll
                                for (int g = 0; g < 16; ++g) v[g] = gelu_erf(v[g]);
                            }
                            if (a.out_bf16) {
                                uint32_t w[8];
#pragma unroll
                                for (int g = 0; g < 8; ++g) {
                                    __nv_bfloat162 h = __floats2bfloat162_rn(v[2 * g], v[2 * g + 1]);
                                    w[g] = *reinterpret_cast<uint32_t *>(&h);
                                }
                                uint4 *yr = reinterpret_cast<uint4 *>(reinterpret_cast<__nv_bfloat16 *>(a.Y) + row * a.ldy + col0);
                                yr[0] = make_uint4(w[0], w[1], w[2], w[3]);
                                yr[1] = make_uint4(w[4], w[5], w[6], w[7]);
                            } else {
                                float4 *yr = reinterpret_cast<float4 *>(a.Y + row * a.ldy + col0);
#pragma unroll
                                for (int g = 0; g < 4; ++g) yr[g] = make_float4(v[4 * g], v[4 * g + 1], v[4 * g + 2], v[4 * g + 3]);
                            }
                        }
                    } else {
                        // top-m: candidates above the running threshold go to this row's buffer
                        const int64_t col0 = (int64_t)nc * a.bn + c;
                        if (col0 >= a.k) return;
                        float sv[16];
#pragma unroll
                        for (int g = 0; g < 4; ++g) {
                            const float4 b4 = a.bias ? __ldg(reinterpret_cast<const float4 *>(a.bias + col0) + g)
                                                     : make_float4(0.f, 0.f, 0.f, 0.f);
                            sv[4 * g] = __uint_as_float(r[4 * g]) + b4.x;
                            sv[4 * g + 1] = __uint_as_float(r[4 * g + 1]) + b4.y;
                            sv[4 * g + 2] = __uint_as_float(r[4 * g + 2]) + b4.z;
                            sv[4 * g + 3] = __uint_as_float(r[4 * g + 3]) + b4.w;
                        }
                        uint32_t m = 0;
#pragma unroll
                        for (int g = 0; g < 16; ++g)
                            if (sv[g] > tau && col0 + g < a.k) m |= 1u << g;
                        while (m) {
                            const int g = __ffs(m) - 1;
                            m &= m - 1;
                            float sg = 0.f;
#pragma unroll
                            for (int h = 0; h < 16; ++h)
                                if (h == g) sg = sv[h];
                            if (tcnt == TOPBUF) {
                                const uint32_t T = topm_threshold(tbv, et, tcnt, a.topm);
                                int nw = 0;
                                for (int i = 0; i < tcnt; ++i) {
                                    const float bvv = tbv[i * 128 + et];
                                    if (fkey(bvv) >= T) {
                                        tbv[nw * 128 + et] = bvv;
                                        tbi[nw * 128 + et] = tbi[i * 128 + et];
                                        ++nw;
                                    }
                                }
                                tcnt = nw;
                                tau = fkey_inv(T);
                                if (!(sg > tau) || tcnt == TOPBUF) continue;
                            }
                            tbv[tcnt * 128 + et] = sg;
                            tbi[tcnt * 128 + et] = (int32_t)(col0 + g);
                            ++tcnt;
                        }
                    }
                };
                uint32_t ra[16], rb[16];
                tmem_ld16(tbase, ra);
                tmem_wait_ld(ra);
                for (int c = 0; c < a.bn; c += 32) {
                    const bool has_b = c + 16 < a.bn;
                    if (has_b) tmem_ld16(tbase + (uint32_t)(c + 16), rb);
                    process(ra, c);
                    if (has_b) {
                        tmem_wait_ld(rb);
                        if (c + 32 < a.bn) tmem_ld16(tbase + (uint32_t)(c + 32), ra);
                        process(rb, c + 16);
                        if (c + 32 < a.bn) tmem_wait_ld(ra);
                    }
                }
                if constexpr (EPI == E_ARGMIN) {
                    if (nc == units_per_tile - 1) {
                        // the point's final top-2: label, expanded min distance, certified near-tie flag
                        const float xn = valid ? a.xnorm[row] : 0.f;
                        const float xr = sqrtf(fmaxf(xn, 0.f)) * (1.f + 1.0e-6f);
                        const float E2 = 2.f * (a.err_rel * xr * cm + a.err_abs * cm * cm);
                        const bool flag = valid && !((v1 - v0) > E2);
                        if (valid) {
                            a.labels[row] = i0;
                            if (a.min_d2) a.min_d2[row] = fmaxf(0.f, xn + v0);
                        }
                        if (a.flag_list) {
                            const unsigned m = __ballot_sync(0xffffffffu, flag);
                            if (m) {
                                const int leader = __ffs(m) - 1;
                                int b0 = 0;
                                if (lane == leader) b0 = atomicAdd(a.flag_count, __popc(m));
                                b0 = __shfl_sync(0xffffffffu, b0, leader);
                                const int slot = b0 + __popc(m & lanemask_lt());
                                int32_t *cf = a.cand + (int64_t)slot * CAND_STRIDE;
                                if (flag) a.flag_list[slot] = (int32_t)row;
                                // two candidates when every other center is certified worse (v2 is
                                // the third best score); otherwise the band must be listed
                                const bool pair = flag && (v2 - v0) > E2;
                                const bool need_band = flag && !pair;
                                if (pair) {
                                    cf[0] = 2;
                                    cf[1] = min(i0, i1);
                                    cf[2] = max(i0, i1);
                                }
                                if (units_per_tile == 1 && __any_sync(0xffffffffu, need_band)) {
                                    // a second pass over the accumulator, still resident in TMEM: every
                                    // center whose score lies inside the band is a candidate
                                    int cnt = 0;
                                    auto band = [&](const uint32_t (&r)[16], int c) {
                                        if (!need_band || c >= a.k) return;
                                        float cn[16];
#pragma unroll
                                        for (int g = 0; g < 4; ++g) {
                                            const float4 t4 = __ldg(reinterpret_cast<const float4 *>(a.cnorm + c) + g);
                                            cn[4 * g] = t4.x, cn[4 * g + 1] = t4.y, cn[4 * g + 2] = t4.z, cn[4 * g + 3] = t4.w;
                                        }
                                        uint32_t inband = 0;
#pragma unroll
                                        for (int g = 0; g < 16; ++g) {
                                            float ms = -2.f;
                                            if constexpr (FORM == F_FP8) ms = (c + g < a.k) ? -2.f * sx * a.cscale[c + g] : 0.f;
                                            const float sc = fmaf(ms, __uint_as_float(r[g]), cn[g]);
                                            if (c + g < a.k && sc - v0 <= E2) inband |= 1u << g;
                                        }
                                        while (inband) {
                                            const int g = __ffs(inband) - 1;
                                            inband &= inband - 1;
                                            if (cnt < CAND_MAX) cf[1 + cnt] = c + g;
                                            ++cnt;
                                        }
                                    };
                                    uint32_t ra[16], rb[16];
                                    tmem_ld16(tbase, ra);
                                    tmem_wait_ld(ra);
                                    for (int c = 0; c < a.bn; c += 32) {
                                        const bool has_b = c + 16 < a.bn;
                                        if (has_b) tmem_ld16(tbase + (uint32_t)(c + 16), rb);
                                        band(ra, c);
                                        if (has_b) {
                                            tmem_wait_ld(rb);
                                            if (c + 32 < a.bn) tmem_ld16(tbase + (uint32_t)(c + 32), ra);
                                            band(rb, c + 16);
                                            if (c + 32 < a.bn) tmem_wait_ld(ra);
                                        }
                                    }
                                    if (need_band) cf[0] = cnt <= CAND_MAX ? cnt : -1;
                                } else if (need_band) {
                                    cf[0] = -1;
                                }
                            }
                        }
                    }
                }
                tc_fence_before();
                __syncwarp();
                if (lane == 0) mbar_arrive(&acce[ab]);
                if (++ab == 2) {
                    ab = 0;
                    aph ^= 1;
                }
            }
            if constexpr (EPI == E_TOPM) {
                // exactly m outputs: keys above the m-th largest, then ties at it, -1 padding
                if (valid) {
                    const int m = a.topm;
                    const uint32_t T = tcnt >= m ? topm_threshold(tbv, et, tcnt, m) : 0u;
                    int w = 0;
                    for (int pass = 0; pass < 2; ++pass)
                        for (int i = 0; i < tcnt && w < m; ++i) {
                            const float bvv = tbv[i * 128 + et];
                            const uint32_t kk = fkey(bvv);
                            if ((pass == 0 && kk > T) || (pass == 1 && kk == T)) {
                                a.top_idx[row * m + w] = tbi[i * 128 + et];
                                if (a.top_val) a.top_val[row * m + w] = bvv;
                                ++w;
                            }
                        }
                    for (; w < m; ++w) {
                        a.top_idx[row * m + w] = -1;
                        if (a.top_val) a.top_val[row * m + w] = -__int_as_float(0x7f800000);
                    }
                }
            }
        }
    epi_done:;
    }
    __syncthreads();
    if (*abort_flag && threadIdx.x == 0) status_raise(a.status, ST_TIMEOUT);
    if (warp == 2) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem_base),
                     "r"((uint32_t)a.tmem_cols)
                     : "memory");
    }
}

// ---------------------------------------------------------------- batched kernel
// The same pipeline over a work list of (problem, row tile) items: every CTA walks items
// blockIdx.x, blockIdx.x + gridDim.x, ...; each item runs its problem's center chunks in order with
// that problem's tensor maps (3 per problem in global memory), K-block count and instruction
// descriptor.  The centers of a problem's seeds are concatenated along N (seeds x kps columns), so
// one read of X serves every seed; the epilogue keeps a separate top-2 per seed (seed boundaries
// fall on 16-column groups) and emits a label and a certified near-tie flag per (seed, point).
template <int FORM>
__global__ void __launch_bounds__(FORM == F_TF32X3 ? 384 : 256, 1)
    k_tcb(const CUtensorMap *__restrict__ maps, const BProb *__restrict__ probs,
          const int32_t *__restrict__ tile_prob, int ntiles, int stages, uint32_t a_bytes, uint32_t b_bytes,
          uint32_t stage_bytes, int32_t *__restrict__ flags, int32_t *__restrict__ flag_count, int *status) {
    constexpr bool X3 = (FORM == F_TF32X3);
    constexpr int BKE = 128 / (FORM == F_BF16 ? 2 : (FORM == F_FP8 ? 1 : 4));
    extern __shared__ uint8_t smem_raw[];
    uint8_t *base = smem_raw + ((1024u - (smem_u32(smem_raw) & 1023u)) & 1023u);
    uint64_t *bars = reinterpret_cast<uint64_t *>(base + (size_t)stages * stage_bytes);
    uint64_t *full = bars, *tfull = bars + MAX_STAGES, *empty = bars + 2 * MAX_STAGES;
    uint64_t *accf = bars + 3 * MAX_STAGES, *acce = accf + 2;
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(acce + 2);
    volatile int *abort_flag = reinterpret_cast<volatile int *>(tmem_slot + 1);
    constexpr uint32_t TMEM_COLS = 512, BN_ALLOC = 256;

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (threadIdx.x == 0) {
        for (int q = 0; q < stages; ++q) {
            mbar_init(&full[q], 1);
            mbar_init(&tfull[q], 4);
            mbar_init(&empty[q], 1);
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(&accf[b], 1);
            mbar_init(&acce[b], 4);
        }
        *abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 2) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                     "r"(TMEM_COLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem_base = *tmem_slot;

    if (warp == 0) {
        if (lane == 0) {
            int st = 0;
            uint32_t ph = 0, issued = 0, last_par = 0;
            for (int it = blockIdx.x; it < ntiles && !*abort_flag; it += gridDim.x) {
                const int p = tile_prob[it];
                const BProb &P = probs[p];
                const int ltile = it - (int)P.tile0;
                const CUtensorMap *tm = maps + 3 * p;
                for (int nc = 0; nc < P.n_chunks; ++nc) {
                    for (int kb = 0; kb < P.kb; ++kb) {
                        if (!mbar_wait(&empty[st], ph ^ 1, abort_flag)) goto producer_done;
                        uint8_t *sb = base + (size_t)st * stage_bytes;
                        mbar_expect_tx(&full[st], P.tx_bytes);
                        tma_load_2d(sb, tm, &full[st], kb * BKE, ltile * BM);
                        uint8_t *bdst = sb + (X3 ? 2 : 1) * a_bytes;
                        tma_load_2d(bdst, tm + 1, &full[st], kb * BKE, nc * P.bn);
                        if constexpr (X3) tma_load_2d(bdst + b_bytes, tm + 2, &full[st], kb * BKE, nc * P.bn);
                        issued |= 1u << st;
                        last_par = (last_par & ~(1u << st)) | (ph << st);
                        if (++st == stages) {
                            st = 0;
                            ph ^= 1;
                        }
                    }
                }
            }
        producer_done:
            if (*abort_flag)
                for (int q = 0; q < stages; ++q)
                    if (issued & (1u << q)) mbar_drain(&full[q], (last_par >> q) & 1, 500000000ull);
        }
    } else if (warp == 1) {
        if (lane == 0) {
            int st = 0, ab = 0;
            uint32_t ph = 0, aph = 0;
            uint64_t *last_bar = nullptr;
            uint32_t last_parity = 0;
            for (int it = blockIdx.x; it < ntiles && !*abort_flag; it += gridDim.x) {
                const BProb &P = probs[tile_prob[it]];
                for (int nc = 0; nc < P.n_chunks; ++nc) {
                    if (!mbar_wait(&acce[ab], aph ^ 1, abort_flag)) goto mma_done;
                    tc_fence_after();
                    const uint32_t d_tmem = tmem_base + (uint32_t)(ab * BN_ALLOC);
                    for (int kb = 0; kb < P.kb; ++kb) {
                        if (!mbar_wait(X3 ? &tfull[st] : &full[st], ph, abort_flag)) goto mma_done;
                        tc_fence_after();
                        uint8_t *sb = base + (size_t)st * stage_bytes;
                        const uint64_t adesc = sw128_desc(sb);
                        const uint64_t bdesc = sw128_desc(sb + (X3 ? 2 : 1) * a_bytes);
#pragma unroll
                        for (int kk = 0; kk < 4; ++kk) {
                            const uint32_t acc = (kb > 0 || kk > 0) ? 1u : 0u;
                            const uint64_t off = (uint64_t)(kk * 2);
                            if constexpr (X3) {
                                const uint64_t alo = sw128_desc(sb + a_bytes);
                                const uint64_t blo = sw128_desc(sb + 2 * a_bytes + b_bytes);
                                tc_mma<FORM>(d_tmem, alo + off, bdesc + off, P.idesc, acc);
                                tc_mma<FORM>(d_tmem, adesc + off, blo + off, P.idesc, 1u);
                                tc_mma<FORM>(d_tmem, adesc + off, bdesc + off, P.idesc, 1u);
                            } else {
                                tc_mma<FORM>(d_tmem, adesc + off, bdesc + off, P.idesc, acc);
                            }
                        }
                        tc_commit(&empty[st]);
                        last_bar = &empty[st];
                        last_parity = ph;
                        if (++st == stages) {
                            st = 0;
                            ph ^= 1;
                        }
                    }
                    tc_commit(&accf[ab]);
                    last_bar = &accf[ab];
                    last_parity = aph;
                    if (++ab == 2) {
                        ab = 0;
                        aph ^= 1;
                    }
                }
            }
        mma_done:
            if (*abort_flag && last_bar) mbar_drain(last_bar, last_parity, 500000000ull);
        }
    } else if (X3 && warp >= 8) {
        const int t = threadIdx.x - 256;
        int st = 0;
        uint32_t ph = 0;
        for (int it = blockIdx.x; it < ntiles && !*abort_flag; it += gridDim.x) {
            const BProb &P = probs[tile_prob[it]];
            for (int nc = 0; nc < P.n_chunks; ++nc) {
                for (int kb = 0; kb < P.kb; ++kb) {
                    if (!mbar_wait(&full[st], ph, abort_flag)) goto split_done;
                    uint8_t *sb = base + (size_t)st * stage_bytes;
                    uint4 *hi = reinterpret_cast<uint4 *>(sb);
                    uint4 *lo = reinterpret_cast<uint4 *>(sb + a_bytes);
#pragma unroll 4
                    for (int e = t; e < (int)(a_bytes / 16); e += 128) {
                        uint4 v = hi[e], h, l;
                        h.x = v.x & 0xffffe000u;
                        h.y = v.y & 0xffffe000u;
                        h.z = v.z & 0xffffe000u;
                        h.w = v.w & 0xffffe000u;
                        l.x = __float_as_uint(__fsub_rn(__uint_as_float(v.x), __uint_as_float(h.x))) & 0xffffe000u;
                        l.y = __float_as_uint(__fsub_rn(__uint_as_float(v.y), __uint_as_float(h.y))) & 0xffffe000u;
                        l.z = __float_as_uint(__fsub_rn(__uint_as_float(v.z), __uint_as_float(h.z))) & 0xffffe000u;
                        l.w = __float_as_uint(__fsub_rn(__uint_as_float(v.w), __uint_as_float(h.w))) & 0xffffe000u;
                        hi[e] = h;
                        lo[e] = l;
                    }
                    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                    __syncwarp();
                    if (lane == 0) mbar_arrive(&tfull[st]);
                    if (++st == stages) {
                        st = 0;
                        ph ^= 1;
                    }
                }
            }
        }
    split_done:;
    } else if (warp >= 4 && warp < 8) {
        const int q = warp - 4;
        int ab = 0;
        uint32_t aph = 0;
        for (int it = blockIdx.x; it < ntiles && !*abort_flag; it += gridDim.x) {
            const int p = tile_prob[it];
            const BProb &P = probs[p];
            const int64_t row = (int64_t)(it - P.tile0) * BM + q * 32 + lane;
            const bool valid = row < P.n;
            const float xn = valid ? P.xnorm[row] : 0.f;
            const float cm = __uint_as_float(*P.cmax);
            const float xr = sqrtf(fmaxf(xn, 0.f)) * (1.f + 1.0e-6f);
            const float E2 = 2.f * (P.err_rel * xr * cm + P.err_abs * cm * cm);
            const int64_t ncols = (int64_t)P.seeds * P.kps;
            float v0 = __int_as_float(0x7f800000), v1 = v0, v2 = v0;
            int i0 = 0, i1 = 0, cur = 0;
            // emit the finished seed s of this point: label, certified near-tie flag, candidates
            auto finish = [&](int s) {
                const bool flag = valid && !((v1 - v0) > E2);
                if (valid) P.labels[(int64_t)s * P.n + row] = i0;
                const unsigned m = __ballot_sync(0xffffffffu, flag);
                if (m) {
                    const int leader = __ffs(m) - 1;
                    int b0 = 0;
                    if (lane == leader) b0 = atomicAdd(flag_count, __popc(m));
                    b0 = __shfl_sync(0xffffffffu, b0, leader);
                    if (flag) {
                        int32_t *f = flags + (int64_t)(b0 + __popc(m & lanemask_lt())) * BFLAG_STRIDE;
                        f[0] = p;
                        f[1] = s;
                        f[2] = (int32_t)row;
                        const bool pair = (v2 - v0) > E2;
                        f[3] = pair ? 2 : -1;
                        f[4] = min(i0, i1);
                        f[5] = max(i0, i1);
                    }
                }
                v0 = v1 = v2 = __int_as_float(0x7f800000);
                i0 = i1 = 0;
            };
            for (int nc = 0; nc < P.n_chunks; ++nc) {
                if (!mbar_wait(&accf[ab], aph, abort_flag)) goto epi_done;
                tc_fence_after();
                const uint32_t tbase = tmem_base + ((uint32_t)(q * 32) << 16) + (uint32_t)(ab * BN_ALLOC);
                auto process = [&](const uint32_t (&r)[16], int c) {
                    const int64_t j0 = (int64_t)nc * P.bn + c;  // column among all seeds' centers
                    if (j0 >= ncols) return;
                    const int s = (int)(j0 / P.kps);
                    const int jl0 = (int)(j0 - (int64_t)s * P.kps);
                    if (s != cur) {
                        finish(cur);
                        cur = s;
                    }
                    if (jl0 >= P.k) return;
                    float cn[16];
#pragma unroll
                    for (int g = 0; g < 4; ++g) {
                        const float4 t4 = __ldg(reinterpret_cast<const float4 *>(P.cnorm + j0) + g);
                        cn[4 * g] = t4.x, cn[4 * g + 1] = t4.y, cn[4 * g + 2] = t4.z, cn[4 * g + 3] = t4.w;
                    }
#pragma unroll
                    for (int g = 0; g < 16; ++g) {
                        const int j = jl0 + g;
                        const float sc = (j < P.k) ? fmaf(-2.f, __uint_as_float(r[g]), cn[g]) : __int_as_float(0x7f800000);
                        const bool lt0 = sc < v0, lt1 = sc < v1;
                        const float m0 = fmaxf(v0, sc), m1 = fmaxf(v1, sc);
                        v2 = fminf(v2, m1);
                        v1 = fminf(v1, m0);
                        v0 = fminf(v0, sc);
                        i1 = lt0 ? i0 : (lt1 ? j : i1);
                        i0 = lt0 ? j : i0;
                    }
                };
                uint32_t ra[16], rb[16];
                tmem_ld16(tbase, ra);
                tmem_wait_ld(ra);
                for (int c = 0; c < P.bn; c += 32) {
                    const bool has_b = c + 16 < P.bn;
                    if (has_b) tmem_ld16(tbase + (uint32_t)(c + 16), rb);
                    process(ra, c);
                    if (has_b) {
                        tmem_wait_ld(rb);
                        if (c + 32 < P.bn) tmem_ld16(tbase + (uint32_t)(c + 32), ra);
                        process(rb, c + 16);
                        if (c + 32 < P.bn) tmem_wait_ld(ra);
                    }
                }
                tc_fence_before();
                __syncwarp();
                if (lane == 0) mbar_arrive(&acce[ab]);
                if (++ab == 2) {
                    ab = 0;
                    aph ^= 1;
                }
            }
            finish(cur);
        }
    epi_done:;
    }
    __syncthreads();
    if (*abort_flag && threadIdx.x == 0) status_raise(status, ST_TIMEOUT);
    if (warp == 2) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem_base), "r"(TMEM_COLS)
                     : "memory");
    }
}

// ---------------------------------------------------------------- host side
typedef CUresult (*EncodeTiledFn)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                  const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

static EncodeTiledFn encode_fn() {
    static EncodeTiledFn fn = nullptr;
    static bool tried = false;
    if (!tried) {
        tried = true;
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<EncodeTiledFn>(p);
        else
            cudaGetLastError();
    }
    return fn;
}

// 2D row-major tensor [outer x inner] of `esize`-byte elements, box = 128 bytes x box_rows, 128B swizzle,
// out-of-range elements read as zero
static bool make_tmap(CUtensorMap *m, CUtensorMapDataType dt, const void *ptr, uint64_t inner, uint64_t outer,
                      uint32_t esize, uint32_t box_rows) {
    EncodeTiledFn fn = encode_fn();
    if (!fn) return false;
    cuuint64_t dims[2] = {inner, outer};
    cuuint64_t strides[1] = {inner * esize};
    cuuint32_t box[2] = {128u / esize, box_rows};
    cuuint32_t es[2] = {1, 1};
    return fn(m, dt, 2, const_cast<void *>(ptr), dims, strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
              CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
              CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

static uint32_t make_idesc(int form, int M, int N) {
    uint32_t ab = (form == F_BF16) ? 1u : (form == F_FP8 ? 0u : 2u);
    uint32_t d = 0;
    d |= 1u << 4;           // D = FP32
    d |= ab << 7;           // A format
    d |= ab << 10;          // B format
    d |= (uint32_t)(N >> 3) << 17;
    d |= (uint32_t)(M >> 4) << 24;
    return d;
}

struct Plan {
    int n_chunks, bn, kb, stages, tmem_cols;
    uint32_t a_bytes, b_bytes, stage_bytes, tx_bytes;
    size_t smem;
};

static Plan plan(int form, int64_t d, int64_t k_pad, int bn_cap = 256, int extra_smem = 0) {
    Plan p;
    const int esize = (form == F_BF16) ? 2 : (form == F_FP8 ? 1 : 4);
    p.n_chunks = (int)ceil_div(k_pad, bn_cap);
    p.bn = (int)(ceil_div(ceil_div(k_pad, p.n_chunks), 16) * 16);
    p.kb = (int)ceil_div(d * esize, 128);
    const bool x3 = form == F_TF32X3;
    p.a_bytes = BM * 128;
    p.b_bytes = (uint32_t)p.bn * 128;
    p.stage_bytes = (x3 ? 2 : 1) * p.a_bytes + (x3 ? 2 : 1) * p.b_bytes;
    p.tx_bytes = p.a_bytes + (x3 ? 2 : 1) * p.b_bytes;
    p.stages = (int)std::min<int64_t>(MAX_STAGES, (SMEM_BUDGET - extra_smem) / p.stage_bytes);
    p.tmem_cols = (2 * p.bn <= 256) ? 256 : 512;
    p.smem = (size_t)p.stages * p.stage_bytes + 1024 + 1024 + extra_smem;
    return p;
}

template <int FORM, int EPI>
static int launch(gbkm_ctx *c, const CUtensorMap &A, const CUtensorMap &B, const CUtensorMap &B2, Args &args,
                  const Plan &p) {
    auto kern = k_tc<FORM, EPI>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)p.smem);
    if (e != cudaSuccess) return cuda_check(c, e, "tcgen05 smem attribute");
    const int threads = (FORM == F_TF32X3) ? 384 : 256;
    const int grid = (int)std::min<int64_t>(c->sm_count, args.m_tiles);
    kern<<<grid, threads, p.smem, c->stream>>>(A, B, B2, args);
    GBKM_LAUNCHED(c);
    return cuda_check(c, cudaGetLastError(), "tcgen05 kernel launch");
}

}  // namespace tc

bool tc_assign_supported(int dtype, int64_t d, int64_t k) {
    if (k < 1 || k > 65536) return false;
    if (!tc::encode_fn()) return false;
    if (dtype == GBKM_BF16) return d % 8 == 0;
    if (dtype == GBKM_F32) return d % 4 == 0;
    if (dtype == GBKM_FP8E4M3) return d % 16 == 0 && d <= 128;
    return false;
}

int launch_assign_tc(gbkm_ctx *c, int dtype, const void *Xop, const float *Xscales, const float *X,
                     const float *xnorm, int64_t n, int64_t d, const CenterPrep &cp, int64_t k, int64_t k_pad,
                     float err_rel, float err_abs, const AssignOut &o) {
    using namespace tc;
    const int form = (dtype == GBKM_BF16) ? F_BF16 : (dtype == GBKM_FP8E4M3 ? F_FP8 : F_TF32X3);
    const Plan p = plan(form, d, k_pad, c->bn_cap > 0 ? c->bn_cap : 256);
    const CUtensorMapDataType dt = (form == F_BF16)  ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16
                                   : (form == F_FP8) ? CU_TENSOR_MAP_DATA_TYPE_UINT8
                                                     : CU_TENSOR_MAP_DATA_TYPE_FLOAT32;
    const uint32_t es = (form == F_BF16) ? 2 : (form == F_FP8 ? 1 : 4);
    CUtensorMap tA, tB, tB2;
    if (!make_tmap(&tA, dt, Xop, (uint64_t)d, (uint64_t)n, es, BM) ||
        !make_tmap(&tB, dt, cp.cop, (uint64_t)d, (uint64_t)k_pad, es, (uint32_t)p.bn))
        return set_error(c, GBKM_ECUDA, "cuTensorMapEncodeTiled failed for the assign operands");
    tB2 = tB;
    if (form == F_TF32X3 && !make_tmap(&tB2, dt, cp.cop_lo, (uint64_t)d, (uint64_t)k_pad, es, (uint32_t)p.bn))
        return set_error(c, GBKM_ECUDA, "cuTensorMapEncodeTiled failed for the TF32 low part");
    Args a{};
    a.n = n, a.d = d, a.k = k, a.k_pad = k_pad;
    a.n_chunks = p.n_chunks, a.bn = p.bn, a.kb = p.kb, a.stages = p.stages, a.tmem_cols = p.tmem_cols;
    a.m_tiles = (int)ceil_div(n, BM);
    a.a_bytes = p.a_bytes, a.b_bytes = p.b_bytes, a.stage_bytes = p.stage_bytes, a.tx_bytes = p.tx_bytes;
    a.idesc = make_idesc(form, BM, p.bn);
    a.cnorm = cp.cnorm, a.cscale = cp.cscale, a.xscale = Xscales, a.xnorm = xnorm, a.cmax = cp.cmax;
    a.err_rel = err_rel, a.err_abs = err_abs;
    a.labels = o.labels, a.min_d2 = o.min_d2, a.flag_list = o.flag_list, a.cand = o.cand, a.flag_count = o.flag_count;
    a.status = c->status;
    if (form == F_BF16) return launch<F_BF16, E_ARGMIN>(c, tA, tB, tB2, a, p);
    if (form == F_FP8) return launch<F_FP8, E_ARGMIN>(c, tA, tB, tB2, a, p);
    return launch<F_TF32X3, E_ARGMIN>(c, tA, tB, tB2, a, p);
}

// V (d x r, FP32) -> V^T (r x d) in the operand format of the projection
__global__ void k_vt(const float *__restrict__ V, int64_t d, int64_t r, int dtype, void *out) {
    const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e >= d * r) return;
    const int64_t q = e / d, t = e % d;  // out[q][t] = V[t][q]
    const float v = V[t * r + q];
    if (dtype == GBKM_BF16)
        static_cast<__nv_bfloat16 *>(out)[e] = __float2bfloat16_rn(v);
    else
        static_cast<float *>(out)[e] = v;
}

bool tc_project_supported(int dtype, int64_t d, int64_t r) {
    if (!tc::encode_fn()) return false;
    if (r % 16 != 0 || r < 16 || r > 256) return false;
    if (dtype == GBKM_BF16) return d % 8 == 0;
    if (dtype == GBKM_F32) return d % 4 == 0;
    return false;
}

int launch_project_tc(gbkm_ctx *c, int dtype, const void *X, int64_t n, int64_t d, const float *V, int64_t r,
                      float *Y) {
    using namespace tc;
    const int form = (dtype == GBKM_BF16) ? F_BF16 : F_TF32;
    const uint32_t es = (form == F_BF16) ? 2 : 4;
    int rc = GBKM_OK;
    void *ws = ws_reserve(c, (size_t)r * d * es + 256, &rc);
    if (!ws) return rc;
    k_vt<<<(unsigned)ceil_div(r * d, 256), 256, 0, c->stream>>>(V, d, r, dtype, ws);
    GBKM_LAUNCHED(c);
    const Plan p = plan(form, d, r);
    const CUtensorMapDataType dt = (form == F_BF16) ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32;
    CUtensorMap tA, tB;
    if (!make_tmap(&tA, dt, X, (uint64_t)d, (uint64_t)n, es, BM) ||
        !make_tmap(&tB, dt, ws, (uint64_t)d, (uint64_t)r, es, (uint32_t)p.bn))
        return set_error(c, GBKM_ECUDA, "cuTensorMapEncodeTiled failed for the projection operands");
    Args a{};
    a.n = n, a.d = d, a.k = r, a.k_pad = r;
    a.n_chunks = p.n_chunks, a.bn = p.bn, a.kb = p.kb, a.stages = p.stages, a.tmem_cols = p.tmem_cols;
    a.m_tiles = (int)ceil_div(n, BM);
    a.a_bytes = p.a_bytes, a.b_bytes = p.b_bytes, a.stage_bytes = p.stage_bytes, a.tx_bytes = p.tx_bytes;
    a.idesc = make_idesc(form, BM, p.bn);
    a.Y = Y, a.ldy = r;
    a.status = c->status;
    if (form == F_BF16) return launch<F_BF16, E_STORE>(c, tA, tB, tB, a, p);
    return launch<F_TF32, E_STORE>(c, tA, tB, tB, a, p);
}


bool tc_batched_supported(int dtype, int64_t d, int64_t k, int64_t seeds) {
    if (!tc::encode_fn()) return false;
    if (dtype != GBKM_BF16 && dtype != GBKM_F32) return false;
    if (d % 16 != 0 || k < 1 || k > 1024 || seeds < 1 || seeds > 8) return false;
    return true;
}

int make_batch_tmaps(gbkm_ctx *c, int dtype, const BProb &P, void *host_maps3) {
    using namespace tc;
    CUtensorMap *m = static_cast<CUtensorMap *>(host_maps3);
    const bool bf = dtype == GBKM_BF16;
    const CUtensorMapDataType dt = bf ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32;
    const uint32_t es = bf ? 2 : 4;
    const uint64_t rows_b = (uint64_t)P.seeds * (uint64_t)P.kps;
    if (!make_tmap(&m[0], dt, P.Xop, (uint64_t)P.d, (uint64_t)P.n, es, BM) ||
        !make_tmap(&m[1], dt, P.cop, (uint64_t)P.d, rows_b, es, (uint32_t)P.bn))
        return set_error(c, GBKM_ECUDA, "cuTensorMapEncodeTiled failed for a batched problem");
    m[2] = m[1];
    if (!bf && !make_tmap(&m[2], dt, P.cop_lo, (uint64_t)P.d, rows_b, es, (uint32_t)P.bn))
        return set_error(c, GBKM_ECUDA, "cuTensorMapEncodeTiled failed for a batched TF32 low part");
    return GBKM_OK;
}

int launch_assign_tc_batched(gbkm_ctx *c, int dtype, const void *maps, const BProb *probs, int64_t nprob,
                             const int32_t *tile_prob, int64_t ntiles, int parity, int bn_max, int32_t *flags,
                             int32_t *flag_count) {
    using namespace tc;
    (void)nprob;
    (void)parity;
    const bool x3 = dtype == GBKM_F32;
    const uint32_t a_bytes = BM * 128, b_bytes = (uint32_t)bn_max * 128;
    const uint32_t stage_bytes = (x3 ? 2 : 1) * a_bytes + (x3 ? 2 : 1) * b_bytes;
    const int stages = (int)std::min<int64_t>(MAX_STAGES, SMEM_BUDGET / stage_bytes);
    const size_t smem = (size_t)stages * stage_bytes + 2048;
    const int threads = x3 ? 384 : 256;
    const int grid = (int)std::min<int64_t>(c->sm_count, ntiles);
    cudaError_t e;
    if (x3) {
        e = cudaFuncSetAttribute(k_tcb<F_TF32X3>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return cuda_check(c, e, "batched smem attribute");
        k_tcb<F_TF32X3><<<grid, threads, smem, c->stream>>>(static_cast<const CUtensorMap *>(maps), probs, tile_prob,
                                                            (int)ntiles, stages, a_bytes, b_bytes, stage_bytes,
                                                            flags, flag_count, c->status);
    } else {
        e = cudaFuncSetAttribute(k_tcb<F_BF16>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return cuda_check(c, e, "batched smem attribute");
        k_tcb<F_BF16><<<grid, threads, smem, c->stream>>>(static_cast<const CUtensorMap *>(maps), probs, tile_prob,
                                                          (int)ntiles, stages, a_bytes, b_bytes, stage_bytes,
                                                          flags, flag_count, c->status);
    }
    GBKM_LAUNCHED(c);
    return cuda_check(c, cudaGetLastError(), "batched tcgen05 launch");
}


// D = A B^T on tcgen05 (BF16 operands, FP32 accumulation) with a fused epilogue: store
// act(D + bias) in FP32 or BF16 (and optionally the FP32 pre-activation), or, when top_idx is
// given, the indices of the topm largest entries of every row of D + bias (D never written).
// A: M x K, B: N x K, row-major BF16, K % 8 == 0, N % 16 == 0, 16-byte aligned.
int launch_gemm_bf16_tc(gbkm_ctx *c, const void *A, const void *B, int64_t M, int64_t N, int64_t K,
                        const float *bias, int act, int out_bf16, void *Y, int64_t ldy, float *Ypre, int64_t ldpre,
                        int32_t *top_idx, float *top_val, int topm) {
    using namespace tc;
    if (M < 1 || N < 16 || N % 16 || K < 8 || K % 8 || !tc::encode_fn())
        return set_error(c, GBKM_EUNSUPPORTED, "gemm: shape unsupported by the tcgen05 GEMM");
    const bool topk = top_idx != nullptr;
    if (topk && (topm < 1 || topm > TOPBUF / 2)) return set_error(c, GBKM_EINVAL, "gemm: topm must be in [1, 32]");
    const int extra = topk ? TOPBUF * 128 * 8 : 0;
    const Plan p = plan(F_BF16, K, N, 256, extra);
    CUtensorMap tA, tB;
    if (!make_tmap(&tA, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, A, (uint64_t)K, (uint64_t)M, 2, BM) ||
        !make_tmap(&tB, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, B, (uint64_t)K, (uint64_t)N, 2, (uint32_t)p.bn))
        return set_error(c, GBKM_ECUDA, "cuTensorMapEncodeTiled failed for the GEMM operands");
    Args a{};
    a.n = M, a.d = K, a.k = N, a.k_pad = N;
    a.n_chunks = p.n_chunks, a.bn = p.bn, a.kb = p.kb, a.stages = p.stages, a.tmem_cols = p.tmem_cols;
    a.m_tiles = (int)ceil_div(M, BM);
    a.a_bytes = p.a_bytes, a.b_bytes = p.b_bytes, a.stage_bytes = p.stage_bytes, a.tx_bytes = p.tx_bytes;
    a.idesc = make_idesc(F_BF16, BM, p.bn);
    a.Y = static_cast<float *>(Y), a.ldy = ldy;
    a.bias = bias, a.act = act, a.out_bf16 = out_bf16, a.Ypre = Ypre, a.ldpre = ldpre;
    a.top_idx = top_idx, a.top_val = top_val, a.topm = topm;
    a.status = c->status;
    if (topk) return launch<F_BF16, E_TOPM>(c, tA, tB, tB, a, p);
    return launch<F_BF16, E_STORE>(c, tA, tB, tB, a, p);
}

}  // namespace gbkm
