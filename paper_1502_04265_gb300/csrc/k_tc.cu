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
constexpr uint64_t WAIT_LIMIT_NS = 2000000000ull;  // 2 s per wait unless the context sets another limit
constexpr uint64_t DRAIN_LIMIT_NS = 500000000ull;  // 0.5 s for the copies in flight on the abort path
constexpr int SMEM_BUDGET = 200 * 1024;      // stage ring of the batched kernel
constexpr int MAX_DYN_SMEM = 227 * 1024;     // dynamic shared memory a CTA may use

// F_BF16X2: BF16 points against centers split into two BF16 terms (hi + lo), two MMAs per step
enum Form : int { F_BF16 = 0, F_TF32X3 = 1, F_FP8 = 2, F_TF32 = 3, F_BF16X2 = 4 };
enum Epi : int { E_ARGMIN = 0, E_STORE = 1, E_TOPM = 2, E_TOPG = 3 };
constexpr int TOPBUF = 64;  // per-row candidate buffer of the top-m epilogue (shared memory)
constexpr int TROW = TOPBUF + 1;  // its row stride in floats
// argmin epilogue shared memory: two groups' band lists, the hand-over slots and their barriers
constexpr int ARGMIN_EXTRA_SMEM = 2 * 2 * CAND_MAX * 128 * 4 + 128 * 16 + 8 * 8;

struct Args {
    int64_t n, d, k, k_pad;
    const int32_t *n_dev;  // if set, the rows are the first min(n, *n_dev) (a count on the device)
    const int32_t *row_map;  // if set, outputs of row i go to index row_map[i] (argmin epilogue)
    int n_chunks, bn, kb, stages, tmem_cols, m_tiles;
    uint32_t a_bytes, b_bytes, stage_bytes, tx_bytes;
    uint32_t idesc;
    // 3xTF32 with bn <= 128: the centers' hi and lo tiles are adjacent in the stage, so one MMA of
    // N = 2 bn (instruction descriptor idesc2) gives x.c_hi and x.c_lo side by side in the
    // accumulator, and x_lo.c_hi is added to the first half; the epilogue adds the two halves
    int stack;
    uint32_t idesc2;
    // argmin epilogue
    const float *cnorm, *cscale, *xscale, *xnorm;
    const unsigned *cmax;
    float err_rel, err_abs;
    // one-term BF16 with the operands' actual rounding residuals: ||x_i - bf16(x_i)|| per row and
    // max_j ||c_j - bf16(c_j)|| (null: the worst case u ||x||, u ||c|| in err_rel); acc_g = the FP32
    // accumulation factor d 2^-22, err_u2 = 2u of the score's own FP32 rounding
    const float *xresid;
    const unsigned *emax;
    float acc_g, err_u2;
    // two-term BF16 centers: band width A (D_j + D_0) + Bc with A = pair_a ||x||,
    // Bc = pair_rel ||x|| cmax + pair_abs cmax^2, D = sqrt(XE + s), XE = ||x||^2 + single_rel ||x||
    // cmax + single_abs cmax^2 (pair_a == 0: the constant width 2 (err_rel ||x|| cmax + err_abs cmax^2))
    float pair_a, pair_rel, pair_abs, single_rel, single_abs;
    int32_t *labels;
    float *min_d2;
    int32_t *flag_list;
    int32_t *cand;
    int32_t *flag_count;
    // store epilogue: Y[row, col] = act(acc + bias[col]) in FP32 or BF16; Ypre = acc + bias (FP32)
    float *Y;
    int64_t ldy;
    const float *bias;
    const float *row_w;  // store epilogue: every output row scaled by sqrt(max(row_w[row], 0)) (or null)
    int act;       // 0: none, 1: GELU (erf form)
    int out_bf16;
    float *Ypre;
    int64_t ldpre;
    // bias_mma: the bias enters the accumulator through one more K block per unit (A: the ones
    // operand, tmA2; B: the bias operand, tmB2, columns (bf16(b), bf16(b - bf16(b)), 0, ...)), so the
    // epilogues add none (bias is then null)
    int bias_mma;
    // top-m epilogue: the m largest (acc + bias) of every row, over all N chunks
    int32_t *top_idx;
    float *top_val;
    int topm;
    int *status;
    uint64_t wait_ns;  // limit of every bounded wait (set by launch())
    int stall_loads;   // diagnostics: the producer issues no copy, so the consumers' waits run out
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

// The certified band of one point, tracked by its thread over the score stream: the best score
// v0 with its index i0 (the lowest index on equal scores: centers arrive in increasing order) in
// registers, and every other center whose score was within the band width of the running best when
// it arrived (a former best included, if still that close) in a per-thread list in shared memory
// (slot-major, stride 128).  Entries that fall out of the band as v0 decreases are pruned when the
// list is full; a candidate that finds it full of band members is dropped and only its score is
// kept (dmin, the least dropped score), so the final band {j : s_j <= t(v0)} is complete exactly
// when dmin > t(v0).  A group of W scores costs a minimum tree unless its minimum can enter.
// Band width: a constant Bc (a bound on the error of any score difference), or, for the two-term
// BF16 centers, a bound that grows with the distances, |err(s_j - s_0)| <= A (D_j + D_0) + Bc with
// D the distance bounds sqrt(XE + s); t(v) is the largest s_j that can satisfy it.
template <int CAP>
struct Band {
    float v0, t, dmin, pt;  // pt: the threshold at the last prune (a full list is pruned again
                            // only after the threshold has come down)
    float A, Bc, XE;        // band width parameters (A == 0: constant width Bc)
    int i0, cnt;
    float *lv;
    int32_t *li;
    __device__ __forceinline__ void reset(float bc, float a = 0.f, float xe = 0.f) {
        v0 = t = dmin = pt = __int_as_float(0x7f800000);
        A = a;
        Bc = bc;
        XE = xe;
        i0 = 0;
        cnt = 0;
    }
    // the largest score that can still belong to the band of a best score v
    __device__ __forceinline__ float t_of(float v) const {
        if (A == 0.f) return v + Bc;
        const float d0sq = fmaxf(XE + v, 0.f), d0 = sqrtf(d0sq);
        const float K = d0sq + A * d0 + Bc;
        const float y = 0.5f * (A + sqrtf(fmaf(A, A, 4.f * K)));
        const float w = fmaxf(fmaf(y, y, -d0sq), 0.f);
        // margins for the FP32 evaluation of the bound itself
        return v + w * 1.001f + 1.0e-6f * (d0sq + fabsf(v));
    }
    __device__ __forceinline__ void prune() {
        pt = t;
        int w = 0;
        for (int q = 0; q < cnt; ++q) {
            const float vv = lv[q * 128];
            const int32_t jj = li[q * 128];
            if (vv <= t) {
                lv[w * 128] = vv;
                li[w * 128] = jj;
                ++w;
            }
        }
        cnt = w;
    }
    __device__ __forceinline__ void list_push(float sc, int j) {
        if (cnt == CAP) {
            if (t < pt) prune();
            if (cnt == CAP) {
                dmin = fminf(dmin, sc);
                return;
            }
        }
        lv[cnt * 128] = sc;
        li[cnt * 128] = j;
        ++cnt;
    }
    template <int W>
    __device__ __forceinline__ static float select(const float (&sc)[W], int g) {
        float r = sc[0];
#pragma unroll
        for (int h = 1; h < W; ++h) r = (h == g) ? sc[h] : r;
        return r;
    }
    template <int W>
    __device__ __forceinline__ static float min_tree(const float (&sc)[W]) {
        float m[W / 2];
#pragma unroll
        for (int g = 0; g < W / 2; ++g) m[g] = fminf(sc[2 * g], sc[2 * g + 1]);
#pragma unroll
        for (int w = W / 4; w >= 1; w >>= 1)
#pragma unroll
            for (int g = 0; g < w; ++g) m[g] = fminf(m[2 * g], m[2 * g + 1]);
        return m[0];
    }
    // W scores of centers j0 .. j0 + W - 1 (+inf where there is no center)
    template <int W>
    __device__ __forceinline__ void group(const float (&sc)[W], int j0) {
        const float m = min_tree(sc);
        if (m <= t) {
            // t_of is monotone, so tn < t only when m is a new best
            const float tn = fminf(t, t_of(m));
            uint32_t le = 0;
#pragma unroll
            for (int g = 0; g < W; ++g) le |= (sc[g] <= tn ? 1u : 0u) << g;
            bool found = !(m < v0);
            if (!found && v0 <= tn) list_push(v0, i0);
            t = tn;
            if (!found && (le & (le - 1)) == 0) {
                // a new best that is the group's only member (m <= tn, so the one member is m)
                v0 = m;
                i0 = j0 + __ffs(le) - 1;
                return;
            }
            // the members in index order: the first one equal to a new best m becomes the best
            // (lowest index on ties), the others enter the list
            while (le) {
                const int g = __ffs(le) - 1;
                le &= le - 1;
                const float sg = select(sc, g);
                if (!found && sg == m) {
                    v0 = m;
                    i0 = j0 + g;
                    found = true;
                } else {
                    list_push(sg, j0 + g);
                }
            }
        }
    }
};

// top-m order: larger value first, then lower index; the key is unique per center
__device__ __forceinline__ unsigned long long topm_key(float v, int32_t j) {
    return ((unsigned long long)fkey(v) << 32) | (uint32_t)(~j);
}

// Bitonic sort of 64 keys held two per lane (x at position lane, y at position lane + 32) into
// ascending order across the warp; every lane takes part.
__device__ __forceinline__ void warp_sort64(unsigned long long &x, unsigned long long &y) {
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int k = 2; k <= 64; k <<= 1) {
#pragma unroll
        for (int j = k >> 1; j > 0; j >>= 1) {
            if (j == 32) {
                const unsigned long long lo = min(x, y), hi = max(x, y);
                x = lo;
                y = hi;
            } else {
                const unsigned long long ox = __shfl_xor_sync(0xffffffffu, x, j);
                const unsigned long long oy = __shfl_xor_sync(0xffffffffu, y, j);
                const bool lower = (lane & j) == 0;
                const bool upx = (lane & k) == 0, upy = ((lane + 32) & k) == 0;
                x = (lower == upx) ? min(x, ox) : max(x, ox);
                y = (lower == upy) ? min(y, oy) : max(y, oy);
            }
        }
    }
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
// limit_ns, in which case it raises the flag itself.  Returns false when it gave up.
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity, volatile int *abort_flag,
                                          uint64_t limit_ns) {
    if (mbar_try_wait(bar, parity)) return true;
    const uint64_t t0 = globaltimer_ns();
    for (uint32_t it = 1;; ++it) {
        if (mbar_try_wait(bar, parity)) return true;
        // the clock and the abort flag after 1, 2, 4, ... 32 polls, then every 64
        if ((it & (it - 1)) == 0 || (it & 63) == 0) {
            if (*abort_flag) return false;
            if (globaltimer_ns() - t0 > limit_ns) {
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
    if constexpr (FORM == F_BF16 || FORM == F_BF16X2) {
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
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, uint32_t (&r)[32]) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, "
        "%14, %15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
          "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
          "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr)
        : "memory");
}
__device__ __forceinline__ void tmem_wait_ld(uint32_t (&r)[32]) {
    asm volatile("tcgen05.wait::ld.sync.aligned;"
                 : "+r"(r[0]), "+r"(r[1]), "+r"(r[2]), "+r"(r[3]), "+r"(r[4]), "+r"(r[5]), "+r"(r[6]), "+r"(r[7]),
                   "+r"(r[8]), "+r"(r[9]), "+r"(r[10]), "+r"(r[11]), "+r"(r[12]), "+r"(r[13]), "+r"(r[14]),
                   "+r"(r[15]), "+r"(r[16]), "+r"(r[17]), "+r"(r[18]), "+r"(r[19]), "+r"(r[20]), "+r"(r[21]),
                   "+r"(r[22]), "+r"(r[23]), "+r"(r[24]), "+r"(r[25]), "+r"(r[26]), "+r"(r[27]), "+r"(r[28]),
                   "+r"(r[29]), "+r"(r[30]), "+r"(r[31])
                 :
                 : "memory");
}
// the first 16 columns of a 32-register buffer (the 16-column tail of a column range)
__device__ __forceinline__ void tmem_ld16_into32(uint32_t taddr, uint32_t (&r)[32]) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, "
        "%14, %15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr)
        : "memory");
}
// 16 columns into the upper half of a 32-register buffer (the second half of a stacked accumulator)
__device__ __forceinline__ void tmem_ld16_upper(uint32_t taddr, uint32_t (&r)[32]) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, "
        "%14, %15}, [%16];"
        : "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
          "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
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
// epilogue warpgroups of a k_tc instance: two (each takes half of every chunk's columns) except for
// the top-m epilogues, whose per-row buffers leave room for one
template <int EPI>
constexpr int epi_groups() {
    return (EPI == E_TOPM || EPI == E_TOPG) ? 1 : 2;
}
template <int FORM, int EPI>
constexpr int tc_threads() {
    return FORM == F_TF32X3 ? (epi_groups<EPI>() == 2 ? 512 : 384) : (epi_groups<EPI>() == 2 ? 384 : 256);
}

template <int FORM, int EPI>
__global__ void __launch_bounds__(tc_threads<FORM, EPI>(), 1)
    k_tc(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB,
         const __grid_constant__ CUtensorMap tmB2, const __grid_constant__ CUtensorMap tmA2, const Args a) {
    constexpr bool X3 = (FORM == F_TF32X3);
    constexpr bool TWO_B = X3 || FORM == F_BF16X2;  // a second center operand (lo part)
    constexpr int NG = epi_groups<EPI>();
    extern __shared__ uint8_t smem_raw[];
    // 1024-byte aligned stage base, derived by pointer arithmetic on the shared array so that
    // accesses through it stay shared-memory accesses
    uint8_t *base = smem_raw + ((1024u - (smem_u32(smem_raw) & 1023u)) & 1023u);
    uint64_t *bars = reinterpret_cast<uint64_t *>(base + (size_t)a.stages * a.stage_bytes);
    uint64_t *full = bars, *tfull = bars + MAX_STAGES, *empty = bars + 2 * MAX_STAGES;
    uint64_t *accf = bars + 3 * MAX_STAGES, *acce = accf + 2;
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(acce + 2);
    volatile int *abort_flag = reinterpret_cast<volatile int *>(tmem_slot + 1);

    {
        // a CTA with no tile (the row count may come from the device) leaves before allocating
        const int64_t nr = a.n_dev ? min(a.n, (int64_t)max(0, *a.n_dev)) : a.n;
        if ((int64_t)blockIdx.x * BM >= nr) return;
    }
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (threadIdx.x == 0) {
        for (int s = 0; s < a.stages; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&tfull[s], 4);
            mbar_init(&empty[s], 1);
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(&accf[b], 1);
            mbar_init(&acce[b], 4 * NG);
        }
        if constexpr (EPI == E_ARGMIN && NG == 2) {
            // hand-over of group 1's half of every point's band to group 0 (one pair per lane quarter)
            uint64_t *xfull = reinterpret_cast<uint64_t *>(base + (size_t)a.stages * a.stage_bytes + 1024 +
                                                           NG * 2 * CAND_MAX * 128 * 4 + 128 * 16);
            for (int i = 0; i < 8; ++i) mbar_init(&xfull[i], 1);
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
    // rows of this launch: n, or a count produced on the device by an earlier kernel
    const int64_t n_rows = a.n_dev ? min(a.n, (int64_t)max(0, *a.n_dev)) : a.n;
    const int m_tiles = (int)((n_rows + BM - 1) / BM);

    if (warp == 0) {
        // ------------------------------------------------ TMA producer
        if (lane == 0) {
            int s = 0;
            uint32_t ph = 0;
            uint32_t issued = 0, last_par = 0;  // per-stage: issued bit, parity of the last issue
            if (a.stall_loads) goto producer_done;
            for (int tile = blockIdx.x; tile < m_tiles && !*abort_flag; tile += gridDim.x) {
                for (int nc = 0; nc < units_per_tile; ++nc) {
                    for (int kb = 0; kb < a.kb; ++kb) {
                        if (!mbar_wait(&empty[s], ph ^ 1, abort_flag, a.wait_ns)) goto producer_done;
                        uint8_t *st = base + (size_t)s * a.stage_bytes;
                        mbar_expect_tx(&full[s], a.tx_bytes);
                        const int32_t kx =
                            kb * (int32_t)(128 / ((FORM == F_BF16 || FORM == F_BF16X2) ? 2 : (FORM == F_FP8 ? 1 : 4)));
                        tma_load_2d(st, &tmA, &full[s], kx, tile * BM);
                        uint8_t *bdst = st + (X3 ? 2 : 1) * a.a_bytes;
                        tma_load_2d(bdst, &tmB, &full[s], kx, nc * a.bn);
                        if constexpr (TWO_B) tma_load_2d(bdst + a.b_bytes, &tmB2, &full[s], kx, nc * a.bn);
                        issued |= 1u << s;
                        last_par = (last_par & ~(1u << s)) | (ph << s);
                        if (++s == a.stages) {
                            s = 0;
                            ph ^= 1;
                        }
                    }
                    if constexpr (FORM == F_BF16) {
                        if (a.bias_mma) {
                            // the bias block: the ones operand (the same tile for every row tile) and
                            // this chunk's rows of the bias operand
                            if (!mbar_wait(&empty[s], ph ^ 1, abort_flag, a.wait_ns)) goto producer_done;
                            uint8_t *st = base + (size_t)s * a.stage_bytes;
                            mbar_expect_tx(&full[s], a.tx_bytes);
                            tma_load_2d(st, &tmA2, &full[s], 0, 0);
                            tma_load_2d(st + a.a_bytes, &tmB2, &full[s], 0, nc * a.bn);
                            issued |= 1u << s;
                            last_par = (last_par & ~(1u << s)) | (ph << s);
                            if (++s == a.stages) {
                                s = 0;
                                ph ^= 1;
                            }
                        }
                    }
                }
            }
        producer_done:
            if (*abort_flag) {
                // let every bulk copy still in flight land before the CTA exits
                for (int q = 0; q < a.stages; ++q)
                    if (issued & (1u << q)) mbar_drain(&full[q], (last_par >> q) & 1, DRAIN_LIMIT_NS);
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
            for (int tile = blockIdx.x; tile < m_tiles && !*abort_flag; tile += gridDim.x) {
                for (int nc = 0; nc < units_per_tile; ++nc) {
                    if (!mbar_wait(&acce[ab], aph ^ 1, abort_flag, a.wait_ns)) goto mma_done;
                    tc_fence_after();
                    const uint32_t d_tmem = tmem_base + (uint32_t)(ab * bn_alloc);
                    for (int kb = 0; kb < a.kb; ++kb) {
                        // 3xTF32: the products of the staged tile itself (x.c_hi and x.c_lo) need only the
                        // copies, so they are issued first and the split's low part overlaps them
                        if (!mbar_wait(&full[s], ph, abort_flag, a.wait_ns)) goto mma_done;
                        tc_fence_after();
                        uint8_t *st = base + (size_t)s * a.stage_bytes;
                        const uint64_t adesc = sw128_desc(st);
                        const uint64_t bdesc = sw128_desc(st + (X3 ? 2 : 1) * a.a_bytes);
                        if constexpr (X3) {
                            const uint64_t blo = sw128_desc(st + 2 * a.a_bytes + a.b_bytes);
#pragma unroll
                            for (int kk = 0; kk < 4; ++kk) {
                                const uint32_t acc = (kb > 0 || kk > 0) ? 1u : 0u;
                                const uint64_t off = (uint64_t)(kk * 2);  // 32 bytes per MMA step
                                if (a.stack) {
                                    tc_mma<FORM>(d_tmem, adesc + off, bdesc + off, a.idesc2, acc);
                                } else {
                                    tc_mma<FORM>(d_tmem, adesc + off, blo + off, a.idesc, acc);
                                    tc_mma<FORM>(d_tmem, adesc + off, bdesc + off, a.idesc, 1u);
                                }
                            }
                            if (!mbar_wait(&tfull[s], ph, abort_flag, a.wait_ns)) {
                                // the products above are in flight: commit them so the abort path drains them
                                tc_commit(&empty[s]);
                                committed = true;
                                last_bar = &empty[s];
                                last_parity = ph;
                                goto mma_done;
                            }
                            tc_fence_after();
                            const uint64_t alo = sw128_desc(st + a.a_bytes);
#pragma unroll
                            for (int kk = 0; kk < 4; ++kk)
                                tc_mma<FORM>(d_tmem, alo + (uint64_t)(kk * 2), bdesc + (uint64_t)(kk * 2), a.idesc, 1u);
                        }
#pragma unroll
                        for (int kk = 0; kk < 4; ++kk) {
                            const uint32_t acc = (kb > 0 || kk > 0) ? 1u : 0u;
                            const uint64_t off = (uint64_t)(kk * 2);  // 32 bytes per MMA step
                            if constexpr (X3) {
                                (void)acc;  // issued above
                            } else if constexpr (FORM == F_BF16X2) {
                                const uint64_t blo = sw128_desc(st + a.a_bytes + a.b_bytes);
                                tc_mma<FORM>(d_tmem, adesc + off, bdesc + off, a.idesc, acc);
                                tc_mma<FORM>(d_tmem, adesc + off, blo + off, a.idesc, 1u);
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
                    if constexpr (FORM == F_BF16) {
                        if (a.bias_mma) {
                            // one K = 16 step: ones x (bias head, bias tail, 0 ...) adds the bias
                            if (!mbar_wait(&full[s], ph, abort_flag, a.wait_ns)) goto mma_done;
                            tc_fence_after();
                            uint8_t *st = base + (size_t)s * a.stage_bytes;
                            tc_mma<FORM>(d_tmem, sw128_desc(st), sw128_desc(st + a.a_bytes), a.idesc, 1u);
                            tc_commit(&empty[s]);
                            last_bar = &empty[s];
                            last_parity = ph;
                            if (++s == a.stages) {
                                s = 0;
                                ph ^= 1;
                            }
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
            if (*abort_flag && committed && last_bar) mbar_drain(last_bar, last_parity, DRAIN_LIMIT_NS);
        }
    } else if (X3 && warp >= 8 && warp < 12) {
        // ------------------------------------------------ 3xTF32 split of the staged X tile: only the low
        // part is written; the tensor cores read the staged FP32 tile itself as the high part (kind::tf32
        // takes the top 19 bits of an FP32 operand, the same truncation as the mask here)
        const int t = threadIdx.x - 256;  // 0..127
        int s = 0;
        uint32_t ph = 0;
        for (int tile = blockIdx.x; tile < m_tiles && !*abort_flag; tile += gridDim.x) {
            for (int nc = 0; nc < units_per_tile; ++nc) {
                for (int kb = 0; kb < a.kb; ++kb) {
                    if (!mbar_wait(&full[s], ph, abort_flag, a.wait_ns)) goto split_done;
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
    } else if (warp >= 4 && (warp < 8 || (NG == 2 && warp >= (X3 ? 12 : 8)))) {
        // ------------------------------------------------ epilogue: one TMEM lane = one point
        const int q = warp & 3;             // TMEM lane quarter of this warp
        const int eg = warp < 8 ? 0 : 1;    // epilogue group: which half of every chunk's columns
        const int g16 = a.bn / 16, h16 = (g16 + NG - 1) / NG;
        const int c_begin = eg * h16 * 16, c_end = min(a.bn, (eg + 1) * h16 * 16);
        int ab = 0;
        uint32_t aph = 0, xph = 0;
        const float cm = (EPI == E_ARGMIN) ? __uint_as_float(*a.cmax) : 0.f;
        const float em = (EPI == E_ARGMIN && FORM == F_BF16 && a.xresid) ? __uint_as_float(*a.emax) : 0.f;
        uint8_t *ex = base + (size_t)a.stages * a.stage_bytes + 1024;  // epilogue shared memory
        for (int tile = blockIdx.x; tile < m_tiles && !*abort_flag; tile += gridDim.x) {
            const int64_t row = (int64_t)tile * BM + q * 32 + lane;
            const bool valid = row < n_rows;
            float sx = 1.f;
            if (EPI == E_ARGMIN && FORM == F_FP8 && valid) sx = a.xscale[row];
            // argmin state: the certified band of this point (its width bounds the error of a score
            // difference)
            const float xn = (EPI == E_ARGMIN && valid) ? a.xnorm[row] : 0.f;
            Band<CAND_MAX> band;
            {
                const float xr = sqrtf(fmaxf(xn, 0.f)) * (1.f + 1.0e-6f);
                if (a.pair_a > 0.f) {
                    // |2 dx.(c_j - c_0)| <= 2 ||dx|| (D_j + D_0): with the row's actual rounding residual
                    // ||dx|| (rounded up) when the quantiser gave it, else its bound u ||x||
                    const float A = a.xresid ? 2.f * (valid ? a.xresid[row] : 0.f) * (1.f + 1.0e-6f) : a.pair_a * xr;
                    band.reset(a.pair_rel * xr * cm + a.pair_abs * cm * cm, A,
                               xn * (1.f + 2.4e-7f) + a.single_rel * xr * cm + a.single_abs * cm * cm);
                } else if (FORM == F_BF16 && a.xresid) {
                    // with dx = x~ - x and e_j = c~_j - c_j: |x~.c~_j - x.c_j| <= ||dx|| (cmax + emax) +
                    // ||x|| emax (Cauchy-Schwarz), plus the FP32 accumulation of d products,
                    // d 2^-22 (||x|| + ||dx||)(cmax + emax); a score difference takes two of these
                    const float dr = valid ? a.xresid[row] : 0.f, ce = cm + em;
                    const float e1 = 2.f * (dr * ce + xr * em + a.acc_g * (xr + dr) * ce) + a.err_u2 * xr * cm +
                                     a.err_abs * cm * cm;
                    band.reset(2.f * e1 * (1.f + 1.0e-3f));
                } else {
                    band.reset(2.f * (a.err_rel * xr * cm + a.err_abs * cm * cm));
                }
                band.lv = reinterpret_cast<float *>(ex) + eg * (2 * CAND_MAX * 128) + q * 32 + lane;
                band.li = reinterpret_cast<int32_t *>(band.lv + CAND_MAX * 128);
            }
            // top-m state: the value a candidate must beat and this row's buffer (row-major, TROW
            // entries per row so that a warp reading one row's entries hits distinct banks)
            float tau = -__int_as_float(0x7f800000);
            int tcnt = 0;
            float *tbv_all = reinterpret_cast<float *>(ex);
            int32_t *tbi_all = reinterpret_cast<int32_t *>(tbv_all + TROW * 128);
            float *tbv = tbv_all + (q * 32 + lane) * TROW;
            int32_t *tbi = tbi_all + (q * 32 + lane) * TROW;
            // warp-cooperative: lane L's full buffer is cut to its topm best (rank order) and its
            // threshold becomes the topm-th best value
            auto compact = [&](int L) {
                float *rv = tbv_all + (q * 32 + L) * TROW;
                int32_t *ri = tbi_all + (q * 32 + L) * TROW;
                const int lc = __shfl_sync(0xffffffffu, tcnt, L);
                unsigned long long x = lane < lc ? topm_key(rv[lane], ri[lane]) : 0ull;
                unsigned long long y = lane + 32 < lc ? topm_key(rv[lane + 32], ri[lane + 32]) : 0ull;
                warp_sort64(x, y);
                const int rk = 31 - lane;  // the rank of y (0 = best)
                if (rk < a.topm) {
                    rv[rk] = fkey_inv((uint32_t)(y >> 32));
                    ri[rk] = ~(int32_t)(uint32_t)y;
                }
                const unsigned long long tk = __shfl_sync(0xffffffffu, y, 32 - a.topm);
                __syncwarp();
                if (lane == L) {
                    tcnt = a.topm;
                    tau = fkey_inv((uint32_t)(tk >> 32));
                }
            };
            if constexpr (EPI == E_ARGMIN && NG == 2) {
                // group 1 reuses its band list only after group 0 has merged the previous point's
                if (eg == 1) {
                    uint64_t *xempty = reinterpret_cast<uint64_t *>(ex + NG * 2 * CAND_MAX * 128 * 4 + 128 * 16) + 4;
                    if (!mbar_wait(&xempty[q], xph ^ 1, abort_flag, a.wait_ns)) goto epi_done;
                }
            }
            for (int nc = 0; nc < units_per_tile; ++nc) {
                if (!mbar_wait(&accf[ab], aph, abort_flag, a.wait_ns)) goto epi_done;
                tc_fence_after();
                const uint32_t tbase = tmem_base + ((uint32_t)(q * 32) << 16) + (uint32_t)(ab * bn_alloc);
                // W accumulator columns starting at chunk column c
                auto process = [&](const auto &r, int c) {
                    constexpr int W = sizeof(r) / sizeof(uint32_t);
                    const int64_t j0 = (int64_t)nc * a.bn + c;
                    if constexpr (EPI == E_ARGMIN) {
                        if (j0 >= a.k) return;
                        float cn[W], sc[W];
                        if (j0 + W <= a.k_pad) {
#pragma unroll
                            for (int g = 0; g < W / 4; ++g) {
                                const float4 t4 = __ldg(reinterpret_cast<const float4 *>(a.cnorm + j0) + g);
                                cn[4 * g] = t4.x, cn[4 * g + 1] = t4.y, cn[4 * g + 2] = t4.z, cn[4 * g + 3] = t4.w;
                            }
                        } else {
#pragma unroll
                            for (int g = 0; g < W; ++g)
                                cn[g] = (j0 + g < a.k_pad) ? a.cnorm[j0 + g] : __int_as_float(0x7f800000);
                        }
                        float ms[W];
#pragma unroll
                        for (int g = 0; g < W; ++g) ms[g] = -2.f;
                        if constexpr (FORM == F_FP8) {
                            // E4M3 scores carry the point's and the center's scales
                            if (j0 + W <= a.k_pad) {
#pragma unroll
                                for (int g = 0; g < W / 4; ++g) {
                                    const float4 t4 = __ldg(reinterpret_cast<const float4 *>(a.cscale + j0) + g);
                                    ms[4 * g] = -2.f * sx * t4.x, ms[4 * g + 1] = -2.f * sx * t4.y;
                                    ms[4 * g + 2] = -2.f * sx * t4.z, ms[4 * g + 3] = -2.f * sx * t4.w;
                                }
                            } else {
#pragma unroll
                                for (int g = 0; g < W; ++g) ms[g] = (j0 + g < a.k_pad) ? -2.f * sx * a.cscale[j0 + g] : -2.f;
                            }
                        }
                        if (j0 + W <= a.k) {
#pragma unroll
                            for (int g = 0; g < W; ++g) sc[g] = fmaf(ms[g], __uint_as_float(r[g]), cn[g]);
                        } else {
                            const int kr = (int)(a.k - j0);  // real centers in this unit (< W)
#pragma unroll
                            for (int g = 0; g < W; ++g)
                                sc[g] = g < kr ? fmaf(ms[g], __uint_as_float(r[g]), cn[g]) : __int_as_float(0x7f800000);
                        }
                        band.group(sc, (int)j0);
                    } else if constexpr (EPI == E_STORE) {
                        if (valid && j0 < a.k) {
#pragma unroll
                            for (int h = 0; h < W / 16; ++h) {
                                const int64_t col0 = j0 + 16 * h;
                                if (col0 >= a.k) break;
                                float v[16];
#pragma unroll
                                for (int g = 0; g < 16; ++g) v[g] = __uint_as_float(r[16 * h + g]);
                                if (a.row_w) {
                                    const float sc = sqrtf(fmaxf(a.row_w[row], 0.f));
#pragma unroll
                                    for (int g = 0; g < 16; ++g) v[g] *= sc;
                                }
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
                                    for (int g = 0; g < 4; ++g)
                                        pr[g] = make_float4(v[4 * g], v[4 * g + 1], v[4 * g + 2], v[4 * g + 3]);
                                }
                                if (a.act == 1) {
#pragma unroll
                                    for (int g = 0; g < 16; ++g) v[g] = gelu_erf(v[g]);
                                }
                                if (a.out_bf16) {
                                    uint32_t w[8];
#pragma unroll
                                    for (int g = 0; g < 8; ++g) {
                                        __nv_bfloat162 hh = __floats2bfloat162_rn(v[2 * g], v[2 * g + 1]);
                                        w[g] = *reinterpret_cast<uint32_t *>(&hh);
                                    }
                                    uint4 *yr = reinterpret_cast<uint4 *>(reinterpret_cast<__nv_bfloat16 *>(a.Y) +
                                                                          row * a.ldy + col0);
                                    yr[0] = make_uint4(w[0], w[1], w[2], w[3]);
                                    yr[1] = make_uint4(w[4], w[5], w[6], w[7]);
                                } else {
                                    float4 *yr = reinterpret_cast<float4 *>(a.Y + row * a.ldy + col0);
#pragma unroll
                                    for (int g = 0; g < 4; ++g)
                                        yr[g] = make_float4(v[4 * g], v[4 * g + 1], v[4 * g + 2], v[4 * g + 3]);
                                }
                            }
                        }
                    } else if constexpr (EPI == E_TOPG) {
                        // grouped proposal: each aligned group of 16 centers offers its best one (lowest
                        // index on equal logits); at most one append per row and group
                        if (j0 >= a.k) return;
                        const int jc = (int)j0;
                        float sv[W];
#pragma unroll
                        for (int g = 0; g < W; ++g) sv[g] = __uint_as_float(r[g]);
                        if (a.bias) {
#pragma unroll
                            for (int g = 0; g < W / 4; ++g) {
                                if (4 * g >= 16 && jc + 16 >= (int)a.k) break;
                                const float4 b4 = __ldg(reinterpret_cast<const float4 *>(a.bias + jc) + g);
                                sv[4 * g] += b4.x, sv[4 * g + 1] += b4.y, sv[4 * g + 2] += b4.z, sv[4 * g + 3] += b4.w;
                            }
                        }
                        if (j0 + W > a.k) {
#pragma unroll
                            for (int g = 0; g < W; ++g)
                                if (jc + g >= (int)a.k) sv[g] = -__int_as_float(0x7f800000);
                        }
                        // a row whose buffer lacks room for this unit's offers is cut first
                        uint32_t fullm = __ballot_sync(0xffffffffu, tcnt > TOPBUF - W / 16);
                        while (fullm) {
                            const int L = __ffs(fullm) - 1;
                            fullm &= fullm - 1;
                            compact(L);
                        }
                        // per group: its maximum and the lowest index holding it (the first quad whose
                        // maximum equals it, then the first entry of that quad), then a branch-free
                        // append: the entry is written at the buffer's end and kept if it beats tau
#pragma unroll
                        for (int h = 0; h < W / 16; ++h) {
                            const float *u = sv + 16 * h;
                            float mq[4];
#pragma unroll
                            for (int t = 0; t < 4; ++t)
                                mq[t] = fmaxf(fmaxf(u[4 * t], u[4 * t + 1]), fmaxf(u[4 * t + 2], u[4 * t + 3]));
                            const float gm = fmaxf(fmaxf(mq[0], mq[1]), fmaxf(mq[2], mq[3]));
                            const int qt = mq[0] == gm ? 0 : (mq[1] == gm ? 1 : (mq[2] == gm ? 2 : 3));
                            float e0 = u[0], e1 = u[1], e2 = u[2];
#pragma unroll
                            for (int t = 1; t < 4; ++t)
                                if (qt == t) e0 = u[4 * t], e1 = u[4 * t + 1], e2 = u[4 * t + 2];
                            const int et = e0 == gm ? 0 : (e1 == gm ? 1 : (e2 == gm ? 2 : 3));
                            tbv[tcnt] = gm;
                            tbi[tcnt] = jc + 16 * h + 4 * qt + et;
                            tcnt += gm > tau ? 1 : 0;
                        }
                    } else {
                        // exact top-m: candidates above the row's threshold go to its buffer; a group of
                        // 16 costs 16 compares unless some lane of the warp has a candidate in it
                        if (j0 >= a.k) return;
                        const int jc = (int)j0;
#pragma unroll
                        for (int h = 0; h < W / 16; ++h) {
                            const int col0 = jc + 16 * h;
                            if (col0 >= (int)a.k) break;
                            float sv[16];
#pragma unroll
                            for (int g = 0; g < 16; ++g) sv[g] = __uint_as_float(r[16 * h + g]);
                            if (a.bias) {
#pragma unroll
                                for (int g = 0; g < 4; ++g) {
                                    const float4 b4 = __ldg(reinterpret_cast<const float4 *>(a.bias + col0) + g);
                                    sv[4 * g] += b4.x, sv[4 * g + 1] += b4.y, sv[4 * g + 2] += b4.z, sv[4 * g + 3] += b4.w;
                                }
                            }
                            if (col0 + 16 > (int)a.k) {
#pragma unroll
                                for (int g = 0; g < 16; ++g)
                                    if (col0 + g >= (int)a.k) sv[g] = -__int_as_float(0x7f800000);
                            }
                            uint32_t msk = 0;
#pragma unroll
                            for (int g = 0; g < 16; ++g) msk |= (sv[g] > tau ? 1u : 0u) << g;
                            uint32_t any = __reduce_or_sync(0xffffffffu, msk);
                            while (any) {
                                const int g = __ffs(any) - 1;
                                any &= any - 1;
                                const float sg = Band<1>::select(sv, g);
                                const bool want = (msk >> g) & 1u;
                                uint32_t fullm = __ballot_sync(0xffffffffu, want && sg > tau && tcnt == TOPBUF);
                                while (fullm) {
                                    const int L = __ffs(fullm) - 1;
                                    fullm &= fullm - 1;
                                    compact(L);
                                }
                                if (want && sg > tau) {
                                    tbv[tcnt] = sg;
                                    tbi[tcnt] = col0 + g;
                                    ++tcnt;
                                }
                            }
                        }
                    }
                };
                // this group's columns in units of 32 (a 16-column tail), the next unit's TMEM load
                // in flight while the current one is processed
                {
                    uint32_t ra[32], rb[32];
                    int c = c_begin;
                    // 32-column units, except 16 for 3xTF32 (its 512-thread CTA leaves 128 registers)
                    constexpr int UW = X3 ? 16 : 32;
                    // (the grouped top-m epilogue runs on chunk widths that are multiples of 32)
                    constexpr bool ONLY32 = EPI == E_TOPG;
                    auto load = [&](uint32_t (&r)[32], int cc) {
                        if (ONLY32 || (UW == 32 && c_end - cc >= 32)) {
                            tmem_ld32(tbase + (uint32_t)cc, r);
                        } else {
                            tmem_ld16_into32(tbase + (uint32_t)cc, r);
                            if (X3 && a.stack) tmem_ld16_upper(tbase + (uint32_t)(a.bn + cc), r);
                        }
                    };
                    auto run = [&](const uint32_t (&r)[32], int cc) {
                        if constexpr (ONLY32) {
                            process(r, cc);
                        } else if (X3 && a.stack) {
                            uint32_t s16[16];
#pragma unroll
                            for (int g = 0; g < 16; ++g)
                                s16[g] = __float_as_uint(__fadd_rn(__uint_as_float(r[g]), __uint_as_float(r[16 + g])));
                            process(s16, cc);
                        } else {
                            if (UW == 32 && c_end - cc >= 32) {
                                process(r, cc);
                            } else {
                                const uint32_t(&r16)[16] = *reinterpret_cast<const uint32_t(*)[16]>(&r[0]);
                                process(r16, cc);
                            }
                        }
                    };
                    if (c < c_end) {
                        load(ra, c);
                        tmem_wait_ld(ra);
                    }
                    while (c < c_end) {
                        const int c1 = c + min(UW, c_end - c);
                        if (c1 < c_end) load(rb, c1);
                        run(ra, c);
                        if (c1 >= c_end) break;
                        tmem_wait_ld(rb);
                        const int c2 = c1 + min(UW, c_end - c1);
                        if (c2 < c_end) load(ra, c2);
                        run(rb, c1);
                        if (c2 >= c_end) break;
                        tmem_wait_ld(ra);
                        c = c2;
                    }
                }
                // the accumulator is free once both groups have read their columns
                tc_fence_before();
                __syncwarp();
                if (lane == 0) mbar_arrive(&acce[ab]);
                if (++ab == 2) {
                    ab = 0;
                    aph ^= 1;
                }
                if constexpr (EPI == E_ARGMIN) {
                    if (nc == units_per_tile - 1) {
                        // group 1 hands its half of the point's band to group 0 through shared memory
                        float4 *xch = reinterpret_cast<float4 *>(ex + NG * 2 * CAND_MAX * 128 * 4);
                        uint64_t *xfull = reinterpret_cast<uint64_t *>(xch + 128), *xempty = xfull + 4;
                        band.prune();
                        if (NG == 2 && eg == 1) {
                            xch[q * 32 + lane] = make_float4(band.v0, __int_as_float(band.i0), __int_as_float(band.cnt),
                                                             band.dmin);
                            __syncwarp();
                            if (lane == 0) mbar_arrive(&xfull[q]);
                            xph ^= 1;
                        } else {
                            float vA = band.v0, vB = __int_as_float(0x7f800000), dB = vB;
                            int iA = band.i0, iB = 0, cB = 0;
                            const float *lvB = band.lv + 2 * CAND_MAX * 128;
                            const int32_t *liB = band.li + 2 * CAND_MAX * 128;
                            if (NG == 2) {
                                if (!mbar_wait(&xfull[q], xph, abort_flag, a.wait_ns)) goto epi_done;
                                const float4 o = xch[q * 32 + lane];
                                vB = o.x, iB = __float_as_int(o.y), cB = __float_as_int(o.z), dB = o.w;
                            }
                            const bool takeB = vB < vA || (vB == vA && iB < iA);
                            const float v = takeB ? vB : vA, vl = takeB ? vA : vB;
                            const int ib = takeB ? iB : iA, il = takeB ? iA : iB;
                            const float t = band.t_of(v);
                            // the band: the best, every listed center within the band width of it,
                            // the other group's best if that close; complete unless something was dropped
                            int cnt = 1 + (vl <= t ? 1 : 0);
                            for (int e = 0; e < band.cnt; ++e) cnt += band.lv[e * 128] <= t ? 1 : 0;
                            for (int e = 0; e < cB; ++e) cnt += lvB[e * 128] <= t ? 1 : 0;
                            const bool over = !(v < __int_as_float(0x7f800000)) || band.dmin <= t || dB <= t ||
                                              cnt > CAND_MAX;
                            const int bc = over ? -1 : cnt;
                            const bool flag = valid && bc != 1;
                            if (valid) {
                                const int64_t dst = a.row_map ? (int64_t)a.row_map[row] : row;
                                a.labels[dst] = ib;
                                if (a.min_d2) a.min_d2[dst] = fmaxf(0.f, xn + v);
                            }
                            if (a.flag_list) {
                                const unsigned m = __ballot_sync(0xffffffffu, flag);
                                if (m) {
                                    const int leader = __ffs(m) - 1;
                                    int b0 = 0;
                                    if (lane == leader) b0 = atomicAdd(a.flag_count, __popc(m));
                                    b0 = __shfl_sync(0xffffffffu, b0, leader);
                                    if (flag) {
                                        const int slot = b0 + __popc(m & lanemask_lt());
                                        a.flag_list[slot] = (int32_t)row;
                                        // the band's centers (the best first), or -1: scan all centers
                                        int32_t *cf = a.cand + (int64_t)slot * CAND_STRIDE;
                                        cf[0] = bc;
                                        if (bc > 0) {
                                            int w = 1;
                                            cf[w++] = ib;
                                            if (vl <= t) cf[w++] = il;
                                            for (int e = 0; e < band.cnt; ++e)
                                                if (band.lv[e * 128] <= t) cf[w++] = band.li[e * 128];
                                            for (int e = 0; e < cB; ++e)
                                                if (lvB[e * 128] <= t) cf[w++] = liB[e * 128];
                                        }
                                    }
                                }
                            }
                            if (NG == 2) {
                                __syncwarp();
                                if (lane == 0) mbar_arrive(&xempty[q]);
                                xph ^= 1;
                            }
                        }
                    }
                }
            }
            if constexpr (EPI == E_TOPM || EPI == E_TOPG) {
                // every row of the warp in turn: its m best in rank order, -1 padding
                for (int L = 0; L < 32; ++L) {
                    const int64_t rowL = (int64_t)tile * BM + q * 32 + L;
                    const float *rv = tbv_all + (q * 32 + L) * TROW;
                    const int32_t *ri = tbi_all + (q * 32 + L) * TROW;
                    const int lc = __shfl_sync(0xffffffffu, tcnt, L);
                    unsigned long long x = lane < lc ? topm_key(rv[lane], ri[lane]) : 0ull;
                    unsigned long long y = lane + 32 < lc ? topm_key(rv[lane + 32], ri[lane + 32]) : 0ull;
                    warp_sort64(x, y);
                    const int rk = 31 - lane;
                    if (rowL < n_rows && rk < a.topm) {
                        a.top_idx[rowL * a.topm + rk] = y ? ~(int32_t)(uint32_t)y : -1;
                        if (a.top_val)
                            a.top_val[rowL * a.topm + rk] = y ? fkey_inv((uint32_t)(y >> 32)) : -__int_as_float(0x7f800000);
                    }
                    __syncwarp();
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
          uint32_t stage_bytes, int32_t *__restrict__ flags, int32_t *__restrict__ flag_count, int *status,
          uint64_t wait_ns) {
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
                        if (!mbar_wait(&empty[st], ph ^ 1, abort_flag, wait_ns)) goto producer_done;
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
                    if (issued & (1u << q)) mbar_drain(&full[q], (last_par >> q) & 1, DRAIN_LIMIT_NS);
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
                    if (!mbar_wait(&acce[ab], aph ^ 1, abort_flag, wait_ns)) goto mma_done;
                    tc_fence_after();
                    const uint32_t d_tmem = tmem_base + (uint32_t)(ab * BN_ALLOC);
                    for (int kb = 0; kb < P.kb; ++kb) {
                        // 3xTF32: the two products of the staged tile itself go first, the split's low part after
                        if (!mbar_wait(&full[st], ph, abort_flag, wait_ns)) goto mma_done;
                        tc_fence_after();
                        uint8_t *sb = base + (size_t)st * stage_bytes;
                        const uint64_t adesc = sw128_desc(sb);
                        const uint64_t bdesc = sw128_desc(sb + (X3 ? 2 : 1) * a_bytes);
#pragma unroll
                        for (int kk = 0; kk < 4; ++kk) {
                            const uint32_t acc = (kb > 0 || kk > 0) ? 1u : 0u;
                            const uint64_t off = (uint64_t)(kk * 2);
                            if constexpr (X3) {
                                const uint64_t blo = sw128_desc(sb + 2 * a_bytes + b_bytes);
                                tc_mma<FORM>(d_tmem, adesc + off, blo + off, P.idesc, acc);
                                tc_mma<FORM>(d_tmem, adesc + off, bdesc + off, P.idesc, 1u);
                            } else {
                                tc_mma<FORM>(d_tmem, adesc + off, bdesc + off, P.idesc, acc);
                            }
                        }
                        if constexpr (X3) {
                            if (!mbar_wait(&tfull[st], ph, abort_flag, wait_ns)) {
                                // the products above are in flight: commit them so the abort path drains them
                                tc_commit(&empty[st]);
                                last_bar = &empty[st];
                                last_parity = ph;
                                goto mma_done;
                            }
                            tc_fence_after();
                            const uint64_t alo = sw128_desc(sb + a_bytes);
#pragma unroll
                            for (int kk = 0; kk < 4; ++kk)
                                tc_mma<FORM>(d_tmem, alo + (uint64_t)(kk * 2), bdesc + (uint64_t)(kk * 2), P.idesc, 1u);
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
            if (*abort_flag && last_bar) mbar_drain(last_bar, last_parity, DRAIN_LIMIT_NS);
        }
    } else if (X3 && warp >= 8) {
        const int t = threadIdx.x - 256;
        int st = 0;
        uint32_t ph = 0;
        for (int it = blockIdx.x; it < ntiles && !*abort_flag; it += gridDim.x) {
            const BProb &P = probs[tile_prob[it]];
            for (int nc = 0; nc < P.n_chunks; ++nc) {
                for (int kb = 0; kb < P.kb; ++kb) {
                    if (!mbar_wait(&full[st], ph, abort_flag, wait_ns)) goto split_done;
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
            Band<BCAND_MAX> band;
            band.lv = reinterpret_cast<float *>(base + (size_t)stages * stage_bytes + 1024) + q * 32 + lane;
            band.li = reinterpret_cast<int32_t *>(band.lv + BCAND_MAX * 128);
            band.reset(E2);
            int cur = 0;
            // emit the finished seed s of this point: label, certified near-tie flag, candidates
            auto finish = [&](int s) {
                band.prune();
                const bool over = !(band.v0 < __int_as_float(0x7f800000)) || band.dmin <= band.t ||
                                  1 + band.cnt > BCAND_MAX;
                const int bc = over ? -1 : 1 + band.cnt;
                const bool flag = valid && bc != 1;
                if (valid) P.labels[(int64_t)s * P.n + row] = band.i0;
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
                        f[3] = bc;
                        if (bc > 0) {
                            f[4] = band.i0;
                            for (int q2 = 0; q2 < band.cnt; ++q2) f[5 + q2] = band.li[q2 * 128];
                        }
                    }
                }
                band.reset(E2);
            };
            for (int nc = 0; nc < P.n_chunks; ++nc) {
                if (!mbar_wait(&accf[ab], aph, abort_flag, wait_ns)) goto epi_done;
                tc_fence_after();
                const uint32_t tbase = tmem_base + ((uint32_t)(q * 32) << 16) + (uint32_t)(ab * BN_ALLOC);
                auto process = [&](const uint32_t (&r)[16], int c) {
                    const int64_t j0 = (int64_t)nc * P.bn + c;  // column among all seeds' centers
                    if (j0 >= ncols) return;
                    const int kps = (int)P.kps;
                    const int s = (int)j0 / kps;
                    const int jl0 = (int)j0 - s * kps;
                    if (s != cur) {
                        finish(cur);
                        cur = s;
                    }
                    if (jl0 >= P.k) return;
                    float cn[16], sc[16];
#pragma unroll
                    for (int g = 0; g < 4; ++g) {
                        const float4 t4 = __ldg(reinterpret_cast<const float4 *>(P.cnorm + j0) + g);
                        cn[4 * g] = t4.x, cn[4 * g + 1] = t4.y, cn[4 * g + 2] = t4.z, cn[4 * g + 3] = t4.w;
                    }
                    if (jl0 + 16 <= P.k) {
#pragma unroll
                        for (int g = 0; g < 16; ++g) sc[g] = fmaf(-2.f, __uint_as_float(r[g]), cn[g]);
                    } else {
#pragma unroll
                        for (int g = 0; g < 16; ++g)
                            sc[g] = (jl0 + g < P.k) ? fmaf(-2.f, __uint_as_float(r[g]), cn[g]) : __int_as_float(0x7f800000);
                    }
                    band.group(sc, jl0);
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

// ---------------------------------------------------------------- transposed contraction over rows
// part[ks] (d x s, FP32) = sum over the rows r of split ks of (sqrt(w_r) A[r, :])^T Q[r, :]: the
// randomised SVD's row reduction Bt = A'^T Q, a contraction over the n rows of A (row-major n x d),
// so A is the MN-major operand.  The tile is transposed in shared memory instead: the producer
// loads a plain 32-row x 128-column box of A (no swizzle), warps 4-7 read it column-wise, scale each
// row by sqrt(w_r), split the values into TF32 hi and lo and write them as the K-major, 128-byte
// swizzled A operand (M = 128 columns of d, K = 32 rows of n); Q^T's hi / lo (s x n, K-major) are the
// B operand.  3xTF32 as in k_tc (lo.hi + hi.lo + hi.hi), FP32 accumulation in TMEM over one split,
// the splits then added in fixed order.  Units (split ks, column tile mt) go to CTAs round-robin;
// two accumulators let the epilogue (warps 8-11, one TMEM lane quarter each) overlap the next unit.
struct TnArgs {
    int64_t n, d, s;
    int mt_count, splits, kb_per_split, stages;
    uint32_t raw_bytes, a_bytes, b_bytes, stage_bytes, tx_bytes, idesc;
    const float *w;
    float *part;
    int *status;
    uint64_t wait_ns;
};

__global__ void __launch_bounds__(384, 1)
    k_tn_tc(const __grid_constant__ CUtensorMap tmRaw, const __grid_constant__ CUtensorMap tmQh,
            const __grid_constant__ CUtensorMap tmQl, const TnArgs a) {
    extern __shared__ uint8_t smem_raw[];
    uint8_t *base = smem_raw + ((1024u - (smem_u32(smem_raw) & 1023u)) & 1023u);
    uint64_t *bars = reinterpret_cast<uint64_t *>(base + (size_t)a.stages * a.stage_bytes);
    uint64_t *full = bars, *tfull = bars + MAX_STAGES, *empty = bars + 2 * MAX_STAGES;
    uint64_t *accf = bars + 3 * MAX_STAGES, *acce = accf + 2;
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(acce + 2);
    volatile int *abort_flag = reinterpret_cast<volatile int *>(tmem_slot + 1);
    const int units = a.mt_count * a.splits;
    if ((int)blockIdx.x >= units) return;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    // stage layout: [A hi | A lo | Q^T hi | Q^T lo | raw A box]
    if (threadIdx.x == 0) {
        for (int q = 0; q < a.stages; ++q) {
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
                     "r"(256u)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem_base = *tmem_slot;
    const int64_t rows_per_split = (int64_t)a.kb_per_split * 32;

    if (warp == 0) {
        if (lane == 0) {
            int st = 0;
            uint32_t ph = 0, issued = 0, last_par = 0;
            for (int u = blockIdx.x; u < units && !*abort_flag; u += gridDim.x) {
                const int ks = u / a.mt_count, mt = u % a.mt_count;
                const int64_t r0 = (int64_t)ks * rows_per_split;
                for (int kb = 0; kb < a.kb_per_split; ++kb) {
                    const int64_t rr = r0 + (int64_t)kb * 32;
                    if (rr >= a.n) break;
                    if (!mbar_wait(&empty[st], ph ^ 1, abort_flag, a.wait_ns)) goto producer_done;
                    uint8_t *sb = base + (size_t)st * a.stage_bytes;
                    mbar_expect_tx(&full[st], a.tx_bytes);
                    tma_load_2d(sb + 2 * a.a_bytes + 2 * a.b_bytes, &tmRaw, &full[st], mt * 128, (int32_t)rr);
                    tma_load_2d(sb + 2 * a.a_bytes, &tmQh, &full[st], (int32_t)rr, 0);
                    tma_load_2d(sb + 2 * a.a_bytes + a.b_bytes, &tmQl, &full[st], (int32_t)rr, 0);
                    issued |= 1u << st;
                    last_par = (last_par & ~(1u << st)) | (ph << st);
                    if (++st == a.stages) {
                        st = 0;
                        ph ^= 1;
                    }
                }
            }
        producer_done:
            if (*abort_flag)
                for (int q = 0; q < a.stages; ++q)
                    if (issued & (1u << q)) mbar_drain(&full[q], (last_par >> q) & 1, DRAIN_LIMIT_NS);
        }
    } else if (warp == 1) {
        if (lane == 0) {
            int st = 0, ab = 0;
            uint32_t ph = 0, aph = 0;
            uint64_t *last_bar = nullptr;
            uint32_t last_parity = 0;
            for (int u = blockIdx.x; u < units && !*abort_flag; u += gridDim.x) {
                const int ks = u / a.mt_count;
                const int64_t r0 = (int64_t)ks * rows_per_split;
                if (!mbar_wait(&acce[ab], aph ^ 1, abort_flag, a.wait_ns)) goto mma_done;
                tc_fence_after();
                const uint32_t d_tmem = tmem_base + (uint32_t)(ab * 128);
                for (int kb = 0; kb < a.kb_per_split; ++kb) {
                    if (r0 + (int64_t)kb * 32 >= a.n) break;
                    if (!mbar_wait(&tfull[st], ph, abort_flag, a.wait_ns)) goto mma_done;
                    tc_fence_after();
                    uint8_t *sb = base + (size_t)st * a.stage_bytes;
                    const uint64_t ahi = sw128_desc(sb), alo = sw128_desc(sb + a.a_bytes);
                    const uint64_t bhi = sw128_desc(sb + 2 * a.a_bytes), blo = sw128_desc(sb + 2 * a.a_bytes + a.b_bytes);
#pragma unroll
                    for (int kk = 0; kk < 4; ++kk) {
                        const uint32_t acc = (kb > 0 || kk > 0) ? 1u : 0u;
                        const uint64_t off = (uint64_t)(kk * 2);
                        tc_mma<F_TF32X3>(d_tmem, alo + off, bhi + off, a.idesc, acc);
                        tc_mma<F_TF32X3>(d_tmem, ahi + off, blo + off, a.idesc, 1u);
                        tc_mma<F_TF32X3>(d_tmem, ahi + off, bhi + off, a.idesc, 1u);
                    }
                    tc_commit(&empty[st]);
                    last_bar = &empty[st];
                    last_parity = ph;
                    if (++st == a.stages) {
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
        mma_done:
            if (*abort_flag && last_bar) mbar_drain(last_bar, last_parity, DRAIN_LIMIT_NS);
        }
    } else if (warp >= 4 && warp < 8) {
        // transposing split: thread t takes column mt * 128 + t of the box (one output row of the
        // K-major operand); rows of the box beyond n were zero-filled by the copy
        const int t = threadIdx.x - 128;
        int st = 0;
        uint32_t ph = 0;
        for (int u = blockIdx.x; u < units && !*abort_flag; u += gridDim.x) {
            const int ks = u / a.mt_count;
            const int64_t r0 = (int64_t)ks * rows_per_split;
            for (int kb = 0; kb < a.kb_per_split; ++kb) {
                const int64_t rr = r0 + (int64_t)kb * 32;
                if (rr >= a.n) break;
                if (!mbar_wait(&full[st], ph, abort_flag, a.wait_ns)) goto split_done;
                uint8_t *sb = base + (size_t)st * a.stage_bytes;
                const float *raw = reinterpret_cast<const float *>(sb + 2 * a.a_bytes + 2 * a.b_bytes);
                uint8_t *hi_row = sb + (t >> 3) * 1024 + (t & 7) * 128;
                uint8_t *lo_row = hi_row + a.a_bytes;
#pragma unroll
                for (int c = 0; c < 8; ++c) {
                    float h4[4], l4[4];
#pragma unroll
                    for (int e = 0; e < 4; ++e) {
                        const int r = 4 * c + e;
                        float v = raw[r * 128 + t];
                        if (a.w) {
                            const int64_t gr = rr + r;
                            v *= gr < a.n ? sqrtf(fmaxf(__ldg(a.w + gr), 0.f)) : 0.f;
                        }
                        const float h = __uint_as_float(__float_as_uint(v) & 0xffffe000u);
                        h4[e] = h;
                        l4[e] = __uint_as_float(__float_as_uint(__fsub_rn(v, h)) & 0xffffe000u);
                    }
                    const int pc = (c ^ (t & 7)) * 16;
                    *reinterpret_cast<float4 *>(hi_row + pc) = make_float4(h4[0], h4[1], h4[2], h4[3]);
                    *reinterpret_cast<float4 *>(lo_row + pc) = make_float4(l4[0], l4[1], l4[2], l4[3]);
                }
                asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                __syncwarp();
                if (lane == 0) mbar_arrive(&tfull[st]);
                if (++st == a.stages) {
                    st = 0;
                    ph ^= 1;
                }
            }
        }
    split_done:;
    } else if (warp >= 8) {
        // epilogue: TMEM lane = column j of d; s accumulator columns per lane
        const int q = warp & 3;
        int ab = 0;
        uint32_t aph = 0;
        for (int u = blockIdx.x; u < units && !*abort_flag; u += gridDim.x) {
            const int ks = u / a.mt_count, mt = u % a.mt_count;
            if (!mbar_wait(&accf[ab], aph, abort_flag, a.wait_ns)) goto epi_done;
            tc_fence_after();
            const int64_t j = (int64_t)mt * 128 + q * 32 + lane;
            const uint32_t tb = tmem_base + ((uint32_t)(q * 32) << 16) + (uint32_t)(ab * 128);
            float *dst = a.part + ((int64_t)ks * a.d + j) * a.s;
            for (int c = 0; c < (int)a.s; c += 16) {
                uint32_t r[16];
                tmem_ld16(tb + (uint32_t)c, r);
                tmem_wait_ld(r);
                if (j < a.d) {
#pragma unroll
                    for (int g = 0; g < 4; ++g)
                        reinterpret_cast<float4 *>(dst + c)[g] =
                            make_float4(__uint_as_float(r[4 * g]), __uint_as_float(r[4 * g + 1]),
                                        __uint_as_float(r[4 * g + 2]), __uint_as_float(r[4 * g + 3]));
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
    epi_done:;
    }
    __syncthreads();
    if (*abort_flag && threadIdx.x == 0) status_raise(a.status, ST_TIMEOUT);
    if (warp == 2) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem_base), "r"(256u) : "memory");
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

__device__ __forceinline__ uint32_t make_idesc_dev(int form) {
    const uint32_t ab = (form == F_BF16 || form == F_BF16X2) ? 1u : (form == F_FP8 ? 0u : 2u);
    return (1u << 4) | (ab << 7) | (ab << 10) | ((uint32_t)(256 >> 3) << 17) | ((uint32_t)(128 >> 4) << 24);
}

// 2D FP32 tensor [outer x inner] with a row stride of stride_bytes (a multiple of 16), an arbitrary
// box and swizzle; out-of-range elements read as zero
static bool make_tmap_f32(CUtensorMap *m, const void *ptr, uint64_t inner, uint64_t outer, uint64_t stride_bytes,
                          uint32_t box_inner, uint32_t box_outer, CUtensorMapSwizzle sw) {
    EncodeTiledFn fn = encode_fn();
    if (!fn) return false;
    cuuint64_t dims[2] = {inner, outer};
    cuuint64_t strides[1] = {stride_bytes};
    cuuint32_t box[2] = {box_inner, box_outer};
    cuuint32_t es[2] = {1, 1};
    return fn(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<void *>(ptr), dims, strides, box, es,
              CU_TENSOR_MAP_INTERLEAVE_NONE, sw, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
              CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

static uint32_t make_idesc(int form, int M, int N) {
    uint32_t ab = (form == F_BF16 || form == F_BF16X2) ? 1u : (form == F_FP8 ? 0u : 2u);
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

static Plan plan(int form, int64_t d, int64_t k_pad, int bn_cap = 256, int extra_smem = 0, int bn_align = 16,
                 int stage_cap = 0) {
    Plan p;
    const int esize = (form == F_BF16 || form == F_BF16X2) ? 2 : (form == F_FP8 ? 1 : 4);
    p.n_chunks = (int)ceil_div(k_pad, bn_cap);
    p.bn = (int)(ceil_div(ceil_div(k_pad, p.n_chunks), bn_align) * bn_align);
    p.kb = (int)ceil_div(d * esize, 128);
    const bool x3 = form == F_TF32X3, two_b = x3 || form == F_BF16X2;
    p.a_bytes = BM * 128;
    p.b_bytes = (uint32_t)p.bn * 128;
    p.stage_bytes = (x3 ? 2 : 1) * p.a_bytes + (two_b ? 2 : 1) * p.b_bytes;
    p.tx_bytes = p.a_bytes + (two_b ? 2 : 1) * p.b_bytes;
    p.stages = (int)std::min<int64_t>(MAX_STAGES, (MAX_DYN_SMEM - 2048 - extra_smem) / p.stage_bytes);
    if (stage_cap >= 2) p.stages = std::min(p.stages, stage_cap);
    p.tmem_cols = (2 * p.bn <= 256) ? 256 : 512;
    p.smem = (size_t)p.stages * p.stage_bytes + 1024 + 1024 + extra_smem;
    return p;
}

// the stacked 3xTF32 MMA (x.[c_hi | c_lo] in one instruction of N = 2 bn) where a chunk has at most 128
// centers: two accumulators of 2 bn columns each must fit the 512 TMEM columns
static void set_stack(Args &a, int form, int bn) {
    if (form == F_TF32X3 && bn <= 128) {
        a.stack = 1;
        a.idesc2 = make_idesc(F_TF32X3, BM, 2 * bn);
        a.tmem_cols = (4 * bn <= 256) ? 256 : 512;
    }
}

template <int FORM, int EPI>
static int launch(gbkm_ctx *c, const CUtensorMap &A, const CUtensorMap &B, const CUtensorMap &B2, Args &args,
                  const Plan &p, const CUtensorMap *A2 = nullptr) {
    auto kern = k_tc<FORM, EPI>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)p.smem);
    if (e != cudaSuccess) return cuda_check(c, e, "tcgen05 smem attribute");
    const int threads = tc_threads<FORM, EPI>();
    const int grid = (int)std::min<int64_t>(c->sm_count, args.m_tiles);
    args.wait_ns = c->wait_ns ? c->wait_ns : WAIT_LIMIT_NS;
    args.stall_loads = c->stall_loads;
    kern<<<grid, threads, p.smem, c->stream>>>(A, B, B2, A2 ? *A2 : A, args);
    GBKM_LAUNCHED(c);
    return cuda_check(c, cudaGetLastError(), "tcgen05 kernel launch");
}

// ---------------------------------------------------------------- peak probes (diagnostics)
// Throughput of the tensor-core shape the engine issues (cta_group::1, M = 128, N = 256, one 32-byte
// K step: K = 16 BF16, 8 TF32 or 32 E4M3 elements): one CTA per SM, operands a fixed pattern of
// values in [0.5, 1) in shared memory, one thread issuing `iters` MMAs into two TMEM accumulators,
// then one commit and a bounded wait.  Each CTA writes its elapsed %globaltimer nanoseconds.
template <int FORM>
__global__ void __launch_bounds__(128, 1) k_probe_mma(int iters, uint64_t *__restrict__ t_out, int *status) {
    extern __shared__ uint8_t smem_raw[];
    uint8_t *base = smem_raw + ((1024u - (smem_u32(smem_raw) & 1023u)) & 1023u);
    constexpr uint32_t A_BYTES = 128 * 128, B_BYTES = 256 * 128;
    uint64_t *bar = reinterpret_cast<uint64_t *>(base + A_BYTES + B_BYTES);
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(bar + 1);
    volatile int *abort_flag = reinterpret_cast<volatile int *>(tmem_slot + 1);
    uint32_t *w = reinterpret_cast<uint32_t *>(base);
    for (uint32_t i = threadIdx.x; i < (A_BYTES + B_BYTES) / 4; i += blockDim.x) {
        const uint32_t h = (i * 2654435761u) ^ (i >> 7);
        uint32_t v;
        if (FORM == F_BF16)
            v = 0x3F003F00u | (h & 0x007F007Fu);        // two BF16 values in [0.5, 1)
        else if (FORM == F_FP8)
            v = 0x30303030u | (h & 0x07070707u);        // four E4M3 values in [0.5, 1)
        else
            v = 0x3F000000u | (h & 0x007FE000u);        // a TF32 value in [0.5, 1)
        w[i] = v;
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    if (threadIdx.x == 0) {
        mbar_init(bar, 1);
        *abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (threadIdx.x < 32) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                     "r"(512u)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;
    if (threadIdx.x == 0) {
        const uint32_t idesc = make_idesc_dev(FORM);
        const uint64_t adesc = sw128_desc(base), bdesc = sw128_desc(base + A_BYTES);
        const uint64_t t0 = globaltimer_ns();
        for (int it = 0; it < iters; ++it) {
            const uint64_t off = (uint64_t)((it & 3) * 2);
            tc_mma<FORM>(tmem + (uint32_t)((it & 1) * 256), adesc + off, bdesc + off, idesc, it >= 2 ? 1u : 0u);
        }
        tc_commit(bar);
        const bool ok = mbar_wait(bar, 0, abort_flag, WAIT_LIMIT_NS);
        const uint64_t t1 = globaltimer_ns();
        t_out[blockIdx.x] = t1 - t0;
        if (!ok) {
            // the MMAs still read shared memory and write TMEM: let them finish before the exit
            mbar_drain(bar, 0, DRAIN_LIMIT_NS);
            status_raise(status, ST_TIMEOUT);
        }
    }
    __syncthreads();
    if (threadIdx.x < 32) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(512u) : "memory");
    }
}

// CUDA-core FMA throughput: CHAINS independent FMA chains per thread
template <class T, int CHAINS>
__global__ void __launch_bounds__(256) k_probe_fma(int iters, T *__restrict__ sink) {
    T a[CHAINS];
#pragma unroll
    for (int i = 0; i < CHAINS; ++i) a[i] = (T)(threadIdx.x + 1) * (T)1e-3 + (T)i;
    const T m = (T)0.999999, c = (T)1e-6;
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int i = 0; i < CHAINS; ++i) a[i] = fma(a[i], m, c);
    }
    T s = 0;
#pragma unroll
    for (int i = 0; i < CHAINS; ++i) s += a[i];
    if (s == (T)-1) sink[blockIdx.x * blockDim.x + threadIdx.x] = s;  // never true; keeps the chains live
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
                     float err_rel, float err_abs, const AssignOut &o, const int32_t *n_dev, const int32_t *row_map) {
    using namespace tc;
    // BF16 with a low part of the centers: the two-term form
    const int form = (dtype == GBKM_BF16) ? (cp.cop_lo ? F_BF16X2 : F_BF16)
                                          : (dtype == GBKM_FP8E4M3 ? F_FP8 : F_TF32X3);
    const bool bf = form == F_BF16 || form == F_BF16X2;
    const Plan p = plan(form, d, k_pad, c->bn_cap > 0 ? c->bn_cap : 256, ARGMIN_EXTRA_SMEM, 16, c->stage_cap);
    const CUtensorMapDataType dt = bf                ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16
                                   : (form == F_FP8) ? CU_TENSOR_MAP_DATA_TYPE_UINT8
                                                     : CU_TENSOR_MAP_DATA_TYPE_FLOAT32;
    const uint32_t es = bf ? 2 : (form == F_FP8 ? 1 : 4);
    CUtensorMap tA, tB, tB2;
    if (!make_tmap(&tA, dt, Xop, (uint64_t)d, (uint64_t)n, es, BM) ||
        !make_tmap(&tB, dt, cp.cop, (uint64_t)d, (uint64_t)k_pad, es, (uint32_t)p.bn))
        return set_error(c, GBKM_ECUDA, "cuTensorMapEncodeTiled failed for the assign operands");
    tB2 = tB;
    if ((form == F_TF32X3 || form == F_BF16X2) &&
        !make_tmap(&tB2, dt, cp.cop_lo, (uint64_t)d, (uint64_t)k_pad, es, (uint32_t)p.bn))
        return set_error(c, GBKM_ECUDA, "cuTensorMapEncodeTiled failed for the centers' low part");
    Args a{};
    a.n = n, a.d = d, a.k = k, a.k_pad = k_pad;
    a.n_chunks = p.n_chunks, a.bn = p.bn, a.kb = p.kb, a.stages = p.stages, a.tmem_cols = p.tmem_cols;
    a.m_tiles = (int)ceil_div(n, BM);
    a.a_bytes = p.a_bytes, a.b_bytes = p.b_bytes, a.stage_bytes = p.stage_bytes, a.tx_bytes = p.tx_bytes;
    a.idesc = make_idesc(form, BM, p.bn);
    a.n_dev = n_dev;
    a.row_map = row_map;
    a.cnorm = cp.cnorm, a.cscale = cp.cscale, a.xscale = Xscales, a.xnorm = xnorm, a.cmax = cp.cmax;
    a.err_rel = err_rel, a.err_abs = err_abs;
    if (form == F_BF16 && Xscales && cp.emax) {
        // BF16 scales are the rows' rounding residuals (kmeans_quantize)
        a.xresid = Xscales, a.emax = cp.emax;
        a.acc_g = (float)((double)d * ldexp(1.0, -22) * (1 + 1e-6));
        a.err_u2 = (float)(2.0 * ldexp(1.0, -24) * (1 + 1e-6));
    }
    if (form == F_BF16X2) {
        // the rows' rounding residuals ||x~ - x|| (kmeans_quantize's side data), when given, replace
        // u ||x|| in the pair term of the band
        if (Xscales) a.xresid = Xscales;
        // |x~ - x| <= u |x| with u = 2^-8 (BF16, nearest even), |c^ - c| <= u^2 |c| for hi + lo, FP32
        // accumulation of 2d products bounded by 2d 2^-22 relative (4x the textbook 2d 2^-24)
        const double u = ldexp(1.0, -8), g = 2.0 * (double)d * ldexp(1.0, -22) * (1 + u) * (1 + u);
        a.pair_a = (float)(2 * u * (1 + 1e-6));
        a.pair_rel = (float)((4 * g + 2 * u * 2 * u * u + 4 * u * u) * (1 + 1e-6));
        a.pair_abs = (float)(ldexp(1.0, -23) * (1 + 1e-6));
        a.single_rel = (float)((2 * g + 2 * u * (1 + u * u) + 2 * u * u) * (1 + 1e-6));
        a.single_abs = (float)(ldexp(1.0, -24) * (1 + 1e-6));
    }
    a.labels = o.labels, a.min_d2 = o.min_d2, a.flag_list = o.flag_list, a.cand = o.cand, a.flag_count = o.flag_count;
    a.status = c->status;
    set_stack(a, form, p.bn);
    if (form == F_BF16X2) return launch<F_BF16X2, E_ARGMIN>(c, tA, tB, tB2, a, p);
    if (form == F_BF16) return launch<F_BF16, E_ARGMIN>(c, tA, tB, tB2, a, p);
    if (form == F_FP8) return launch<F_FP8, E_ARGMIN>(c, tA, tB, tB2, a, p);
    return launch<F_TF32X3, E_ARGMIN>(c, tA, tB, tB2, a, p);
}

// V (d x r, FP32) -> V^T (r x d) in the operand format of the projection: BF16, or FP32 split into
// TF32 hi and lo parts (hi = the top 19 bits of v, lo = those of v - hi) for the 3xTF32 form
__global__ void k_vt(const float *__restrict__ V, int64_t d, int64_t r, int dtype, void *out, float *out_lo) {
    const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e >= d * r) return;
    const int64_t q = e / d, t = e % d;  // out[q][t] = V[t][q]
    const float v = V[t * r + q];
    if (dtype == GBKM_BF16) {
        static_cast<__nv_bfloat16 *>(out)[e] = __float2bfloat16_rn(v);
    } else {
        const float hi = __uint_as_float(__float_as_uint(v) & 0xffffe000u);
        static_cast<float *>(out)[e] = hi;
        out_lo[e] = __uint_as_float(__float_as_uint(__fsub_rn(v, hi)) & 0xffffe000u);
    }
}

// V (d x r, FP32, row-major: already the N x K, K-major operand of the lift) split into TF32 hi / lo
__global__ void k_split_tf32(const float *__restrict__ V, int64_t count, float *__restrict__ hi,
                             float *__restrict__ lo) {
    const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e >= count) return;
    const float v = V[e];
    const float h = __uint_as_float(__float_as_uint(v) & 0xffffe000u);
    hi[e] = h;
    lo[e] = __uint_as_float(__float_as_uint(__fsub_rn(v, h)) & 0xffffe000u);
}

bool tc_project_supported(int dtype, int64_t d, int64_t r) {
    if (!tc::encode_fn()) return false;
    if (r % 16 != 0 || r < 16 || r > 256) return false;
    if (dtype == GBKM_BF16) return d % 8 == 0;
    if (dtype == GBKM_F32) return d % 4 == 0;
    return false;
}

// a store-epilogue GEMM Out[M x N] = A[M x K] B^T (B: N x K) on the engine, operands already in place
static int launch_store_gemm(gbkm_ctx *c, int form, const void *A, const void *B, const void *B_lo, int64_t M,
                             int64_t N, int64_t K, float *Out, const float *row_w = nullptr) {
    using namespace tc;
    const uint32_t es = (form == F_BF16) ? 2 : 4;
    const Plan p = plan(form, K, N);
    const CUtensorMapDataType dt = (form == F_BF16) ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32;
    CUtensorMap tA, tB, tB2;
    if (!make_tmap(&tA, dt, A, (uint64_t)K, (uint64_t)M, es, BM) ||
        !make_tmap(&tB, dt, B, (uint64_t)K, (uint64_t)N, es, (uint32_t)p.bn))
        return set_error(c, GBKM_ECUDA, "cuTensorMapEncodeTiled failed for the projection operands");
    tB2 = tB;
    if (form == F_TF32X3 && !make_tmap(&tB2, dt, B_lo, (uint64_t)K, (uint64_t)N, es, (uint32_t)p.bn))
        return set_error(c, GBKM_ECUDA, "cuTensorMapEncodeTiled failed for the projection's low part");
    Args a{};
    a.n = M, a.d = K, a.k = N, a.k_pad = N;
    a.n_chunks = p.n_chunks, a.bn = p.bn, a.kb = p.kb, a.stages = p.stages, a.tmem_cols = p.tmem_cols;
    a.m_tiles = (int)ceil_div(M, BM);
    a.a_bytes = p.a_bytes, a.b_bytes = p.b_bytes, a.stage_bytes = p.stage_bytes, a.tx_bytes = p.tx_bytes;
    a.idesc = make_idesc(form, BM, p.bn);
    a.Y = Out, a.ldy = N;
    a.row_w = row_w;
    a.status = c->status;
    set_stack(a, form, p.bn);
    if (form == F_BF16) return launch<F_BF16, E_STORE>(c, tA, tB, tB2, a, p);
    return launch<F_TF32X3, E_STORE>(c, tA, tB, tB2, a, p);
}

// The randomised SVD's sketch Y = diag(sqrt(w)) A Omega on the tensor cores (3xTF32): A (n x d) is
// the K-major A operand, Omega^T (s x d, split into TF32 hi / lo by k_vt into omt, 2 s d floats of
// workspace) the B operand; the row weights enter in the store epilogue.  d % 4 == 0, s % 16 == 0.
int launch_sketch_tc(gbkm_ctx *c, const float *A, const float *w, int64_t n, int64_t d, const float *Omega, int64_t s,
                     float *omt, float *Y) {
    k_vt<<<(unsigned)ceil_div(s * d, 256), 256, 0, c->stream>>>(Omega, d, s, GBKM_F32, omt, omt + s * d);
    GBKM_LAUNCHED(c);
    return launch_store_gemm(c, tc::F_TF32X3, A, omt, omt + s * d, n, s, d, Y, w);
}

// Y = X V: BF16 X against BF16 V, or FP32 X in the 3xTF32 form (the staged X tile split into TF32 hi
// and lo in shared memory, V^T split in the workspace; three MMAs per step: FP32-faithful products)
int launch_project_tc(gbkm_ctx *c, int dtype, const void *X, int64_t n, int64_t d, const float *V, int64_t r,
                      float *Y) {
    using namespace tc;
    const int form = (dtype == GBKM_BF16) ? F_BF16 : F_TF32X3;
    const uint32_t es = (form == F_BF16) ? 2 : 4;
    int rc = GBKM_OK;
    WsPlan wp;
    const size_t o_hi = wp.take<char>((size_t)r * d * es), o_lo = wp.take<float>(form == F_BF16 ? 0 : (size_t)r * d);
    void *ws = ws_reserve(c, wp.off, &rc);
    if (!ws) return rc;
    k_vt<<<(unsigned)ceil_div(r * d, 256), 256, 0, c->stream>>>(V, d, r, dtype, ws_at<void>(ws, o_hi),
                                                                 ws_at<float>(ws, o_lo));
    GBKM_LAUNCHED(c);
    return launch_store_gemm(c, form, X, ws_at<void>(ws, o_hi), ws_at<void>(ws, o_lo), n, r, d, Y);
}

bool tc_lift_supported(int64_t d, int64_t r) {
    return tc::encode_fn() && d % 16 == 0 && d >= 16 && r % 4 == 0 && r >= 4;
}

// X_lift = Y V^T (n x d) in the 3xTF32 form: A = Y (n x r, K = r), B = V itself (d x r row-major is the
// N x K, K-major operand), split into TF32 hi / lo in the workspace
int launch_lift_tc(gbkm_ctx *c, const float *Y, int64_t n, int64_t r, const float *V, int64_t d, float *X_lift) {
    using namespace tc;
    int rc = GBKM_OK;
    WsPlan wp;
    const size_t o_hi = wp.take<float>((size_t)d * r), o_lo = wp.take<float>((size_t)d * r);
    void *ws = ws_reserve(c, wp.off, &rc);
    if (!ws) return rc;
    k_split_tf32<<<(unsigned)ceil_div(d * r, 256), 256, 0, c->stream>>>(V, d * r, ws_at<float>(ws, o_hi),
                                                                        ws_at<float>(ws, o_lo));
    GBKM_LAUNCHED(c);
    return launch_store_gemm(c, F_TF32X3, Y, ws_at<void>(ws, o_hi), ws_at<void>(ws, o_lo), n, d, r, X_lift);
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
    const size_t smem = (size_t)stages * stage_bytes + 2048 + BCAND_MAX * 128 * 8;
    const int threads = x3 ? 384 : 256;
    const int grid = (int)std::min<int64_t>(c->sm_count, ntiles);
    const uint64_t wait_ns = c->wait_ns ? c->wait_ns : WAIT_LIMIT_NS;
    cudaError_t e;
    if (x3) {
        e = cudaFuncSetAttribute(k_tcb<F_TF32X3>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return cuda_check(c, e, "batched smem attribute");
        k_tcb<F_TF32X3><<<grid, threads, smem, c->stream>>>(static_cast<const CUtensorMap *>(maps), probs, tile_prob,
                                                            (int)ntiles, stages, a_bytes, b_bytes, stage_bytes,
                                                            flags, flag_count, c->status, wait_ns);
    } else {
        e = cudaFuncSetAttribute(k_tcb<F_BF16>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return cuda_check(c, e, "batched smem attribute");
        k_tcb<F_BF16><<<grid, threads, smem, c->stream>>>(static_cast<const CUtensorMap *>(maps), probs, tile_prob,
                                                          (int)ntiles, stages, a_bytes, b_bytes, stage_bytes,
                                                          flags, flag_count, c->status, wait_ns);
    }
    GBKM_LAUNCHED(c);
    return cuda_check(c, cudaGetLastError(), "batched tcgen05 launch");
}


// Operands of the bias K block: ones (BM x 64 BF16, columns 0 and 1 = 1) and, per output column j,
// (bf16(b_j), bf16(b_j - bf16(b_j)), 0, ..., 0): the MMA adds b_j to within 2^-17 |b_j|.
__global__ void k_bias_operands(const float *__restrict__ bias, int64_t N, __nv_bfloat16 *__restrict__ ones,
                                __nv_bfloat16 *__restrict__ bb) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < (int64_t)tc::BM * 64) ones[i] = __float2bfloat16_rn((i % 64) < 2 ? 1.f : 0.f);
    if (i < N * 64) {
        const int64_t j = i / 64, col = i % 64;
        const float b = bias[j];
        const __nv_bfloat16 hi = __float2bfloat16_rn(b);
        bb[i] = col == 0 ? hi : (col == 1 ? __float2bfloat16_rn(b - __bfloat162float(hi)) : __float2bfloat16_rn(0.f));
    }
}

// D = A B^T on tcgen05 (BF16 operands, FP32 accumulation) with a fused epilogue: store
// act(D + bias) in FP32 or BF16 (and optionally the FP32 pre-activation), or, when top_idx is
// given, the indices of the topm largest entries of every row of D + bias (D never written).
// A: M x K, B: N x K, row-major BF16, K % 8 == 0, N % 16 == 0, 16-byte aligned.
int launch_gemm_bf16_tc(gbkm_ctx *c, const void *A, const void *B, int64_t M, int64_t N, int64_t K,
                        const float *bias, int act, int out_bf16, void *Y, int64_t ldy, float *Ypre, int64_t ldpre,
                        int32_t *top_idx, float *top_val, int topm, int group) {
    using namespace tc;
    if (M < 1 || N < 16 || N % 16 || K < 8 || K % 8 || !tc::encode_fn())
        return set_error(c, GBKM_EUNSUPPORTED, "gemm: shape unsupported by the tcgen05 GEMM");
    const bool topk = top_idx != nullptr;
    if (topk && (topm < 1 || topm > TOPBUF / 2)) return set_error(c, GBKM_EINVAL, "gemm: topm must be in [1, 32]");
    const int extra = topk ? TROW * 128 * 8 : 0;
    const bool grouped = topk && group == 16;
    const Plan p = plan(F_BF16, K, N, 256, extra, grouped ? 32 : 16);
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
    // the bias through the MMA (one more K block per unit) instead of loads and adds in the epilogue
    CUtensorMap tA2 = tA, tB2 = tB;
    void *bops = nullptr;
    if (bias) {
        const size_t ones_n = (size_t)BM * 64, bb_n = (size_t)N * 64;
        cudaError_t e = cudaMallocAsync(&bops, sizeof(__nv_bfloat16) * (ones_n + bb_n), c->stream);
        if (e != cudaSuccess) {
            cudaGetLastError();
            return set_error(c, GBKM_ENOMEM, "gemm: bias operand allocation failed");
        }
        __nv_bfloat16 *ones = static_cast<__nv_bfloat16 *>(bops), *bb = ones + ones_n;
        k_bias_operands<<<(unsigned)ceil_div((int64_t)std::max(ones_n, bb_n), 256), 256, 0, c->stream>>>(bias, N, ones,
                                                                                                      bb);
        GBKM_LAUNCHED(c);
        if (!make_tmap(&tA2, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, ones, 64, (uint64_t)BM, 2, BM) ||
            !make_tmap(&tB2, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, bb, 64, (uint64_t)N, 2, (uint32_t)p.bn)) {
            cudaFreeAsync(bops, c->stream);
            return set_error(c, GBKM_ECUDA, "cuTensorMapEncodeTiled failed for the bias operands");
        }
        a.bias = nullptr;
        a.bias_mma = 1;
    }
    int rc;
    if (grouped)
        rc = launch<F_BF16, E_TOPG>(c, tA, tB, tB2, a, p, &tA2);
    else if (topk)
        rc = launch<F_BF16, E_TOPM>(c, tA, tB, tB2, a, p, &tA2);
    else
        rc = launch<F_BF16, E_STORE>(c, tA, tB, tB2, a, p, &tA2);
    if (bops) cudaFreeAsync(bops, c->stream);
    return rc;
}

}  // namespace gbkm

// ---------------------------------------------------------------- peak probes: host entry
extern "C" int gbkm_probe_peak(gbkm_ctx *c, int32_t unit, double *tflops_out) {
    using namespace gbkm;
    using namespace gbkm::tc;
    if (!c || !tflops_out || unit < 0 || unit > 4) return GBKM_EINVAL;
    int prev = -1;
    cudaGetDevice(&prev);
    if (prev != c->device) cudaSetDevice(c->device);
    int rc = GBKM_OK;
    const int sms = c->sm_count;
    void *buf = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaError_t e = cudaMalloc(&buf, sizeof(uint64_t) * (size_t)sms * 8 * 256);
    if (e == cudaSuccess) e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    if (e != cudaSuccess) {
        cudaGetLastError();
        rc = set_error(c, GBKM_ENOMEM, "probe: buffers");
    }
    double flops = 0.0, secs = 0.0;
    if (rc == GBKM_OK && unit <= 2) {
        const int form = unit == 0 ? F_BF16 : (unit == 1 ? F_TF32 : F_FP8);
        const int kstep = unit == 0 ? 16 : (unit == 1 ? 8 : 32);
        // about 100k MMAs of 1-2 MFLOP per SM: tens of milliseconds, well inside the wait limit
        const int iters = 100000;
        const size_t smem = 1024 + 128 * 128 + 256 * 128 + 64;
        auto kern = form == F_BF16 ? k_probe_mma<F_BF16> : (form == F_TF32 ? k_probe_mma<F_TF32> : k_probe_mma<F_FP8>);
        e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e == cudaSuccess) {
            kern<<<sms, 128, smem, c->stream>>>(iters / 10, static_cast<uint64_t *>(buf), c->status);  // warm-up
            kern<<<sms, 128, smem, c->stream>>>(iters, static_cast<uint64_t *>(buf), c->status);
            GBKM_LAUNCHED(c);
            GBKM_LAUNCHED(c);
            e = cudaStreamSynchronize(c->stream);
        }
        std::vector<uint64_t> t((size_t)sms);
        if (e == cudaSuccess) e = cudaMemcpy(t.data(), buf, sizeof(uint64_t) * sms, cudaMemcpyDeviceToHost);
        if (e != cudaSuccess) {
            rc = cuda_check(c, e, "probe: tensor-core launch");
        } else {
            uint64_t tmax = 0;
            for (uint64_t v : t) tmax = std::max(tmax, v);
            flops = 2.0 * 128 * 256 * kstep * (double)iters * sms;
            secs = (double)tmax * 1e-9;
        }
    } else if (rc == GBKM_OK) {
        const int blocks = sms * 8, iters = unit == 3 ? 20000 : 2000;
        for (int rep = 0; rep < 2 && e == cudaSuccess; ++rep) {
            // the first pass warms up, the second is timed
            cudaEventRecord(e0, c->stream);
            if (unit == 3)
                k_probe_fma<float, 16><<<blocks, 256, 0, c->stream>>>(iters, static_cast<float *>(buf));
            else
                k_probe_fma<double, 8><<<blocks, 256, 0, c->stream>>>(iters, static_cast<double *>(buf));
            GBKM_LAUNCHED(c);
            cudaEventRecord(e1, c->stream);
            e = cudaEventSynchronize(e1);
        }
        float ms = 0.f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
        if (e != cudaSuccess) {
            rc = cuda_check(c, e, "probe: FMA launch");
        } else {
            flops = 2.0 * (unit == 3 ? 16 : 8) * (double)iters * blocks * 256;
            secs = ms * 1e-3;
        }
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (buf) cudaFree(buf);
    if (prev >= 0 && prev != c->device) cudaSetDevice(prev);
    if (rc != GBKM_OK) return rc;
    if (!(secs > 0.0)) return set_error(c, GBKM_ECUDA, "probe: no elapsed time");
    *tflops_out = flops / secs * 1e-12;
    return GBKM_OK;
}

// ---------------------------------------------------------------- the SVD's row reduction on the tensor cores
namespace gbkm {

// Q (n x s, row-major) -> Q^T split into TF32 hi / lo, s x ld each (ld >= n, columns n..ld-1 zero)
__global__ void __launch_bounds__(256) k_qt_split(const float *__restrict__ Q, int64_t n, int64_t s, int64_t ld,
                                                  float *__restrict__ hi, float *__restrict__ lo) {
    __shared__ float tile[32][33];
    const int64_t r0 = (int64_t)blockIdx.x * 32, c0 = (int64_t)blockIdx.y * 32;
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
    for (int i = ty; i < 32; i += 8) {
        const int64_t r = r0 + i, c = c0 + tx;
        tile[i][tx] = (r < n && c < s) ? Q[r * s + c] : 0.f;
    }
    __syncthreads();
    for (int i = ty; i < 32; i += 8) {
        const int64_t c = c0 + i, r = r0 + tx;
        if (c < s && r < ld) {
            const float v = tile[tx][i];
            const float h = __uint_as_float(__float_as_uint(v) & 0xffffe000u);
            hi[c * ld + r] = h;
            lo[c * ld + r] = __uint_as_float(__float_as_uint(__fsub_rn(v, h)) & 0xffffe000u);
        }
    }
}

// Bt = the splits' partials added in split order, in double-float
__global__ void __launch_bounds__(256) k_tn_reduce_f32(const float *__restrict__ part, int64_t ds, int splits,
                                                       float *__restrict__ Bt) {
    const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e >= ds) return;
    DF acc;
    for (int g = 0; g < splits; ++g) acc.add(part[(int64_t)g * ds + e]);
    Bt[e] = (float)acc.value();
}

bool tc_rows_supported(int64_t d, int64_t s) {
    return tc::encode_fn() && d % 4 == 0 && s % 16 == 0 && s >= 16 && s <= 128;
}

// splits of the n rows: about four units per SM, 32-row K blocks
void tc_rows_shape(int64_t n, int64_t d, int sm_count, int *splits, int *kb_per_split) {
    const int64_t mt = ceil_div(d, (int64_t)128);
    int64_t want = std::max<int64_t>(1, ceil_div(4 * (int64_t)sm_count, mt));
    const int64_t kb_total = ceil_div(n, (int64_t)32);
    const int64_t kbs = std::max<int64_t>(1, ceil_div(kb_total, want));
    *kb_per_split = (int)kbs;
    *splits = (int)ceil_div(kb_total, kbs);
}

// Bt (d x s) = (diag(sqrt(w)) A)^T Q on the tensor cores.  qt: 2 s ld floats (ld = n rounded up to 4),
// part: splits x d x s floats, from tc_rows_shape.
int launch_rows_tc(gbkm_ctx *c, const float *A, const float *w, int64_t n, int64_t d, const float *Q, int64_t s,
                   float *qt, float *part, float *Bt) {
    using namespace tc;
    int splits = 0, kbs = 0;
    tc_rows_shape(n, d, c->sm_count, &splits, &kbs);
    const int64_t ld = ceil_div(n, (int64_t)4) * 4;
    float *qhi = qt, *qlo = qt + s * ld;
    k_qt_split<<<dim3((unsigned)ceil_div(ld, (int64_t)32), (unsigned)ceil_div(s, (int64_t)32)), 256, 0, c->stream>>>(
        Q, n, s, ld, qhi, qlo);
    GBKM_LAUNCHED(c);
    CUtensorMap tRaw, tQh, tQl;
    if (!make_tmap_f32(&tRaw, A, (uint64_t)d, (uint64_t)n, (uint64_t)d * 4, 128, 32, CU_TENSOR_MAP_SWIZZLE_NONE) ||
        !make_tmap_f32(&tQh, qhi, (uint64_t)n, (uint64_t)s, (uint64_t)ld * 4, 32, (uint32_t)s, CU_TENSOR_MAP_SWIZZLE_128B) ||
        !make_tmap_f32(&tQl, qlo, (uint64_t)n, (uint64_t)s, (uint64_t)ld * 4, 32, (uint32_t)s, CU_TENSOR_MAP_SWIZZLE_128B))
        return set_error(c, GBKM_ECUDA, "cuTensorMapEncodeTiled failed for the row reduction");
    TnArgs a{};
    a.n = n, a.d = d, a.s = s;
    a.mt_count = (int)ceil_div(d, (int64_t)128);
    a.splits = splits, a.kb_per_split = kbs;
    a.a_bytes = 128 * 128;
    a.b_bytes = (uint32_t)s * 128;
    a.raw_bytes = 32 * 128 * 4;
    a.stage_bytes = 2 * a.a_bytes + 2 * a.b_bytes + a.raw_bytes;
    a.tx_bytes = a.raw_bytes + 2 * a.b_bytes;
    a.stages = (int)std::min<int64_t>(MAX_STAGES, (MAX_DYN_SMEM - 2048) / a.stage_bytes);
    a.idesc = make_idesc(F_TF32X3, 128, (int)s);
    a.w = w;
    a.part = part;
    a.status = c->status;
    a.wait_ns = c->wait_ns ? c->wait_ns : WAIT_LIMIT_NS;
    const size_t smem = (size_t)a.stages * a.stage_bytes + 2048;
    cudaError_t e = cudaFuncSetAttribute(k_tn_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return cuda_check(c, e, "row reduction smem attribute");
    const int units = a.mt_count * splits;
    k_tn_tc<<<(unsigned)std::min<int64_t>(c->sm_count, units), 384, smem, c->stream>>>(tRaw, tQh, tQl, a);
    GBKM_LAUNCHED(c);
    k_tn_reduce_f32<<<(unsigned)ceil_div(d * s, (int64_t)256), 256, 0, c->stream>>>(part, d * s, splits, Bt);
    GBKM_LAUNCHED(c);
    return cuda_check(c, cudaGetLastError(), "row reduction launch");
}

}  // namespace gbkm
