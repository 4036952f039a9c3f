// internal.cuh -- context, workspace and device helpers shared by the kernels.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp8.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <cstdarg>
#include <cstdio>
#include <vector>

#include "../../include/gbkm.h"
#include "../../include/gbkm_diag.h"

// ---------------------------------------------------------------- device status word bits
enum : int {
    ST_TIMEOUT = 1,      // a bounded wait gave up
    ST_DEGENERATE = 2,   // k-means++ ran out of points with positive D^2
    ST_BADLABEL = 4,     // a label outside [0, k) reached the update
    ST_BOUNDS = 8,       // an internal index check failed (access skipped)
};

struct ProfRec {
    const char *name;
    cudaEvent_t a, b;
};

struct gbkm_ctx {
    int device = 0;
    bool prof = false;              // per-kernel CUDA-event timing on the context's stream
    std::vector<ProfRec> recs;
    std::vector<size_t> prof_open;  // indices of the open brackets in recs (innermost last)
    std::vector<cudaEvent_t> pool;
    size_t pool_used = 0;
    cudaStream_t stream = nullptr;
    char err[512] = {0};
    void *ws = nullptr;          // grow-only workspace
    size_t ws_bytes = 0;
    int *status = nullptr;       // device status word
    int sm_count = 0;
    int64_t launches = 0;
    void *tmap_scratch = nullptr;  // device copy of tensor maps (128 B aligned, 16 slots)
    void *graph_exec = nullptr;    // last instantiated batched-run graph (cudaGraphExec_t)
    uint64_t ws_epoch = 0;         // bumped by every ws_reserve (any call that writes the workspace)
    uint64_t graph_epoch = 0;      // ws_epoch when graph_exec was recorded (its tables live in ws)
    int64_t graph_launches = 0;    // kernels recorded into graph_exec (counted again at every replay)
    cudaStream_t cap_stream = nullptr;  // private stream the batched run is recorded on
    int bn_cap = 0;                // center-chunk width of the tcgen05 assignment (0: 256); autotuner knob
    int stage_cap = 0;             // stage-ring depth cap of the tcgen05 assignment (0: as many as fit); autotuner knob
    uint64_t wait_ns = 0;          // limit of every bounded device wait (0: the default, 2 s)
    int fail_alloc = 0;            // diagnostics: the next fail_alloc workspace growths fail as if out of memory
    int stall_loads = 0;           // diagnostics: tensor-core launches issue no copies (their waits run out)
};

int set_error(gbkm_ctx *c, int code, const char *fmt, ...);
int cuda_check(gbkm_ctx *c, cudaError_t e, const char *what);
// returns a pointer to >= bytes of workspace (grows, synchronising the stream, if needed)
void *ws_reserve(gbkm_ctx *c, size_t bytes, int *rc);

// bump sub-allocator over a workspace block, 256-byte aligned slices
struct WsPlan {
    size_t off = 0;
    template <class T>
    size_t take(size_t count) {
        size_t o = off;
        off += ((count * sizeof(T) + 255) / 256) * 256;
        return o;
    }
};
template <class T>
static inline T *ws_at(void *base, size_t off) {
    return reinterpret_cast<T *>(static_cast<char *>(base) + off);
}

#define GBKM_LAUNCHED(ctx) ((ctx)->launches += 1)

// bracket a kernel (or a short sequence of kernels) with events when profiling is on
void prof_begin(gbkm_ctx *c, const char *name);
void prof_end(gbkm_ctx *c);

// ---------------------------------------------------------------- device helpers
__device__ __forceinline__ uint64_t globaltimer_ns() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ void status_raise(int *status, int bit) {
    if (status) atomicOr(status, bit);
}

// Knuth's TwoSum: s + e == a + b exactly.
__device__ __forceinline__ void two_sum(float a, float b, float &s, float &e) {
    s = __fadd_rn(a, b);
    float bb = __fsub_rn(s, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

// double-float accumulator: hi + lo carries the running sum
struct DF {
    float hi = 0.f, lo = 0.f;
    __device__ __forceinline__ void add(float v) {
        float s, e;
        two_sum(hi, v, s, e);
        hi = s;
        lo = __fadd_rn(lo, e);
    }
    // add the exact product a*b (TwoProd via fma)
    __device__ __forceinline__ void add_prod(float a, float b) {
        float p = __fmul_rn(a, b);
        float pe = __fmaf_rn(a, b, -p);
        add(p);
        lo = __fadd_rn(lo, pe);
    }
    // add (x - c)^2 with the difference and the square resolved error-free
    __device__ __forceinline__ void add_sqdiff(float x, float c) {
        float s, e;
        two_sum(x, -c, s, e);           // x - c == s + e exactly
        float p = __fmul_rn(s, s);
        float pe = __fmaf_rn(s, s, -p);  // s*s == p + pe exactly
        float q = __fmul_rn(__fmul_rn(2.f, s), e);
        add(p);
        lo = __fadd_rn(lo, __fadd_rn(pe, q));
    }
    __device__ __forceinline__ double value() const { return (double)hi + (double)lo; }
};

// warp-wide sum of double-float values with error-free TwoSum at every butterfly step; the result
// is bitwise identical on every lane (TwoSum's error term is exact whichever operand comes first)
__device__ __forceinline__ double warp_sum_df(DF a) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const float h2 = __shfl_xor_sync(0xffffffffu, a.hi, o);
        const float l2 = __shfl_xor_sync(0xffffffffu, a.lo, o);
        float s, e;
        two_sum(a.hi, h2, s, e);
        a.hi = s;
        a.lo = __fadd_rn(__fadd_rn(a.lo, l2), e);
    }
    return a.value();
}

// deterministic tree sum of blockDim.x doubles in shared memory (blockDim.x a power of two);
// every thread must call it; returns the total to every thread
__device__ __forceinline__ double block_tree_sum_d(double v, double *sh) {
    sh[threadIdx.x] = v;
    __syncthreads();
    for (int o = blockDim.x >> 1; o > 0; o >>= 1) {
        if ((int)threadIdx.x < o) sh[threadIdx.x] += sh[threadIdx.x + o];
        __syncthreads();
    }
    const double r = sh[0];
    __syncthreads();
    return r;
}

__device__ __forceinline__ float warp_sum_f(float v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}
__device__ __forceinline__ double warp_sum_d(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// exclusive scan of one int32 per thread across the block (blockDim.x a multiple of 32, <= 1024);
// `total` receives the block's sum; sh holds 32 ints
__device__ __forceinline__ int32_t block_excl_scan(int32_t v, int32_t *sh, int32_t &total) {
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

// ---------------------------------------------------------------- host-side launch helpers
static inline int64_t ceil_div(int64_t a, int64_t b) { return (a + b - 1) / b; }

// kernel entry points implemented in the .cu files (host launchers)
namespace gbkm {
int launch_row_norms(gbkm_ctx *c, const float *X, int64_t n, int64_t d, float *xnorm);
int launch_quantize(gbkm_ctx *c, const float *X, int64_t n, int64_t d, int dtype, void *Xq,
                    float *scales);
// center preparation: ||c||^2 (FP32 from FP64 sums), max ||c|| (as float bits), optional
// operand copies (bf16 / fp8 with per-row scale / tf32 hi-lo split)
struct CenterPrep {
    float *cnorm;       // k
    unsigned *cmax;     // 1: max ||c_j|| as float bits
    unsigned *emax;     // 1: max ||c_j - bf16(c_j)|| as float bits (one-term BF16 operand), or null
    void *cop;          // operand copy (k_pad x d) or null
    void *cop_lo;       // tf32 low part or null
    float *cscale;      // fp8 per-row scales or null
    float *esc_hi;      // 3xTF32 split of the centers for the escalation pass (k_pad x d), or null
    float *esc_lo;
};
// (cp.cmax and cp.emax are maxima by atomics: the caller zeroes them first)
int launch_center_prep(gbkm_ctx *c, const float *C, int64_t k, int64_t d, int dtype,
                       int64_t k_pad, const CenterPrep &cp);

constexpr int CAND_MAX = 8, CAND_STRIDE = CAND_MAX + 1;

struct AssignOut {
    int32_t *labels;
    float *min_d2;
    int32_t *flag_list;   // n entries max: rows whose argmin is a certified near-tie
    int32_t *cand;        // per flag slot, CAND_STRIDE ints: count (-1 = scan all k), then the
                          // centers inside the certified band in increasing index order
    int32_t *flag_count;  // 1
};
int launch_assign_simt(gbkm_ctx *c, const float *X, const float *xnorm, int64_t n, int64_t d,
                       const float *C, const float *cnorm, const unsigned *cmax, int64_t k,
                       float err_rel, float err_abs, const AssignOut &o);
// Out[M x N] = A[M x K] B^T with B[nn * sbn + kk * sbk]
int launch_gemm_simt_strided(gbkm_ctx *c, const float *A, const float *B, int64_t M, int64_t N,
                             int64_t K, int64_t sbn, int64_t sbk, float *Out);
// Escalation of flagged rows whose band is not listed (count <= 0): the recheck appends each to
// list (count) and copies the row and its norm into the dense block Xe / xne, for the next
// precision's pass over that block, instead of scanning all k centers.
struct Escalation {
    int32_t *list;
    int32_t *count;
    float *Xe;
    float *xne;
    const float *xnorm;
};
// exact re-resolution of the flagged rows (X rows; labels / min_d2 of row i go to index
// row_map[i] when row_map is set)
int launch_recheck(gbkm_ctx *c, const float *X, int64_t n, int64_t d, const float *C, int64_t k,
                   const AssignOut &o, int64_t *n_rechecked, const Escalation *esc = nullptr,
                   const int32_t *row_map = nullptr);

// device-wide exclusive scan of L int32 (totals < 2^31); bsum holds ceil(L / 4096) ints
void scan_excl(cudaStream_t st, const int32_t *in, int64_t L, int32_t *bsum, int32_t *out);
int update_impl(gbkm_ctx *c, const float *X, int64_t n, int64_t d, const float *w,
                const int32_t *labels, int64_t k, const float *C_old, float *C_new,
                double *counts, double *cost_old, double *cost_new, int64_t *n_empty);
int seed_impl(gbkm_ctx *c, const float *X, int64_t n, int64_t d, const float *w, int64_t k,
              const double *u, int64_t *idx_out, float *C_out, const void *Xq = nullptr,
              const float *xresid = nullptr);
// worst-case error coefficients of the distance scores of an operand format and engine
void score_error_coeffs(int dtype, int engine_tc, int64_t d, float &err_rel, float &err_abs);
bool tc_assign_supported(int dtype, int64_t d, int64_t k);
int launch_assign_tc(gbkm_ctx *c, int dtype, const void *Xop, const float *Xscales,
                     const float *X, const float *xnorm, int64_t n, int64_t d,
                     const CenterPrep &cp, int64_t k, int64_t k_pad, float err_rel,
                     float err_abs, const AssignOut &o, const int32_t *n_dev = nullptr,
                     const int32_t *row_map = nullptr);
int launch_gemm_bf16_tc(gbkm_ctx *c, const void *A, const void *B, int64_t M, int64_t N, int64_t K,
                        const float *bias, int act, int out_bf16, void *Y, int64_t ldy, float *Ypre, int64_t ldpre,
                        int32_t *top_idx, float *top_val, int topm, int group = 1);
int64_t mlp_param_count(const gbkm_mlp *m);
int mlp_forward(gbkm_ctx *c, const gbkm_mlp *m, const void *Xh, int64_t n, float *logits, int32_t *top_idx, int topm,
                int group = 1);
int mlp_train_step(gbkm_ctx *c, gbkm_mlp *m, const void *Xh, const int32_t *labels, int64_t B, float lr, float wd,
                   float *loss_rows, float *grad_out);
int center_separation(gbkm_ctx *c, const float *C, int64_t k, int64_t d, float *s2);
int learned_assign(gbkm_ctx *c, const gbkm_mlp *m, const float *X, const void *Xh, int64_t n, int64_t d,
                   const float *C, int64_t k, const float *s2, int topm, int32_t *labels, int64_t *n_fallback,
                   int32_t *cand_out);
bool tc_project_supported(int dtype, int64_t d, int64_t r);
int launch_project_tc(gbkm_ctx *c, int dtype, const void *X, int64_t n, int64_t d,
                      const float *V, int64_t r, float *Y);
// X_lift = Y V^T on the tensor cores (3xTF32); d % 16 == 0, r % 4 == 0, Y and X_lift 16-byte aligned
bool tc_lift_supported(int64_t d, int64_t r);
// the randomised SVD's two passes over a piece on the tensor cores (3xTF32)
int launch_sketch_tc(gbkm_ctx *c, const float *A, const float *w, int64_t n, int64_t d, const float *Omega, int64_t s,
                     float *omt, float *Y);
bool tc_rows_supported(int64_t d, int64_t s);
void tc_rows_shape(int64_t n, int64_t d, int sm_count, int *splits, int *kb_per_split);
int launch_rows_tc(gbkm_ctx *c, const float *A, const float *w, int64_t n, int64_t d, const float *Q, int64_t s,
                   float *qt, float *part, float *Bt);
int launch_lift_tc(gbkm_ctx *c, const float *Y, int64_t n, int64_t r, const float *V, int64_t d, float *X_lift);
// ---------------------------------------------------------------- batched problems
// device-side descriptor of one problem of a batched run (all pointers are device pointers)
struct BProb {
    const float *X;          // n x d FP32
    int64_t n, d, k, kps;    // kps: per-seed stride of the centers in the operand (k rounded up to 16)
    int32_t seeds, m_tiles, n_chunks, bn, kb, nb;  // nb: sampling blocks of 128 rows
    uint32_t idesc, tx_bytes;
    float err_rel, err_abs;
    const void *Xop;         // operand copy of X (BF16) or X itself (FP32)
    float *xnorm;            // n
    float *C[2];             // seeds x k x d, ping-pong centers
    float *cnorm;            // seeds x kps
    unsigned *cmax;          // 1
    void *cop, *cop_lo;      // (seeds x kps) x d operand copies of the centers
    int32_t *labels;         // seeds x n
    double *D2;              // seeds x n
    int32_t *A;              // seeds x n: nearest chosen center so far (k-means++ skip test)
    float *D2f;              // seeds x n: D2 rounded up to FP32 (the certified tests' copy)
    float *ccf;              // seeds x k: squared distances of the newest center to the earlier ones, rounded down
    int64_t *dirty;          // seeds: the block of the last pick (its sum is refreshed in the next round)
    double *bsum;            // seeds x nb
    int32_t *stop;           // seeds
    const double *u;         // seeds x k uniforms
    int64_t pair0;           // index of (this problem, seed 0) among all pairs
    int64_t crow0;           // first row of this problem among all centers rows (seeds x kps each)
    int64_t tile0;           // first global row tile
};
constexpr int BCAND_MAX = 4;     // candidates listed per flagged (problem, seed, point)
constexpr int BFLAG_STRIDE = 4 + BCAND_MAX;  // flag entry: problem, seed, row, count (-1: all), candidates

// batched tcgen05 distance GEMM over the (problem, row tile) work list; maps: 3 tensor maps per
// problem (X operand, center operand, TF32 low part) in global memory, 64-byte aligned
int launch_assign_tc_batched(gbkm_ctx *c, int dtype, const void *maps, const BProb *probs, int64_t nprob,
                             const int32_t *tile_prob, int64_t ntiles, int parity, int bn_max,
                             int32_t *flags, int32_t *flag_count);
bool tc_batched_supported(int dtype, int64_t d, int64_t k, int64_t seeds);
int batch_run(gbkm_ctx *c, const gbkm_problem *up, int64_t count, int64_t seeds, int64_t iters, int dtype,
              int flags, const int *bn_caps);
// fastest center-chunk width (64, 128 or 256 columns) of the tcgen05 assignment for this shape
int autotune_bn(gbkm_ctx *c, int dtype, int64_t d, int64_t ncols, int *bn_out);
// the single-problem assignment's tuned configuration: engine (GBKM_ENGINE_SIMT or _TCGEN05), center-chunk
// width and stage-ring depth (0: as many as fit)
struct TuneChoice {
    int engine, bn, stages;
};
// times the candidates for this shape (or returns the cached choice)
int autotune_assign(gbkm_ctx *c, int dtype, int64_t d, int64_t ncols, TuneChoice *out);
// the cached choice for this shape, without timing anything; false when the shape was never tuned
bool tuned_assign(gbkm_ctx *c, int dtype, int64_t d, int64_t ncols, TuneChoice *out);
int make_batch_tmaps(gbkm_ctx *c, int dtype, const BProb &P, void *host_maps3);
}  // namespace gbkm
