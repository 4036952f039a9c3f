/*
 * gbkm_diag.h -- diagnostics of the GB300 k-means library (no paper counterpart).
 *
 * Per-kernel timing with CUDA events recorded on the context's own stream, so
 * that a caller can measure one kernel's device time inside a longer sequence
 * without a profiler.  Host-side calls; ctx as in gbkm.h.
 */
#ifndef GBKM_DIAG_H
#define GBKM_DIAG_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

struct gbkm_ctx;

/* enable (1) or disable (0) event timing around the library's main kernels:
 * "row_norms", "quantize", "assign_simt", "assign_tc", "recheck", "escalate", "update" (part
 * "segsum": the segmented sums), "seed" (part "seed_d2": the rounds, each one launch), "project", "lift", "bico_take",
 * "piecy_lift", "rsvd" (parts "rsvd_sketch", "rsvd_qr", "rsvd_rows", "rsvd_small"),
 * "center_prep", "gemm", "mlp_forward", "mlp_hidden", "mlp_topm", "mlp_logits", "mlp_train_step",
 * "learned_assign", "cand_check", "fallback", "batch_run" and, for a batched run
 * that is not recorded into a graph, "seed_batched", "assign_batched",
 * "recheck_batched", "update_batched".  Brackets nest: a composite call is timed as a
 * whole and by its parts (so the parts' times also count in the whole's).
 * Enabling clears earlier records. */
int gbkm_profile_enable(struct gbkm_ctx *ctx, int enable);

/* Synchronise the stream, then write one line per kernel name,
 * "<name> <launches> <total_ms>\n", into buf (host, len bytes, NUL-terminated,
 * truncated if short) and clear the records.  Returns the number of names or a
 * negative gbkm_status. */
int gbkm_profile_read(struct gbkm_ctx *ctx, char *buf, int64_t len);

/* Failure detection without a GPU fault.
 *
 * gbkm_debug_set_wait_limit: every bounded device-side wait of the tensor-core kernels launched
 * on ctx afterwards gives up after ns nanoseconds instead of the default 2 s (0 restores the
 * default).  A wait that gives up makes its CTA stop issuing work, wait (at most 0.5 s) for its
 * copies and tensor-core operations in flight, free its tensor memory and exit; the outputs of
 * that call are then undefined, and the next gbkm_sync returns GBKM_ETIMEOUT and clears the
 * status, after which the context is usable again.
 *
 * gbkm_debug_stall_loads: with on != 0, the tensor-core kernels launched on ctx afterwards issue
 * none of their shared-memory copies, so the tensor-core issuer's first wait (for a copy that is
 * never made) runs out after the wait limit and the whole launch takes the path above: the way a
 * test makes a bounded wait give up without faulting the GPU.  0 turns it off.
 *
 * gbkm_debug_fail_alloc: the next `count` growths of ctx's workspace fail as a failed
 * cudaMalloc would (GBKM_ENOMEM, nothing queued by that call); 0 clears it.  Host-side only. */
/* Measured peak of one arithmetic unit on ctx's device, in TFLOP/s (host *tflops_out):
 *   unit 0: tcgen05.mma kind::f16 (BF16 operands, FP32 accumulation), 1: kind::tf32, 2: kind::f8f6f4
 *   (E4M3), each at the shape the library's tensor-core kernels issue (one CTA per SM,
 *   cta_group::1, M = 128, N = 256, operands resident in shared memory);
 *   3: FP32 FMA on the CUDA cores; 4: FP64 FMA.
 * A 3xTF32 product costs three kind::tf32 MMAs, so its peak is unit 1's figure / 3.
 * Runs a few tens of milliseconds of work and synchronises ctx's stream. */
int gbkm_probe_peak(struct gbkm_ctx *ctx, int32_t unit, double *tflops_out);

int gbkm_debug_set_wait_limit(struct gbkm_ctx *ctx, uint64_t ns);
int gbkm_debug_stall_loads(struct gbkm_ctx *ctx, int on);
int gbkm_debug_fail_alloc(struct gbkm_ctx *ctx, int count);

#ifdef __cplusplus
}
#endif
#endif /* GBKM_DIAG_H */
