// api.cu -- the C ABI declared in include/gbkm.h: context, workspace, argument checks and the
// orchestration of the kernels of one call on the context's stream.
#include <math.h>
#include <string.h>

#include <map>
#include <mutex>
#include <new>
#include <vector>

#include "internal.cuh"

#define GBKM_VERSION 10000

int set_error(gbkm_ctx *c, int code, const char *fmt, ...) {
    if (c) {
        va_list ap;
        va_start(ap, fmt);
        vsnprintf(c->err, sizeof(c->err), fmt, ap);
        va_end(ap);
    }
    return code;
}

int cuda_check(gbkm_ctx *c, cudaError_t e, const char *what) {
    if (e == cudaSuccess) return GBKM_OK;
    return set_error(c, GBKM_ECUDA, "%s: %s", what, cudaGetErrorString(e));
}

void *ws_reserve(gbkm_ctx *c, size_t bytes, int *rc) {
    c->ws_epoch++;
    if (bytes <= c->ws_bytes) return c->ws;
    cudaError_t e = cudaStreamSynchronize(c->stream);  // the old block may still be in use
    if (e != cudaSuccess) {
        *rc = cuda_check(c, e, "workspace sync");
        return nullptr;
    }
    if (c->ws) cudaFree(c->ws);
    c->ws = nullptr;
    c->ws_bytes = 0;
    size_t want = bytes + (bytes >> 3) + (1 << 20);
    if (c->fail_alloc > 0) {
        // a failure injected by gbkm_debug_fail_alloc: the same path as a failed cudaMalloc
        c->fail_alloc--;
        *rc = set_error(c, GBKM_ENOMEM, "workspace of %zu bytes: allocation failure injected", want);
        return nullptr;
    }
    e = cudaMalloc(&c->ws, want);
    if (e != cudaSuccess) {
        cudaGetLastError();
        *rc = set_error(c, GBKM_ENOMEM, "workspace of %zu bytes: %s", want, cudaGetErrorString(e));
        return nullptr;
    }
    c->ws_bytes = want;
    return c->ws;
}

void prof_begin(gbkm_ctx *c, const char *name) {
    if (!c->prof) return;
    while (c->pool.size() < c->pool_used + 2) {
        cudaEvent_t e;
        if (cudaEventCreate(&e) != cudaSuccess) {
            cudaGetLastError();
            c->prof_open.push_back(SIZE_MAX);  // keeps begin/end pairs matched
            return;
        }
        c->pool.push_back(e);
    }
    ProfRec r{name, c->pool[c->pool_used], c->pool[c->pool_used + 1]};
    c->pool_used += 2;
    cudaEventRecord(r.a, c->stream);
    c->recs.push_back(r);
    c->prof_open.push_back(c->recs.size() - 1);
}

// closes the innermost open bracket (brackets nest: a composite call may time its parts)
void prof_end(gbkm_ctx *c) {
    if (!c->prof || c->prof_open.empty()) return;
    const size_t i = c->prof_open.back();
    c->prof_open.pop_back();
    if (i != SIZE_MAX) cudaEventRecord(c->recs[i].b, c->stream);
}

namespace {
struct DeviceGuard {
    int prev = -1;
    explicit DeviceGuard(int dev) {
        cudaGetDevice(&prev);
        if (prev != dev) cudaSetDevice(dev);
    }
    ~DeviceGuard() {
        int cur = -1;
        cudaGetDevice(&cur);
        if (prev >= 0 && cur != prev) cudaSetDevice(prev);
    }
};

bool aligned16(const void *p) { return (reinterpret_cast<uintptr_t>(p) & 15) == 0; }

// page-locked, device-mapped host blocks handed out by gbkm_host_alloc: base address -> bytes
std::mutex g_host_mu;
std::map<uintptr_t, size_t> g_host_blocks;

// the gbkm_host_alloc block holding all of [p, p + bytes), or 0
uintptr_t host_block_of(const void *p, size_t bytes) {
    std::lock_guard<std::mutex> lock(g_host_mu);
    const uintptr_t q = reinterpret_cast<uintptr_t>(p);
    auto it = g_host_blocks.upper_bound(q);
    if (it == g_host_blocks.begin()) return 0;
    --it;
    const uintptr_t b = it->first;
    const size_t sz = it->second;
    if (q - b >= sz || bytes > sz - (q - b)) return 0;
    return b;
}

}  // namespace

namespace gbkm {
int rsvd_impl(gbkm_ctx *c, const float *A, int64_t n, int64_t d, const float *w, const float *Omega, int64_t s,
              int64_t ell, float *V, float *sigma, int32_t *info);
int launch_ingest(gbkm_ctx *c, const float *src, int64_t n, int64_t d, float *xdev, float *xnorm, void *xq,
                  float *resid);
}

namespace gbkm {
// worst-case relative error coefficients of the distance scores of each operand format:
// |score_err| <= err_rel ||x|| max||c|| + err_abs max||c||^2 (see the certified near-tie rule)
void score_error_coeffs(int dtype, int engine_tc, int64_t d, float &err_rel, float &err_abs) {
    const double u = ldexp(1.0, -24);
    double dot;
    if (!engine_tc) {
        // FP32 FFMA chain: gamma_d = d u / (1 - d u)
        dot = (double)d * u / (1.0 - (double)d * u);
    } else if (dtype == GBKM_F32) {
        // 3xTF32: representation error 3.01 * 2^-20, accumulation of 3d terms at 2^-22 each
        dot = 3.01 * ldexp(1.0, -20) + 3.0 * (double)d * ldexp(1.0, -22) * 1.003;
    } else if (dtype == GBKM_BF16) {
        const double uq = ldexp(1.0, -8);
        dot = 2 * uq + uq * uq + (double)d * ldexp(1.0, -22) * (1 + uq) * (1 + uq);
    } else {
        // E4M3 with power-of-two per-row scales, d <= 128: normal range 2^-4, subnormal absolute
        // term folded in via max|x|/448 <= ||x||/224; accumulation assumed no better than 14 bits
        const double uq = ldexp(1.0, -4);
        dot = 2 * uq + uq * uq + 2.0 * ldexp(1.0, -10) * sqrt((double)d) / 224.0 * (1 + uq) +
              ldexp(1.0, -20) * (double)d / (224.0 * 224.0) + (double)d * ldexp(1.0, -13) * 1.3;
    }
    err_rel = (float)((2.0 * dot + 2.0 * u) * (1.0 + 1e-3));
    err_abs = (float)(3.0 * u * (1.0 + 1e-3));
}
}  // namespace gbkm

extern "C" {

int gbkm_version(void) { return GBKM_VERSION; }

int gbkm_create(gbkm_ctx **out, int device, void *cuda_stream) {
    if (!out) return GBKM_EINVAL;
    *out = nullptr;
    gbkm_ctx *c = new (std::nothrow) gbkm_ctx();
    if (!c) return GBKM_ENOMEM;
    c->device = device;
    c->stream = (cudaStream_t)cuda_stream;
    DeviceGuard g(device);
    cudaError_t e = cudaDeviceGetAttribute(&c->sm_count, cudaDevAttrMultiProcessorCount, device);
    if (e == cudaSuccess) e = cudaMalloc(&c->status, 256);
    if (e == cudaSuccess) e = cudaMemset(c->status, 0, 256);
    if (e != cudaSuccess) {
        cudaGetLastError();
        if (c->status) cudaFree(c->status);
        delete c;
        return GBKM_ECUDA;
    }
    *out = c;
    return GBKM_OK;
}

int gbkm_profile_enable(gbkm_ctx *c, int enable) {
    if (!c) return GBKM_EINVAL;
    c->prof = enable != 0;
    c->recs.clear();
    c->prof_open.clear();
    c->pool_used = 0;
    return GBKM_OK;
}

int gbkm_profile_read(gbkm_ctx *c, char *buf, int64_t len) {
    if (!c || !buf || len < 1) return GBKM_EINVAL;
    DeviceGuard g(c->device);
    cudaError_t e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return cuda_check(c, e, "profile sync");
    struct Acc {
        const char *name;
        int64_t launches;
        double ms;
    };
    std::vector<Acc> acc;
    for (const ProfRec &r : c->recs) {
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, r.a, r.b) != cudaSuccess) {
            cudaGetLastError();
            continue;
        }
        size_t q = 0;
        while (q < acc.size() && strcmp(acc[q].name, r.name) != 0) ++q;
        if (q == acc.size()) acc.push_back({r.name, 0, 0.0});
        acc[q].launches += 1;
        acc[q].ms += ms;
    }
    c->recs.clear();
    c->prof_open.clear();
    c->pool_used = 0;
    int64_t off = 0;
    buf[0] = 0;
    for (const Acc &a : acc) {
        int w = snprintf(buf + off, (size_t)(len - off), "%s %lld %.6f\n", a.name, (long long)a.launches, a.ms);
        if (w < 0 || off + w >= len) break;
        off += w;
    }
    return (int)acc.size();
}

int gbkm_debug_set_wait_limit(gbkm_ctx *c, uint64_t ns) {
    if (!c) return GBKM_EINVAL;
    c->wait_ns = ns;
    return GBKM_OK;
}

int gbkm_debug_stall_loads(gbkm_ctx *c, int on) {
    if (!c) return GBKM_EINVAL;
    c->stall_loads = on != 0;
    return GBKM_OK;
}

int gbkm_debug_fail_alloc(gbkm_ctx *c, int count) {
    if (!c || count < 0) return GBKM_EINVAL;
    c->fail_alloc = count;
    return GBKM_OK;
}

int gbkm_destroy(gbkm_ctx *c) {
    if (!c) return GBKM_OK;
    DeviceGuard g(c->device);
    cudaStreamSynchronize(c->stream);
    if (c->graph_exec) cudaGraphExecDestroy((cudaGraphExec_t)c->graph_exec);
    if (c->cap_stream) cudaStreamDestroy(c->cap_stream);
    for (cudaEvent_t e : c->pool) cudaEventDestroy(e);
    if (c->ws) cudaFree(c->ws);
    if (c->status) cudaFree(c->status);
    if (c->tmap_scratch) cudaFree(c->tmap_scratch);
    delete c;
    return GBKM_OK;
}

int gbkm_set_stream(gbkm_ctx *c, void *cuda_stream) {
    if (!c) return GBKM_EINVAL;
    c->stream = (cudaStream_t)cuda_stream;
    return GBKM_OK;
}

const char *gbkm_last_error(const gbkm_ctx *c) { return c ? c->err : "null context"; }

int64_t gbkm_launch_count(const gbkm_ctx *c) { return c ? c->launches : 0; }

int gbkm_sync(gbkm_ctx *c) {
    if (!c) return GBKM_EINVAL;
    DeviceGuard g(c->device);
    cudaError_t e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return cuda_check(c, e, "stream synchronize");
    int st = 0;
    e = cudaMemcpy(&st, c->status, sizeof(int), cudaMemcpyDeviceToHost);
    if (e == cudaSuccess) e = cudaMemset(c->status, 0, sizeof(int));
    if (e != cudaSuccess) return cuda_check(c, e, "status read");
    if (st & ST_TIMEOUT) return set_error(c, GBKM_ETIMEOUT, "a bounded device wait timed out");
    if (st & ST_BADLABEL) return set_error(c, GBKM_EINVAL, "a label outside [0, k) reached kmeans_update");
    if (st & ST_BOUNDS) return set_error(c, GBKM_ECUDA, "an internal index check failed");
    if (st & ST_DEGENERATE)
        return set_error(c, GBKM_EDEGENERATE, "k-means++: fewer than k points with positive D^2");
    return GBKM_OK;
}

int kmeans_row_norms(gbkm_ctx *c, const float *X, int64_t n, int64_t d, float *xnorm) {
    if (!c) return GBKM_EINVAL;
    if (n < 1 || d < 1 || !X || !xnorm) return set_error(c, GBKM_EINVAL, "row_norms: bad arguments");
    DeviceGuard g(c->device);
    prof_begin(c, "row_norms");
    const int rc = gbkm::launch_row_norms(c, X, n, d, xnorm);
    prof_end(c);
    return rc;
}

int kmeans_quantize(gbkm_ctx *c, const float *X, int64_t n, int64_t d, int32_t dtype, void *Xq,
                    float *scales) {
    if (!c) return GBKM_EINVAL;
    if (n < 1 || d < 1 || !X || !Xq) return set_error(c, GBKM_EINVAL, "quantize: bad arguments");
    if (dtype != GBKM_BF16 && dtype != GBKM_FP8E4M3)
        return set_error(c, GBKM_EINVAL, "quantize: dtype must be BF16 or FP8E4M3");
    if (dtype == GBKM_FP8E4M3 && !scales) return set_error(c, GBKM_EINVAL, "quantize: FP8 needs scales");
    if (!aligned16(Xq)) return set_error(c, GBKM_EINVAL, "quantize: Xq must be 16-byte aligned");
    DeviceGuard g(c->device);
    prof_begin(c, "quantize");
    const int rc = gbkm::launch_quantize(c, X, n, d, dtype, Xq, scales);
    prof_end(c);
    return rc;
}

int gbkm_host_alloc(size_t bytes, void **out) {
    if (!out || bytes == 0) return GBKM_EINVAL;
    *out = nullptr;
    void *p = nullptr;
    const cudaError_t e = cudaHostAlloc(&p, bytes, cudaHostAllocMapped | cudaHostAllocPortable);
    if (e != cudaSuccess || !p) {
        cudaGetLastError();
        return GBKM_ENOMEM;
    }
    {
        std::lock_guard<std::mutex> lock(g_host_mu);
        g_host_blocks[reinterpret_cast<uintptr_t>(p)] = bytes;
    }
    *out = p;
    return GBKM_OK;
}

int gbkm_host_free(void *p) {
    if (!p) return GBKM_OK;
    {
        std::lock_guard<std::mutex> lock(g_host_mu);
        auto it = g_host_blocks.find(reinterpret_cast<uintptr_t>(p));
        if (it == g_host_blocks.end()) return GBKM_EINVAL;
        g_host_blocks.erase(it);
    }
    if (cudaFreeHost(p) != cudaSuccess) {
        cudaGetLastError();
        return GBKM_ECUDA;
    }
    return GBKM_OK;
}

int kmeans_ingest(gbkm_ctx *c, const float *X_src, int64_t n, int64_t d, float *X_dev, float *xnorm,
                  void *Xq, float *resid) {
    if (!c) return GBKM_EINVAL;
    if (n < 1 || d < 1 || !X_src) return set_error(c, GBKM_EINVAL, "ingest: bad arguments");
    if (resid && !Xq) return set_error(c, GBKM_EINVAL, "ingest: resid needs Xq");
    if (Xq && !aligned16(Xq)) return set_error(c, GBKM_EINVAL, "ingest: Xq must be 16-byte aligned");
    if (X_dev && !aligned16(X_dev)) return set_error(c, GBKM_EINVAL, "ingest: X_dev must be 16-byte aligned");
    if (X_dev == X_src) return set_error(c, GBKM_EINVAL, "ingest: X_dev may not be X_src");
    if ((uint64_t)n > (uint64_t)INT64_MAX / 4 / (uint64_t)d)
        return set_error(c, GBKM_EINVAL, "ingest: n x d overflows");
    DeviceGuard g(c->device);
    const size_t bytes = (size_t)n * (size_t)d * sizeof(float);
    const float *src = nullptr;
    if (const uintptr_t b = host_block_of(X_src, bytes)) {
        // the block's address in this device's address space
        void *dbase = nullptr;
        const cudaError_t e = cudaHostGetDevicePointer(&dbase, reinterpret_cast<void *>(b), 0);
        if (e != cudaSuccess || !dbase) return cuda_check(c, e != cudaSuccess ? e : cudaErrorInvalidValue, "ingest: mapped host block");
        src = reinterpret_cast<const float *>(static_cast<char *>(dbase) + (reinterpret_cast<uintptr_t>(X_src) - b));
    } else {
        cudaPointerAttributes at;
        const cudaError_t e = cudaPointerGetAttributes(&at, X_src);
        if (e != cudaSuccess) {
            cudaGetLastError();
            return set_error(c, GBKM_EINVAL, "ingest: X_src is neither device memory nor a gbkm_host_alloc block");
        }
        if (at.type != cudaMemoryTypeDevice && at.type != cudaMemoryTypeManaged)
            return set_error(c, GBKM_EINVAL, "ingest: X_src is neither device memory nor a gbkm_host_alloc block");
        src = X_src;
    }
    prof_begin(c, "ingest");
    const int rc = gbkm::launch_ingest(c, src, n, d, X_dev, xnorm, Xq, resid);
    prof_end(c);
    return rc;
}

int kmeans_rsvd(gbkm_ctx *c, const float *A, int64_t n, int64_t d, const float *w, const float *Omega,
                int64_t s, int64_t ell, float *V, float *sigma, int32_t *info) {
    if (!c) return GBKM_EINVAL;
    if (!A || !Omega || !V || n < 1 || d < 1) return set_error(c, GBKM_EINVAL, "rsvd: bad arguments");
    if (s < 16 || s > 128 || s % 16 != 0 || ell < 1 || ell > s || s > n || s > d)
        return set_error(c, GBKM_EINVAL, "rsvd: need 16 <= s <= 128, s %% 16 == 0, 1 <= ell <= s <= min(n, d)");
    if (n >= ((int64_t)1 << 31) || d >= ((int64_t)1 << 31)) return set_error(c, GBKM_EUNSUPPORTED, "rsvd: n or d too large");
    DeviceGuard g(c->device);
    prof_begin(c, "rsvd");
    const int rc = gbkm::rsvd_impl(c, A, n, d, w, Omega, s, ell, V, sigma, info);
    prof_end(c);
    return rc;
}

int kmeans_project_block(gbkm_ctx *c, const void *X, int32_t xt, int64_t n, int64_t d,
                         const float *V, int64_t r, float *Y, float *X_lift) {
    if (!c) return GBKM_EINVAL;
    if (n < 1 || d < 1 || r < 1 || r > d || !X || !V || !Y)
        return set_error(c, GBKM_EINVAL, "project_block: bad arguments");
    if (xt != GBKM_F32 && xt != GBKM_BF16)
        return set_error(c, GBKM_EINVAL, "project_block: X dtype must be F32 or BF16");
    DeviceGuard g(c->device);
    int rc;
    prof_begin(c, "project");
    if (gbkm::tc_project_supported(xt, d, r) && aligned16(X)) {
        rc = gbkm::launch_project_tc(c, xt, X, n, d, V, r, Y);
    } else if (xt == GBKM_F32) {
        // Y[n x r] = X V: B addressed as V[kk * r + nn]
        rc = gbkm::launch_gemm_simt_strided(c, (const float *)X, V, n, r, d, 1, r, Y);
    } else {
        prof_end(c);
        return set_error(c, GBKM_EUNSUPPORTED, "project_block: BF16 X needs r %% 16 == 0, r <= 256, d %% 64 == 0");
    }
    prof_end(c);
    if (rc != GBKM_OK || !X_lift) return rc;
    // X_lift[n x d] = Y V^T: B = V as an N x K (d x r) row-major matrix
    prof_begin(c, "lift");
    if (gbkm::tc_lift_supported(d, r) && aligned16(Y) && aligned16(X_lift))
        rc = gbkm::launch_lift_tc(c, Y, n, r, V, d, X_lift);
    else
        rc = gbkm::launch_gemm_simt_strided(c, Y, V, n, d, r, r, 1, X_lift);
    prof_end(c);
    return rc;
}

int kmeans_seed_pp(gbkm_ctx *c, const float *X, int64_t n, int64_t d, const float *w, int64_t k,
                   const double *u, int64_t *idx_out, float *C_out) {
    if (!c) return GBKM_EINVAL;
    if (n < 1 || d < 1 || k < 1 || k > n || !X || !u || !idx_out || !C_out)
        return set_error(c, GBKM_EINVAL, "seed_pp: bad arguments (need 1 <= k <= n)");
    DeviceGuard g(c->device);
    prof_begin(c, "seed");
    int rc = gbkm::seed_impl(c, X, n, d, w, k, u, idx_out, C_out);
    prof_end(c);
    return rc;
}

int kmeans_seed_pp_q(gbkm_ctx *c, const float *X, const void *Xq, const float *xresid, int64_t n, int64_t d,
                     const float *w, int64_t k, const double *u, int64_t *idx_out, float *C_out) {
    if (!c) return GBKM_EINVAL;
    if (n < 1 || d < 1 || k < 1 || k > n || !X || !u || !idx_out || !C_out || !Xq || !xresid)
        return set_error(c, GBKM_EINVAL, "seed_pp_q: bad arguments (need 1 <= k <= n, Xq and xresid)");
    DeviceGuard g(c->device);
    prof_begin(c, "seed");
    int rc = gbkm::seed_impl(c, X, n, d, w, k, u, idx_out, C_out, Xq, xresid);
    prof_end(c);
    return rc;
}

int kmeans_assign(gbkm_ctx *c, const void *Xop, const float *Xop_scales, const float *X,
                  const float *xnorm, int64_t n, int64_t d, const float *C, int64_t k,
                  const gbkm_assign_opts *opts, int32_t *labels, float *min_d2, int64_t *n_rechecked) {
    if (!c) return GBKM_EINVAL;
    gbkm_assign_opts o = {GBKM_F32, GBKM_ENGINE_AUTO, 1, 1};
    if (opts) o = *opts;
    if (n < 1 || d < 1 || k < 1 || k > 65536 || !X || !C || !labels)
        return set_error(c, GBKM_EINVAL, "assign: bad arguments");
    if (o.compute != GBKM_F32 && o.compute != GBKM_BF16 && o.compute != GBKM_FP8E4M3)
        return set_error(c, GBKM_EINVAL, "assign: unknown compute dtype %d", o.compute);
    if (o.compute != GBKM_F32 && !Xop) return set_error(c, GBKM_EINVAL, "assign: Xop required");
    if (o.compute == GBKM_FP8E4M3 && (!Xop_scales || d > 128))
        return set_error(c, GBKM_EINVAL, "assign: FP8 needs per-row scales and d <= 128");
    if (!Xop) Xop = X;
    const bool tc_ok = gbkm::tc_assign_supported(o.compute, d, k) && aligned16(Xop);
    bool use_tc;
    if (o.engine == GBKM_ENGINE_SIMT) {
        if (o.compute != GBKM_F32) return set_error(c, GBKM_EUNSUPPORTED, "assign: SIMT engine is FP32 only");
        use_tc = false;
    } else if (o.engine == GBKM_ENGINE_TCGEN05) {
        if (!tc_ok) return set_error(c, GBKM_EUNSUPPORTED, "assign: shape/dtype not supported by tcgen05 engine");
        use_tc = true;
    } else {
        use_tc = tc_ok;
        if (!use_tc && o.compute != GBKM_F32)
            return set_error(c, GBKM_EUNSUPPORTED, "assign: low-precision forms need the tcgen05 engine");
    }
    // a configuration the autotuner chose for this shape (kmeans_autotune_assign) replaces the default
    // one under GBKM_ENGINE_AUTO: the engine, the center-chunk width and the stage-ring depth
    gbkm::TuneChoice tuned{0, 0, 0};
    const bool has_tune = o.engine == GBKM_ENGINE_AUTO && gbkm::tuned_assign(c, o.compute, d, k, &tuned) &&
                          (tuned.engine == GBKM_ENGINE_SIMT ? o.compute == GBKM_F32 : tc_ok);
    if (has_tune) use_tc = tuned.engine == GBKM_ENGINE_TCGEN05;
    struct CapGuard {
        gbkm_ctx *c;
        int bn, st;
        ~CapGuard() { c->bn_cap = bn, c->stage_cap = st; }
    } capg{c, c->bn_cap, c->stage_cap};
    if (has_tune && use_tc) c->bn_cap = tuned.bn, c->stage_cap = tuned.stages;
    DeviceGuard g(c->device);
    const int64_t k_pad = use_tc ? ceil_div(k, 16) * 16 : k;
    // BF16 centers as two BF16 terms (hi + lo) on request: the near-tie bound then grows with the
    // point's distances to the two centers instead of with max ||c||
    const bool split = use_tc && o.compute == GBKM_BF16 && o.center_terms == 2;
    const size_t esz = o.compute == GBKM_BF16 ? 2 : (o.compute == GBKM_FP8E4M3 ? 1 : 4);
    // escalation: rows of a low-precision form whose near-tie band is too wide to list go through the
    // 3xTF32 form (a far smaller error bound), then through the exact recheck
    const bool esc = use_tc && o.recheck && o.compute != GBKM_F32 && gbkm::tc_assign_supported(GBKM_F32, d, k) &&
                     aligned16(X) && (d % 4) == 0;
    const int64_t ne = esc ? n : 0;
    WsPlan p;
    // o_cm: the call's counters, zeroed by one memset: cmax, emax, flag count, escalation count (2)
    size_t o_xn = p.take<float>(xnorm ? 0 : n), o_cn = p.take<float>(k_pad), o_cm = p.take<unsigned>(8),
           o_cop = p.take<char>(use_tc ? k_pad * d * esz : 0),
           o_clo = p.take<float>(use_tc && (o.compute == GBKM_F32 || split) ? k_pad * d : 0),
           o_cs = p.take<float>(k_pad), o_fl = p.take<int32_t>(n), o_cd = p.take<int32_t>(n * gbkm::CAND_STRIDE),
           o_fc = o_cm + 2 * sizeof(unsigned);
    size_t o_el = p.take<int32_t>(ne), o_ec = o_cm + 3 * sizeof(unsigned), o_xe = p.take<float>(ne * d),
           o_xne = p.take<float>(ne), o_ehi = p.take<float>(esc ? k_pad * d : 0),
           o_elo = p.take<float>(esc ? k_pad * d : 0), o_fl2 = p.take<int32_t>(ne),
           o_cd2 = p.take<int32_t>(ne * gbkm::CAND_STRIDE);
    int rc = GBKM_OK;
    void *ws = ws_reserve(c, p.off, &rc);
    if (!ws) return rc;
    float *xn = xnorm ? const_cast<float *>(xnorm) : ws_at<float>(ws, o_xn);
    if (!xnorm && (rc = gbkm::launch_row_norms(c, X, n, d, xn)) != GBKM_OK) return rc;
    gbkm::CenterPrep cp;
    cp.cnorm = ws_at<float>(ws, o_cn);
    cp.cmax = ws_at<unsigned>(ws, o_cm);
    if (cudaError_t e0 = cudaMemsetAsync(cp.cmax, 0, 8 * sizeof(unsigned), c->stream); e0 != cudaSuccess)
        return cuda_check(c, e0, "memset counters");
    // one-term BF16 with the rows' rounding residuals: the centers' largest residual as well
    cp.emax = (use_tc && o.compute == GBKM_BF16 && !split && Xop_scales) ? cp.cmax + 1 : nullptr;
    cp.cop = use_tc ? ws_at<void>(ws, o_cop) : nullptr;
    cp.cop_lo = (use_tc && (o.compute == GBKM_F32 || split)) ? ws_at<void>(ws, o_clo) : nullptr;
    cp.cscale = ws_at<float>(ws, o_cs);
    cp.esc_hi = esc ? ws_at<float>(ws, o_ehi) : nullptr;
    cp.esc_lo = esc ? ws_at<float>(ws, o_elo) : nullptr;
    prof_begin(c, "center_prep");
    rc = gbkm::launch_center_prep(c, C, k, d, o.compute, k_pad, cp);
    prof_end(c);
    if (rc != GBKM_OK) return rc;
    gbkm::AssignOut out;
    out.labels = labels;
    out.min_d2 = min_d2;
    out.flag_list = o.recheck ? ws_at<int32_t>(ws, o_fl) : nullptr;
    out.cand = ws_at<int32_t>(ws, o_cd);
    out.flag_count = ws_at<int32_t>(ws, o_fc);
    cudaError_t e = cudaSuccess;
    float err_rel, err_abs;
    gbkm::score_error_coeffs(o.compute, use_tc, d, err_rel, err_abs);
    prof_begin(c, use_tc ? "assign_tc" : "assign_simt");
    if (use_tc)
        rc = gbkm::launch_assign_tc(c, o.compute, Xop, Xop_scales, X, xn, n, d, cp, k, k_pad, err_rel,
                                    err_abs, out);
    else
        rc = gbkm::launch_assign_simt(c, X, xn, n, d, C, cp.cnorm, cp.cmax, k, err_rel, err_abs, out);
    prof_end(c);
    if (rc != GBKM_OK) return rc;
    if (o.recheck && esc) {
        gbkm::Escalation es;
        es.list = ws_at<int32_t>(ws, o_el);
        es.count = ws_at<int32_t>(ws, o_ec);
        es.Xe = ws_at<float>(ws, o_xe);
        es.xne = ws_at<float>(ws, o_xne);
        es.xnorm = xn;
        prof_begin(c, "recheck");
        rc = gbkm::launch_recheck(c, X, n, d, C, k, out, n_rechecked, &es);
        prof_end(c);
        if (rc != GBKM_OK) return rc;
        // the escalated rows: 3xTF32 assignment of the gathered block (row count on the device),
        // then the exact recheck of its own near-ties; results go straight to the rows' slots
        prof_begin(c, "escalate");
        gbkm::CenterPrep cp2 = cp;
        cp2.cop = cp.esc_hi;
        cp2.cop_lo = cp.esc_lo;
        cp2.cscale = nullptr;
        gbkm::AssignOut out2;
        out2.labels = labels;
        out2.min_d2 = min_d2;
        out2.flag_list = ws_at<int32_t>(ws, o_fl2);
        out2.cand = ws_at<int32_t>(ws, o_cd2);
        out2.flag_count = es.count + 1;
        float er2, ea2;
        gbkm::score_error_coeffs(GBKM_F32, 1, d, er2, ea2);
        if ((rc = gbkm::launch_assign_tc(c, GBKM_F32, es.Xe, nullptr, es.Xe, es.xne, n, d, cp2, k, k_pad, er2, ea2,
                                         out2, es.count, es.list)) == GBKM_OK)
            rc = gbkm::launch_recheck(c, es.Xe, n, d, C, k, out2, nullptr, nullptr, es.list);
        prof_end(c);
        return rc;
    }
    if (o.recheck) {
        prof_begin(c, "recheck");
        rc = gbkm::launch_recheck(c, X, n, d, C, k, out, n_rechecked);
        prof_end(c);
        return rc;
    }
    if (n_rechecked) {
        e = cudaMemsetAsync(n_rechecked, 0, sizeof(int64_t), c->stream);
        if (e != cudaSuccess) return cuda_check(c, e, "memset n_rechecked");
    }
    return GBKM_OK;
}

int kmeans_update(gbkm_ctx *c, const float *X, int64_t n, int64_t d, const float *w,
                  const int32_t *labels, int64_t k, const float *C_old, float *C_new, double *counts,
                  double *cost_old, double *cost_new, int64_t *n_empty) {
    if (!c) return GBKM_EINVAL;
    if (n < 1 || d < 1 || k < 1 || k > 65536 || !X || !labels || !C_old || !C_new || C_old == C_new)
        return set_error(c, GBKM_EINVAL, "update: bad arguments");
    if (n >= ((int64_t)1 << 31)) return set_error(c, GBKM_EUNSUPPORTED, "update: n >= 2^31");
    DeviceGuard g(c->device);
    prof_begin(c, "update");
    int rc = gbkm::update_impl(c, X, n, d, w, labels, k, C_old, C_new, counts, cost_old, cost_new, n_empty);
    prof_end(c);
    return rc;
}

int kmeans_batch_run(gbkm_ctx *c, const gbkm_problem *probs, int64_t count, int64_t seeds, int64_t iters,
                     int32_t compute, int32_t flags) {
    if (!c) return GBKM_EINVAL;
    if (!probs || count < 1 || seeds < 1 || seeds > 8 || iters < 0)
        return set_error(c, GBKM_EINVAL, "batch_run: bad arguments");
    if (compute != GBKM_F32 && compute != GBKM_BF16)
        return set_error(c, GBKM_EINVAL, "batch_run: compute must be F32 or BF16");
    for (int64_t p = 0; p < count; ++p) {
        const gbkm_problem &q = probs[p];
        if (!q.X || !q.u || !q.C_out || q.n < 1 || q.k < 1 || q.k > q.n || q.n >= ((int64_t)1 << 31) ||
            !aligned16(q.X))
            return set_error(c, GBKM_EINVAL, "batch_run: problem %lld has bad arguments", (long long)p);
        if (!gbkm::tc_batched_supported(compute, q.d, q.k, seeds))
            return set_error(c, GBKM_EUNSUPPORTED, "batch_run: problem %lld needs d %% 16 == 0 and k <= 1024",
                             (long long)p);
    }
    DeviceGuard g(c->device);
    std::vector<int> caps(count, 256);
    if (flags & GBKM_BATCH_AUTOTUNE) {
        for (int64_t p = 0; p < count; ++p) {
            int bn = 256;
            const int64_t ncols = seeds * ((probs[p].k + 15) / 16 * 16);
            int rc = gbkm::autotune_bn(c, compute, probs[p].d, ncols, &bn);
            if (rc != GBKM_OK) return rc;
            caps[p] = bn;
        }
    }
    prof_begin(c, "batch_run");
    int rc = gbkm::batch_run(c, probs, count, seeds, iters, compute, flags, caps.data());
    prof_end(c);
    return rc;
}

int kmeans_batch_replay(gbkm_ctx *c) {
    if (!c) return GBKM_EINVAL;
    if (!c->graph_exec || c->graph_epoch != c->ws_epoch)
        return set_error(c, GBKM_EINVAL, "batch_replay: no recorded batched graph, or the workspace was reused since");
    DeviceGuard g(c->device);
    prof_begin(c, "batch_run");
    cudaError_t e = cudaGraphLaunch((cudaGraphExec_t)c->graph_exec, c->stream);
    prof_end(c);
    if (e == cudaSuccess) c->launches += c->graph_launches;  // every recorded kernel runs again
    return cuda_check(c, e, "graph launch");
}

int kmeans_autotune(gbkm_ctx *c, int32_t compute, int64_t d, int64_t ncols, int32_t *bn_out) {
    if (!c) return GBKM_EINVAL;
    if (!bn_out || d < 1 || ncols < 1) return set_error(c, GBKM_EINVAL, "autotune: bad arguments");
    DeviceGuard g(c->device);
    int bn = 256;
    int rc = gbkm::autotune_bn(c, compute, d, ncols, &bn);
    *bn_out = bn;
    return rc;
}

int kmeans_autotune_assign(gbkm_ctx *c, int32_t compute, int64_t d, int64_t k, int32_t *engine_out, int32_t *bn_out,
                           int32_t *stages_out) {
    if (!c) return GBKM_EINVAL;
    if (d < 1 || k < 1 || k > 65536 || (compute != GBKM_F32 && compute != GBKM_BF16))
        return set_error(c, GBKM_EINVAL, "autotune_assign: bad arguments (F32 or BF16, 1 <= k <= 65536)");
    DeviceGuard g(c->device);
    gbkm::TuneChoice t{0, 0, 0};
    const int rc = gbkm::autotune_assign(c, compute, d, k, &t);
    if (rc != GBKM_OK) return rc;
    if (engine_out) *engine_out = t.engine;
    if (bn_out) *bn_out = t.bn;
    if (stages_out) *stages_out = t.stages;
    return GBKM_OK;
}

int64_t kmeans_mlp_param_count(int64_t d_in, int64_t hidden, int64_t k) {
    gbkm_mlp m{};
    m.d_in = d_in, m.hidden = hidden, m.k = k;
    return gbkm::mlp_param_count(&m);
}

int kmeans_gemm_bf16(gbkm_ctx *c, const void *A, const void *B, int64_t M, int64_t N, int64_t K, const float *bias,
                     int32_t act, int32_t out_bf16, void *Y, int64_t ldy) {
    if (!c) return GBKM_EINVAL;
    if (!A || !B || !Y || M < 1 || ldy < N || !aligned16(A) || !aligned16(B) || !aligned16(Y) || (act != 0 && act != 1))
        return set_error(c, GBKM_EINVAL, "gemm: bad arguments");
    DeviceGuard g(c->device);
    prof_begin(c, "gemm");
    int rc = gbkm::launch_gemm_bf16_tc(c, A, B, M, N, K, bias, act, out_bf16, Y, ldy, nullptr, 0, nullptr, nullptr, 0);
    prof_end(c);
    return rc;
}

int kmeans_mlp_forward(gbkm_ctx *c, const gbkm_mlp *mlp, const void *Xh, int64_t n, float *logits, int32_t *top_idx,
                       int32_t topm, int32_t group) {
    if (!c) return GBKM_EINVAL;
    DeviceGuard g(c->device);
    prof_begin(c, "mlp_forward");
    int rc = gbkm::mlp_forward(c, mlp, Xh, n, logits, top_idx, topm, group);
    prof_end(c);
    return rc;
}

int kmeans_mlp_train_step(gbkm_ctx *c, gbkm_mlp *mlp, const void *Xh, const int32_t *labels, int64_t B, float lr,
                          float wd, float *loss_rows, float *grad_out) {
    if (!c) return GBKM_EINVAL;
    DeviceGuard g(c->device);
    prof_begin(c, "mlp_train_step");
    int rc = gbkm::mlp_train_step(c, mlp, Xh, labels, B, lr, wd, loss_rows, grad_out);
    prof_end(c);
    return rc;
}

int kmeans_center_separation(gbkm_ctx *c, const float *C, int64_t k, int64_t d, float *s2) {
    if (!c) return GBKM_EINVAL;
    if (!C || !s2 || k < 2 || d < 1) return set_error(c, GBKM_EINVAL, "center_separation: bad arguments");
    DeviceGuard g(c->device);
    return gbkm::center_separation(c, C, k, d, s2);
}

int kmeans_learned_assign(gbkm_ctx *c, const gbkm_mlp *mlp, const float *X, const void *Xh, int64_t n, int64_t d,
                          const float *C, int64_t k, const float *s2, int32_t topm, int32_t *labels,
                          int64_t *n_fallback, int32_t *cand_out) {
    if (!c) return GBKM_EINVAL;
    if (!X || !Xh || !C || !s2 || !labels || n < 1) return set_error(c, GBKM_EINVAL, "learned_assign: bad arguments");
    DeviceGuard g(c->device);
    prof_begin(c, "learned_assign");
    int rc = gbkm::learned_assign(c, mlp, X, Xh, n, d, C, k, s2, topm, labels, n_fallback, cand_out);
    prof_end(c);
    return rc;
}

int kmeans_cost(gbkm_ctx *c, const float *X, int64_t n, int64_t d, const float *w, const float *C,
                int64_t k, double *cost) {
    if (!c) return GBKM_EINVAL;
    if (n < 1 || d < 1 || k < 1 || k > 65536 || !X || !C || !cost)
        return set_error(c, GBKM_EINVAL, "cost: bad arguments");
    DeviceGuard g(c->device);
    // private scratch for the labels and a throwaway center copy, kept in its own allocation so
    // that the update's workspace plan does not overlap it
    int32_t *labels = nullptr;
    float *Cn = nullptr;
    cudaError_t e = cudaMallocAsync(&labels, sizeof(int32_t) * n, c->stream);
    if (e == cudaSuccess) e = cudaMallocAsync(&Cn, sizeof(float) * k * d, c->stream);
    if (e != cudaSuccess) {
        cudaGetLastError();
        if (labels) cudaFreeAsync(labels, c->stream);
        return set_error(c, GBKM_ENOMEM, "cost: scratch allocation failed");
    }
    gbkm_assign_opts o = {GBKM_F32, GBKM_ENGINE_AUTO, 1, 1};
    int rc = kmeans_assign(c, X, nullptr, X, nullptr, n, d, C, k, &o, labels, nullptr, nullptr);
    if (rc == GBKM_OK) rc = kmeans_update(c, X, n, d, w, labels, k, C, Cn, nullptr, cost, nullptr, nullptr);
    cudaFreeAsync(labels, c->stream);
    cudaFreeAsync(Cn, c->stream);
    return rc;
}

}  // extern "C"
