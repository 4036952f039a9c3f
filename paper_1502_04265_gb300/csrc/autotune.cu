// autotune.cu -- the project's tile autotuner.  For one (compute dtype, d, number of centers) shape it
// times real assignments on a synthetic problem and keeps the fastest configuration: for the batched
// engine the center-chunk width (64, 128 or 256 columns); for the single-problem assignment the engine
// (CUDA cores or tcgen05, FP32), the chunk width and the depth of the shared-memory stage ring.
// Choices are cached per process and optionally in a text file (GBKM_TUNE_CACHE), one
// "gpu|dtype|d|ncols_pow2 bn" or "assign|gpu|dtype|d|ncols_pow2 engine:bn:stages" line per shape.
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "internal.cuh"

namespace gbkm {

namespace {
std::mutex g_tune_mu;
std::map<std::string, int> g_tune;
bool g_tune_loaded = false;

// deterministic pseudo-random fill (a hash of the index), values in [-8, 8)
__global__ void k_fill_synth(float *p, int64_t m, uint32_t salt) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= m) return;
    uint32_t h = (uint32_t)i * 2654435761u ^ salt;
    h ^= h >> 16;
    h *= 2246822519u;
    h ^= h >> 13;
    p[i] = (float)(h & 0xffffu) * (16.f / 65536.f) - 8.f;
}

std::map<int, std::string> g_dev_name;  // device ordinal -> name (looked up once)
std::map<std::string, TuneChoice> g_tune_assign;

// (called with g_tune_mu held)
std::string tune_key(gbkm_ctx *c, int dtype, int64_t d, int64_t ncols) {
    auto it = g_dev_name.find(c->device);
    if (it == g_dev_name.end()) {
        cudaDeviceProp prop;
        cudaGetDeviceProperties(&prop, c->device);
        it = g_dev_name.emplace(c->device, std::string(prop.name)).first;
    }
    int64_t p2 = 16;
    while (p2 < ncols) p2 <<= 1;
    return it->second + "|" + std::to_string(dtype) + "|" + std::to_string(d) + "|" + std::to_string(p2);
}

void load_file_cache() {
    if (g_tune_loaded) return;
    g_tune_loaded = true;
    const char *path = getenv("GBKM_TUNE_CACHE");
    if (!path) return;
    FILE *f = fopen(path, "r");
    if (!f) return;
    char line[512];
    while (fgets(line, sizeof line, f)) {
        char *sp = strrchr(line, ' ');
        if (!sp) continue;
        *sp = 0;
        if (strncmp(line, "assign|", 7) == 0) {
            TuneChoice t{0, 0, 0};
            if (sscanf(sp + 1, "%d:%d:%d", &t.engine, &t.bn, &t.stages) == 3) g_tune_assign[line] = t;
        } else {
            g_tune[line] = atoi(sp + 1);
        }
    }
    fclose(f);
}

void store_file_cache(const std::string &key, int bn) {
    const char *path = getenv("GBKM_TUNE_CACHE");
    if (!path) return;
    FILE *f = fopen(path, "a");
    if (!f) return;
    fprintf(f, "%s %d\n", key.c_str(), bn);
    fclose(f);
}
}  // namespace

int autotune_bn(gbkm_ctx *c, int dtype, int64_t d, int64_t ncols, int *bn_out) {
    std::string key;
    {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        key = tune_key(c, dtype, d, ncols);
        load_file_cache();
        auto it = g_tune.find(key);
        if (it != g_tune.end()) {
            *bn_out = it->second;
            return GBKM_OK;
        }
    }
    const int64_t kp = ceil_div(ncols, 16) * 16;
    if (kp <= 64 || !tc_assign_supported(dtype, d, ncols)) {  // one chunk whatever the cap
        *bn_out = 256;
        return GBKM_OK;
    }
    const int64_t n = 16384;
    float *X = nullptr, *C = nullptr, *xn = nullptr;
    void *Xop = nullptr;
    int32_t *lab = nullptr;
    cudaError_t e = cudaMalloc(&X, sizeof(float) * n * d);
    if (e == cudaSuccess) e = cudaMalloc(&C, sizeof(float) * ncols * d);
    if (e == cudaSuccess) e = cudaMalloc(&xn, sizeof(float) * n);
    if (e == cudaSuccess) e = cudaMalloc(&Xop, (size_t)n * d * 2);
    if (e == cudaSuccess) e = cudaMalloc(&lab, sizeof(int32_t) * n);
    int rc = GBKM_OK;
    std::vector<std::pair<float, int>> res;
    if (e == cudaSuccess) {
        k_fill_synth<<<(unsigned)ceil_div(n * d, 256), 256, 0, c->stream>>>(X, n * d, 0x1234u);
        k_fill_synth<<<(unsigned)ceil_div(ncols * d, 256), 256, 0, c->stream>>>(C, ncols * d, 0x9876u);
        c->launches += 2;
        rc = launch_row_norms(c, X, n, d, xn);
        if (rc == GBKM_OK && dtype == GBKM_BF16) rc = launch_quantize(c, X, n, d, GBKM_BF16, Xop, nullptr);
        cudaEvent_t a, b;
        cudaEventCreate(&a);
        cudaEventCreate(&b);
        gbkm_assign_opts o = {dtype, GBKM_ENGINE_TCGEN05, 0, 0};
        const int saved = c->bn_cap;
        for (int cap : {64, 128, 256}) {
            if (rc != GBKM_OK) break;
            if (cap > 64 && ceil_div(kp, cap) == ceil_div(kp, cap / 2)) continue;  // same chunking
            c->bn_cap = cap;
            float best = 1e30f;
            for (int rep = 0; rep < 4 && rc == GBKM_OK; ++rep) {
                cudaEventRecord(a, c->stream);
                rc = kmeans_assign(c, dtype == GBKM_BF16 ? Xop : X, nullptr, X, xn, n, d, C, ncols, &o, lab, nullptr,
                                   nullptr);
                cudaEventRecord(b, c->stream);
                cudaEventSynchronize(b);
                float ms = 0.f;
                cudaEventElapsedTime(&ms, a, b);
                if (rep > 0) best = std::min(best, ms);
            }
            res.push_back({best, cap});
        }
        c->bn_cap = saved;
        cudaEventDestroy(a);
        cudaEventDestroy(b);
    } else {
        cudaGetLastError();
        rc = set_error(c, GBKM_ENOMEM, "autotune: synthetic problem allocation failed");
    }
    cudaStreamSynchronize(c->stream);
    cudaFree(X);
    cudaFree(C);
    cudaFree(xn);
    cudaFree(Xop);
    cudaFree(lab);
    if (rc != GBKM_OK) return rc;
    int bn = 256;
    float bt = 1e30f;
    for (auto &r : res)
        if (r.first < bt) {
            bt = r.first;
            bn = r.second;
        }
    {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        g_tune[key] = bn;
        store_file_cache(key, bn);
    }
    *bn_out = bn;
    return GBKM_OK;
}

bool tuned_assign(gbkm_ctx *c, int dtype, int64_t d, int64_t ncols, TuneChoice *out) {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    load_file_cache();
    if (g_tune_assign.empty()) return false;
    auto it = g_tune_assign.find("assign|" + tune_key(c, dtype, d, ncols));
    if (it == g_tune_assign.end()) return false;
    *out = it->second;
    return true;
}

// The single-problem assignment's search: the tcgen05 engine over center-chunk widths {64, 128, 256}
// (distinct chunkings only) x stage rings {2, 3, as many as fit}, and for FP32 also the CUDA-core
// engine; each candidate timed on a synthetic 32,768-point problem of this shape (best of 3 after a
// warm-up), the fastest kept.
int autotune_assign(gbkm_ctx *c, int dtype, int64_t d, int64_t ncols, TuneChoice *out) {
    if (tuned_assign(c, dtype, d, ncols, out)) return GBKM_OK;
    std::string key;
    {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        key = "assign|" + tune_key(c, dtype, d, ncols);
    }
    const bool tc = tc_assign_supported(dtype, d, ncols) && (dtype != GBKM_BF16 || d % 8 == 0);
    if (!tc && dtype != GBKM_F32) return set_error(c, GBKM_EUNSUPPORTED, "autotune: no engine takes this shape");
    const int64_t n = 32768, kp = ceil_div(ncols, 16) * 16;
    float *X = nullptr, *C = nullptr, *xn = nullptr;
    void *Xop = nullptr;
    int32_t *lab = nullptr;
    cudaError_t e = cudaMalloc(&X, sizeof(float) * n * d);
    if (e == cudaSuccess) e = cudaMalloc(&C, sizeof(float) * ncols * d);
    if (e == cudaSuccess) e = cudaMalloc(&xn, sizeof(float) * n);
    if (e == cudaSuccess) e = cudaMalloc(&Xop, (size_t)n * d * 2);
    if (e == cudaSuccess) e = cudaMalloc(&lab, sizeof(int32_t) * n);
    int rc = GBKM_OK;
    TuneChoice best{tc ? (int)GBKM_ENGINE_TCGEN05 : (int)GBKM_ENGINE_SIMT, 256, 0};
    float best_ms = 1e30f;
    if (e == cudaSuccess) {
        k_fill_synth<<<(unsigned)ceil_div(n * d, 256), 256, 0, c->stream>>>(X, n * d, 0x4321u);
        k_fill_synth<<<(unsigned)ceil_div(ncols * d, 256), 256, 0, c->stream>>>(C, ncols * d, 0x6789u);
        c->launches += 2;
        rc = launch_row_norms(c, X, n, d, xn);
        if (rc == GBKM_OK && dtype == GBKM_BF16) rc = launch_quantize(c, X, n, d, GBKM_BF16, Xop, nullptr);
        cudaEvent_t a, b;
        cudaEventCreate(&a);
        cudaEventCreate(&b);
        const int saved_bn = c->bn_cap, saved_st = c->stage_cap;
        std::vector<TuneChoice> cand;
        if (tc)
            for (int cap : {64, 128, 256}) {
                if (cap > 64 && ceil_div(kp, cap) == ceil_div(kp, cap / 2)) continue;  // same chunking
                for (int st : {2, 3, 0}) cand.push_back({(int)GBKM_ENGINE_TCGEN05, cap, st});
            }
        if (dtype == GBKM_F32) cand.push_back({(int)GBKM_ENGINE_SIMT, 0, 0});
        for (const TuneChoice &t : cand) {
            if (rc != GBKM_OK) break;
            c->bn_cap = t.bn;
            c->stage_cap = t.stages;
            gbkm_assign_opts o = {dtype, t.engine, 0, 0};
            float tbest = 1e30f;
            for (int rep = 0; rep < 4 && rc == GBKM_OK; ++rep) {
                cudaEventRecord(a, c->stream);
                rc = kmeans_assign(c, dtype == GBKM_BF16 ? Xop : X, nullptr, X, xn, n, d, C, ncols, &o, lab, nullptr,
                                   nullptr);
                cudaEventRecord(b, c->stream);
                cudaEventSynchronize(b);
                float ms = 0.f;
                cudaEventElapsedTime(&ms, a, b);
                if (rep > 0) tbest = std::min(tbest, ms);
            }
            if (rc == GBKM_OK && tbest < best_ms) {
                best_ms = tbest;
                best = t;
            }
        }
        c->bn_cap = saved_bn;
        c->stage_cap = saved_st;
        cudaEventDestroy(a);
        cudaEventDestroy(b);
    } else {
        cudaGetLastError();
        rc = set_error(c, GBKM_ENOMEM, "autotune: synthetic problem allocation failed");
    }
    cudaStreamSynchronize(c->stream);
    cudaFree(X);
    cudaFree(C);
    cudaFree(xn);
    cudaFree(Xop);
    cudaFree(lab);
    if (rc != GBKM_OK) return rc;
    {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        g_tune_assign[key] = best;
        const char *path = getenv("GBKM_TUNE_CACHE");
        if (path) {
            if (FILE *f = fopen(path, "a")) {
                fprintf(f, "%s %d:%d:%d\n", key.c_str(), best.engine, best.bn, best.stages);
                fclose(f);
            }
        }
    }
    *out = best;
    return GBKM_OK;
}

}  // namespace gbkm
