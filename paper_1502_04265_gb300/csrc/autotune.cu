// autotune.cu -- the project's tile autotuner: for one (compute dtype, d, number of centers) shape it
// times the tcgen05 assignment with center-chunk widths of 64, 128 and 256 columns on a synthetic
// problem and keeps the fastest.  Choices are cached per process and optionally in a text file
// (GBKM_TUNE_CACHE), one "gpu|dtype|d|ncols_pow2 bn" line per shape.
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

std::string tune_key(gbkm_ctx *c, int dtype, int64_t d, int64_t ncols) {
    cudaDeviceProp prop;
    cudaGetDeviceProperties(&prop, c->device);
    int64_t p2 = 16;
    while (p2 < ncols) p2 <<= 1;
    return std::string(prop.name) + "|" + std::to_string(dtype) + "|" + std::to_string(d) + "|" + std::to_string(p2);
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
        g_tune[line] = atoi(sp + 1);
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
    const std::string key = tune_key(c, dtype, d, ncols);
    {
        std::lock_guard<std::mutex> lk(g_tune_mu);
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

}  // namespace gbkm
