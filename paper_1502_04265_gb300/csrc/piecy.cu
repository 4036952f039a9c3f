// piecy.cu -- per-piece bases with the d-dimensional lift (Section 2.2, piecy): the input is cut into
// pieces of consecutive rows; each piece gets its own best-fit basis from the randomised SVD and is
// replaced by its projection onto that basis, A_l = A V V^T, which keeps the d coordinates (so the
// pieces can be clustered together) but has intrinsic dimension l.  Host orchestration only: the
// work runs in the SVD kernels and the tensor-core projection and lift.
#include <algorithm>

#include "internal.cuh"

extern "C" int kmeans_piecy_lift(gbkm_ctx *c, const float *X, int64_t n, int64_t d, const float *w,
                                 int64_t piece_rows, const float *Omegas, int64_t s, int64_t ell, float *X_lift,
                                 float *V_out, float *sigma_out, int32_t *info_out) {
    if (!c) return GBKM_EINVAL;
    if (!X || !Omegas || !X_lift || !V_out || n < 1 || d < 1 || piece_rows < 1)
        return set_error(c, GBKM_EINVAL, "piecy_lift: bad arguments");
    if (s < 16 || s > 128 || s % 16 != 0 || ell < 1 || ell > s || s > d)
        return set_error(c, GBKM_EINVAL, "piecy_lift: need 16 <= s <= 128, s %% 16 == 0, 1 <= ell <= s <= d");
    const int64_t pieces = ceil_div(n, piece_rows);
    const int64_t last = n - (pieces - 1) * piece_rows;
    if (piece_rows < s || last < s)
        return set_error(c, GBKM_EINVAL, "piecy_lift: every piece (the last has %lld rows) needs at least s = %lld rows",
                         (long long)last, (long long)s);
    if (X_lift == X) return set_error(c, GBKM_EINVAL, "piecy_lift: X_lift may not alias X");
    int prev = -1;
    cudaGetDevice(&prev);
    if (prev != c->device) cudaSetDevice(c->device);
    // the r-dimensional coordinates of one piece between its projection and its lift
    float *Y = nullptr;
    int rc = GBKM_OK;
    cudaError_t e = cudaMallocAsync(&Y, sizeof(float) * (size_t)std::min(piece_rows, n) * (size_t)ell, c->stream);
    if (e != cudaSuccess) {
        cudaGetLastError();
        rc = set_error(c, GBKM_ENOMEM, "piecy_lift: coordinates buffer");
    }
    prof_begin(c, "piecy_lift");
    for (int64_t q = 0; q < pieces && rc == GBKM_OK; ++q) {
        const int64_t r0 = q * piece_rows, rows = std::min(piece_rows, n - r0);
        float *Vq = V_out + q * d * ell;
        rc = kmeans_rsvd(c, X + r0 * d, rows, d, w ? w + r0 : nullptr, Omegas + q * d * s, s, ell, Vq,
                         sigma_out ? sigma_out + q * ell : nullptr, info_out ? info_out + q : nullptr);
        if (rc == GBKM_OK) rc = kmeans_project_block(c, X + r0 * d, GBKM_F32, rows, d, Vq, ell, Y, X_lift + r0 * d);
    }
    prof_end(c);
    if (Y) cudaFreeAsync(Y, c->stream);
    if (prev >= 0 && prev != c->device) cudaSetDevice(prev);
    return rc;
}
