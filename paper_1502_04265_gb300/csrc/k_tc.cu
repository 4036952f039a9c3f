// k_tc.cu -- tcgen05 engines (placeholder until the tensor-core kernels land).
#include "internal.cuh"

namespace gbkm {
bool tc_assign_supported(int, int64_t, int64_t) { return false; }
int launch_assign_tc(gbkm_ctx *c, int, const void *, const float *, const float *, const float *, int64_t,
                     int64_t, const CenterPrep &, int64_t, int64_t, float, float, const AssignOut &) {
    return set_error(c, GBKM_EUNSUPPORTED, "tcgen05 assign not built");
}
bool tc_project_supported(int, int64_t, int64_t) { return false; }
int launch_project_tc(gbkm_ctx *c, int, const void *, int64_t, int64_t, const float *, int64_t, float *) {
    return set_error(c, GBKM_EUNSUPPORTED, "tcgen05 projection not built");
}
}  // namespace gbkm
