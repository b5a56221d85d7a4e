#include "fmm.cuh"

namespace bgl {

struct FmmPlan {
    int dummy;
};

FmmPlan *fmm_create(bgl_graph *, const bgl_params *, int64_t) {
    fail(BGL_EINVAL, "fmm: not available in this build");
}
void fmm_destroy(FmmPlan *pl) { delete pl; }
void fmm_repulsion(FmmPlan *, const float2 *, int64_t, float2 *, int64_t) {}

}  // namespace bgl
