// Tensor-core X-engine (placeholder until the tcgen05 kernel lands).
#include "xengine_tc.h"

namespace gbcorr {

struct TcPlan {
    int dummy;
};

int tc_plan_create(TcPlan** out, int, int, int, std::string& err) {
    *out = nullptr;
    err = "the tensor-core X-engine is not built yet; use CORR_FP32_SIMT";
    return CORR_EUNSUPPORTED;
}
int tc_plan_update(TcPlan*, void*, int64_t, int, int, int, std::string&) { return CORR_EUNSUPPORTED; }
int tc_run(TcPlan*, int64_t, float2*, const float*, int*, cudaStream_t, std::string&) {
    return CORR_EUNSUPPORTED;
}
int tc_num_partials(const TcPlan*, int64_t) { return 0; }
void tc_plan_destroy(TcPlan* p) { delete p; }

}  // namespace gbcorr
