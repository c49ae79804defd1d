// Fused FP32 path (placeholder until the persistent kernel is written).
#include "fused.h"
#include "solver.h"

namespace fewha {

struct FusedPlan {};

FusedPlan* fused_create(const HostSetup&, const DevGeo<float>&, const FusedBuffers&, std::string& err) {
    err = "fused path not available";
    return nullptr;
}
void fused_destroy(FusedPlan* plan) { delete plan; }
int fused_solve(FusedPlan*, const float*, int, int, int, long long, cudaStream_t, std::string& err, long long&) {
    err = "fused path not available";
    return FEWHA_ERR_STATE;
}

}  // namespace fewha
