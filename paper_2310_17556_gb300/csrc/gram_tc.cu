// Placeholder: tensor-core Gram not built yet.
#include "kernels.cuh"

namespace dfs {
int gram_tc_supported(int, int) { return 0; }
GramTcPlan gram_tc_plan(int, int kind, int64_t, int64_t, int) {
    GramTcPlan p{};
    p.kind = kind;
    return p;
}
cudaError_t launch_gram_tc(const GramTcPlan&, int, const void*, int64_t, int64_t, int64_t, void*, DevStatus*,
                           cudaStream_t) {
    return cudaErrorNotSupported;
}
cudaError_t launch_gram_tc_finalize(const GramTcPlan&, const void*, int64_t, int64_t, double, void*, int64_t,
                                    cudaStream_t) {
    return cudaErrorNotSupported;
}
}  // namespace dfs
