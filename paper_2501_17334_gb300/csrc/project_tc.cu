// tcgen05 BF16x3 projector contraction (placeholder until the tensor-core kernel lands).
#include "qst_internal.cuh"

namespace qst {

struct TcPlan {
    int dummy;
};

int tc_column_tile(int KD) { (void)KD; return 0; }
int tc_ngroups(const ProblemView &p, int64_t rows) { (void)p; (void)rows; return 1; }
cudaError_t tc_plan_create(const ProblemView &, const __nv_bfloat16 *, int64_t, TcPlan **plan) {
    *plan = nullptr;
    return cudaErrorNotSupported;
}
void tc_plan_destroy(TcPlan *plan) { delete plan; }
cudaError_t launch_project_tc(const TcPlan *, const ProblemView &, int64_t, double *, float *, uint32_t *,
                              cudaStream_t) {
    return cudaErrorNotSupported;
}

}  // namespace qst
