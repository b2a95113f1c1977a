// Split-precision near-field contraction (placeholder until the sliced path lands).
#include <cuda_runtime.h>

#include <vector>

#include "plan.h"
#include "vp_internal.h"

namespace vp {

int build_split(vp_tables_s*, cudaStream_t) { return VP_ERR_ARG; }

int split_plan_build(vp_tree_s*, const TreePlan&, const std::vector<long long>&, cudaStream_t) { return VP_ERR_ARG; }
int split_near_run(vp_tree_s*, const double*, cudaStream_t) { return VP_ERR_ARG; }
void split_plan_free(vp_tree_s*) {}
int split_launches(const vp_tree_s*) { return 0; }

}  // namespace vp
