// Mixed-precision (bf16 / fp16 hi+lo on tcgen05 tensor cores) exchange mode products.
#include "internal.cuh"

namespace cc {

cc_status mixed_workspace_alloc(cc_tables) { return CC_OK; }
void mixed_workspace_free(cc_tables) {}
cc_status exchange_mixed(cc_tables, int, int, float*, double*, cudaStream_t) {
  return CC_ERR_NOTSUPP;
}

}  // namespace cc
