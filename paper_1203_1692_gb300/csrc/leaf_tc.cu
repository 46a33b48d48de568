// Stage 4 on the tcgen05 tensor cores (placeholder until the kernel lands).
#include "spamm_internal.cuh"

namespace spamm {

cudaError_t launch_leaf_tc(spamm_ctx*, const spamm_tree*, const spamm_tree*, float, float,
                           float*, int64_t) {
    return cudaErrorNotSupported;
}

}  // namespace spamm
