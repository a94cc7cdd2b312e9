// gf_train.cu -- reverse-KL training step (in progress).
#include "gf_flow.cuh"

extern "C" {
size_t gf_train_workspace_bytes(const gf_flow*, int64_t) { return 0; }
gf_status gf_flow_train_step(gf_flow*, const gf_phi4*, int64_t, uint64_t, uint64_t, const float*,
                             double*, float*, float, float, float, float, float*, float*, int64_t,
                             void*, size_t, cudaStream_t) {
    return GF_EUNSUPPORTED;
}
}
