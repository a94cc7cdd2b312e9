// gf_flow_bf16.cu -- BF16 tensor-core variant of the fused coupling stack.
// Not built yet: flows requested with GF_PREC_BF16CONV_FP64RED are refused
// with GF_EUNSUPPORTED at creation.
#include "gf_flow.cuh"

namespace gf {

bool bf16_supported(const gf_flow_shape*) { return false; }
gf_status bf16_configure(gf_flow*) { return GF_EUNSUPPORTED; }
gf_status repack_bf16(gf_flow*, cudaStream_t) { return GF_EUNSUPPORTED; }
gf_status launch_flow_bf16(const gf_flow*, bool, const gf_phi4*, int64_t, uint64_t, uint64_t,
                           const float*, float*, const float*, float*, double*, double*, double*,
                           cudaStream_t) {
    return GF_EUNSUPPORTED;
}

}  // namespace gf
