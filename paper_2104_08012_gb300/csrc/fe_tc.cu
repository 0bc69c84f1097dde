// bf16 tensor-core operator apply (placeholder until the tcgen05 kernel lands).
#include "fe_internal.cuh"

bool bf16_supported() { return false; }

void apply_bf16_enqueue(const Level&, const float*, float*, cudaStream_t) {
  FE_FAIL(FE_ERR_UNSUPPORTED, "bf16 tensor-core apply not available");
}
