// k_batch_rat6.cu -- the batched conversion kernels for the fitted cube-root
// rationals of degree up to (6, 6).  One translation unit per cube-root form,
// so the forms compile in parallel.
#include "k_batch.cuh"

namespace mact {
MACT_BATCH_FORM(false, 6)
}  // namespace mact
