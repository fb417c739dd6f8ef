// k_batch_exact.cu -- the batched conversion kernels for the exact form
// (cbrtf, atanf, atan2f and acosf).  One translation unit per cube-root form,
// so the forms compile in parallel.
#include "k_batch.cuh"

namespace mact {
MACT_BATCH_FORM(true, 4)
}  // namespace mact
