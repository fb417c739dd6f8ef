// k_batch_poly.cu -- the batched conversion kernels for the cube-root
// polynomials, evaluated in FP64.  One translation unit per cube-root form,
// so the forms compile in parallel.
#include "k_batch.cuh"

namespace mact {
MACT_BATCH_FORM(false, 0)
}  // namespace mact
