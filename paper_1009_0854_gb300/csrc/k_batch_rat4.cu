// k_batch_rat4.cu -- the batched conversion kernels for the cube-root
// rationals up to degree (4, 4): the printed table and the fitted low
// degrees.  One translation unit per cube-root form, so the forms compile in
// parallel.
#include "k_batch.cuh"

namespace mact {
MACT_BATCH_FORM(false, 4)
}  // namespace mact
