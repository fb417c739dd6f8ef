// k_batch_inst.cu -- one (cube-root form, launch shape) pair of the batched
// conversion kernels.  The build compiles this file once per pair, naming it
// with -DMACT_FORM_EXACT=<0|1> -DMACT_FORM_RDEG=<0|4|6> -DMACT_SHAPE_T=<threads>
// -DMACT_SHAPE_S=<sub-blocks>; the forms are the exact one (libm), the
// rationals with Horner degree 4 (printed table, low fitted degrees) and 6
// (fitted up to (6, 6)), and the FP64 cube-root polynomials; the shapes are
// those of MACT_BATCH_SHAPES (convert_common.cuh).
#include "k_batch.cuh"

#if !defined(MACT_FORM_EXACT) || !defined(MACT_FORM_RDEG) || !defined(MACT_SHAPE_T) || !defined(MACT_SHAPE_S)
#error "k_batch_inst.cu is compiled once per form and shape with -DMACT_FORM_* -DMACT_SHAPE_*"
#endif

namespace mact {
MACT_BATCH_SHAPE(MACT_FORM_EXACT != 0, MACT_FORM_RDEG, MACT_SHAPE_T, MACT_SHAPE_S)
}  // namespace mact
