// k_lut_inst.cu -- the interpolation kernels of one LUT method.  The build
// compiles this file once per method, naming it with
// -DMACT_LUT_METHOD_ID=<0 trilinear | 1 prism | 2 pyramid | 3 tetrahedral>.
#include "k_lut_interp.cuh"

#if !defined(MACT_LUT_METHOD_ID)
#error "k_lut_inst.cu is compiled once per method with -DMACT_LUT_METHOD_ID"
#endif

namespace mact {
MACT_LUT_METHOD(MACT_LUT_METHOD_ID)
}  // namespace mact
