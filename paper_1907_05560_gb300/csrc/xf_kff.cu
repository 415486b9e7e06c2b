// xf_kff.cu -- XF_FP32X2 instantiations of the persistent integrator kernel:
// FP64 state, tables and sums, the predictor-corrector's propagator in
// float-float (xf_ff.cuh).
#include "xf_kernels.h"

namespace xf {

RunKernel run_kernel_ff(int nfm, int stepper)
{
    if (stepper != STEP_EXPH) return {nullptr, 0};
    if (nfm == 2) return {(const void *)xf_run_kernel<2, STEP_EXPH, double, 256, VAR_FF>, 256};
    if (nfm == 3) return {(const void *)xf_run_kernel<3, STEP_EXPH, double, 128, VAR_FF>, 128};
    if (nfm == 0) return {(const void *)xf_run_kernel<0, STEP_EXPH, double, 128, VAR_FF>, 128};
    return {nullptr, 0};
}

} // namespace xf
