// xf_k64.cu -- FP64 instantiations of the persistent integrator kernel.
#include "xf_kernels.h"

namespace xf {

RunKernel run_kernel_fp64(int nfm, int stepper)
{
    if (stepper == STEP_RK4) {
        if (nfm == 2) return {(const void *)xf_run_kernel<2, STEP_RK4, double, 256, VAR_PLAIN>, 256};
        if (nfm == 3) return {(const void *)xf_run_kernel<3, STEP_RK4, double, 128, VAR_PLAIN>, 128};
        if (nfm == 0) return {(const void *)xf_run_kernel<0, STEP_RK4, double, 128, VAR_PLAIN>, 128};
    } else if (stepper == STEP_EXPH) {
        if (nfm == 2) return {(const void *)xf_run_kernel<2, STEP_EXPH, double, 256, VAR_PLAIN>, 256};
        if (nfm == 3) return {(const void *)xf_run_kernel<3, STEP_EXPH, double, 128, VAR_PLAIN>, 128};
        if (nfm == 0) return {(const void *)xf_run_kernel<0, STEP_EXPH, double, 128, VAR_PLAIN>, 128};
    }
    return {nullptr, 0};
}

} // namespace xf
