// xf_k64.cu -- FP64 instantiations of the persistent integrator kernel.
#include "xf_kernels.h"

namespace xf {

RunKernel run_kernel_fp64(int nf, int stepper)
{
    if (nf == 2 && stepper == STEP_RK4) return {(const void *)xf_run_kernel<2, STEP_RK4, double, 256>, 256};
    if (nf == 2 && stepper == STEP_EXPH) return {(const void *)xf_run_kernel<2, STEP_EXPH, double, 256>, 256};
    if (nf == 3 && stepper == STEP_RK4) return {(const void *)xf_run_kernel<3, STEP_RK4, double, 128>, 128};
    if (nf == 3 && stepper == STEP_EXPH) return {(const void *)xf_run_kernel<3, STEP_EXPH, double, 128>, 128};
    return {nullptr, 0};
}

} // namespace xf
