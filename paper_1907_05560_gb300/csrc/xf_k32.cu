// xf_k32.cu -- FP32 instantiations (per-bin arithmetic and storage in FP32;
// moments, radius, path length and phases in FP64).
#include "xf_kernels.h"

namespace xf {

RunKernel run_kernel_fp32(int nf, int stepper)
{
    if (nf == 2 && stepper == STEP_RK4) return {(const void *)xf_run_kernel<2, STEP_RK4, float, 256>, 256};
    if (nf == 2 && stepper == STEP_EXPH) return {(const void *)xf_run_kernel<2, STEP_EXPH, float, 256>, 256};
    if (nf == 3 && stepper == STEP_RK4) return {(const void *)xf_run_kernel<3, STEP_RK4, float, 128>, 128};
    if (nf == 3 && stepper == STEP_EXPH) return {(const void *)xf_run_kernel<3, STEP_EXPH, float, 128>, 128};
    return {nullptr, 0};
}

} // namespace xf
