// xf_k32.cu -- FP32 instantiations (per-bin arithmetic and storage in FP32; moments above
// the warp, radius, path length and phases in FP64).
#include "xf_kernels.h"

namespace xf {

RunKernel run_kernel_fp32(int nfm, int stepper)
{
    if (stepper == STEP_RK4) {
        if (nfm == 2) return {(const void *)xf_run_kernel<2, STEP_RK4, float, 256>, 256};
        if (nfm == 3) return {(const void *)xf_run_kernel<3, STEP_RK4, float, 128>, 128};
        if (nfm == 0) return {(const void *)xf_run_kernel<0, STEP_RK4, float, 128>, 128};
    } else if (stepper == STEP_EXPH) {
        if (nfm == 2) return {(const void *)xf_run_kernel<2, STEP_EXPH, float, 256>, 256};
        if (nfm == 3) return {(const void *)xf_run_kernel<3, STEP_EXPH, float, 128>, 128};
        if (nfm == 0) return {(const void *)xf_run_kernel<0, STEP_EXPH, float, 128>, 128};
    }
    return {nullptr, 0};
}

} // namespace xf
