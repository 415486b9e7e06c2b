// xf_k32.cu -- FP32 instantiations (per-bin arithmetic and storage in FP32; moments above
// the warp, radius, path length and phases in FP64), plain variant; the compensated and
// renormalising variants are instantiated in xf_k32c.cu and xf_k32r.cu.
#include "xf_kernels.h"

namespace xf {

RunKernel run_kernel_fp32_comp(int nfm, int stepper);
RunKernel run_kernel_fp32_renorm(int nfm, int stepper);

RunKernel run_kernel_fp32(int nfm, int stepper, int var)
{
    if (var == VAR_COMP) return run_kernel_fp32_comp(nfm, stepper);
    if (var == VAR_RENORM) return run_kernel_fp32_renorm(nfm, stepper);
    if (var != VAR_PLAIN) return {nullptr, 0};
    if (stepper == STEP_RK4) {
        if (nfm == 2) return {(const void *)xf_run_kernel<2, STEP_RK4, float, 256, VAR_PLAIN>, 256};
        if (nfm == 3) return {(const void *)xf_run_kernel<3, STEP_RK4, float, 128, VAR_PLAIN>, 128};
        if (nfm == 0) return {(const void *)xf_run_kernel<0, STEP_RK4, float, 128, VAR_PLAIN>, 128};
    } else if (stepper == STEP_EXPH) {
        if (nfm == 2) return {(const void *)xf_run_kernel<2, STEP_EXPH, float, 256, VAR_PLAIN>, 256};
        if (nfm == 3) return {(const void *)xf_run_kernel<3, STEP_EXPH, float, 128, VAR_PLAIN>, 128};
        if (nfm == 0) return {(const void *)xf_run_kernel<0, STEP_EXPH, float, 128, VAR_PLAIN>, 128};
    }
    return {nullptr, 0};
}

} // namespace xf
