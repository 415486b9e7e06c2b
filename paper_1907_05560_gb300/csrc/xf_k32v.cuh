// xf_k32v.cuh -- FP32 instantiations of one arithmetic variant (VAR_COMP in
// xf_k32c.cu, VAR_RENORM in xf_k32r.cu; separate units so they compile in
// parallel).
#pragma once

#include "xf_kernels.h"

namespace xf {

template <int VAR>
RunKernel run_kernel_fp32_var(int nfm, int stepper)
{
    if (stepper == STEP_RK4) {
        if (nfm == 2) return {(const void *)xf_run_kernel<2, STEP_RK4, float, 256, VAR>, 256};
        if (nfm == 3) return {(const void *)xf_run_kernel<3, STEP_RK4, float, 128, VAR>, 128};
        if (nfm == 0) return {(const void *)xf_run_kernel<0, STEP_RK4, float, 128, VAR>, 128};
    } else if (stepper == STEP_EXPH) {
        if (nfm == 2) return {(const void *)xf_run_kernel<2, STEP_EXPH, float, 256, VAR>, 256};
        if (nfm == 3) return {(const void *)xf_run_kernel<3, STEP_EXPH, float, 128, VAR>, 128};
        if (nfm == 0) return {(const void *)xf_run_kernel<0, STEP_EXPH, float, 128, VAR>, 128};
    }
    return {nullptr, 0};
}

} // namespace xf
