// xf_kaz.cu -- the integrator kernel with the extended bulb model's four
// moments (Eq. 3.18), FP64 and FP32 bins, plain arithmetic.
#include "xf_kernels.h"

namespace xf {

template <typename Real>
static RunKernel pick_azimuth(int nfm, int stepper)
{
    constexpr int P = VAR_PLAIN;
    if (stepper == STEP_RK4) {
        if (nfm == 2) return {(const void *)xf_run_kernel<2, STEP_RK4, Real, 256, P, 4>, 256};
        if (nfm == 3) return {(const void *)xf_run_kernel<3, STEP_RK4, Real, 128, P, 4>, 128};
        if (nfm == 0) return {(const void *)xf_run_kernel<0, STEP_RK4, Real, 128, P, 4>, 128};
    } else if (stepper == STEP_EXPH) {
        if (nfm == 2) return {(const void *)xf_run_kernel<2, STEP_EXPH, Real, 256, P, 4>, 256};
        if (nfm == 3) return {(const void *)xf_run_kernel<3, STEP_EXPH, Real, 128, P, 4>, 128};
        if (nfm == 0) return {(const void *)xf_run_kernel<0, STEP_EXPH, Real, 128, P, 4>, 128};
    }
    return {nullptr, 0};
}

RunKernel run_kernel_azimuth(int nfm, int stepper, bool fp64)
{
    return fp64 ? pick_azimuth<double>(nfm, stepper) : pick_azimuth<float>(nfm, stepper);
}

} // namespace xf
