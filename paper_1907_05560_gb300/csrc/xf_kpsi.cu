// xf_kpsi.cu -- the integrator kernel in the wavefunction form (one psi per
// initial flavor), FP64 and FP32 bins, plain arithmetic, two moments.
#include "xf_kernels.h"

namespace xf {

template <typename Real>
static RunKernel pick_psi(int nfm, int stepper)
{
    constexpr int P = VAR_PLAIN;
    if (stepper == STEP_RK4) {
        if (nfm == 2) return {(const void *)xf_run_kernel<2, STEP_RK4, Real, 256, P, 2, FORM_PSI>, 256};
        if (nfm == 3) return {(const void *)xf_run_kernel<3, STEP_RK4, Real, 128, P, 2, FORM_PSI>, 128};
        if (nfm == 0) return {(const void *)xf_run_kernel<0, STEP_RK4, Real, 128, P, 2, FORM_PSI>, 128};
    } else if (stepper == STEP_EXPH) {
        if (nfm == 2) return {(const void *)xf_run_kernel<2, STEP_EXPH, Real, 256, P, 2, FORM_PSI>, 256};
        if (nfm == 3) return {(const void *)xf_run_kernel<3, STEP_EXPH, Real, 128, P, 2, FORM_PSI>, 128};
        if (nfm == 0) return {(const void *)xf_run_kernel<0, STEP_EXPH, Real, 128, P, 2, FORM_PSI>, 128};
    }
    return {nullptr, 0};
}

RunKernel run_kernel_psi(int nfm, int stepper, bool fp64)
{
    return fp64 ? pick_psi<double>(nfm, stepper) : pick_psi<float>(nfm, stepper);
}

} // namespace xf
