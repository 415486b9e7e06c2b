// xf_kcyl.cu -- the cylinder/line model's integrator kernel (Eq. 3.20),
// FP64 and FP32 bins, two and three flavors.
#include "xf_cyl.cuh"
#include "xf_kernels.h"

namespace xf {

template <typename Real>
static RunKernel pick_cyl(int nf, int stepper)
{
    if (stepper == STEP_RK4) {
        if (nf == 2) return {(const void *)xf_cyl_kernel<2, STEP_RK4, Real>, CYL_NT};
        if (nf == 3) return {(const void *)xf_cyl_kernel<3, STEP_RK4, Real>, CYL_NT};
    } else if (stepper == STEP_EXPH) {
        if (nf == 2) return {(const void *)xf_cyl_kernel<2, STEP_EXPH, Real>, CYL_NT};
        if (nf == 3) return {(const void *)xf_cyl_kernel<3, STEP_EXPH, Real>, CYL_NT};
    }
    return {nullptr, 0};
}

RunKernel run_kernel_cyl(int nf, int stepper, bool fp64)
{
    return fp64 ? pick_cyl<double>(nf, stepper) : pick_cyl<float>(nf, stepper);
}

} // namespace xf
