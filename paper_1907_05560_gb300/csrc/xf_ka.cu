// xf_ka.cu -- instantiations of the error-controlled step kernel (xf_adapt.cuh).
#include "xf_adapt.cuh"
#include "xf_kernels.h"

namespace xf {

RunKernel run_kernel_adapt(int nfm, bool fp64)
{
    if (fp64) {
        if (nfm == 2) return {(const void *)xf_adapt_kernel<2, double, 256>, 256};
        if (nfm == 3) return {(const void *)xf_adapt_kernel<3, double, 128>, 128};
        if (nfm == 0) return {(const void *)xf_adapt_kernel<0, double, 128>, 128};
    } else {
        if (nfm == 2) return {(const void *)xf_adapt_kernel<2, float, 256>, 256};
        if (nfm == 3) return {(const void *)xf_adapt_kernel<3, float, 128>, 128};
        if (nfm == 0) return {(const void *)xf_adapt_kernel<0, float, 128>, 128};
    }
    return {nullptr, 0};
}

} // namespace xf
