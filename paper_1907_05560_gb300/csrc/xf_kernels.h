// xf_kernels.h -- host-visible handles of the persistent integrator kernels
// (instantiated in xf_k64.cu and xf_k32.cu, compiled in parallel).
#pragma once

#include "xf_run.cuh"

namespace xf {

struct RunKernel {
    const void *fn; // __global__ void (RunArgs)
    int nt;         // threads per CTA it was compiled for
};

// nf in {2, 3}, stepper STEP_RK4 / STEP_EXPH; fn == nullptr if not built.
RunKernel run_kernel_fp64(int nf, int stepper);
RunKernel run_kernel_fp32(int nf, int stepper);

} // namespace xf
