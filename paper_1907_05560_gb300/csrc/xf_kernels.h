// xf_kernels.h -- host-visible handles of the persistent integrator kernels
// (instantiated in xf_k64.cu, xf_kff.cu, xf_k32*.cu, xf_ka.cu, xf_kaz.cu, xf_kpsi.cu and
// xf_kcyl.cu, compiled in parallel).
#pragma once

#include "xf_run.cuh"

namespace xf {

struct RunKernel {
    const void *fn; // __global__ void (RunArgs)
    int nt;         // threads per CTA it was compiled for
};

// nfm: 2 or 3 (all instances of the pack have that many flavors) or 0
// (mixed pack); stepper STEP_RK4 / STEP_EXPH; var VAR_PLAIN / VAR_COMP /
// VAR_RENORM (FP32 only; mixed packs plain only).  fn == nullptr if not built.
RunKernel run_kernel_fp64(int nfm, int stepper);
RunKernel run_kernel_fp32(int nfm, int stepper, int var);
// XF_FP32X2: FP64 storage and sums, float-float propagator (predictor-corrector only)
RunKernel run_kernel_ff(int nfm, int stepper);
// the error-controlled step (xf_adapt_kernel), FP64 or FP32 bins
RunKernel run_kernel_adapt(int nfm, bool fp64);
// the extended bulb model (four moments), plain arithmetic, FP64 or FP32 bins
RunKernel run_kernel_azimuth(int nfm, int stepper, bool fp64);
// the wavefunction form, plain arithmetic, FP64 or FP32 bins
RunKernel run_kernel_psi(int nfm, int stepper, bool fp64);
// the cylinder/line model (one problem per launch), FP64 or FP32 bins
RunKernel run_kernel_cyl(int nf, int stepper, bool fp64);

} // namespace xf
