// xf_k32r.cu -- FP32 bins with the per-step restoration of tr(T^2).
#include "xf_k32v.cuh"

namespace xf {

RunKernel run_kernel_fp32_renorm(int nfm, int stepper) { return run_kernel_fp32_var<VAR_RENORM>(nfm, stepper); }

} // namespace xf
