// xf_k32c.cu -- FP32 bins with compensated (TwoSum) moment sums.
#include "xf_k32v.cuh"

namespace xf {

RunKernel run_kernel_fp32_comp(int nfm, int stepper) { return run_kernel_fp32_var<VAR_COMP>(nfm, stepper); }

} // namespace xf
