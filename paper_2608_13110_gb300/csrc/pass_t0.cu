// Pass kernels of shape P_FWD for window sizes 5..10 (see pass_kernel.cuh).
#include "pass_kernel.cuh"

namespace tb {
TB_DEFINE_LAUNCH_PASS(P_FWD, launch_pass_t0)
}  // namespace tb
