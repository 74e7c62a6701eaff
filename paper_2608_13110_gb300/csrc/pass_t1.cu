// Pass kernels of shape P_REV for window sizes 5..10 (see pass_kernel.cuh).
#include "pass_kernel.cuh"

namespace tb {
TB_DEFINE_LAUNCH_PASS(P_REV, launch_pass_t1)
}  // namespace tb
