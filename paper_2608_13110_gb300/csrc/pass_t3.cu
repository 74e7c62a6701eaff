// Pass kernels of shape P_BOT for window sizes 5..10 (see pass_kernel.cuh).
#include "pass_kernel.cuh"

namespace tb {
TB_DEFINE_LAUNCH_PASS(P_BOT, launch_pass_t3)
}  // namespace tb
