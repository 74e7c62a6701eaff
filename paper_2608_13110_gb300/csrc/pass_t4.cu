// Pass kernels of shape P_BOT_START for window sizes 5..10 (see pass_kernel.cuh).
#include "pass_kernel.cuh"

namespace tb {
TB_DEFINE_LAUNCH_PASS(P_BOT_START, launch_pass_t4)
}  // namespace tb
