// Pass kernels of shape P_TOP for window sizes 5..10 (see pass_kernel.cuh).
#include "pass_kernel.cuh"

namespace tb {
TB_DEFINE_LAUNCH_PASS(P_TOP, launch_pass_t2)
}  // namespace tb
