// FP32 state, history and accumulation (plain or Kahan; forward and adjoint).
#include "fd_kernels.h"

namespace fdk {
const void *kernel_f32(bool kahan, bool adj)
{
    if (adj) return kahan ? nullptr : (const void *)engine_kernel<float, float, float, false, true>;
    return kahan ? (const void *)engine_kernel<float, float, float, true, false>
                 : (const void *)engine_kernel<float, float, float, false, false>;
}
}  // namespace fdk
