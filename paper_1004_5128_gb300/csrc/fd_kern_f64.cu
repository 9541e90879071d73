// FP64 state, history and accumulation (tolerance 1e-12 against the FP64 oracle).
#include "fd_kernels.h"

namespace fdk {
const void *kernel_f64(bool kahan, bool adj)
{
    if (kahan) return nullptr;  // FP64 accumulation needs no compensation at these lengths
    return adj ? (const void *)engine_kernel<double, double, double, false, true>
               : (const void *)engine_kernel<double, double, double, false, false>;
}
}  // namespace fdk
