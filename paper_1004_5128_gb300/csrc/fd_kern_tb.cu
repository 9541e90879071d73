// FP32 temporally blocked kernels (blocks of 4, 8 and 16 steps).
#include "fd_kernels.h"

namespace fdk {
const void *kernel_tb(int tb)
{
    switch (tb) {
    case 4: return (const void *)engine_tb_kernel<4>;
    case 8: return (const void *)engine_tb_kernel<8>;
    case 16: return (const void *)engine_tb_kernel<16>;
    default: return nullptr;
    }
}
}  // namespace fdk
