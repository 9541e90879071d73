// Temporally blocked kernels with BF16 or FP16 (row-tile scaled) history, FP32 state and
// accumulation: forward only, blocks of 4, 8 and 16 steps.
#include "fd_kernels.h"

namespace fdk {
const void *kernel_tb_lowp(int tb, int hist)
{
    if (hist == 2) {
        switch (tb) {
        case 4: return (const void *)engine_tb_kernel<4, false, __nv_bfloat16>;
        case 8: return (const void *)engine_tb_kernel<8, false, __nv_bfloat16>;
        case 16: return (const void *)engine_tb_kernel<16, false, __nv_bfloat16>;
        default: return nullptr;
        }
    }
    if (hist == 3) {
        switch (tb) {
        case 4: return (const void *)engine_tb_kernel<4, false, __half>;
        case 8: return (const void *)engine_tb_kernel<8, false, __half>;
        case 16: return (const void *)engine_tb_kernel<16, false, __half>;
        default: return nullptr;
        }
    }
    return nullptr;
}
}  // namespace fdk
