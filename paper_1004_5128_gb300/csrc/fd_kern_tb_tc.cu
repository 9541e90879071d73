// Temporally blocked kernels whose far units run on the tensor cores (tcgen05): BF16 or FP16
// (row-tile scaled) history at blocks of 16, 32 and 64 steps, and FP32 history (split into FP16
// hi and lo parts in shared memory) at blocks of 32 and 64; FP32 state and accumulation, forward.
#include "fd_kernels.h"

namespace fdk {
const void *kernel_tb_tc(int tb, int hist)
{
    if (hist == 2) {
        switch (tb) {
        case 16: return (const void *)engine_tb_kernel<16, false, __nv_bfloat16, true>;
        case 32: return (const void *)engine_tb_kernel<32, false, __nv_bfloat16, true>;
        case 64: return (const void *)engine_tb_kernel<64, false, __nv_bfloat16, true>;
        default: return nullptr;
        }
    }
    if (hist == 3) {
        switch (tb) {
        case 16: return (const void *)engine_tb_kernel<16, false, __half, true>;
        case 32: return (const void *)engine_tb_kernel<32, false, __half, true>;
        case 64: return (const void *)engine_tb_kernel<64, false, __half, true>;
        default: return nullptr;
        }
    }
    if (hist == 1) {
        switch (tb) {
        case 32: return (const void *)engine_tb_kernel<32, false, float, true>;
        case 64: return (const void *)engine_tb_kernel<64, false, float, true>;
        default: return nullptr;
        }
    }
    return nullptr;
}
}  // namespace fdk
