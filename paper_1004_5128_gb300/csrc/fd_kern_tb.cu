// FP32 temporally blocked kernels: forward (blocks of 4, 8, 16 steps) and adjoint (4, 8).
#include "fd_kernels.h"

namespace fdk {
const void *kernel_tb(int tb, bool adj, int hist, bool tc)
{
    if (tc) return adj ? nullptr : kernel_tb_tc(tb, hist);
    if (hist != 1) return adj ? nullptr : kernel_tb_lowp(tb, hist);
    if (adj) {  // two accumulator sets: blocks of at most 8 steps fit the register budget
        switch (tb) {
        case 4: return (const void *)engine_tb_kernel<4, true>;
        case 8: return (const void *)engine_tb_kernel<8, true>;
        default: return nullptr;
        }
    }
    switch (tb) {
    case 4: return (const void *)engine_tb_kernel<4, false>;
    case 8: return (const void *)engine_tb_kernel<8, false>;
    case 16: return (const void *)engine_tb_kernel<16, false>;
    default: return nullptr;
    }
}
}  // namespace fdk
