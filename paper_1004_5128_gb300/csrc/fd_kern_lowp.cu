// FP32 state with BF16 or FP16 (per row-tile scaled) history, FP32 (Kahan) accumulation.
#include "fd_kernels.h"

namespace fdk {
const void *kernel_lowp(int hist, bool kahan, bool adj)
{
    if (adj) return nullptr;
    if (hist == 2)
        return kahan ? (const void *)engine_kernel<float, __nv_bfloat16, float, true, false>
                     : (const void *)engine_kernel<float, __nv_bfloat16, float, false, false>;
    if (hist == 3)
        return kahan ? (const void *)engine_kernel<float, __half, float, true, false>
                     : (const void *)engine_kernel<float, __half, float, false, false>;
    return nullptr;
}

const void *kernel_for(int state, int hist, int acc, bool kahan, bool adj)
{
    if (state == 0 && hist == 0 && acc == 0) return kernel_f64(kahan, adj);
    if (state == 1 && hist == 1 && acc == 1) return kernel_f32(kahan, adj);
    if (state == 1 && acc == 1 && (hist == 2 || hist == 3)) return kernel_lowp(hist, kahan, adj);
    return nullptr;
}
}  // namespace fdk
