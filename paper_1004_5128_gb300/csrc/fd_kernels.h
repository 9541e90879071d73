// fd_kernels.h -- registry of the engine's template instantiations (internal).
#pragma once
#include "fd_engine.cuh"
#include "fd_engine_tb.cuh"

namespace fdk {
// Kernel for (state, history, accumulator) dtypes (FD_F64/FD_F32/FD_BF16/FD_F16 codes),
// Kahan accumulation and adjoint mode; nullptr when the combination is not built.
const void *kernel_for(int state, int hist, int acc, bool kahan, bool adj);
const void *kernel_f64(bool kahan, bool adj);
const void *kernel_f32(bool kahan, bool adj);
const void *kernel_lowp(int hist, bool kahan, bool adj);
// Temporally blocked kernel (FP32 state and accumulation) for a block of tb steps and a history
// dtype (FD_F32: forward 4/8/16, adjoint 4/8; FD_BF16 / FD_F16: forward 4/8/16), else nullptr.
// With tc (forward; BF16 or FP16 history at blocks of 16, 32, 64, FP32 history at 32, 64) the far
// rows run on the tensor cores.
const void *kernel_tb(int tb, bool adj = false, int hist = 1, bool tc = false);
const void *kernel_tb_lowp(int tb, int hist);
const void *kernel_tb_tc(int tb, int hist);
}  // namespace fdk
