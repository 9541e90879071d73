// fd_tc.cuh -- fifth-generation tensor core (tcgen05) and tensor-map bulk copy primitives,
// written as inline PTX for sm_103a.
//
// The temporally blocked far product is a contraction: T steps x P points x R rows per unit
// (the Toeplitz form of the memory sum, eq. frac_norxn).  With 16-bit history it runs as
//     D[p][t] += sum_r H[r][p] * C[r][t]        (M = 128 points, N = T steps, K = 16 rows)
// with the history tile H^T as the MN-major A operand, loaded by the tensor-map unit with a
// 128-byte swizzle, the coefficient block C as the K-major B operand written by the CTA with the
// same swizzle, and D accumulated in FP32 in tensor memory.
//
// Layouts (16-bit elements, 128-byte swizzle: the 16-byte chunk c of a 128-byte row at byte
// offset o is stored at chunk c ^ ((o >> 7) & 7), so an atom is 8 rows x 128 bytes = 1 KB and
// every atom starts 1 KB-aligned):
//  * A, MN-major: an atom holds 64 consecutive points (one 128-byte row) for 8 consecutive
//    history rows.  Atoms adjacent in the point direction are LBO bytes apart, atoms adjacent
//    in the row (K) direction SBO bytes apart.
//  * B, K-major: an atom holds 8 steps (N) x 64 rows (K, one 128-byte row per step).  Atoms
//    adjacent in N are SBO bytes apart; a K slice of 16 starts 32 bytes further into the atom.
//
// FP32 history runs as the same FP16 product, three MMAs per K slice (hi.hi + hi.lo + lo.hi): each
// row is stored as two FP16 planes, hi = fp16(delta 2^e) and lo = fp16(delta 2^e - hi), with a
// power-of-two scale 2^-e per (row, tile) that joins the coefficients (about 22 significant bits).
#pragma once

#include <stdint.h>

namespace fdk {
namespace tc {

__device__ __forceinline__ uint32_t saddr(const void *p) { return static_cast<uint32_t>(__cvta_generic_to_shared(p)); }

// Shared-memory matrix descriptor: start address, leading / stride byte offsets (16-byte units),
// descriptor version 1 (bits 46-47), base offset 0 (atoms 1 KB-aligned), 128-byte swizzle (2).
__device__ __forceinline__ uint64_t desc_sw128(uint32_t addr, uint32_t lbo, uint32_t sbo)
{
    return (uint64_t)((addr >> 4) & 0x3FFFu) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) |
           ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | (1ull << 46) | (2ull << 61);
}

// Instruction descriptor of kind::f16 with FP32 accumulation: A and B both BF16 (bf16 = true) or
// both FP16, A MN-major, B K-major, N at bits 17-22 (N / 8), M at bits 24-28 (M / 16).
__host__ __device__ constexpr uint32_t idesc_f16_amn(int M, int N, bool bf16)
{
    return (1u << 4) | ((bf16 ? 1u : 0u) << 7) | ((bf16 ? 1u : 0u) << 10) | (1u << 15) |
           ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

// D (tensor memory) = A B + (acc ? D : 0), issued by one thread.
__device__ __forceinline__ void mma_f16(uint32_t d, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc)
{
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d),
        "l"(a), "l"(b), "r"(idesc), "r"(acc)
        : "memory");
}

// The mbarrier receives one arrival once every tcgen05 operation this thread issued before has
// completed (and their shared-memory operands are no longer read).
__device__ __forceinline__ void commit(uint64_t *bar)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(saddr(bar))
                 : "memory");
}

__device__ __forceinline__ void fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// Warp-wide: allocate ncols (a power of two >= 32) tensor-memory columns; the address is written
// to *dst in shared memory.  The permit is released at once, as this CTA allocates only here.
__device__ __forceinline__ void tmem_alloc(uint32_t *dst, uint32_t ncols)
{
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(saddr(dst)), "r"(ncols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols)
{
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}

// Warp-wide: 32 lanes x 16 consecutive 32-bit columns from taddr (lane in bits 16-31); thread i
// receives lane (taddr's lane + i).  Waits for the load.
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float *v)
{
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, "
        "%14, %15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

// Tensor-map tile copy of a 2-D box at element coordinates (x, y) into shared memory, completing
// on the mbarrier's transaction count.  x times the element size must be a multiple of 16 bytes.
__device__ __forceinline__ void tma_load_2d(void *dst, const void *tmap, int x, int y, uint64_t *bar)
{
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], "
        "[%4];" ::"r"(saddr(dst)),
        "l"(tmap), "r"(x), "r"(y), "r"(saddr(bar))
        : "memory");
}

// The same for a 3-D box at (x, y, z).
__device__ __forceinline__ void tma_load_3d(void *dst, const void *tmap, int x, int y, int z, uint64_t *bar)
{
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, "
        "%4}], [%5];" ::"r"(saddr(dst)),
        "l"(tmap), "r"(x), "r"(y), "r"(z), "r"(saddr(bar))
        : "memory");
}

}  // namespace tc
}  // namespace fdk
