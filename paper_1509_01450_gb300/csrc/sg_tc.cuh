// Fifth-generation tensor-core primitives (tcgen05, sm_100 family) for the
// dense DFT-matrix form of short azimuthal transforms: tensor-memory
// allocation, shared-memory matrix descriptors, the single-CTA TF32 MMA, its
// completion on an mbarrier, and the 32-lane tensor-memory loads.  Every
// instruction is issued as written in the PTX ISA; nothing here is generated.
#pragma once
#include <stdint.h>

// ---- host and device: descriptors -------------------------------------------

// Shared-memory matrix descriptor (64 bits) of an operand stored K-major
// without swizzling.  The operand is a grid of core matrices of 8 rows x 16
// bytes (8 x 4 TF32 values), each 128 contiguous bytes; lbo is the byte
// distance between core matrices adjacent along K, sbo between core matrices
// adjacent along M (or N).  Field layout: start address >> 4 in bits 0-13,
// lbo >> 4 in 16-29, sbo >> 4 in 32-45, the descriptor version 1 in bits
// 46-48, base offset 0, swizzle mode 0 (none) in bits 61-63.
__host__ __device__ inline uint64_t sg_tc_smem_desc(uint32_t smem_addr, uint32_t lbo, uint32_t sbo)
{
    return (uint64_t)((smem_addr & 0x3FFFFu) >> 4) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) |
           ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | (1ull << 46);
}

// Instruction descriptor (32 bits) of kind::tf32 with an FP32 accumulator,
// both operands K-major, no negation or sparsity: D format F32 (1) in bits
// 4-5, A and B format TF32 (2) in bits 7-9 and 10-12, N >> 3 in bits 17-22,
// M >> 4 in bits 24-28.  M = 128 with N a multiple of 16 in [16, 256].
__host__ __device__ inline uint32_t sg_tc_idesc_tf32(int M, int N)
{
    return (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

// Round an FP32 value to the nearest TF32 value (10 stored fraction bits;
// ties away from zero): add half of the 13 dropped bits' weight to the
// magnitude and clear them.  The result has its low 13 bits zero, so the
// tensor core reads it exactly whatever its own conversion does.
__host__ __device__ inline uint32_t sg_tf32_bits(uint32_t u) { return (u + 0x1000u) & 0xFFFFE000u; }

#ifdef __CUDACC__
// ---- device: tensor memory ----------------------------------------------------

// Allocate ncols (a power of two, 32 .. 512) tensor-memory columns of all 128
// lanes for this CTA; one full warp executes it.  The allocated address is
// written to *dst in shared memory.
__device__ __forceinline__ void sg_tc_alloc(uint32_t* dst, uint32_t ncols)
{
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     (uint32_t)__cvta_generic_to_shared(dst)),
                 "r"(ncols)
                 : "memory");
}
// Give up this CTA's right to allocate again, so that a waiting CTA on the
// SM may allocate; one full warp.
__device__ __forceinline__ void sg_tc_relinquish()
{
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void sg_tc_dealloc(uint32_t taddr, uint32_t ncols)
{
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}
// Order tensor-core operations across a thread barrier.
__device__ __forceinline__ void sg_tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void sg_tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
// One arrival (no transaction bytes) on an mbarrier's current phase.
__device__ __forceinline__ void sg_mbar_arrive(uint64_t* bar)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"((uint32_t)__cvta_generic_to_shared(bar))
                 : "memory");
}
// Make this thread's ordinary shared-memory stores visible to the tensor
// core's (asynchronous proxy) reads.
__device__ __forceinline__ void sg_fence_proxy_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

// D (tensor memory, 128 lanes x N columns of FP32) = A B + (acc ? D : 0),
// A: 128 x 8 and B: N x 8 TF32 values given by their descriptors.  One
// thread issues it.
__device__ __forceinline__ void sg_tc_mma_tf32(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                               uint32_t acc)
{
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(d_tmem),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(acc)
        : "memory");
}
// Arrive once on the mbarrier when every tensor-core operation this thread
// has issued so far has completed.
__device__ __forceinline__ void sg_tc_commit(uint64_t* bar)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                     (uint32_t)__cvta_generic_to_shared(bar))
                 : "memory");
}

// 32 consecutive FP32 columns of this warp's 32 lanes (lane = thread's lane
// within the warp's quarter of tensor memory): taddr = base + (lane0 << 16) +
// column.  Complete after sg_tc_wait_ld.
__device__ __forceinline__ void sg_tc_ld32(uint32_t taddr, float (&v)[32])
{
    uint32_t r[32];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
        "%15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
          "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
          "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr)
        : "memory");
#pragma unroll
    for (int i = 0; i < 32; i++) v[i] = __uint_as_float(r[i]);
}
__device__ __forceinline__ void sg_tc_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }
#endif
