// Fifth-generation tensor-core primitives of sm_100-class GPUs (tcgen05), written as inline PTX:
// tensor-memory (TMEM) allocation, the single-thread matrix multiply-accumulate with operands in
// shared memory and the accumulator in TMEM, its completion signalled on an mbarrier, and the
// warp-wide TMEM -> register loads of the accumulator.
//
// Operand layout used throughout: K-major tiles with the 128-byte swizzle.  A tile of `rows` rows
// (M or N) by 64 sixteen-bit K elements occupies rows x 128 bytes, 1024-byte aligned; row r starts at
// byte (r / 8) 1024 + (r % 8) 128 and its eight 16-byte chunks (K elements 8c .. 8c+7) are stored at
// chunk position c ^ (r % 8).  Longer K is a sequence of such 64-element K blocks.  An MMA step of
// K = 16 starting at K element k0 of a block takes the block's descriptor with its start address
// advanced by 2 k0 bytes.
//
// Every wait on an mbarrier is bounded: after about a second the caller gets `false` and must
// report an error instead of waiting longer.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>

namespace lsm {
namespace umma {

constexpr uint64_t kWaitLimitNs = 1000000000ull;  // a wait on an mbarrier gives up after one second
constexpr uint32_t kSpinLimit = 1u << 30;          // and after this many polls in any case

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ uint64_t globaltimer_ns() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;\n" : "=l"(t));
    return t;
}

// ---------------------------------------------------------------------------------------- mbarrier

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

// true once the phase with the given parity has completed; false after about a second
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity) {
    const uint32_t addr = smem_u32(bar);
    uint64_t t0 = 0;
    for (uint32_t i = 0; i < kSpinLimit; ++i) {
        uint32_t done;
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}\n"
            : "=r"(done)
            : "r"(addr), "r"(parity)
            : "memory");
        if (done) return true;
        if ((i & 255u) == 0) {
            const uint64_t t = globaltimer_ns();
            if (i == 0) t0 = t;
            else if (t - t0 > kWaitLimitNs) return false;
        }
    }
    return false;
}

// --------------------------------------------------------------------------------- tensor memory

// Allocate `ncols` TMEM columns (a power of two, 32 .. 512) for the CTA; the base address is
// written to *slot (shared memory).  Called by one whole warp.
__device__ __forceinline__ void tmem_alloc(uint32_t* slot, uint32_t ncols) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(smem_u32(slot)),
                 "r"(ncols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::: "memory");
}

// Free the CTA's columns; called by one whole warp after every MMA and TMEM access has finished.
__device__ __forceinline__ void tmem_free(uint32_t base, uint32_t ncols) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(base), "r"(ncols) : "memory");
}

__device__ __forceinline__ void fence_before_sync() { asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory"); }
__device__ __forceinline__ void fence_after_sync() { asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory"); }

// generic-proxy shared-memory writes made visible to the tensor core (the async proxy)
__device__ __forceinline__ void fence_smem_to_async() { asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory"); }

// ------------------------------------------------------------------------------- descriptors

// Shared-memory matrix descriptor: K-major, 128-byte swizzle, 8-row groups 1024 bytes apart.
__device__ __forceinline__ uint64_t desc_sw128(uint32_t smem_addr) {
    uint64_t d = 0;
    d |= (uint64_t)((smem_addr & 0x3FFFFu) >> 4);  // start address, 16-byte units
    d |= (uint64_t)1 << 16;                         // leading-dimension byte offset (unused for this layout)
    d |= (uint64_t)(1024u >> 4) << 32;              // stride-dimension byte offset: next 8-row group
    d |= (uint64_t)1 << 46;                         // descriptor version of sm_100-class GPUs
    d |= (uint64_t)2 << 61;                         // swizzle mode: 128 bytes
    return d;
}

// Instruction descriptor of kind::f16 with FP32 accumulation, both operands K-major.
//   ab_bf16: operands are bf16 (true) or fp16 (false); M = 128; N a multiple of 16 up to 256.
__host__ __device__ constexpr uint32_t idesc_f16(bool ab_bf16, int M, int N) {
    return (1u << 4)                              // accumulator format: F32
           | ((ab_bf16 ? 1u : 0u) << 7)           // A format
           | ((ab_bf16 ? 1u : 0u) << 10)          // B format
           | ((uint32_t)(N >> 3) << 17)           // N / 8
           | ((uint32_t)(M >> 4) << 24);          // M / 16
}

// D[tmem] (+)= A[smem] . B[smem]^T for one K = 16 step; issued by a single thread.
__device__ __forceinline__ void mma_f16(uint32_t d_tmem, uint64_t a_desc, uint64_t b_desc, uint32_t idesc,
                                        bool accumulate) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(d_tmem),
        "l"(a_desc), "l"(b_desc), "r"(idesc), "r"((uint32_t)accumulate)
        : "memory");
}

// Arrive once on `bar` when every MMA this thread has issued so far has completed.
__device__ __forceinline__ void mma_commit(uint64_t* bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(
                     smem_u32(bar))
                 : "memory");
}

// ------------------------------------------------------------------------- TMEM -> registers

// 32 consecutive 32-bit columns of this thread's TMEM lane (warp w reads lanes 32 (w % 4) ..).  The
// wait for the load is part of the same statement, so no use of the registers can be scheduled
// before the data has arrived.
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float (&v)[32]) {
    uint32_t r[32];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
        "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
        "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];\n\t"
        "tcgen05.wait::ld.sync.aligned;\n"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
          "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
          "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr)
        : "memory");
#pragma unroll
    for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}

// 16 consecutive 32-bit columns of this thread's TMEM lane (as tmem_ld32)
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float (&v)[16]) {
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 "
        "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];\n\t"
        "tcgen05.wait::ld.sync.aligned;\n"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr)
        : "memory");
#pragma unroll
    for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

// byte offset of 16-bit K element k of row r in a K-major 128-byte-swizzled block (rows x 64)
__host__ __device__ constexpr uint32_t sw128_offset(uint32_t r, uint32_t k) {
    return (r >> 3) * 1024u + (r & 7u) * 128u + ((((k >> 3) ^ r) & 7u) << 4) + ((k & 7u) << 1);
}

}  // namespace umma
}  // namespace lsm
