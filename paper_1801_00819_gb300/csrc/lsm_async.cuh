// Asynchronous global -> shared copies (cp.async, 16 bytes per thread and copy) used to stage the
// coefficient rows of the next depth step while the current one runs.
#pragma once

#include <cuda_runtime.h>

namespace lsm {

__device__ __forceinline__ void cp_async16(void* smem_dst, const void* gmem_src) {
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem_dst);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gmem_src) : "memory");
}
// The same copy, bypassing L1 and marked evict-first in L2: for rows that stream through once per
// launch, so that they do not push out data a later kernel reads back from L2.
__device__ __forceinline__ unsigned long long l2_evict_first_policy() {
    unsigned long long pol;
    asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;\n" : "=l"(pol));
    return pol;
}
__device__ __forceinline__ void cp_async16_stream(void* smem_dst, const void* gmem_src, unsigned long long pol) {
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem_dst);
    asm volatile("cp.async.cg.shared.global.L2::cache_hint [%0], [%1], 16, %2;\n" ::"r"(s), "l"(gmem_src), "l"(pol)
                 : "memory");
}
// A 16-byte store marked evict-last in L2: for data that a kernel launched right after this one
// reads back (and then drops with discard.global.L2), so that streamed loads do not push it out.
__device__ __forceinline__ void st_global_keep_l2(float4* dst, float4 v) {
    unsigned long long pol;
    asm volatile("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;\n" : "=l"(pol));
    asm volatile("st.global.L2::cache_hint.v4.f32 [%0], {%1, %2, %3, %4}, %5;\n" ::"l"(dst), "f"(v.x), "f"(v.y),
                 "f"(v.z), "f"(v.w), "l"(pol)
                 : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;\n" ::: "memory"); }

}  // namespace lsm
