// Shared-memory addresses and bounded mbarrier waits of the kernels that take
// their operands by TMA bulk copies (cp.async.bulk completing on an mbarrier).
// Every wait polls a bounded number of times and reports whether the phase
// completed, so that a copy that never lands ends the CTA with an error status
// instead of a hang.
#pragma once
#include <cuda_runtime.h>

namespace dnsk {

__device__ __forceinline__ unsigned su32(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }

// Wait on phase `parity` of the mbarrier at shared address bar (at most 2^22
// polls); false if it did not complete.
__device__ __forceinline__ bool mbar_wait(unsigned bar, unsigned parity) {
    for (int it = 0; it < (1 << 22); ++it) {
        unsigned done;
        asm volatile(
            "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
            : "=r"(done) : "r"(bar), "r"(parity) : "memory");
        if (done) return true;
    }
    return false;
}

}  // namespace dnsk
