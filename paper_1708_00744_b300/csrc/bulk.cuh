// bulk.cuh -- device helpers shared by libqmcdu's kernels: the global timer,
// and bulk asynchronous copies global -> shared memory whose completion is
// counted on an mbarrier (transaction bytes), with time-bounded waits that
// report ST_TIMEOUT instead of spinning forever.
#pragma once

#include <cuda_runtime.h>

#include "qmcdu_internal.cuh"

namespace qmcdu {

__device__ __forceinline__ unsigned long long globaltimer()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// ---- bulk asynchronous copy global -> shared, completion on an mbarrier
__device__ __forceinline__ unsigned smem_addr(const void *p)
{
    return (unsigned)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(unsigned long long *bar)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_addr(bar)) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void mbar_expect(unsigned long long *bar, unsigned bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;"
                 ::"r"(smem_addr(bar)), "r"(bytes) : "memory");
}

__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, unsigned bytes,
                                         unsigned long long *bar)
{
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
        ::"r"(smem_addr(dst)), "l"(src), "r"(bytes), "r"(smem_addr(bar)) : "memory");
}

// Bounded wait for phase `parity` of the mbarrier; false on timeout.
__device__ __forceinline__ bool mbar_wait(unsigned long long *bar, unsigned parity, int *status,
                                          long long budget_ns)
{
    const unsigned long long t0 = globaltimer();
    for (;;) {
        unsigned done;
        asm volatile(
            "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
            " selp.u32 %0, 1, 0, p;\n}\n"
            : "=r"(done) : "r"(smem_addr(bar)), "r"(parity) : "memory");
        if (done) return true;
        if ((long long)(globaltimer() - t0) > budget_ns) {
            atomicOr(status, ST_TIMEOUT);
            return false;
        }
    }
}

// Arrive on an mbarrier (no transaction bytes).
__device__ __forceinline__ void mbar_arrive(unsigned long long *bar)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_addr(bar)) : "memory");
}

// pivot-search key of x: the bit pattern of |x|, which orders non-negative
// doubles as their values do, compared on the integer pipe; NaN gives -2, below
// the empty key -1, so that it never wins (as an fp64 comparison leaves it)
__device__ __forceinline__ long long gj_key(double x)
{
    const long long b = __double_as_longlong(x) & 0x7FFFFFFFFFFFFFFFll;
    return b > 0x7FF0000000000000ll ? -2ll : b;
}

__device__ __forceinline__ void mbar_init_count(unsigned long long *bar, unsigned count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}

}  // namespace qmcdu
