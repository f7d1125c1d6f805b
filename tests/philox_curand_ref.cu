// Test-only reference: cuRAND's own Philox4x32-10 (curand_philox4x32_x.h),
// used to pin the library's generator and the numpy input generator.
#include <curand_kernel.h>

__global__ void curand_philox_kernel(const uint4 *ctr, unsigned k0, unsigned k1, uint4 *out, int n)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] = curand_Philox4x32_10(ctr[i], make_uint2(k0, k1));
}

extern "C" int curand_philox_ref(const void *ctr, unsigned k0, unsigned k1, void *out, int n)
{
    if (n <= 0) return 0;
    curand_philox_kernel<<<(n + 255) / 256, 256>>>((const uint4 *)ctr, k0, k1, (uint4 *)out, n);
    return (int)cudaDeviceSynchronize();
}
