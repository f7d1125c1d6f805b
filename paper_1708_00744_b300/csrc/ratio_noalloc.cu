// ratio_noalloc.cu -- determinant ratio of one proposed move through a delay
// queue that the caller holds, computed without allocating device memory.
//
// Same arithmetic as the handle's ratio kernel (kernels_move.cu), in the
// change form of Eq. 1-3 (u = v - a_j, V rows the queued changes):
//   d = u . a,  b = P u,  c = V a,  r = 1 + (d - b' Kinv c)
// with the chunk partial sums of the CTAs and their arrival counter kept in one
// fixed, file-scope device array instead of memory owned by a handle. Every
// call on a device shares that array; it keeps the last call's contents, so
// the arrival counter is cleared (a memset, no allocation) before each launch,
// and calls whose executions overlap on the GPU race on it.
#include <mutex>
#include <string>

#include "qmcdu_internal.cuh"

namespace qmcdu {

namespace {

constexpr int NA_CHUNK = 256;                            // elements of N per CTA
constexpr int NA_THREADS = 256;
constexpr int NA_MAX_SPLIT = QMCDU_MAX_N / NA_CHUNK;     // 32 CTAs at N = 8192
constexpr int NA_MAX_JOBS = 2 * QMCDU_MAX_K + 1;         // 513 dot products at k = 256
constexpr size_t NA_COUNTER_BYTES = 256;
constexpr size_t NA_SCRATCH_BYTES =
    NA_COUNTER_BYTES + sizeof(double) * (size_t)NA_MAX_SPLIT * NA_MAX_JOBS;   // 131,584 bytes

// The scratch: [0, 256) arrival counter, then NA_MAX_SPLIT x NA_MAX_JOBS fp64
// partial sums. Every GPU that loads the library holds it until exit.
static __device__ __align__(256) unsigned char qmcdu_noalloc_scratch[NA_SCRATCH_BYTES];

constexpr int NA_MAX_DEVICES = 128;
std::mutex na_mutex;
void *na_scratch_addr[NA_MAX_DEVICES] = {};

__device__ __forceinline__ double na_warp_sum(double v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Grid: ceil(N / 256) CTAs; CTA s forms the 2k+1 partial dot products of its
// chunk; the last CTA to arrive sums them in chunk order and forms r.
__global__ void __launch_bounds__(NA_THREADS) ratio_noalloc_kernel(
    int N, int k, const double *__restrict__ a, const double *__restrict__ u,
    const double *__restrict__ P, const double *__restrict__ V, const double *__restrict__ Kinv,
    double *ratio_out, unsigned char *scratch)
{
    unsigned *arrive = (unsigned *)scratch;
    double *partial = (double *)(scratch + NA_COUNTER_BYTES);
    const int split = blockIdx.x, nsplit = gridDim.x;
    const int i0 = split * NA_CHUNK, n = min(NA_CHUNK, N - i0);
    const int nj = 2 * k + 1;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int job = warp; job < nj; job += NA_THREADS / 32) {
        const double *src, *with;
        if (job == 0) { src = a; with = u; }
        else if (job <= k) { src = P + (size_t)(job - 1) * N; with = u; }
        else { src = V + (size_t)(job - 1 - k) * N; with = a; }
        double s = 0.0;
        for (int t = lane; t < n; t += 32) s += src[i0 + t] * with[i0 + t];
        s = na_warp_sum(s);
        if (lane == 0) partial[(size_t)split * NA_MAX_JOBS + job] = s;
    }
    __threadfence();
    __syncthreads();
    __shared__ unsigned ticket;
    if (threadIdx.x == 0) ticket = atomicAdd(arrive, 1u);
    __syncthreads();
    if (ticket != (unsigned)(nsplit - 1)) return;
    __threadfence();
    __shared__ double red[NA_MAX_JOBS];
    __shared__ double xs[QMCDU_MAX_K];
    for (int job = threadIdx.x; job < nj; job += NA_THREADS) {
        double s = 0.0;
        for (int q = 0; q < nsplit; ++q) s += __ldcg(partial + (size_t)q * NA_MAX_JOBS + job);
        red[job] = s;
    }
    __syncthreads();
    const double *bv = red + 1, *cv = red + 1 + k;
    for (int m = threadIdx.x; m < k; m += NA_THREADS) {
        double x = 0.0;
        for (int q = 0; q < k; ++q) x += Kinv[(size_t)m * k + q] * cv[q];
        xs[m] = x;
    }
    __syncthreads();
    if (warp == 0) {
        double s = 0.0;
        for (int m = lane; m < k; m += 32) s += bv[m] * xs[m];
        s = na_warp_sum(s);
        if (lane == 0) {
            *ratio_out = 1.0 + (red[0] - s);
            *arrive = 0u;
        }
    }
}

}  // namespace

}  // namespace qmcdu

using namespace qmcdu;

extern "C" int qmcdu_ratio_noalloc(int N, int k, const double *ainv_col, const double *u,
                                   const double *P, const double *V, const double *Kinv,
                                   double *ratio_out, void *stream)
{
    if (N < 1 || N > QMCDU_MAX_N || k < 0 || k > QMCDU_MAX_K || k > N) {
        set_handleless_error(
            "qmcdu_ratio_noalloc: N=" + std::to_string(N) + ", k=" + std::to_string(k) +
            " outside the fixed scratch (1 <= N <= 8192, 0 <= k <= min(N, 256))");
        return QMCDU_ERR_ARG;
    }
    if (!ainv_col || !u || !ratio_out || (k > 0 && (!P || !V || !Kinv))) {
        set_handleless_error("qmcdu_ratio_noalloc: null pointer argument");
        return QMCDU_ERR_ARG;
    }
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess || dev < 0 || dev >= NA_MAX_DEVICES) {
        set_handleless_error(std::string("qmcdu_ratio_noalloc: no usable current device: ") +
                             cudaGetErrorString(e));
        return QMCDU_ERR_CUDA;
    }
    void *scratch = nullptr;
    {
        // set-up, once per device, with that device current
        std::lock_guard<std::mutex> lock(na_mutex);
        if (!na_scratch_addr[dev]) {
            e = cudaGetSymbolAddress(&na_scratch_addr[dev], qmcdu_noalloc_scratch);
            if (e != cudaSuccess) {
                na_scratch_addr[dev] = nullptr;
                set_handleless_error(std::string("qmcdu_ratio_noalloc: cudaGetSymbolAddress: ") +
                                     cudaGetErrorString(e));
                return QMCDU_ERR_CUDA;
            }
        }
        scratch = na_scratch_addr[dev];
    }
    cudaStream_t s = (cudaStream_t)stream;
    e = cudaMemsetAsync(scratch, 0, sizeof(unsigned), s);
    if (e == cudaSuccess) {
        const int nsplit = (N + NA_CHUNK - 1) / NA_CHUNK;
        ratio_noalloc_kernel<<<nsplit, NA_THREADS, 0, s>>>(N, k, ainv_col, u, P, V, Kinv, ratio_out,
                                                          (unsigned char *)scratch);
        e = cudaGetLastError();
    }
    if (e != cudaSuccess) {
        set_handleless_error(std::string("qmcdu_ratio_noalloc: ") + cudaGetErrorString(e));
        return QMCDU_ERR_CUDA;
    }
    return QMCDU_OK;
}
