// kernels_tc.cu -- the fp32 flush contraction (Eq. 4) on the 5th-generation
// tensor cores: split-bf16 x3 with fp32 accumulation in tensor memory.
//
//   C = alpha * A B' + beta * C,   A: M x K,  B: N x K (or K x N), fp32.
//
// Each fp32 operand x is split as x = hi + lo with hi = bf16(x) and
// lo = bf16(x - hi); the product is hi*hi + hi*lo + lo*hi (the lo*lo term,
// ~2^-16 of the product, is dropped), each bf16 x bf16 product exact in the
// fp32 accumulator. One CTA computes a 128 x BN tile of C:
//   * 256 threads stage a K-block of both operands from global memory, split
//     them and write bf16 "core matrices" (8 rows x 16 bytes, K-major, no
//     swizzle) into shared memory, double buffered;
//   * one thread issues tcgen05.mma (M = 128, N = BN, K = 16) into a tensor
//     memory accumulator and commits to an mbarrier;
//   * four warps read the accumulator back with tcgen05.ld (warp w owns
//     lanes 32w..32w+31, i.e. rows of the tile) and apply alpha / beta.
// Every wait is bounded; on expiry the kernel records ST_TIMEOUT, still waits
// (bounded) for its issued MMAs, frees its tensor memory and returns.
#include <cuda_bf16.h>
#include <stdint.h>

#include "qmcdu_internal.cuh"

namespace qmcdu {

namespace tc {

constexpr int THREADS = 256;
constexpr int BM = 128;         // tile rows = TMEM lanes
constexpr int BK = 32;          // K-block staged per step (two MMA K-steps of 16)
constexpr int STAGES = 2;

__device__ __forceinline__ uint32_t su32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ unsigned long long gtimer()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Shared-memory matrix descriptor of the 5th-generation tensor cores: start
// address, leading byte offset (between core matrices along K), stride byte
// offset (between 8-row groups), all in 16-byte units; descriptor version 1;
// no swizzle.
__device__ __forceinline__ uint64_t sdesc(uint32_t saddr, uint32_t lbo, uint32_t sbo)
{
    return (uint64_t)((saddr >> 4) & 0x3FFFu) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) |
           ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | (1ull << 46);
}

// Instruction descriptor of kind::f16: D fp32, A and B bf16, both K-major,
// N >> 3 at bit 17, M >> 4 at bit 24.
__host__ __device__ constexpr uint32_t idesc_bf16(int M, int N)
{
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void mma_bf16(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc,
                                         uint32_t accumulate)
{
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n"
        ::"r"(d_tmem), "l"(a), "l"(b), "r"(idesc), "r"(accumulate) : "memory");
}

__device__ __forceinline__ void mma_commit(uint64_t *bar)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];"
                 ::"r"(su32(bar)) : "memory");
}

__device__ __forceinline__ void bar_init(uint64_t *bar, unsigned count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(su32(bar)), "r"(count) : "memory");
}

// Bounded wait for the completion of phase `parity`.
__device__ __forceinline__ bool bar_wait(uint64_t *bar, unsigned parity, long long budget_ns)
{
    const unsigned long long t0 = gtimer();
    for (;;) {
        unsigned done;
        asm volatile(
            "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
            " selp.u32 %0, 1, 0, p;\n}\n"
            : "=r"(done) : "r"(su32(bar)), "r"(parity) : "memory");
        if (done) return true;
        if ((long long)(gtimer() - t0) > budget_ns) return false;
    }
}

// Byte offset of element (row r, column k) of a K-major bf16 tile of BK
// columns laid out as 8 x 8 core matrices: core matrix (r/8, k/8) at
// ((r/8) * (BK/8) + k/8) * 128, row r%8 at 16 bytes, column k%8 at 2 bytes.
__device__ __forceinline__ uint32_t core_off(int r, int k)
{
    return (uint32_t)((((r >> 3) * (BK / 8) + (k >> 3)) << 7) + ((r & 7) << 4) + ((k & 7) << 1));
}
constexpr uint32_t LBO = 128;                 // next core matrix along K
constexpr uint32_t SBO = (BK / 8) * 128;      // next 8-row group

struct Args {
    int M, N, K;                 // nominal sizes (K, N may be replaced per batch by kdyn)
    const float *A; long long lda, sA;        // A(m, k) = A[m*lda + k]
    const float *B; long long ldb, sB;        // B(n, k) = B[n*ldb + k], or B[k*ldb + n] if b_trans
    int b_trans;
    float *C; long long ldc, sC;              // C(m, n) = C[m*ldc + n]
    float alpha, beta;
    const int *kdyn;             // per-batch k (device) or null
    int kdyn_is_n;               // 1: k replaces N (rounded up to 16); 0: k replaces K
    int kthresh;                 // batches with k < kthresh are skipped (when kdyn)
    const int *fix_idx;          // C(m, n) -= [m == fix_idx[b*fix_stride + n]]
    int fix_stride;
    int *status;
    long long budget_ns;
};

template <int BN>
struct Smem {
    __nv_bfloat16 a_hi[STAGES][BM * BK], a_lo[STAGES][BM * BK];
    __nv_bfloat16 b_hi[STAGES][BN * BK], b_lo[STAGES][BN * BK];
    uint64_t bar[STAGES];
    uint32_t tmem_base;
};

// Stage K-block k0 of both operands into buffer s (split into hi / lo).
template <int BN>
__device__ __forceinline__ void stage(const Args &g, Smem<BN> &sm, int s, int m0, int n0, int k0,
                                      int M, int N, int K, const float *A, const float *B)
{
    for (int e = threadIdx.x; e < BM * BK; e += THREADS) {
        const int r = e / BK, kk = e - r * BK;
        const int gm = m0 + r, gk = k0 + kk;
        const float x = (gm < M && gk < K) ? __ldcg(A + gm * g.lda + gk) : 0.f;
        const __nv_bfloat16 hi = __float2bfloat16_rn(x);
        const __nv_bfloat16 lo = __float2bfloat16_rn(x - __bfloat162float(hi));
        const uint32_t o = core_off(r, kk) >> 1;
        sm.a_hi[s][o] = hi;
        sm.a_lo[s][o] = lo;
    }
    for (int e = threadIdx.x; e < BN * BK; e += THREADS) {
        int r, kk;
        if (g.b_trans) { kk = e / BN; r = e - kk * BN; }   // consecutive threads along n
        else { r = e / BK; kk = e - r * BK; }               // consecutive threads along k
        const int gn = n0 + r, gk = k0 + kk;
        float x = 0.f;
        if (gn < N && gk < K) x = g.b_trans ? __ldcg(B + gk * g.ldb + gn) : __ldcg(B + gn * g.ldb + gk);
        const __nv_bfloat16 hi = __float2bfloat16_rn(x);
        const __nv_bfloat16 lo = __float2bfloat16_rn(x - __bfloat162float(hi));
        const uint32_t o = core_off(r, kk) >> 1;
        sm.b_hi[s][o] = hi;
        sm.b_lo[s][o] = lo;
    }
}

template <int BN>
__global__ void __launch_bounds__(THREADS, 1) gemm_bf16x3_kernel(Args g)
{
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    Smem<BN> &sm = *reinterpret_cast<Smem<BN> *>(smem_raw);
    const int b = blockIdx.z;
    int M = g.M, N = g.N, K = g.K;
    if (g.kdyn) {
        const int kb = g.kdyn[b];
        if (kb < g.kthresh || kb <= 0) return;
        if (g.kdyn_is_n) N = kb; else K = kb;
    }
    const int m0 = blockIdx.x * BM, n0 = blockIdx.y * BN;
    if (m0 >= M || n0 >= N) return;
    const float *A = g.A + b * g.sA;
    const float *B = g.B + b * g.sB;
    float *C = g.C + b * g.sC;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

    // tensor memory: BN fp32 columns x 128 lanes (one warp allocates)
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
                     ::"r"(su32(&sm.tmem_base)), "r"((uint32_t)BN) : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (threadIdx.x == 0) {
        for (int s = 0; s < STAGES; ++s) bar_init(&sm.bar[s], 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = sm.tmem_base;
    const int nb = (min(N - n0, BN) + 15) / 16 * 16;        // MMA N for this tile
    const uint32_t idesc = idesc_bf16(BM, nb);
    const int nk = (K + BK - 1) / BK;
    unsigned phase[STAGES] = {0, 0};
    int issued[STAGES] = {0, 0};
    bool ok = true;
    __shared__ int ok_s;

    for (int kb = 0; kb < nk; ++kb) {
        const int s = kb % STAGES;
        // buffer s is free once the MMAs that read it (issued STAGES blocks ago) are done
        if (issued[s]) {
            if (threadIdx.x == 0) ok_s = bar_wait(&sm.bar[s], phase[s], g.budget_ns) ? 1 : 0;
            __syncthreads();
            phase[s] ^= 1u;
            issued[s] = 0;
            if (!ok_s) { ok = false; break; }
        }
        stage<BN>(g, sm, s, m0, n0, kb * BK, M, N, K, A, B);
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        __syncthreads();
        if (threadIdx.x == 0) {
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
#pragma unroll
            for (int ks = 0; ks < BK / 16; ++ks) {
                const uint32_t koff = (uint32_t)(2 * ks) * 128u;   // two core matrices per K-step
                const uint64_t ah = sdesc(su32(sm.a_hi[s]) + koff, LBO, SBO);
                const uint64_t al = sdesc(su32(sm.a_lo[s]) + koff, LBO, SBO);
                const uint64_t bh = sdesc(su32(sm.b_hi[s]) + koff, LBO, SBO);
                const uint64_t bl = sdesc(su32(sm.b_lo[s]) + koff, LBO, SBO);
                const uint32_t first = (kb == 0 && ks == 0) ? 0u : 1u;
                mma_bf16(tmem, ah, bh, idesc, first);
                mma_bf16(tmem, ah, bl, idesc, 1u);
                mma_bf16(tmem, al, bh, idesc, 1u);
            }
            mma_commit(&sm.bar[s]);
        }
        issued[s] = 1;
    }
    // drain: wait for every issued commit (bounded even after a failure)
    for (int s = 0; s < STAGES; ++s) {
        if (issued[s]) {
            if (threadIdx.x == 0) ok_s = bar_wait(&sm.bar[s], phase[s], g.budget_ns) ? 1 : 0;
            __syncthreads();
            if (!ok_s) ok = false;
        }
    }
    if (!ok && threadIdx.x == 0 && g.status) atomicOr(g.status, ST_TIMEOUT);
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");

    if (ok && warp < 4) {
        const bool have_acc = nk > 0;   // K = 0: the product is zero
        // epilogue: warp w owns tile rows 32w .. 32w+31 (TMEM lanes)
        const int row = m0 + warp * 32 + lane;
        for (int c0 = 0; c0 < nb; c0 += 16) {
            uint32_t r[16] = {0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0};
            const uint32_t taddr = tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0;
            if (have_acc) asm volatile(
                "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,"
                "%13,%14,%15}, [%16];"
                : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
                  "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]),
                  "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
                : "r"(taddr));
            if (have_acc) asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
            if (row < M) {
#pragma unroll
                for (int j = 0; j < 16; ++j) {
                    const int col = n0 + c0 + j;
                    if (col >= N) continue;
                    float v = g.alpha * __uint_as_float(r[j]);
                    float *dst = C + row * g.ldc + col;
                    if (g.beta != 0.f) v += g.beta * *dst;
                    if (g.fix_idx && g.fix_idx[(size_t)b * g.fix_stride + col] == row) v -= 1.f;
                    *dst = v;
                }
            }
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;"
                     ::"r"(tmem), "r"((uint32_t)BN) : "memory");
}

template <int BN>
static cudaError_t launch_bn(const Args &g, int batch, cudaStream_t s)
{
    const size_t smem = sizeof(Smem<BN>);
    cudaError_t e = cudaFuncSetAttribute(gemm_bf16x3_kernel<BN>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    dim3 grid((g.M + BM - 1) / BM, (g.N + BN - 1) / BN, batch);
    gemm_bf16x3_kernel<BN><<<grid, THREADS, smem, s>>>(g);
    return cudaGetLastError();
}

}  // namespace tc

// C = alpha A B' + beta C in split-bf16 x3 on tcgen05 (see the file comment).
cudaError_t launch_gemm_bf16x3(int M, int N, int K, const float *A, long long lda, long long sA,
                               const float *B, long long ldb, long long sB, int b_trans, float *C,
                               long long ldc, long long sC, float alpha, float beta, int batch,
                               const int *kdyn, int kdyn_is_n, int kthresh, const int *fix_idx,
                               int fix_stride, int *status, long long budget_ns, cudaStream_t s)
{
    tc::Args g;
    g.M = M; g.N = N; g.K = K;
    g.A = A; g.lda = lda; g.sA = sA;
    g.B = B; g.ldb = ldb; g.sB = sB; g.b_trans = b_trans;
    g.C = C; g.ldc = ldc; g.sC = sC;
    g.alpha = alpha; g.beta = beta;
    g.kdyn = kdyn; g.kdyn_is_n = kdyn_is_n; g.kthresh = kthresh;
    g.fix_idx = fix_idx; g.fix_stride = fix_stride;
    g.status = status; g.budget_ns = budget_ns;
    if (M <= 0 || N <= 0 || K < 0 || batch <= 0) return cudaSuccess;
    // narrow N (a short queue) takes a narrower tile
    if (N <= 64) return tc::launch_bn<64>(g, batch, s);
    if (N <= 128) return tc::launch_bn<128>(g, batch, s);
    return tc::launch_bn<256>(g, batch, s);
}

}  // namespace qmcdu
