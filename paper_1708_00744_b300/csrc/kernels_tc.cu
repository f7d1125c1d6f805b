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

#include <algorithm>
#include <map>
#include <mutex>

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

// ---------------------------------------------------------------------------
// The plain contraction (one matrix, no per-batch k) with operands split once:
//   * tc2_split_kernel writes each fp32 operand as bf16 hi and lo planes,
//     already in the tensor cores' K-major core-matrix layout, tile by tile
//     (A: 128-row tiles, B: 256-row tiles, 32 columns of K each; a tile's hi
//     plane, then its lo plane, contiguous), zero-padded to whole tiles;
//   * tc2_gemm_kernel streams those tiles into a 4-stage shared-memory ring
//     with one bulk copy per operand per stage (producer warp, "full"
//     mbarriers counting bytes), one thread issues the three MMAs per K-step of
//     16 into a 128 x 256 fp32 accumulator in tensor memory and commits each
//     stage to its "empty" mbarrier, and four warps apply alpha / beta.
namespace tc2 {

constexpr int BM = 128, BN = 256, BK = 32, STAGES = 4;
constexpr int THREADS = 192;    // warp 0 producer, warp 1 MMA, warps 2..5 epilogue
constexpr uint32_t A_TILE = BM * BK * 2;          // bytes of one bf16 plane of an A tile
constexpr uint32_t B_TILE = BN * BK * 2;
constexpr uint32_t STAGE_BYTES = 2 * A_TILE + 2 * B_TILE;
constexpr size_t SMEM = (size_t)STAGES * STAGE_BYTES + 256;

// Split rows x cols of X (row r, column k at X[r * ldr + k * ldc]) into tiles of
// R rows: tile (r / R, k / BK) at ((r / R) * nkb + k / BK) * 2 * R * BK * 2 bytes.
// One thread per 8 consecutive k of a row: one 16-byte row of a core matrix
// in each plane, written with one vector store.
template <int R>
__global__ void tc2_split_kernel(const float *X, long long ldr, long long ldc, int rows, int cols,
                                 int nkb, unsigned char *out, long long total)
{
    const long long per_row = (long long)nkb * (BK / 8);
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
         e += (long long)gridDim.x * blockDim.x) {
        const int r = (int)(e / per_row);
        const int k0 = (int)(e - (long long)r * per_row) * 8;
        uint32_t hw[4], lw[4];
#pragma unroll
        for (int j = 0; j < 8; j += 2) {
            const int k = k0 + j;
            const float x0 = (r < rows && k < cols) ? __ldg(X + r * ldr + (long long)k * ldc) : 0.f;
            const float x1 = (r < rows && k + 1 < cols) ? __ldg(X + r * ldr + (long long)(k + 1) * ldc) : 0.f;
            const __nv_bfloat16 h0 = __float2bfloat16_rn(x0), h1 = __float2bfloat16_rn(x1);
            const __nv_bfloat16 l0 = __float2bfloat16_rn(x0 - __bfloat162float(h0));
            const __nv_bfloat16 l1 = __float2bfloat16_rn(x1 - __bfloat162float(h1));
            hw[j / 2] = (uint32_t)__bfloat16_as_ushort(h0) | ((uint32_t)__bfloat16_as_ushort(h1) << 16);
            lw[j / 2] = (uint32_t)__bfloat16_as_ushort(l0) | ((uint32_t)__bfloat16_as_ushort(l1) << 16);
        }
        const int rt = r / R, rr = r - rt * R, kt = k0 / BK, kk = k0 - kt * BK;
        unsigned char *tile = out + ((size_t)rt * nkb + kt) * (size_t)(2 * R * BK * 2);
        const uint32_t o = tc::core_off(rr, kk);
        *reinterpret_cast<uint4 *>(tile + o) = make_uint4(hw[0], hw[1], hw[2], hw[3]);
        *reinterpret_cast<uint4 *>(tile + R * BK * 2 + o) = make_uint4(lw[0], lw[1], lw[2], lw[3]);
    }
}

struct Args2 {
    int M, N, K, nkb;
    const __nv_bfloat16 *At, *Bt;     // split tiles
    float *C;
    long long ldc;
    float alpha, beta;
    int *status;
    long long budget_ns;
};

__device__ __forceinline__ void bulk_copy(void *dst, const void *src, uint32_t bytes, uint64_t *bar)
{
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
        ::"r"(tc::su32(dst)), "l"(src), "r"(bytes), "r"(tc::su32(bar)) : "memory");
}

__device__ __forceinline__ void expect_tx(uint64_t *bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;"
                 ::"r"(tc::su32(bar)), "r"(bytes) : "memory");
}

__global__ void __launch_bounds__(THREADS, 1) tc2_gemm_kernel(Args2 g)
{
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    unsigned char *ring = smem_raw;                                        // [STAGES][STAGE_BYTES]
    uint64_t *full = reinterpret_cast<uint64_t *>(smem_raw + (size_t)STAGES * STAGE_BYTES);
    uint64_t *empty = full + STAGES;
    uint64_t *done = empty + STAGES;
    uint32_t *tmem_s = reinterpret_cast<uint32_t *>(done + 1);
    __shared__ int abort_s, issued_s;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int m0 = blockIdx.x * BM, n0 = blockIdx.y * BN;
    const int nk = g.nkb;

    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
                     ::"r"(tc::su32(tmem_s)), "r"((uint32_t)BN) : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (threadIdx.x == 0) {
        for (int s = 0; s < STAGES; ++s) {
            tc::bar_init(&full[s], 1);
            tc::bar_init(&empty[s], 1);
        }
        tc::bar_init(done, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        abort_s = 0;
        issued_s = 0;
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = *tmem_s;

    if (warp == 0 && lane == 0) {
        // producer
        const unsigned char *Ab = reinterpret_cast<const unsigned char *>(g.At) +
                                  (size_t)blockIdx.x * nk * (2 * A_TILE);
        const unsigned char *Bb = reinterpret_cast<const unsigned char *>(g.Bt) +
                                  (size_t)blockIdx.y * nk * (2 * B_TILE);
        int kb = 0;
        for (; kb < nk; ++kb) {
            const int s = kb % STAGES;
            if (kb >= STAGES && !tc::bar_wait(&empty[s], ((kb / STAGES) - 1) & 1, g.budget_ns)) {
                abort_s = 1;
                break;
            }
            if (*(volatile int *)&abort_s) break;
            unsigned char *st = ring + (size_t)s * STAGE_BYTES;
            expect_tx(&full[s], STAGE_BYTES);
            bulk_copy(st, Ab + (size_t)kb * (2 * A_TILE), 2 * A_TILE, &full[s]);
            bulk_copy(st + 2 * A_TILE, Bb + (size_t)kb * (2 * B_TILE), 2 * B_TILE, &full[s]);
        }
        issued_s = kb;
    } else if (warp == 1 && lane == 0) {
        // MMA issuer
        const uint32_t idesc = tc::idesc_bf16(BM, BN);
        int kb = 0;
        for (; kb < nk; ++kb) {
            const int s = kb % STAGES;
            if (!tc::bar_wait(&full[s], (kb / STAGES) & 1, g.budget_ns) || *(volatile int *)&abort_s) {
                abort_s = 1;
                break;
            }
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const uint32_t st = tc::su32(ring + (size_t)s * STAGE_BYTES);
            const uint32_t ah = st, al = st + A_TILE, bh = st + 2 * A_TILE, bl = bh + B_TILE;
#pragma unroll
            for (int ks = 0; ks < BK / 16; ++ks) {
                const uint32_t koff = (uint32_t)(2 * ks) * 128u;
                const uint32_t first = (kb == 0 && ks == 0) ? 0u : 1u;
                tc::mma_bf16(tmem, tc::sdesc(ah + koff, tc::LBO, tc::SBO),
                             tc::sdesc(bh + koff, tc::LBO, tc::SBO), idesc, first);
                tc::mma_bf16(tmem, tc::sdesc(ah + koff, tc::LBO, tc::SBO),
                             tc::sdesc(bl + koff, tc::LBO, tc::SBO), idesc, 1u);
                tc::mma_bf16(tmem, tc::sdesc(al + koff, tc::LBO, tc::SBO),
                             tc::sdesc(bh + koff, tc::LBO, tc::SBO), idesc, 1u);
            }
            tc::mma_commit(&empty[s]);
        }
        tc::mma_commit(done);      // arrives once every MMA issued above has completed
    }

    // epilogue warps wait for the accumulator; everyone then meets
    bool ok = true;
    if (warp >= 2) ok = tc::bar_wait(done, 0, g.budget_ns);
    __syncthreads();
    if (!ok || abort_s) {
        // let every issued copy and MMA finish (bounded) before the memory goes away
        if (threadIdx.x == 0) {
            const int n = issued_s;
            for (int kb = (n > STAGES ? n - STAGES : 0); kb < n; ++kb)
                tc::bar_wait(&full[kb % STAGES], (kb / STAGES) & 1, g.budget_ns);
            tc::bar_wait(done, 0, g.budget_ns);
            if (g.status) atomicOr(g.status, ST_TIMEOUT);
        }
    } else if (warp >= 2) {
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        const int q = warp & 3;                    // TMEM lanes 32q .. 32q+31
        const int row = m0 + q * 32 + lane;
        for (int c0 = 0; c0 < BN; c0 += 16) {
            if (n0 + c0 >= g.N) break;
            uint32_t r[16];
            const uint32_t taddr = tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)c0;
            asm volatile(
                "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,"
                "%13,%14,%15}, [%16];"
                : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
                  "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]),
                  "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
                : "r"(taddr));
            asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
            if (row < g.M) {
                float *dst = g.C + (size_t)row * g.ldc + n0 + c0;
#pragma unroll
                for (int j = 0; j < 16; ++j) {
                    if (n0 + c0 + j >= g.N) break;
                    float v = g.alpha * __uint_as_float(r[j]);
                    if (g.beta != 0.f) v += g.beta * dst[j];
                    dst[j] = v;
                }
            }
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 1)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;"
                     ::"r"(tmem), "r"((uint32_t)BN) : "memory");
}

// Workspace of the split operands: a memory pool of the library's own per device
// that keeps what it has reserved (release threshold unbounded), so that
// repeated calls neither synchronise nor map memory again.
static cudaError_t workspace_pool(cudaMemPool_t *out)
{
    static std::mutex mu;
    static std::map<int, cudaMemPool_t> pools;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    std::lock_guard<std::mutex> lock(mu);
    auto it = pools.find(dev);
    if (it != pools.end()) {
        *out = it->second;
        return cudaSuccess;
    }
    cudaMemPoolProps props = {};
    props.allocType = cudaMemAllocationTypePinned;
    props.location.type = cudaMemLocationTypeDevice;
    props.location.id = dev;
    cudaMemPool_t pool;
    e = cudaMemPoolCreate(&pool, &props);
    if (e != cudaSuccess) return e;
    uint64_t keep = ~0ull;
    e = cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep);
    if (e != cudaSuccess) return e;
    pools[dev] = pool;
    *out = pool;
    return cudaSuccess;
}

static cudaError_t launch(int M, int N, int K, const float *A, long long lda, const float *B,
                          long long ldb, int b_trans, float *C, long long ldc, float alpha,
                          float beta, int *status, long long budget_ns, cudaStream_t s)
{
    const int mt = (M + BM - 1) / BM, nt = (N + BN - 1) / BN, nkb = (K + BK - 1) / BK;
    const size_t a_elems = (size_t)mt * nkb * 2 * BM * BK, b_elems = (size_t)nt * nkb * 2 * BN * BK;
    __nv_bfloat16 *ws = nullptr;
    cudaMemPool_t pool;
    cudaError_t e = workspace_pool(&pool);
    if (e == cudaSuccess)
        e = cudaMallocFromPoolAsync(reinterpret_cast<void **>(&ws),
                                    (a_elems + b_elems) * sizeof(__nv_bfloat16), pool, s);
    if (e != cudaSuccess) return e;
    // one thread per 8 elements of a row
    const long long at = (long long)mt * BM * nkb * (BK / 8), bt = (long long)nt * BN * nkb * (BK / 8);
    unsigned char *wa = reinterpret_cast<unsigned char *>(ws);
    unsigned char *wb = reinterpret_cast<unsigned char *>(ws + a_elems);
    tc2_split_kernel<BM><<<(int)std::min<long long>((at + 255) / 256, 148 * 16), 256, 0, s>>>(
        A, lda, 1, M, K, nkb, wa, at);
    if (b_trans)    // B(n, k) at B[k * ldb + n]
        tc2_split_kernel<BN><<<(int)std::min<long long>((bt + 255) / 256, 148 * 16), 256, 0, s>>>(
            B, 1, ldb, N, K, nkb, wb, bt);
    else
        tc2_split_kernel<BN><<<(int)std::min<long long>((bt + 255) / 256, 148 * 16), 256, 0, s>>>(
            B, ldb, 1, N, K, nkb, wb, bt);
    e = cudaGetLastError();
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(tc2_gemm_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)SMEM);
    if (e == cudaSuccess) {
        Args2 g{M, N, K, nkb, ws, ws + a_elems, C, ldc, alpha, beta, status, budget_ns};
        tc2_gemm_kernel<<<dim3(mt, nt), THREADS, SMEM, s>>>(g);
        e = cudaGetLastError();
    }
    cudaError_t f = cudaFreeAsync(ws, s);
    return e != cudaSuccess ? e : f;
}

}  // namespace tc2

// C = alpha A B' + beta C in split-bf16 x3 on tcgen05 (see the file comment).
cudaError_t launch_gemm_bf16x3(int M, int N, int K, const float *A, long long lda, long long sA,
                               const float *B, long long ldb, long long sB, int b_trans, float *C,
                               long long ldc, long long sC, float alpha, float beta, int batch,
                               const int *kdyn, int kdyn_is_n, int kthresh, int *status,
                               long long budget_ns, cudaStream_t s)
{
    tc::Args g;
    g.M = M; g.N = N; g.K = K;
    g.A = A; g.lda = lda; g.sA = sA;
    g.B = B; g.ldb = ldb; g.sB = sB; g.b_trans = b_trans;
    g.C = C; g.ldc = ldc; g.sC = sC;
    g.alpha = alpha; g.beta = beta;
    g.kdyn = kdyn; g.kdyn_is_n = kdyn_is_n; g.kthresh = kthresh;
    g.status = status; g.budget_ns = budget_ns;
    if (M <= 0 || N <= 0 || K < 0 || batch <= 0) return cudaSuccess;
    // one plain matrix: operands split once, a TMA-fed pipeline
    if (batch == 1 && !kdyn && K > 0 && N > 128)
        return tc2::launch(M, N, K, A, lda, B, ldb, b_trans, C, ldc, alpha, beta, status,
                           budget_ns, s);
    // narrow N (a short queue) takes a narrower tile
    if (N <= 64) return tc::launch_bn<64>(g, batch, s);
    if (N <= 128) return tc::launch_bn<128>(g, batch, s);
    return tc::launch_bn<256>(g, batch, s);
}

}  // namespace qmcdu
