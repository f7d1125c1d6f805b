// kernels_sweep.cu -- one Metropolis sweep per walker in a single persistent,
// cooperative kernel launch (ratio, decision, accept and flush fused).
//
// Each walker is served by a group of Gf CTAs. The first Gr of them (the ratio
// CTAs) each own a chunk of rows of the N-vectors and advance the proposals in
// lock step, exchanging tagged partial dot products (polled in global memory,
// no counter barrier) once per proposal; all Gf CTAs (ratio CTAs and
// helpers) apply the flush of Eq. 4, each to its own block of columns of
// A^{-1}. Groups never wait on one another.
//
// Delay queue, in the paper's change form (Eq. 1-4). A move of electron j to
// the new row v changes A by the rank-1 term e_j u' with u = v - a_j; the
// queue keeps the changes of the k accepted moves as the rows of V (Delta'),
// the columns P = A^{-1}[:, idx] of the inverse at the last flush and, instead
// of the k x k inverse Kinv = (I + V'P)^{-1} of Eq. 3, its product with the
// panel, W = P Kinv (N x k), which is the operand the flush needs. With
// a = A^{-1}[:, j], d = u.a, y = W'u, c = V'a the bordered-inverse algebra gives
//   r  = 1 + (d - y.c)                      (ratio of the proposal, Eq. 1/3)
//   z  = a - W c,   W <- [W - z y'/r, z/r]   (append on accept)
// so every step is an N-parallel dot product or axpy over the row chunks, with
// no k x k work on the critical path. When a ratio CTA's rows of W and V fit,
// they stay in its shared memory for the whole sweep (RES) and are written to
// global memory only for a flush.
//
// Flush (column c of the column-major A^{-1}, T = V'A^{-1}, Eq. 4):
//   t_m = V[m] . A^{-1}[:, c],   A^{-1}[:, c] -= sum_m t_m W[m].
// Four implementations, chosen per flush: flush_columns_small (k < 4, K = 1's
// Sherman-Morrison), flush_block (fp64 column blocks >= 64 wide: a
// register-tiled GEMM), flush_tc (split-bf16 walkers: tcgen05 with the
// accumulators in tensor memory), flush_columns (the rest: column tiles brought
// into shared memory by bulk asynchronous copies, completion on an mbarrier).
//
// The proposal Gaussians and Metropolis uniforms of the sweep are drawn up
// front by a fully parallel kernel (sweep_draw_kernel), and the running
// log|det A| is brought up to date after the sweep from the recorded ratios,
// so that neither costs time on the sequential chain of proposals.
//
// Every spin-wait has a time budget (globaltimer); on expiry the kernel sets
// ST_TIMEOUT in the status word and returns. Data written by other CTAs is read
// with ld.global.cg (L2, not the SM's L1).
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <math.h>

#include <algorithm>
#include <type_traits>

#include "philox.cuh"
#include "bulk.cuh"
#include "qmcdu_internal.cuh"

namespace qmcdu {

constexpr int STHREADS = 256;
constexpr int SWARPS = STHREADS / 32;
constexpr int MAX_CB = 8;
constexpr int SYNC_STRIDE = 96;   // unsigned words per walker group: three 128-byte lines
// flush implementations of a sweep kernel instance
constexpr int FM_SIMT = 0;   // flush_columns_small / flush_block / flush_columns
constexpr int FM_TC = 1;     // flush_tc (split-bf16 walkers)
constexpr int FM_OZ = 2;     // flush_oz (fp64 walkers, emulated on the tensor cores)

template <typename T>
struct SweepParams {
    int N, K, ld, batch;
    int Gf, Gr, ngroups, chunk, cb;
    double *A;
    T *Ainv, *W, *V;
    int *idx, *kglob;
    const double *gauss;    // [batch][N][ld] proposal Gaussians of this sweep
    const double *unif;     // [batch][N] Metropolis uniforms of this sweep
    double *partial;        // [ngroups][2][Gr][2K+2] tagged (hi, lo) words (slot 2K+1: row padding)
    unsigned *sync;         // [ngroups][SYNC_STRIDE]: a spare line (the proposals exchange tagged
                            // partials instead of a barrier), the flush barrier and the flush
                            // command, each on its own 128-byte line
    int *status;
    double sigma;
    const signed char *override_;
    unsigned char *acc_out;
    double *ratio_out;
    long long *ties;
    long long budget_ns;    // per wait
    int stall;              // test hook: the first ratio barrier waits for one CTA too many
    int off_vs, off_as, off_vd, off_red, off_ts, off_xs, off_wsm, off_vsm, off_bar;
    int kp;                         // tensor-core flush: K rounded up to 16 (<= 64)
    int block_ok;                   // the xs region holds flush_block's tiles
    unsigned long long *phase_ns;   // optional [11]: time per phase, group 0 rank 0 thread 0
    const int *wlist;               // optional [nw]: the walkers this launch sweeps (else 0..nw)
    int nw;
    unsigned char *oz;              // emulated-fp64 flush: per-group scratch (ozf::layout)
    size_t oz_stride;               // bytes per walker group
    int off_tcbar;                  // the tensor-core flush's mbarriers (offset in shared memory)
    int off_cl;                     // cluster mode: [2][2K+1] partial dot products, then a flag
    int fixed_slot;                 // rejected proposals take queue slots (zero changes)
};

__device__ __forceinline__ unsigned ld_acquire(const unsigned *p)
{
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}



// Arrival on a group counter (after all of this CTA's prior writes): the CTA
// barrier orders every thread's writes before thread 0's release-add, whose
// release semantics (cumulative) publish them at gpu scope.
__device__ __forceinline__ void group_arrive(unsigned *ctr)
{
    __syncthreads();
    if (threadIdx.x == 0)
        asm volatile("red.release.gpu.global.add.u32 [%0], 1;" ::"l"(ctr) : "memory");
}

// Wait until a group counter reaches `target`. Returns false, uniformly for
// the CTA, when the budget runs out or another CTA has reported a timeout.
__device__ bool group_wait_for(unsigned *ctr, unsigned target, int *status, long long budget_ns,
                               unsigned backoff_ns = 0)
{
    __shared__ int ok_s;
    __syncthreads();
    if (threadIdx.x == 0) {
        int ok = 1;
        const unsigned long long t0 = globaltimer();
        unsigned spins = 0;
        while (ld_acquire(ctr) < target) {
            if (backoff_ns) __nanosleep(backoff_ns);
            if ((++spins & 63u) == 0) {
                if ((long long)(globaltimer() - t0) > budget_ns) {
                    atomicOr(status, ST_TIMEOUT);
                    ok = 0;
                    break;
                }
                if (*(volatile const int *)status & ST_TIMEOUT) {
                    ok = 0;
                    break;
                }
            }
        }
        // (the acquire load orders the CTA's later reads, through the barrier below)
        ok_s = ok;
    }
    __syncthreads();
    return ok_s != 0;
}

__device__ __forceinline__ bool group_barrier(unsigned *ctr, unsigned target, int *status,
                                              long long budget_ns)
{
    group_arrive(ctr);
    return group_wait_for(ctr, target, status, budget_ns);
}

// ---- distributed shared memory of a thread-block cluster (cluster mode: the
// ratio CTAs of a walker form one cluster and exchange their partial dot
// products through each other's shared memory)
__device__ __forceinline__ uint32_t cl_map(const void *local, int rank)
{
    uint32_t r;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;"
                 : "=r"(r) : "r"((uint32_t)__cvta_generic_to_shared(local)), "r"(rank));
    return r;
}
__device__ __forceinline__ unsigned cl_ld_acquire(uint32_t addr)
{
    unsigned v;
    asm volatile("ld.acquire.cluster.shared::cluster.u32 %0, [%1];" : "=r"(v) : "r"(addr) : "memory");
    return v;
}
__device__ __forceinline__ double cl_ld_f64(uint32_t addr)
{
    double v;
    asm volatile("ld.shared::cluster.f64 %0, [%1];" : "=d"(v) : "r"(addr) : "memory");
    return v;
}
__device__ __forceinline__ void cl_st_release(unsigned *local, unsigned v)
{
    asm volatile("st.release.cluster.shared::cta.u32 [%0], %1;"
                 ::"r"((uint32_t)__cvta_generic_to_shared(local)), "r"(v) : "memory");
}
__device__ __forceinline__ void cl_barrier()
{
    asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}
// Wait until the flags of cluster ranks 0 .. n - 1 reach `target` (threads
// 0 .. n - 1 poll one each), with a time budget; uniform result for the CTA.
__device__ bool cl_wait_flags(const unsigned *flag, unsigned target, int n, int *status,
                              long long budget_ns)
{
    bool ok = true;
    if ((int)threadIdx.x < n) {
        const uint32_t a = cl_map(flag, threadIdx.x);
        const unsigned long long t0 = globaltimer();
        unsigned spins = 0;
        while (cl_ld_acquire(a) < target) {
            if ((++spins & 63u) == 0 && (long long)(globaltimer() - t0) > budget_ns) {
                atomicOr(status, ST_TIMEOUT);
                ok = false;
                break;
            }
        }
    }
    return __syncthreads_and(ok) != 0;
}

__device__ __forceinline__ float2 cl_ld_f2(uint32_t addr)
{
    float2 v;
    asm volatile("ld.shared::cluster.v2.f32 {%0, %1}, [%2];" : "=f"(v.x), "=f"(v.y) : "r"(addr) : "memory");
    return v;
}
// ---- double-fp32 pairs (hi + lo): the ratio CTAs each sum all Gr x (2k + 1)
// partial dot products of a proposal. B300's fp64 pipe retires two lanes per
// clock per SM (a warp-wide fp64 add costs 16 cycles), so those sums run on
// the fp32 pipe as error-free two-sums (Knuth's TwoSum) on (hi, lo) pairs:
// about 48 bits, far below the path's other errors.
__device__ __forceinline__ float2 df_split(double x)
{
    const float hi = __double2float_rn(x);
    return make_float2(hi, __double2float_rn(x - (double)hi));
}
__device__ __forceinline__ float2 df_add(float2 a, float2 b)
{
    const float s = __fadd_rn(a.x, b.x);
    const float bb = __fsub_rn(s, a.x);
    const float e = __fadd_rn(__fsub_rn(a.x, __fsub_rn(s, bb)), __fsub_rn(b.x, bb));
    return make_float2(s, __fadd_rn(__fadd_rn(a.y, b.y), e));
}

// ---- tagged partials: a (hi, lo) pair travels as one 64-bit word, the two
// lowest bits of lo replaced by the proposal's tag (1 + p mod 3, p the
// group's count of proposals in this launch; 0 after the clearing memset that
// precedes every launch). One single-copy-atomic 64-bit store publishes the
// value and its readiness together, so the readers poll the data itself: no
// CTA barrier, release fence or counter round trip per proposal. Proposal p
// reads the slots of its 2k + 1 dot products in buffer p & 1 (by the launch's
// proposal count, not the walker's electron index: walkers of odd N follow
// one another in a launch); k grows by at most one per proposal, so besides
// its own slots every proposal tags the next four (zero values) in its
// buffer: then every slot that proposal p reads was last written by p - 2,
// and three tags tell the current value from every stale one. The two bits
// cost under 4 ulp of lo (about 2^-45 of the value).
__device__ __forceinline__ void st_tagged(double *dst, float2 v, unsigned tag)
{
    const unsigned lo = (__float_as_uint(v.y) & ~3u) | tag;
    const unsigned long long w = ((unsigned long long)lo << 32) | __float_as_uint(v.x);
    asm volatile("st.relaxed.gpu.global.b64 [%0], %1;" ::"l"(dst), "l"(w) : "memory");
}
__device__ __forceinline__ unsigned long long ld_tagged(const double *src)
{
    unsigned long long w;
    asm volatile("ld.relaxed.gpu.global.b64 %0, [%1];" : "=l"(w) : "l"(src));
    return w;
}
__device__ __forceinline__ unsigned tag_of(unsigned long long w) { return (unsigned)(w >> 32) & 3u; }
// 16 bytes global -> shared, asynchronous, through L2 only (no stale L1 line
// can answer a repeated copy of a polled word)
__device__ __forceinline__ void cp_async16(void *dst_smem, const void *src)
{
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;"
                 ::"r"((uint32_t)__cvta_generic_to_shared(dst_smem)), "l"(src) : "memory");
}
__device__ __forceinline__ float2 untag(unsigned long long w)
{
    return make_float2(__uint_as_float((unsigned)w), __uint_as_float((unsigned)(w >> 32) & ~3u));
}

// Lanes of this warp that take part in a loop iteration over t < n, where t
// runs lane by lane (t = base + lane, base a multiple of 32). The shuffles
// after a loop name these lanes explicitly: lanes that left a data-dependent
// loop (the polls of tagged partials) at different times need not have
// reconverged, so __activemask() could miss some of them.
__device__ __forceinline__ unsigned lanes_below(int t, int n)
{
    const int rem = n - (t - (int)(threadIdx.x & 31));
    return rem >= 32 ? 0xffffffffu : (rem <= 0 ? 0u : (1u << rem) - 1u);
}

template <typename T>
__device__ __forceinline__ T warp_allsum(T v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Flush for a short queue (k < SMALL_K, including Sherman-Morrison at K = 1).
// The CTA takes its columns in batches of SCB: every thread walks rows
// i = tid, tid + STHREADS, ... of all the batch's columns, so that each V and W
// element is read once per batch and the reads of the batch's columns are in
// flight together; the column sums are reduced over the warps in shared
// memory, then every thread updates its rows of the batch's columns.
constexpr int SMALL_K = 4;
constexpr int SCB = 8;

template <typename T, int KK>
__device__ void flush_columns_small_k(const SweepParams<T> &p, int w, int c_begin, int c_end)
{
    const int N = p.N, ld = p.ld, K = p.K;
    const size_t wN = (size_t)N * ld, wK = (size_t)K * ld;
    T *Ab = p.Ainv + (size_t)w * wN;
    const T *Vb = p.V + (size_t)w * wK;
    const T *Wb = p.W + (size_t)w * wK;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    __shared__ T part[SWARPS][SCB * SMALL_K];
    __shared__ T tsum[SCB * SMALL_K];
    for (int cb = c_begin; cb < c_end; cb += SCB) {
        const int nc = min(SCB, c_end - cb);
        T t[SCB][KK];
#pragma unroll
        for (int c = 0; c < SCB; ++c)
#pragma unroll
            for (int m = 0; m < KK; ++m) t[c][m] = 0;
#pragma unroll 2
        for (int i = threadIdx.x; i < N; i += STHREADS) {
            T vv[KK];
#pragma unroll
            for (int m = 0; m < KK; ++m) vv[m] = __ldcg(Vb + (size_t)m * ld + i);
#pragma unroll
            for (int c = 0; c < SCB; ++c) {
                if (c < nc) {
                    const T x = __ldcg(Ab + (size_t)(cb + c) * ld + i);
#pragma unroll
                    for (int m = 0; m < KK; ++m) t[c][m] += vv[m] * x;
                }
            }
        }
#pragma unroll
        for (int c = 0; c < SCB; ++c)
#pragma unroll
            for (int m = 0; m < KK; ++m)
                if (c < nc) {
                    const T v = warp_allsum(t[c][m]);
                    if (lane == 0) part[warp][c * SMALL_K + m] = v;
                }
        __syncthreads();
        if (threadIdx.x < SCB * SMALL_K) {
            const int c = threadIdx.x / SMALL_K, m = threadIdx.x - c * SMALL_K;
            T sum = 0;
            if (c < nc && m < KK) {
#pragma unroll
                for (int q = 0; q < SWARPS; ++q) sum += part[q][threadIdx.x];
            }
            tsum[threadIdx.x] = sum;
        }
        __syncthreads();
#pragma unroll 2
        for (int i = threadIdx.x; i < N; i += STHREADS) {
            T ww[KK];
#pragma unroll
            for (int m = 0; m < KK; ++m) ww[m] = __ldcg(Wb + (size_t)m * ld + i);
#pragma unroll
            for (int c = 0; c < SCB; ++c) {
                if (c < nc) {
                    T acc = 0;
#pragma unroll
                    for (int m = 0; m < KK; ++m) acc += ww[m] * tsum[c * SMALL_K + m];
                    T *xc = Ab + (size_t)(cb + c) * ld + i;
                    *xc = __ldcg(xc) - acc;
                }
            }
        }
        __syncthreads();
    }
}

// k = 1, 2 or 3 queued moves: the arithmetic for exactly k terms
template <typename T>
__device__ void flush_columns_small(const SweepParams<T> &p, int w, int k, int c_begin, int c_end)
{
    if (k == 1) flush_columns_small_k<T, 1>(p, w, c_begin, c_end);
    else if (k == 2) flush_columns_small_k<T, 2>(p, w, c_begin, c_end);
    else flush_columns_small_k<T, 3>(p, w, c_begin, c_end);
}
// The same, out of line: the emulated-fp64 sweep calls it only for a queue
// shorter than SMALL_K (end of a sweep), and inlined there its registers would
// press on the proposal chain's, which already fills 255
template <typename T>
__device__ __noinline__ void flush_columns_small_ool(const SweepParams<T> &p, int w, int k, int c_begin, int c_end)
{
    flush_columns_small(p, w, k, c_begin, c_end);
}

// Flush of walker w on a wide column block [c_begin, c_end) (fp64, K <= 64): a
// register-tiled GEMM in two phases per tile of BT = 64 columns, so that the
// queue panels V and W are read once per 64 columns (not once per few columns).
//   T' = V A^{-1}[:, tile]: rows i in chunks of BI1 = 32, V^t and the tile's rows
//        staged in shared memory (row stride BT + 1: the transposing stores hit
//        distinct banks), each thread a 4 x 4 block of (m, c);
//   T  = T' kept in shared memory;
//   A^{-1}[:, tile] -= W^t T: rows i in chunks of BI2 = 64, W staged, each thread
//        a 4 x 4 block of (i, c) with the lanes along i, so that a half-warp's
//        read-modify-write of a column is 64 consecutive rows.
// Shared memory: 2 * 64 * 64 elements of T at off_xs.
constexpr int BT = 64, BI1 = 32, BI2 = 64, SLD = BT + 1;

template <typename T>
__device__ void flush_block(const SweepParams<T> &p, int w, int k, int c_begin, int c_end,
                            unsigned char *smem)
{
    const int N = p.N, ld = p.ld, K = p.K;
    const size_t wN = (size_t)N * ld, wK = (size_t)K * ld;
    T *Ab = p.Ainv + (size_t)w * wN;
    const T *Vb = p.V + (size_t)w * wK;
    const T *Wb = p.W + (size_t)w * wK;
    T *Vs = (T *)(smem + p.off_xs);        // [BI1][SLD] : V^t chunk, Vs[ci][m]
    T *As = Vs + BI1 * SLD;                // [BI1][SLD] : A^{-1} chunk, As[ci][c]
    T *Ts = Vs;                            // [BT][BT]   : T[m][c] (after phase 1)
    T *Ws = Vs + BT * BT;                  // [BT][BI2]  : W chunk, Ws[m][ii]
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;   // 16 x 16 threads
    for (int c0 = c_begin; c0 < c_end; c0 += BT) {
        const int nc = min(BT, c_end - c0);
        T acc[4][4];
#pragma unroll
        for (int a = 0; a < 4; ++a)
#pragma unroll
            for (int b = 0; b < 4; ++b) acc[a][b] = 0;
        // ---- phase 1: T'[m][c] = sum_i V[m][i] A^{-1}[i][c0 + c]   (m = ty*4+u, c = tx*4+v)
        for (int i0 = 0; i0 < N; i0 += BI1) {
            __syncthreads();
            // stage: consecutive threads take consecutive i of one row / column
            for (int e = threadIdx.x; e < BT * BI1; e += STHREADS) {
                const int r = e / BI1, ci = e - r * BI1, i = i0 + ci;
                Vs[ci * SLD + r] = (r < k && i < N) ? __ldcg(Vb + (size_t)r * ld + i) : (T)0;
                As[ci * SLD + r] = (r < nc && i < N) ? __ldcg(Ab + (size_t)(c0 + r) * ld + i) : (T)0;
            }
            __syncthreads();
#pragma unroll 8
            for (int ci = 0; ci < BI1; ++ci) {
                T a[4], b[4];
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    a[q] = Vs[ci * SLD + ty * 4 + q];
                    b[q] = As[ci * SLD + tx * 4 + q];
                }
#pragma unroll
                for (int u = 0; u < 4; ++u)
#pragma unroll
                    for (int v = 0; v < 4; ++v) acc[u][v] += a[u] * b[v];
            }
        }
        __syncthreads();
        // ---- T = Delta' A^{-1} into shared memory
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int m = ty * 4 + u;
#pragma unroll
            for (int v = 0; v < 4; ++v) {
                const int c = tx * 4 + v;
                Ts[m * BT + c] = (m < k && c < nc) ? acc[u][v] : (T)0;
            }
        }
        // ---- phase 2: A^{-1}[i][c0 + c] -= sum_m W[m][i] T[m][c]   (i = tx*4+u, c = ty*4+v)
        for (int i0 = 0; i0 < N; i0 += BI2) {
            __syncthreads();
            for (int e = threadIdx.x; e < BT * BI2; e += STHREADS) {
                const int m = e / BI2, ii = e - m * BI2, i = i0 + ii;
                Ws[m * BI2 + ii] = (m < k && i < N) ? __ldcg(Wb + (size_t)m * ld + i) : (T)0;
            }
            __syncthreads();
#pragma unroll
            for (int u = 0; u < 4; ++u)
#pragma unroll
                for (int v = 0; v < 4; ++v) acc[u][v] = 0;
            for (int m = 0; m < k; ++m) {
                T a[4], b[4];
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    a[q] = Ws[m * BI2 + tx * 4 + q];
                    b[q] = Ts[m * BT + ty * 4 + q];
                }
#pragma unroll
                for (int u = 0; u < 4; ++u)
#pragma unroll
                    for (int v = 0; v < 4; ++v) acc[u][v] += a[u] * b[v];
            }
#pragma unroll
            for (int v = 0; v < 4; ++v) {
                const int c = ty * 4 + v;
                if (c >= nc) continue;
                T *col = Ab + (size_t)(c0 + c) * ld + i0 + tx * 4;
#pragma unroll
                for (int u = 0; u < 4; ++u)
                    if (i0 + tx * 4 + u < N) col[u] = __ldcg(col + u) - acc[u][v];
            }
        }
    }
    __syncthreads();
}

// Flush of walker w on columns [c_begin, c_end): tiles of nc <= cb columns.
// Each column is one bulk copy of ld elements (ld is a multiple of 16, so
// every copy is 16-byte aligned and a multiple of 16 bytes long).
template <typename T>
__device__ bool flush_columns(const SweepParams<T> &p, int w, int k, int c_begin, int c_end,
                              unsigned char *smem, unsigned &bar_phase)
{
    const int N = p.N, ld = p.ld, K = p.K, cb = p.cb;
    T *xs = (T *)(smem + p.off_xs);
    T *ts = (T *)(smem + p.off_ts);
    unsigned long long *bar = (unsigned long long *)(smem + p.off_bar);
    __shared__ int ok_s;
    const size_t wN = (size_t)N * ld, wK = (size_t)K * ld;
    T *Ab = p.Ainv + (size_t)w * wN;
    const T *Vb = p.V + (size_t)w * wK;
    const T *Wb = p.W + (size_t)w * wK;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int c0 = c_begin; c0 < c_end; c0 += cb) {
        const int nc = min(cb, c_end - c0);
        __syncthreads();
        if (threadIdx.x == 0) {
            asm volatile("fence.proxy.async;" ::: "memory");
            const unsigned bytes = (unsigned)(ld * sizeof(T));
            mbar_expect(bar, bytes * nc);
            for (int cc = 0; cc < nc; ++cc)
                bulk_g2s(xs + (size_t)cc * ld, Ab + (size_t)(c0 + cc) * ld, bytes, bar);
            ok_s = mbar_wait(bar, bar_phase, p.status, p.budget_ns) ? 1 : 0;
        }
        bar_phase ^= 1u;
        __syncthreads();
        if (!ok_s) return false;
        // T tile: t[m][cc] = V[m] . A^{-1}[:, c0 + cc] - [idx_m == c0 + cc], four rows per warp
        for (int mb = warp * 4; mb < k; mb += SWARPS * 4) {
            T acc[4][MAX_CB];
#pragma unroll
            for (int r = 0; r < 4; ++r)
#pragma unroll
                for (int cc = 0; cc < MAX_CB; ++cc) acc[r][cc] = 0;
            const T *v0 = Vb + (size_t)mb * ld;
            if (mb + 4 <= k) {
#pragma unroll 2
                for (int i = lane; i < N; i += 32) {
                    T vv[4];
#pragma unroll
                    for (int r = 0; r < 4; ++r) vv[r] = __ldcg(v0 + (size_t)r * ld + i);
#pragma unroll
                    for (int cc = 0; cc < MAX_CB; ++cc) {
                        if (cc < nc) {
                            const T x = xs[(size_t)cc * ld + i];
#pragma unroll
                            for (int r = 0; r < 4; ++r) acc[r][cc] += vv[r] * x;
                        }
                    }
                }
            } else {
                // tail rows one at a time (compile-time indices only)
#pragma unroll
                for (int r = 0; r < 3; ++r) {
                    if (mb + r < k) {
                        for (int i = lane; i < N; i += 32) {
                            const T vv = __ldcg(v0 + (size_t)r * ld + i);
#pragma unroll
                            for (int cc = 0; cc < MAX_CB; ++cc)
                                if (cc < nc) acc[r][cc] += vv * xs[(size_t)cc * ld + i];
                        }
                    }
                }
            }
#pragma unroll
            for (int r = 0; r < 4; ++r) {
                const int m = mb + r;
#pragma unroll
                for (int cc = 0; cc < MAX_CB; ++cc) {
                    const T v = warp_allsum(acc[r][cc]);
                    if (lane == 0 && cc < nc && m < k) ts[m * cb + cc] = v;
                }
            }
        }
        __syncthreads();
        // update: A^{-1}[:, c0 + cc] -= sum_m t[m][cc] W[m], two rows per thread
        for (int i = threadIdx.x; i < N; i += 2 * STHREADS) {
            const int i2 = i + STHREADS;
            const bool two = i2 < N;
            T a0[MAX_CB], a1[MAX_CB];
#pragma unroll
            for (int cc = 0; cc < MAX_CB; ++cc) a0[cc] = a1[cc] = 0;
#pragma unroll 2
            for (int m = 0; m < k; ++m) {
                const T w0 = __ldcg(Wb + (size_t)m * ld + i);
                const T w1 = two ? __ldcg(Wb + (size_t)m * ld + i2) : (T)0;
#pragma unroll
                for (int cc = 0; cc < MAX_CB; ++cc) {
                    if (cc < nc) {
                        const T t = ts[m * cb + cc];
                        a0[cc] += t * w0;
                        a1[cc] += t * w1;
                    }
                }
            }
#pragma unroll
            for (int cc = 0; cc < MAX_CB; ++cc) {
                if (cc < nc) {
                    Ab[(size_t)(c0 + cc) * ld + i] = xs[(size_t)cc * ld + i] - a0[cc];
                    if (two) Ab[(size_t)(c0 + cc) * ld + i2] = xs[(size_t)cc * ld + i2] - a1[cc];
                }
            }
        }
    }
    __syncthreads();
    return true;
}


// ---------------------------------------------------------------------------
// Tensor-core flush (fp32 working precision, split-bf16 x3 on tcgen05), for
// flush CTAs that own at least 128 columns of A^{-1}. Per tile of 128 columns
// (rows of the column-major storage):
//   T' (128 x k) = X V'          K = N, staged 32 at a time, double buffered
//   X (128 x N) -= T' W           K = k, 128 columns of X at a time
// with x = hi + lo, hi = bf16(x), lo = bf16(x - hi), and hi*hi + hi*lo + lo*hi
// accumulated in fp32 tensor memory (columns [0, 128) hold T', [128, 256) the
// update). Operands are written by the CTA's threads as K-major 8 x 8 bf16
// core matrices (no swizzle), which the shared-memory descriptors describe.
namespace tcf {
constexpr int BM = 128, BK = 32;
__device__ __forceinline__ uint32_t su32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }
__device__ __forceinline__ uint64_t sdesc(uint32_t saddr, uint32_t lbo, uint32_t sbo)
{
    return (uint64_t)((saddr >> 4) & 0x3FFFu) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) |
           ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | (1ull << 46);
}
__device__ __forceinline__ uint32_t idesc(int M, int N)
{
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}
// byte offset of (row r, column k) in a K-major tile of `kc` columns
__device__ __forceinline__ uint32_t coff(int r, int k, int kc)
{
    return (uint32_t)((((r >> 3) * (kc >> 3) + (k >> 3)) << 7) + ((r & 7) << 4) + ((k & 7) << 1));
}
__device__ __forceinline__ void mma(uint32_t d, uint64_t a, uint64_t b, uint32_t id, uint32_t acc)
{
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n"
        ::"r"(d), "l"(a), "l"(b), "r"(id), "r"(acc) : "memory");
}
__device__ __forceinline__ void commit(unsigned long long *bar)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];"
                 ::"r"(su32(bar)) : "memory");
}
__device__ __forceinline__ void ld16(uint32_t taddr, uint32_t *r)
{
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15},"
        " [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]),
          "=r"(r[15])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}
// the same load without the wait: several loads in flight, then tmem_wait_ld()
__device__ __forceinline__ void ld16_nw(uint32_t taddr, uint32_t *r)
{
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15},"
        " [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]),
          "=r"(r[15])
        : "r"(taddr));
}
__device__ __forceinline__ void tmem_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }
// shared-memory region of the tensor-core flush, for kp = K rounded up to 16:
// two stages of the T' operands (A^{-1} and V blocks), T as the update's B
// operand, two stages of the update's W block, four mbarriers
__host__ __device__ inline size_t region_bytes(int kp)
{
    return (size_t)2 * 2 * BM * BK * 2 + (size_t)2 * 2 * kp * BK * 2 + (size_t)2 * BM * kp * 2 +
           (size_t)2 * 2 * BM * kp * 2 + 4 * sizeof(unsigned long long);
}
// eight floats as bf16 hi and lo, packed for one 16-byte store per plane
__device__ __forceinline__ void split8(const float *x, uint4 &hi, uint4 &lo)
{
    uint32_t h[4], l[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        const __nv_bfloat16 h0 = __float2bfloat16_rn(x[2 * j]), h1 = __float2bfloat16_rn(x[2 * j + 1]);
        const __nv_bfloat16 l0 = __float2bfloat16_rn(x[2 * j] - __bfloat162float(h0));
        const __nv_bfloat16 l1 = __float2bfloat16_rn(x[2 * j + 1] - __bfloat162float(h1));
        h[j] = (uint32_t)__bfloat16_as_ushort(h0) | ((uint32_t)__bfloat16_as_ushort(h1) << 16);
        l[j] = (uint32_t)__bfloat16_as_ushort(l0) | ((uint32_t)__bfloat16_as_ushort(l1) << 16);
    }
    hi = make_uint4(h[0], h[1], h[2], h[3]);
    lo = make_uint4(l[0], l[1], l[2], l[3]);
}
}  // namespace tcf

// Eq. 4 on the tensor cores for walker w's columns [c_begin, c_end), tiles of
// BM = 128 columns (split-bf16 x3, fp32 accumulators in tensor memory):
//   T'[c][m] = sum_i A^{-1}[i][c] V[m][i]   M = 128 columns, N = kp, K = N in
//       blocks of 32; the CTA splits the next block's operands (eight elements per
//       thread, 16-byte stores) while the MMAs of the current one run;
//   T = T', read back from tensor memory into the B operand of
//   D[i][c] = sum_m W[m][i] T[m][c]        M = 128 rows i, N = 128 columns, K = kp;
//       the W block of the next 128 rows is split while the MMAs run, and with
//       the rows of A^{-1} along the tensor-memory lanes the read-modify-write
//       A^{-1}[c][i] -= D[i][c] is coalesced across each warp.
// Returns false after a wait ran out of budget (ST_TIMEOUT recorded).
template <typename T>
__device__ bool flush_tc(const SweepParams<T> &p, int w, int k, int c_begin, int c_end,
                         unsigned char *smem, uint32_t tmem, unsigned *tph)
{
    using namespace tcf;
    const int N = p.N, ld = p.ld, K = p.K, KP = p.kp;
    unsigned char *reg = smem + p.off_xs;
    __nv_bfloat16 *a1h = (__nv_bfloat16 *)reg;                    // [2][BM*BK]  A^{-1} block
    __nv_bfloat16 *a1l = a1h + 2 * BM * BK;
    __nv_bfloat16 *b1h = a1l + 2 * BM * BK;                      // [2][KP*BK]  V block
    __nv_bfloat16 *b1l = b1h + 2 * KP * BK;
    __nv_bfloat16 *tbh = b1l + 2 * KP * BK;                      // [BM*KP]     T (rows c)
    __nv_bfloat16 *tbl = tbh + BM * KP;
    __nv_bfloat16 *wah = tbl + BM * KP;                          // [2][BM*KP]  W block (rows i)
    __nv_bfloat16 *wal = wah + 2 * BM * KP;
    unsigned long long *bars = (unsigned long long *)(wal + 2 * BM * KP);
    __shared__ int ok_s;
    const size_t wN = (size_t)N * ld, wK = (size_t)K * ld;
    T *Ab = p.Ainv + (size_t)w * wN;
    const T *Vb = p.V + (size_t)w * wK;
    const T *Wb = p.W + (size_t)w * wK;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int kp = (k + 15) / 16 * 16;
    const uint32_t id1 = idesc(BM, kp), id2 = idesc(BM, BM);
    const int nk = (N + BK - 1) / BK;
    const uint32_t sbo2 = (uint32_t)(KP / 8) * 128u;

    // staging of T' block kb: thread t covers 8 consecutive i of A^{-1} column
    // (t / 4 + 64 h) and of V row t / 4 (t % 4 selects the 8-element part)
    auto load1 = [&](int kb, float (&xa)[2][8], float (&xv)[8], int c0, int nrows) {
        const int i = kb * BK + (threadIdx.x & 3) * 8;
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int c = (threadIdx.x >> 2) + 64 * h;
            const bool in = c < nrows && i < ld;     // rows past N are zero padding
            const float4 *src = reinterpret_cast<const float4 *>(Ab + (size_t)(c0 + c) * ld + i);
            const float4 u = in ? __ldcg(src) : make_float4(0.f, 0.f, 0.f, 0.f);
            const float4 v = in ? __ldcg(src + 1) : make_float4(0.f, 0.f, 0.f, 0.f);
            xa[h][0] = u.x; xa[h][1] = u.y; xa[h][2] = u.z; xa[h][3] = u.w;
            xa[h][4] = v.x; xa[h][5] = v.y; xa[h][6] = v.z; xa[h][7] = v.w;
        }
        const int m = threadIdx.x >> 2;
        const bool in = m < k && i < ld;
        const float4 *src = reinterpret_cast<const float4 *>(Vb + (size_t)m * ld + i);
        const float4 u = in ? __ldcg(src) : make_float4(0.f, 0.f, 0.f, 0.f);
        const float4 v = in ? __ldcg(src + 1) : make_float4(0.f, 0.f, 0.f, 0.f);
        xv[0] = u.x; xv[1] = u.y; xv[2] = u.z; xv[3] = u.w;
        xv[4] = v.x; xv[5] = v.y; xv[6] = v.z; xv[7] = v.w;
    };
    auto store1 = [&](int s, const float (&xa)[2][8], const float (&xv)[8]) {
        const int kk = (threadIdx.x & 3) * 8;
        uint4 hi, lo;
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int c = (threadIdx.x >> 2) + 64 * h;
            split8(xa[h], hi, lo);
            const uint32_t o = coff(c, kk, BK) >> 1;
            *reinterpret_cast<uint4 *>(a1h + s * BM * BK + o) = hi;
            *reinterpret_cast<uint4 *>(a1l + s * BM * BK + o) = lo;
        }
        const int m = threadIdx.x >> 2;
        if (m < KP) {
            split8(xv, hi, lo);
            const uint32_t o = coff(m, kk, BK) >> 1;
            *reinterpret_cast<uint4 *>(b1h + s * KP * BK + o) = hi;
            *reinterpret_cast<uint4 *>(b1l + s * KP * BK + o) = lo;
        }
    };
    // staging of the update's W block (rows i0.., all m): thread t covers 4
    // consecutive i (t % 32) and 8 consecutive m (t / 32), transposed in registers
    auto stage2 = [&](int i0, int s) {
        const int ig = (threadIdx.x & 31) * 4, mg = (threadIdx.x >> 5) * 8;
        if (mg >= KP) return;
        float x[4][8];
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            const int m = mg + j, i = i0 + ig;
            const bool in = m < k && i < ld;
            const float4 u = in ? __ldcg(reinterpret_cast<const float4 *>(Wb + (size_t)m * ld + i))
                                : make_float4(0.f, 0.f, 0.f, 0.f);
            x[0][j] = u.x; x[1][j] = u.y; x[2][j] = u.z; x[3][j] = u.w;
        }
        uint4 hi, lo;
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            split8(x[q], hi, lo);
            const uint32_t o = coff(ig + q, mg, KP) >> 1;
            *reinterpret_cast<uint4 *>(wah + s * BM * KP + o) = hi;
            *reinterpret_cast<uint4 *>(wal + s * BM * KP + o) = lo;
        }
    };
    auto wait_bar = [&](int b) -> bool {
        if (threadIdx.x == 0) ok_s = mbar_wait(&bars[b], tph[b], p.status, p.budget_ns) ? 1 : 0;
        __syncthreads();
        tph[b] ^= 1u;
        return ok_s != 0;
    };

    for (int c0 = c_begin; c0 < c_end; c0 += BM) {
        const int nrows = min(BM, c_end - c0);
        // ---- T' = X V' over K = N
        int pend[2] = {0, 0};
        float xa[2][8], xv[8];
        load1(0, xa, xv, c0, nrows);
        for (int kb = 0; kb < nk; ++kb) {
            const int s = kb & 1;
            if (pend[s]) {
                if (!wait_bar(s)) return false;
                pend[s] = 0;
            }
            store1(s, xa, xv);
            if (kb + 1 < nk) load1(kb + 1, xa, xv, c0, nrows);    // in flight during the MMAs
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            __syncthreads();
            if (threadIdx.x == 0) {
                asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
#pragma unroll
                for (int ks = 0; ks < BK / 16; ++ks) {
                    const uint32_t ko = (uint32_t)ks * 256u;
                    const uint64_t ah = sdesc(su32(a1h + s * BM * BK) + ko, 128, 512);
                    const uint64_t al = sdesc(su32(a1l + s * BM * BK) + ko, 128, 512);
                    const uint64_t bh = sdesc(su32(b1h + s * KP * BK) + ko, 128, 512);
                    const uint64_t bl = sdesc(su32(b1l + s * KP * BK) + ko, 128, 512);
                    mma(tmem, ah, bh, id1, (kb == 0 && ks == 0) ? 0u : 1u);
                    mma(tmem, ah, bl, id1, 1u);
                    mma(tmem, al, bh, id1, 1u);
                }
                commit(&bars[s]);
            }
            pend[s] = 1;
        }
        for (int s = 0; s < 2; ++s)
            if (pend[s] && !wait_bar(s)) return false;
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        // ---- T = T' into shared memory (rows c, K = m): the update's B operand
        if (warp < 4) {
            const int c = warp * 32 + lane;
            for (int m0 = 0; m0 < kp; m0 += 16) {
                uint32_t v[16];
                ld16(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)m0, v);
#pragma unroll
                for (int half = 0; half < 2; ++half) {
                    float t[8];
#pragma unroll
                    for (int j = 0; j < 8; ++j) {
                        const int m = m0 + half * 8 + j;
                        t[j] = m < k ? __uint_as_float(v[half * 8 + j]) : 0.f;
                    }
                    uint4 hi, lo;
                    split8(t, hi, lo);
                    const uint32_t o = coff(c, m0 + half * 8, KP) >> 1;
                    *reinterpret_cast<uint4 *>(tbh + o) = hi;
                    *reinterpret_cast<uint4 *>(tbl + o) = lo;
                }
            }
        }
        stage2(0, 0);
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        __syncthreads();
        // ---- X[c][i] -= sum_m W[m][i] T[m][c], 128 rows i at a time
        const int nblk = (N + BM - 1) / BM;
        for (int b = 0; b < nblk; ++b) {
            const int i0 = b * BM, s = b & 1;
            if (threadIdx.x == 0) {
                asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                for (int ks = 0; ks < kp / 16; ++ks) {
                    const uint32_t ko = (uint32_t)ks * 256u;
                    const uint64_t ah = sdesc(su32(wah + s * BM * KP) + ko, 128, sbo2);
                    const uint64_t al = sdesc(su32(wal + s * BM * KP) + ko, 128, sbo2);
                    const uint64_t bh = sdesc(su32(tbh) + ko, 128, sbo2);
                    const uint64_t bl = sdesc(su32(tbl) + ko, 128, sbo2);
                    mma(tmem + 128u, ah, bh, id2, ks == 0 ? 0u : 1u);
                    mma(tmem + 128u, ah, bl, id2, 1u);
                    mma(tmem + 128u, al, bh, id2, 1u);
                }
                commit(&bars[2]);
            }
            if (b + 1 < nblk) stage2(i0 + BM, s ^ 1);                // overlaps the MMAs
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            if (!wait_bar(2)) return false;
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            // lanes = rows i; warps 0-3 take columns 0..63, warps 4-7 columns 64..127
            {
                const int q = warp & 3;
                const int i = i0 + q * 32 + lane;
                const int cbeg = (warp >> 2) * 64;
                for (int j0 = cbeg; j0 < cbeg + 64; j0 += 16) {
                    uint32_t v[16];
                    ld16(tmem + ((uint32_t)(q * 32) << 16) + 128u + (uint32_t)j0, v);
                    if (i < N) {
#pragma unroll
                        for (int j = 0; j < 16; ++j) {
                            const int c = j0 + j;
                            if (c < nrows) {
                                T *x = Ab + (size_t)(c0 + c) * ld + i;
                                *x = __ldcg(x) - (T)__uint_as_float(v[j]);
                            }
                        }
                    }
                }
            }
            asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
            __syncthreads();
        }
    }
    return true;
}

// ------------------------------------------------------------------------
// Emulated-fp64 flush on the tensor cores (fp64 walkers).
//
// Every fp64 operand x of a contraction is cut into NS = 7 signed 8-bit
// integer slices relative to a power of two shared by its row or column
// (Emax: the largest biased exponent of the set):
//   q = round(|x| 2^(1078 - Emax)) < 2^56,  q = sum_j s_j 2^(48 - 8j),
//   x ~ sign(x) 2^(Emax - 1078) q            (56 bits of every operand).
// An element far below the largest of its set keeps few of those bits, which
// matters where its partner in the contraction is correspondingly large (a
// matrix whose orbitals, or electrons, span many binades). So each
// contraction index is first scaled by a power of two on both sides, which
// leaves every product unchanged: row i of A^{-1} by 2^-s_i and column i of
// V by 2^s_i, with s_i chosen to make the scaled queued changes uniform in i
// (oz_colexp_init: a move that changes orbital i by D_i makes A^{-1}'s row i
// carry 1/D_i); queue entry m of W and T by 2^f_m and
// 2^-f_m, with f_m from the column exponent of A^{-1} at the queued electron
// (a scaling of the electrons' rows). The shared exponents are those of the
// scaled values; an element's own slicing exponent adds its index's shift.
// A slice is an integer of magnitude <= 255, exact in fp16, and the product of
// two slices is an integer <= 65025; a tcgen05 MMA with fp32 accumulation sums
// such products without rounding while every partial sum stays below 2^24.
// The slice pairs (j, l) with j + l <= 6 (28 products, issued as 9 or 10 MMAs
// per K-step with the slices of one operand stacked along N) are accumulated
// per diagonal d = j + l in tensor memory and recombined exactly in 64-bit
// integers. The dropped (j + l >= 7) and rounded terms stay near 2^-53 of
// |row| |column|: one flush matches fp64 arithmetic's own error (about 1e-15
// relative for a 200 x 200 walker, against 3e-13 with six slices).
//
// The flush of Eq. 4 runs in three phases over all CTAs of the walker group,
// with a group barrier after each:
//   A  T'[c][m] = sum_i A^{-1}[i][c] V[m][i]: items of 128 columns x 256 rows
//      (the contraction split over row chunks), raw K-blocks of 16 rows
//      brought in by asynchronous copies two blocks ahead and sliced with the
//      column exponents of A^{-1} and the row exponents of V (kept up to date
//      by phase C and by the accepts); one pair per tensor-memory block for
//      d <= 3 (exact: 256 x 65025 < 2^24), d = 4..6 spread over two blocks
//      each (their fp32 rounding lies below 2^-53 of the result); partials as
//      an exact int64 and an fp32 tail.
//   B  T = sum of the partials (integers, fixed order), sliced with one
//      exponent per column c; W = P Kinv sliced with one exponent per row i;
//      the slices are written in the tensor cores' K-major tile layout.
//   C  A^{-1}[i][c] -= sum_m W[m][i] T[m][c]: items of 128 rows x 64 columns,
//      contraction K <= 32 so that all seven diagonals accumulate exactly
//      (7 x 32 x 65025 < 2^24); S = sum_d D_d 2^(8(5-d)) in int64 with the
//      seventh diagonal folded in, turned into fp64 by integer operations, and
//      one fp64 subtraction per element of A^{-1}. The tiles arrive by bulk
//      copies, the next item's T tile while the current one computes.
namespace ozf {
constexpr int NS = 7;
constexpr int AM = 128, AR = 256, AK = 16;      // phase A item: columns, rows; rows per K-block
constexpr int NSLOT = 3;                        // phase A: raw fp64 K-blocks in flight
constexpr int CM = 128, CN = 64;                // phase C item: rows, columns
constexpr int TMEM_COLS = 512;

struct Layout {
    size_t part, partg, wsl, tsl, wex, tex, cex, vex, rex, fex, vsl, bytes;
    int nrc, nca, nrb, nct;
};
// per walker-group scratch: partial T' [nrc][nca*AM][kp] as exact int64 sums
// of the d <= 3 diagonals and fp32 sums of d = 4, 5; slices of W
// [nrb][NS][CM*kp] and of T [nct][NS][CN*kp] fp16; exponents of W rows, T
// columns, A^{-1} columns (cex) and V rows (vex), all of the scaled values;
// the row shifts s_i (rex) and the queue shifts f_m (fex); the slices of V
// [nrc*AR/AK][NS][kp*AK] fp16, one block of AK rows after another in phase
// A's shared-memory layout
__host__ __device__ inline Layout layout(int N, int kp)
{
    Layout L;
    L.nrc = (N + AR - 1) / AR;
    L.nca = (N + AM - 1) / AM;
    L.nrb = (N + CM - 1) / CM;
    L.nct = (N + CN - 1) / CN;
    size_t o = 0;
    L.part = o;  o += (size_t)L.nrc * L.nca * AM * kp * sizeof(long long);
    L.partg = o; o += (size_t)L.nrc * L.nca * AM * kp * sizeof(float);
    L.wsl = o;  o += (size_t)L.nrb * NS * CM * kp * 2;
    L.tsl = o;  o += (size_t)L.nct * NS * CN * kp * 2;
    L.wex = o;  o += (size_t)L.nrb * CM * sizeof(int);
    L.tex = o;  o += (size_t)L.nct * CN * sizeof(int);
    L.cex = o;  o += (size_t)L.nca * AM * sizeof(int);
    L.vex = o;  o += 64 * sizeof(int);
    L.rex = o;  o += ((size_t)L.nca * AM + 2) * sizeof(int);
    L.fex = o;  o += 64 * sizeof(int);
    o = (o + 255) / 256 * 256;
    L.vsl = o;  o += (size_t)L.nrc * (AR / AK) * NS * kp * AK * 2;
    L.bytes = (o + 255) / 256 * 256;
    return L;
}
// shared memory: phase A's NSLOT raw fp64 K-blocks of A^{-1} columns, two
// stages of their slices and NSLOT blocks of V's slices; phase C reuses it for one W tile, two
// T tiles and two blocks of column exponents; then eight mbarriers (0, 1:
// phase A stages free again; 2: phase C MMAs; 3: W tile; 4, 5: T tiles; 6, 7:
// phase A stages full)
constexpr int NBAR = 8;
// arrivals per phase: 6, 7 are phase A's stage-full barriers (one per warp)
__host__ __device__ inline unsigned bar_count(int q) { return q >= 6 ? 8u : 1u; }
// phase A's raw fp64 K-blocks: column stride RS = AK + 2 doubles, so that the
// 16-byte accesses of a warp (lanes 64 bytes apart in the column, two lanes per
// column) spread over the shared-memory banks instead of 16 lanes per bank group
constexpr int RS = AK + 2;
__host__ __device__ inline size_t raw_bytes(int) { return (size_t)AM * RS * sizeof(double); }
__host__ __device__ inline size_t phase_a_bytes(int kp)
{
    return NSLOT * raw_bytes(kp) + (size_t)2 * NS * AM * AK * 2 + (size_t)NSLOT * NS * kp * AK * 2;
}
__host__ __device__ inline size_t phase_c_bytes(int kp)
{
    return (size_t)NS * (CM + 2 * CN) * kp * 2 + 2 * CN * sizeof(int);
}
__host__ __device__ inline size_t bar_offset(int kp)
{
    const size_t a = phase_a_bytes(kp), c = phase_c_bytes(kp);
    return ((a > c ? a : c) + 15) / 16 * 16;
}
__host__ __device__ inline size_t region_bytes(int kp) { return bar_offset(kp) + NBAR * sizeof(unsigned long long); }

__device__ __forceinline__ int bexp(double x) { return (int)((__double_as_longlong(x) >> 52) & 0x7FF); }
// x != 0 as an integer test (an fp64 compare would take the fp64 pipe, which
// retires two lanes per clock per SM)
__device__ __forceinline__ bool nz(double x) { return ((unsigned long long)__double_as_longlong(x) << 1) != 0ull; }

// 56-bit magnitude q = round(|x| 2^(1078 - emax)) of x relative to the set's
// largest biased exponent emax (|x| < 2^(emax - 1022)), clamped to 2^56 - 1,
// and its sign, as two 32-bit words (bits 32..55 and 0..31). Rounding to
// nearest keeps the slicing error unbiased.
__device__ __forceinline__ void mag56(double x, int emax, uint32_t &qhi, uint32_t &qlo, uint32_t &neg)
{
    const unsigned long long b = (unsigned long long)__double_as_longlong(x);
    const int E = (int)((b >> 52) & 0x7FF);
    const int s = E - emax + 3;                 // q = m 2^s, s <= 3
    const unsigned long long m = (b & 0xFFFFFFFFFFFFFull) | (1ull << 52);
    const int r = -s;
    unsigned long long q = s >= 0 ? (m << (s & 63))
                                  : (r > 54 ? 0ull : ((m + (1ull << ((r - 1) & 63))) >> (r & 63)));
    q = E == 0 ? 0ull : (q > 0xFFFFFFFFFFFFFFull ? 0xFFFFFFFFFFFFFFull : q);
    qhi = (uint32_t)(q >> 32);
    qlo = (uint32_t)q;
    neg = (uint32_t)(b >> 63);
}
// slice j (0 = most significant byte) of two magnitudes as a packed pair of
// fp16: the bytes are placed under the exponent of +-1024 (the pair's signs
// already in `base` = 0x6400 per half with the sign bits set; 1024 + b is
// exact in fp16 for b < 1024), and +-1024 is subtracted from both halves at
// once, which leaves +-b
__device__ __forceinline__ uint32_t slice_pair(uint32_t qh0, uint32_t ql0, uint32_t qh1, uint32_t ql1,
                                               int j, uint32_t base)
{
    const bool hi = j < 3;
    const uint32_t a = hi ? qh0 : ql0, b = hi ? qh1 : ql1;
    const uint32_t idx = hi ? (uint32_t)(2 - j) : (uint32_t)(6 - j);      // byte index in the word
    const uint32_t w = (__byte_perm(a, b, idx | ((4u + idx) << 8)) & 0x00FF00FFu) | base;
    __half2 h = *reinterpret_cast<const __half2 *>(&w);
    h = __hsub2(h, *reinterpret_cast<const __half2 *>(&base));
    return *reinterpret_cast<const uint32_t *>(&h);
}
// eight values, value e relative to exponent emax[e]: plane j of the slices
// as eight packed fp16
__device__ __forceinline__ void slice8(const double (&x)[8], const int (&emax)[8], uint4 (&out)[NS])
{
    uint32_t qh[8], ql[8], ng[8];
#pragma unroll
    for (int e = 0; e < 8; ++e) mag56(x[e], emax[e], qh[e], ql[e], ng[e]);
    uint32_t sg[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) sg[q] = 0x64006400u | (ng[2 * q] << 15) | (ng[2 * q + 1] << 31);
#pragma unroll
    for (int j = 0; j < NS; ++j) {
        uint32_t w[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) w[q] = slice_pair(qh[2 * q], ql[2 * q], qh[2 * q + 1], ql[2 * q + 1], j, sg[q]);
        out[j] = make_uint4(w[0], w[1], w[2], w[3]);
    }
}
// S 2^e as fp64 (S rounded to 53 significant bits, halves away from zero),
// built with integer operations: 0 for S = 0 or below the normal range, +-inf
// above it (a carry out of the rounding moves into the exponent field)
__device__ __forceinline__ double scaled_i64(long long S, int e)
{
    const unsigned long long neg = (unsigned long long)S & 0x8000000000000000ull;
    const unsigned long long M = S < 0 ? 0ull - (unsigned long long)S : (unsigned long long)S;
    const int lz = __clzll((long long)M);
    const int be = 63 - lz + e + 1023;                  // biased exponent of the leading bit
    const unsigned long long Mn = M << (lz & 63);
    const unsigned long long frac = (Mn >> 11) + ((Mn >> 10) & 1ull);   // rounded to 53 bits
    unsigned long long bits = neg | (((unsigned long long)(be - 1) << 52) + frac);
    bits = (M == 0 || be <= 0) ? neg : (be >= 2047 ? (neg | 0x7FF0000000000000ull) : bits);
    return __longlong_as_double((long long)bits);
}
// 2^e as fp64 (0 below the normal range, +inf above it)
__device__ __forceinline__ double pow2(int e)
{
    return e < -1022 ? 0.0 : e > 1023 ? __longlong_as_double(0x7FF0000000000000ll)
                                      : __longlong_as_double((long long)(e + 1023) << 52);
}
// instruction descriptor: fp16 x fp16 -> fp32, K-major A and B, M x N
__device__ __forceinline__ uint32_t idesc_f16(int M, int N)
{
    return (1u << 4) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}
// Phase A's MMAs per K-step. The V slices are stacked along N in shared
// memory, so one MMA multiplies A^{-1} slice j by the V slices l_lo .. l_lo +
// nl - 1, and its accumulator block b + t (units of kp columns) receives the
// pair (j, l_lo + t), of diagonal d = j + l_lo + t. Four banks place the
// blocks so that every diagonal d <= 3 block holds exactly one pair (exact
// over 256 rows); the d = 4..6 blocks of banks 0 and 1 take several.
//   bank 0: blocks 0..6 = d 0..6; bank 1: blocks 7..12 = d 1..6;
//   bank 2: blocks 13, 14 = d 2, 3; bank 3: block 15 = d 3.
// (16 blocks of kp <= 32 columns: the 512 columns of tensor memory.)
constexpr int NMMA_A = 9, NMMA_C = 10;
struct MmaA { int j, l, nl, blk, fresh; };
__device__ constexpr MmaA kMmaA[NMMA_A] = {
    {0, 0, 7, 0, 1}, {1, 0, 6, 7, 1}, {2, 0, 2, 13, 1}, {2, 2, 3, 4, 0}, {3, 0, 1, 15, 1},
    {3, 1, 3, 10, 0}, {4, 0, 3, 4, 0}, {5, 0, 2, 11, 0}, {6, 0, 1, 6, 0}};
// Phase C's MMAs per K-step: W slice j times the T slices l .. l + nl - 1,
// accumulator block (units of 64 columns) = diagonal d = j + l; every block
// is exact (at most 7 pairs x 32 terms: 7 x 32 x 65025 < 2^24).
struct MmaC { int j, l, nl, fresh; };
__device__ constexpr MmaC kMmaC[NMMA_C] = {
    {0, 0, 4, 1}, {0, 4, 3, 1}, {1, 0, 4, 0}, {1, 4, 2, 0}, {2, 0, 4, 0},
    {2, 4, 1, 0}, {3, 0, 4, 0}, {4, 0, 3, 0}, {5, 0, 2, 0}, {6, 0, 1, 0}};
}  // namespace ozf

// Slicing exponents of walker w's A^{-1}, computed by all CTAs of the group at
// the start of the walker's sweep (and by the per-call flush): first the row
// shifts s_i, then, after a group barrier, the column exponents of the
// shifted values, max_i (E(x_ic) - s_i) over the nonzero elements. Phase A
// slices 2^-s_i A^{-1}_ic per column and 2^s_i u_i per queued change, so that
// the shift cancels in every product. A term keeps its precision when both
// factors sit near their shared maxima; the shift that achieves this for the
// terms u_i A^{-1}_ic is the one that makes the scaled changes uniform in i:
// s_i = 1023 - max_m E(V[m][i]) over the queued changes (Vq, kq rows), which
// the per-call flush knows when it runs. (Scaling A^{-1}'s rows to a common
// size instead loses the small entries of a row dominated by one large one,
// as ill-conditioned walks make them.) The persistent sweep's changes are
// sigma g for one scalar sigma, already uniform in i: it passes Vq = nullptr
// and s_i = 0. Every emulated flush then keeps the column exponents up to
// date (phase C) with the same shifts. A flush by flush_columns_small, which
// does not, only ends a sweep. Returns false after the barrier's wait ran
// out of budget.
template <typename T>
__device__ bool oz_colexp_init(const SweepParams<T> &p, int w, int grp, int rank, unsigned *flush_ctr,
                               unsigned &n_flush, const double *Vq, int kq)
{
    const int N = p.N, ld = p.ld;
    const ozf::Layout Ly = ozf::layout(N, p.kp);
    unsigned char *scr = p.oz + (size_t)grp * p.oz_stride;
    int *cex = (int *)(scr + Ly.cex);
    int *rex = (int *)(scr + Ly.rex);
    const double *Ab = (const double *)p.Ainv + (size_t)w * N * ld;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    // the queue's row exponents start from zero (the accepts raise them); the
    // scratch is shared with the recompute's update, which lays it out for
    // 32 queue entries
    if (rank == 0 && threadIdx.x < 64) ((int *)(scr + Ly.vex))[threadIdx.x] = 0;
    for (int i = rank * STHREADS + (int)threadIdx.x; i < N; i += p.Gf * STHREADS) {
        int g = 0;
        for (int m = 0; m < kq; ++m) {
            const double x = __ldcg(Vq + (size_t)m * ld + i);
            if (ozf::nz(x)) g = max(g, ozf::bexp(x));
        }
        rex[i] = g ? 1023 - g : 0;
    }
    if (!group_barrier(flush_ctr, (++n_flush) * p.Gf, p.status, p.budget_ns)) return false;
    for (int c = rank * SWARPS + warp; c < N; c += p.Gf * SWARPS) {
        int e = 0;
        for (int i = 2 * lane; i < N; i += 64) {
            const double2 u = __ldcg(reinterpret_cast<const double2 *>(Ab + (size_t)c * ld + i));
            const int2 r = __ldcg(reinterpret_cast<const int2 *>(rex + i));
            if (ozf::nz(u.x)) e = max(e, ozf::bexp(u.x) - r.x);
            if (ozf::nz(u.y)) e = max(e, ozf::bexp(u.y) - r.y);
        }
        e = __reduce_max_sync(0xffffffffu, e);
        if (lane == 0) cex[c] = e;
    }
    return true;
}
template <typename T>
__device__ __forceinline__ int *oz_vex(const SweepParams<T> &p, int grp)
{
    return (int *)(p.oz + (size_t)grp * p.oz_stride + ozf::layout(p.N, p.kp).vex);
}

// V's slices for phase A, cut once per flush by all CTAs of the group: block
// kbg of AK rows (i = kbg AK .. + AK - 1), plane j, in phase A's shared-memory
// layout, so that every row chunk of phase A copies them instead of cutting
// them again. Entry (m, i) is sliced with the row exponent of queue entry m
// (vex) less the row shift s_i; rows past N and entries m >= k are zero.
template <typename T>
__device__ __noinline__ void oz_slice_v(const SweepParams<T> &p, int w, int k, int grp, int rank)
{
    using namespace tcf;
    using namespace ozf;
    const int N = p.N, ld = p.ld, kp = p.kp;
    const Layout Ly = layout(N, kp);
    unsigned char *scr = p.oz + (size_t)grp * p.oz_stride;
    const int *vex = (const int *)(scr + Ly.vex);
    const int *rex = (const int *)(scr + Ly.rex);
    __half *vg = (__half *)(scr + Ly.vsl);
    const double *Vb = (const double *)p.V + (size_t)w * p.K * ld;
    const size_t bplane = (size_t)kp * AK;
    const int units = Ly.nrc * (AR / AK) * kp * 2;    // (block, m, half block): eight values each
    for (int u = rank * STHREADS + (int)threadIdx.x; u < units; u += p.Gf * STHREADS) {
        const int kbg = u / (kp * 2), rem = u - kbg * kp * 2, m = rem >> 1, kk = (rem & 1) * 8;
        const int i0 = kbg * AK + kk;
        const int ev = m < k ? __ldcg(vex + m) : 0;
        double x[8];
        int em[8];
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            const int i = i0 + q;
            const bool in = m < k && i < N;
            x[q] = in ? __ldcg(Vb + (size_t)m * ld + i) : 0.0;
            em[q] = ev - (i < N ? __ldcg(rex + i) : 0);
        }
        uint4 out[NS];
        slice8(x, em, out);
        const uint32_t o = coff(m, kk, AK) >> 1;
#pragma unroll
        for (int j = 0; j < NS; ++j)
            *reinterpret_cast<uint4 *>(vg + ((size_t)kbg * NS + j) * bplane + o) = out[j];
    }
}

// The emulated-fp64 flush of walker w (all Gf CTAs of the group call it; it
// takes three group barriers of its own). Returns false after a wait ran out of
// budget (ST_TIMEOUT recorded).
// Phase A of flush_oz (a function of its own: its register allocation does not
// compete with the rest of the sweep kernel's).
template <typename T>
__device__ __noinline__ bool oz_phase_a(const SweepParams<T> &p, int w, int k, int grp, int rank, unsigned char *smem,
                                uint32_t tmem, unsigned *tph)
{
    using namespace tcf;
    using namespace ozf;
    const int N = p.N, ld = p.ld, K = p.K, kp = p.kp, Gf = p.Gf;
    const Layout Ly = layout(N, kp);
    unsigned char *scr = p.oz + (size_t)grp * p.oz_stride;
    int *cex = (int *)(scr + Ly.cex);
    const int *rex = (const int *)(scr + Ly.rex);
    long long *partS = (long long *)(scr + Ly.part);
    float *partG = (float *)(scr + Ly.partg);
    unsigned char *reg = smem + p.off_xs;
    unsigned long long *bars = (unsigned long long *)(reg + bar_offset(kp));
    __shared__ int ecol[AM], erw[AR], ok_s;
    const size_t wN = (size_t)N * ld, wK = (size_t)K * ld;
    double *Ab = (double *)p.Ainv + (size_t)w * wN;
    const double *Vb = (const double *)p.V + (size_t)w * wK;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int Nc = Ly.nca * AM;     // row stride of the partial T' buffers
    auto wait_bar = [&](int b) -> bool {
        if (tid == 0) ok_s = mbar_wait(&bars[b], tph[b], p.status, p.budget_ns) ? 1 : 0;
        __syncthreads();
        tph[b] ^= 1u;
        return ok_s != 0;
    };

    // the queue shifts f_m for phase B, from the column exponents as they
    // stand (phase B resets them for phase C)
    if (rank == 0 && tid < k) {
        int *fex = (int *)(scr + Ly.fex);
        fex[tid] = 1023 - __ldcg(cex + __ldcg(p.idx + (size_t)w * K + tid));
    }

    // ------------------------------------------------------------ phase A
    {
        // T'[c][m] partial over rows [r0, r0 + AR) of column tile c0: raw fp64
        // K-blocks of AK rows of A^{-1} arrive by asynchronous copies two
        // blocks ahead and are cut into slices with the column exponents of
        // A^{-1} (cex), which every row chunk shares, so that the partials add
        // up exactly as integers; V's slices, cut once per flush
        // (oz_slice_v), arrive by asynchronous copies one block ahead
        const int nA = Ly.nca * Ly.nrc;
        const int nkb = AR / AK;
        const size_t aplane = (size_t)AM * AK, bplane = (size_t)kp * AK;   // fp16 elements
        double *raw = (double *)reg;                                       // [NSLOT][AM][RS]
        __half *sa = (__half *)(reg + NSLOT * raw_bytes(kp));              // [2][NS][AM*AK]
        __half *sv = sa + 2 * NS * aplane;                                 // [NSLOT][NS][kp*AK]
        const __half *vg = (const __half *)(scr + Ly.vsl);                 // [nrc*AR/AK][NS][kp*AK]
        const int vch = (int)(NS * bplane * sizeof(__half) / 16);          // 16-byte chunks per block
        const uint32_t sboA = (AK / 8) * 128;
        for (int it = rank; it < nA; it += Gf) {
            const int ct = it % Ly.nca, rc = it / Ly.nca;
            const int c0 = ct * AM, r0 = rc * AR;
            const int ncol = min(AM, N - c0);
            if (tid < AM) ecol[tid] = tid < ncol ? __ldcg(cex + c0 + tid) : 0;
            for (int t = tid; t < AR; t += STHREADS) erw[t] = r0 + t < N ? __ldcg(rex + r0 + t) : 0;
            // A pipeline without CTA barriers. Thread t copies, with 16-byte
            // asynchronous copies two blocks ahead, exactly the raw data it cuts
            // (rows 8 (t & 1) .. + 7 of column t >> 1 of A^{-1}), and a few
            // chunks of the V slices of the next block; its own wait_group
            // then covers both. Each warp announces stage s on bars[6 + s] (8
            // arrivals), thread 0 issues the stage's MMAs and commits them to
            // bars[s], which every thread waits on before it cuts into stage s
            // (and copies into the V slot of block kb - 2) again. A wait that
            // runs out of budget marks the thread bad; it keeps walking the loop
            // without work and the CTA leaves together after it.
            const int ca = tid >> 1, kk = (tid & 1) * 8;
            const int kbg0 = r0 / AK;
            auto issue = [&](int kb, int kbv) {
                if (kb < nkb) {
                    const int i = r0 + kb * AK;
                    double *dst = raw + (size_t)(kb % NSLOT) * AM * RS;
                    const bool ina = i < ld && ca < ncol;
                    const double *srca = Ab + (size_t)(c0 + (ina ? ca : 0)) * ld + (ina ? i + kk : 0);
#pragma unroll
                    for (int q = 0; q < 4; ++q)
                        asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;"
                                     ::"r"(su32(dst + (size_t)ca * RS + kk + 2 * q)), "l"(ina ? srca + 2 * q : srca),
                                       "r"(ina ? 16 : 0) : "memory");
                }
                if (kbv >= 0 && kbv < nkb) {
                    const uint4 *src = reinterpret_cast<const uint4 *>(vg + (size_t)(kbg0 + kbv) * NS * bplane);
                    uint4 *dst = reinterpret_cast<uint4 *>(sv + (size_t)(kbv % NSLOT) * NS * bplane);
                    for (int c = tid; c < vch; c += STHREADS) cp_async16(dst + c, src + c);
                }
                asm volatile("cp.async.commit_group;" ::: "memory");
            };
            issue(0, 0);
            issue(1, -1);
            __syncthreads();                       // ecol, erw
            bool bad = false;
            for (int kb = 0; kb < nkb; ++kb) {
                const int s = kb & 1, sl = kb % NSLOT;
                if (kb >= 2) {    // the MMAs of block kb - 2 have read stage s and V slot (kb + 1) % NSLOT
                    if (!bad) bad = !mbar_wait(&bars[s], tph[s], p.status, p.budget_ns);
                    tph[s] ^= 1u;
                }
                issue(kb + 2, kb + 1);
                asm volatile("cp.async.wait_group 1;" ::: "memory");     // blocks kb (raw, V) complete
                const int i = r0 + kb * AK;
                const double *rw = raw + (size_t)sl * AM * RS;
                if (!bad) {
                    {
                        double x[8];
                        const bool in = ca < ncol && i < ld;
#pragma unroll
                        for (int q = 0; q < 4; ++q) {
                            const double2 u = in ? *reinterpret_cast<const double2 *>(rw + ca * RS + kk + 2 * q)
                                                 : make_double2(0.0, 0.0);
                            x[2 * q] = u.x;
                            x[2 * q + 1] = u.y;
                        }
                        int em[8];
#pragma unroll
                        for (int q = 0; q < 8; ++q) em[q] = ecol[ca] + erw[kb * AK + kk + q];
                        uint4 out[NS];
                        slice8(x, em, out);
                        const uint32_t o = coff(ca, kk, AK) >> 1;
#pragma unroll
                        for (int j = 0; j < NS; ++j)
                            *reinterpret_cast<uint4 *>(sa + (s * NS + j) * aplane + o) = out[j];
                    }
                }
                asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                __syncwarp();
                if (lane == 0) mbar_arrive(&bars[6 + s]);
                if (tid == 0) {
                    if (!bad) bad = !mbar_wait(&bars[6 + s], tph[6 + s], p.status, p.budget_ns);
                    tph[6 + s] ^= 1u;
                    if (!bad) {
                        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
#pragma unroll
                        for (int q = 0; q < NMMA_A; ++q) {
                            const MmaA mm = kMmaA[q];
                            const uint64_t ad = sdesc(su32(sa + (s * NS + mm.j) * aplane), 128, sboA);
                            const uint64_t bd = sdesc(su32(sv + (sl * NS + mm.l) * bplane), 128, sboA);
                            const bool first = kb == 0 && mm.fresh;
                            mma(tmem + (uint32_t)(mm.blk * kp), ad, bd, idesc_f16(AM, mm.nl * kp), first ? 0u : 1u);
                        }
                        commit(&bars[s]);
                    }
                }
            }
            for (int kb = nkb - 2; kb < nkb; ++kb) {     // the last two blocks' MMAs
                const int s = kb & 1;
                if (!bad) bad = !mbar_wait(&bars[s], tph[s], p.status, p.budget_ns);
                tph[s] ^= 1u;
            }
            if (__syncthreads_or(bad)) return false;
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            // readout: lanes = columns c, 16 values of m per warp; the d <= 3
            // diagonals as one exact int64, d = 4..6 as an fp32 tail in units
            // of 2^-8 of it
            {
                const int q = warp & 3, m0 = (warp >> 2) * 16;
                const int c = q * 32 + lane;
                if (m0 < kp) {
                    const uint32_t lanebase = tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)m0;
                    long long S[16];
                    float g[16], g5[16];
                    uint32_t v[16];
#pragma unroll
                    for (int e = 0; e < 16; ++e) S[e] = 0;
                    // blocks of diagonal d (bank layout of kMmaA): d <= 3 exact
                    constexpr int nblk[4] = {1, 2, 3, 4};
                    constexpr int blks[4][4] = {{0, 0, 0, 0}, {1, 7, 0, 0}, {2, 8, 13, 0}, {3, 9, 14, 15}};
#pragma unroll
                    for (int d = 0; d <= 3; ++d) {
                        int Dd[16];
#pragma unroll
                        for (int e = 0; e < 16; ++e) Dd[e] = 0;
#pragma unroll
                        for (int t = 0; t < nblk[d]; ++t) {
                            ld16(lanebase + (uint32_t)(blks[d][t] * kp), v);
#pragma unroll
                            for (int e = 0; e < 16; ++e) Dd[e] += __float2int_rz(__uint_as_float(v[e]));
                        }
#pragma unroll
                        for (int e = 0; e < 16; ++e) S[e] = S[e] * 256 + Dd[e];
                    }
                    // the tail: g = D4 + D5 / 2^8 + D6 / 2^16 (blocks 4, 10; 5, 11; 6, 12)
                    ld16(lanebase + (uint32_t)(6 * kp), v);
#pragma unroll
                    for (int e = 0; e < 16; ++e) g5[e] = __uint_as_float(v[e]);
                    ld16(lanebase + (uint32_t)(12 * kp), v);
#pragma unroll
                    for (int e = 0; e < 16; ++e) g5[e] = (g5[e] + __uint_as_float(v[e])) * (1.0f / 256.0f);
                    ld16(lanebase + (uint32_t)(5 * kp), v);
#pragma unroll
                    for (int e = 0; e < 16; ++e) g5[e] += __uint_as_float(v[e]);
                    ld16(lanebase + (uint32_t)(11 * kp), v);
#pragma unroll
                    for (int e = 0; e < 16; ++e) g5[e] = (g5[e] + __uint_as_float(v[e])) * (1.0f / 256.0f);
                    ld16(lanebase + (uint32_t)(4 * kp), v);
#pragma unroll
                    for (int e = 0; e < 16; ++e) g[e] = g5[e] + __uint_as_float(v[e]);
                    ld16(lanebase + (uint32_t)(10 * kp), v);
#pragma unroll
                    for (int e = 0; e < 16; ++e) g[e] += __uint_as_float(v[e]);
                    if (c < ncol) {
                        const size_t o = ((size_t)rc * Nc + c0 + c) * kp + m0;
#pragma unroll
                        for (int e = 0; e < 16; e += 2)
                            *reinterpret_cast<longlong2 *>(partS + o + e) = make_longlong2(S[e], S[e + 1]);
#pragma unroll
                        for (int e = 0; e < 16; e += 4)
                            *reinterpret_cast<float4 *>(partG + o + e) = make_float4(g[e], g[e + 1], g[e + 2], g[e + 3]);
                    }
                }
            }
            asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
            __syncthreads();
        }
    }
    return true;
}

// Phase B of flush_oz.
template <typename T>
__device__ __noinline__ bool oz_phase_b(const SweepParams<T> &p, int w, int k, int grp, int rank, unsigned char *smem,
                                uint32_t tmem, unsigned *tph)
{
    using namespace tcf;
    using namespace ozf;
    const int N = p.N, ld = p.ld, K = p.K, kp = p.kp, Gf = p.Gf;
    const Layout Ly = layout(N, kp);
    unsigned char *scr = p.oz + (size_t)grp * p.oz_stride;
    int *cex = (int *)(scr + Ly.cex);
    int *vex = (int *)(scr + Ly.vex);
    long long *partS = (long long *)(scr + Ly.part);
    float *partG = (float *)(scr + Ly.partg);
    __half *wsl = (__half *)(scr + Ly.wsl);
    __half *tsl = (__half *)(scr + Ly.tsl);
    int *wex = (int *)(scr + Ly.wex);
    int *tex = (int *)(scr + Ly.tex);
    const size_t wK = (size_t)K * ld;
    const double *Wb = (const double *)p.W + (size_t)w * wK;
    const int Nc = Ly.nca * AM;     // row stride of the partial T' buffers
    const int tid = threadIdx.x;
    __shared__ int fs[32];          // queue shifts f_m (from phase A)
    if (tid < 32) fs[tid] = tid < k ? __ldcg((const int *)(scr + Ly.fex) + tid) : 0;
    __syncthreads();

    // ------------------------------------------------------------ phase B
    {
        // T = sum_rc T'_rc, eight consecutive m per thread, the kp / 8
        // threads of a column adjacent in the warp. Chunks of 32 tasks go to
        // the group's warps round-robin over its CTAs (chunk cn to CTA cn mod Gf),
        // so that every SM takes a share
        const int ng = kp / 8;
        const int totT = N * ng;
        const int warp = tid >> 5, lane = tid & 31;
        for (int cn = rank + Gf * warp; cn * 32 < totT; cn += Gf * SWARPS) {
            const int e = cn * 32 + lane;
            const bool in = e < totT;
            const int c = in ? e / ng : 0, m0 = (e - (e / ng) * ng) * 8;
            double t[8];
#pragma unroll
            for (int q = 0; q < 8; ++q) t[q] = 0.0;
            const int ec = in ? __ldcg(cex + c) : 0;
            __syncwarp();
            if (in) {
                if (m0 == 0) cex[c] = 0;        // phase C records the new column exponents
                long long S[8];
                float g[8];
#pragma unroll
                for (int q = 0; q < 8; ++q) {
                    S[q] = 0;
                    g[q] = 0.f;
                }
#pragma unroll 4
                for (int rc = 0; rc < Ly.nrc; ++rc) {
                    const size_t o = ((size_t)rc * Nc + c) * kp + m0;
                    const longlong2 *s2 = reinterpret_cast<const longlong2 *>(partS + o);
                    const float4 *g4 = reinterpret_cast<const float4 *>(partG + o);
#pragma unroll
                    for (int q = 0; q < 4; ++q) {
                        const longlong2 u = __ldcg(s2 + q);
                        S[2 * q] += u.x;
                        S[2 * q + 1] += u.y;
                    }
#pragma unroll
                    for (int q = 0; q < 2; ++q) {
                        const float4 u = __ldcg(g4 + q);
                        g[4 * q] += u.x;
                        g[4 * q + 1] += u.y;
                        g[4 * q + 2] += u.z;
                        g[4 * q + 3] += u.w;
                    }
                }
#pragma unroll
                for (int q = 0; q < 8; ++q) {
                    const int m = m0 + q;
                    if (m < k) {
                        const int e = ec + __ldcg(vex + m) - 2084;
                        t[q] = fma((double)g[q], pow2(e - 8), (double)S[q] * pow2(e));
                    }
                }
            }
            // T's column exponent over the scaled entries T[m][c] 2^-f_m
            int em = 0;
#pragma unroll
            for (int q = 0; q < 8; ++q)
                if (nz(t[q])) em = max(em, bexp(t[q]) - fs[m0 + q]);
            for (int o = 1; o < ng; o <<= 1) em = max(em, __shfl_xor_sync(0xffffffffu, em, o));
            if (in) {
                int emq[8];
#pragma unroll
                for (int q = 0; q < 8; ++q) emq[q] = em + fs[m0 + q];
                uint4 sl[NS];
                slice8(t, emq, sl);
                const int ct = c / CN;
                const uint32_t o = coff(c - ct * CN, m0, kp) >> 1;
#pragma unroll
                for (int j = 0; j < NS; ++j)
                    *reinterpret_cast<uint4 *>(tsl + ((size_t)ct * NS + j) * CN * kp + o) = sl[j];
                if (m0 == 0) tex[c] = em;
            }
        }
        // W: the kp / 8 threads of a row i adjacent in the warp, eight values
        // of m each (chunks of 32 tasks round-robin over the CTAs as for T);
        // the row exponent over the scaled entries W[m][i] 2^f_m
        const int totW = N * ng;
        for (int cn = rank + Gf * warp; cn * 32 < totW; cn += Gf * SWARPS) {
            const int e = cn * 32 + lane;
            const bool in = e < totW;
            const int i = in ? e / ng : 0, g = e - (e / ng) * ng;
            double y[8];
            int em = 0;
#pragma unroll
            for (int q = 0; q < 8; ++q) {
                const int m = g * 8 + q;
                y[q] = (in && m < k) ? __ldcg(Wb + (size_t)m * ld + i) : 0.0;
                if (nz(y[q])) em = max(em, bexp(y[q]) + fs[m]);
            }
            for (int o = 1; o < ng; o <<= 1) em = max(em, __shfl_xor_sync(0xffffffffu, em, o));
            if (in) {
                int emq[8];
#pragma unroll
                for (int q = 0; q < 8; ++q) emq[q] = em - fs[g * 8 + q];
                uint4 sl[NS];
                slice8(y, emq, sl);
                const int rb = i / CM;
                const uint32_t o = coff(i - rb * CM, g * 8, kp) >> 1;
#pragma unroll
                for (int j = 0; j < NS; ++j)
                    *reinterpret_cast<uint4 *>(wsl + ((size_t)rb * NS + j) * CM * kp + o) = sl[j];
                if (g == 0) wex[i] = em;
            }
        }
    }
    return true;
}

// Phase C of flush_oz.
template <typename T>
__device__ __noinline__ bool oz_phase_c(const SweepParams<T> &p, int w, int k, int grp, int rank, unsigned char *smem,
                                uint32_t tmem, unsigned *tph)
{
    using namespace tcf;
    using namespace ozf;
    const int N = p.N, ld = p.ld, K = p.K, kp = p.kp, Gf = p.Gf;
    const Layout Ly = layout(N, kp);
    unsigned char *scr = p.oz + (size_t)grp * p.oz_stride;
    int *cex = (int *)(scr + Ly.cex);
    int *vex = (int *)(scr + Ly.vex);
    __half *wsl = (__half *)(scr + Ly.wsl);
    __half *tsl = (__half *)(scr + Ly.tsl);
    int *wex = (int *)(scr + Ly.wex);
    int *tex = (int *)(scr + Ly.tex);
    const int *rex = (const int *)(scr + Ly.rex);
    __shared__ int ok_s;
    unsigned char *reg = smem + p.off_xs;
    unsigned long long *bars = (unsigned long long *)(reg + bar_offset(kp));
    const size_t wN = (size_t)N * ld;
    double *Ab = (double *)p.Ainv + (size_t)w * wN;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    auto wait_bar = [&](int b) -> bool {
        if (tid == 0) ok_s = mbar_wait(&bars[b], tph[b], p.status, p.budget_ns) ? 1 : 0;
        __syncthreads();
        tph[b] ^= 1u;
        return ok_s != 0;
    };

    // ------------------------------------------------------------ phase C
    {
        // each CTA takes a contiguous run of items, row-block major, so that
        // consecutive items share the W tile; the next item's T tile and column
        // exponents arrive by bulk copy while the current one computes
        const int nC = Ly.nrb * Ly.nct;
        const int per = (nC + Gf - 1) / Gf;
        const int it0 = min(nC, rank * per), it1 = min(nC, it0 + per);
        const uint32_t sbo = (uint32_t)(kp / 8) * 128u;
        const unsigned wbytes = (unsigned)(NS * CM * kp * 2), tbytes = (unsigned)(NS * CN * kp * 2);
        __half *swt = (__half *)reg;                               // [NS][CM*kp]
        __half *stt = swt + NS * CM * kp;                          // [2][NS][CN*kp]
        int *stx = (int *)(stt + 2 * NS * CN * kp);                // [2][CN]
        auto load_t = [&](int it, int b) {
            const int ct = it % Ly.nct;
            mbar_expect(&bars[4 + b], tbytes + CN * sizeof(int));
            bulk_g2s(stt + (size_t)b * NS * CN * kp, tsl + (size_t)ct * NS * CN * kp, tbytes, &bars[4 + b]);
            bulk_g2s(stx + b * CN, tex + ct * CN, CN * sizeof(int), &bars[4 + b]);
        };
        auto load_w = [&](int it) {
            const int rb = it / Ly.nct;
            mbar_expect(&bars[3], wbytes);
            bulk_g2s(swt, wsl + (size_t)rb * NS * CM * kp, wbytes, &bars[3]);
        };
        if (rank == 0 && tid < 64) vex[tid] = 0;    // the next queue records its own
        if (it0 < it1 && tid == 0) {
            load_w(it0);
            load_t(it0, 0);
        }
        bool wpend = it0 < it1;
        for (int it = it0; it < it1; ++it) {
            const int q = it - it0, b = q & 1;
            const int rb = it / Ly.nct, ct = it - rb * Ly.nct;
            const int i0 = rb * CM, c0 = ct * CN;
            if (wpend) {
                if (!wait_bar(3)) return false;
                wpend = false;
            }
            if (!wait_bar(4 + b)) return false;
            if (tid == 0) {
                if (it + 1 < it1) load_t(it + 1, b ^ 1);   // its buffer's last MMAs completed
                asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                for (int ks = 0; ks < kp / 16; ++ks) {
                    const uint32_t ko = (uint32_t)ks * 256u;
#pragma unroll
                    for (int u = 0; u < NMMA_C; ++u) {
                        const MmaC mm = kMmaC[u];
                        const uint64_t ad = sdesc(su32(swt + (size_t)mm.j * CM * kp) + ko, 128, sbo);
                        const uint64_t bd = sdesc(su32(stt + ((size_t)b * NS + mm.l) * CN * kp) + ko, 128, sbo);
                        mma(tmem + (uint32_t)((mm.j + mm.l) * CN), ad, bd, idesc_f16(CM, mm.nl * CN),
                            (ks == 0 && mm.fresh) ? 0u : 1u);
                    }
                }
                commit(&bars[2]);
            }
            // lanes = rows i; warps 0-3 take columns 0..31, warps 4-7 columns 32..63;
            // the first 16 values of A^{-1} are read while the MMAs run
            const int qw = warp & 3;
            const int i = i0 + qw * 32 + lane;
            const int cb = (warp >> 2) * 32;
            const bool rowin = i < N;
            const int ei = rowin ? __ldcg(wex + i) : 0;
            const int ri = rowin ? __ldcg(rex + i) : 0;     // the row's shift s_i
            double xa[16];
            auto load_x = [&](int j0) {
#pragma unroll
                for (int e = 0; e < 16; ++e) {
                    const int c = c0 + j0 + e;
                    xa[e] = (rowin && c < N) ? __ldcg(Ab + (size_t)c * ld + i) : 0.0;
                }
            };
            load_x(cb);
            if (!wait_bar(2)) return false;
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            if (it + 1 < it1 && (it + 1) / Ly.nct != rb) {
                if (tid == 0) load_w(it + 1);              // the W tile's MMAs completed
                wpend = true;
            }
            for (int j0 = cb; j0 < cb + 32; j0 += 16) {
                long long S[16];
                uint32_t v[3][16];
                const uint32_t lrow = tmem + ((uint32_t)(qw * 32) << 16) + (uint32_t)j0;
#pragma unroll
                for (int e = 0; e < 16; ++e) S[e] = 0;
                // the diagonals three loads at a time, one wait per three
#pragma unroll
                for (int d0 = 0; d0 < NS - 1; d0 += 3) {
#pragma unroll
                    for (int t = 0; t < 3; ++t) ld16_nw(lrow + (uint32_t)((d0 + t) * CN), v[t]);
                    tmem_wait_ld();
#pragma unroll
                    for (int t = 0; t < 3; ++t)
#pragma unroll
                        for (int e = 0; e < 16; ++e) S[e] = S[e] * 256 + __float2int_rz(__uint_as_float(v[t][e]));
                }
                // S = sum_{d <= 5} D_d 2^(8(5 - d)) < 2^61.02; the d = 6 diagonal
                // joins as 2 S + round(D_6 / 2^7) (an error of 2^-63 of the leading term)
                ld16(lrow + (uint32_t)((NS - 1) * CN), v[0]);
#pragma unroll
                for (int e = 0; e < 16; ++e) S[e] = 2 * S[e] + ((__float2int_rz(__uint_as_float(v[0][e])) + 64) >> 7);
                double y[16];
#pragma unroll
                for (int e = 0; e < 16; ++e) y[e] = xa[e] - scaled_i64(S[e], ei + stx[b * CN + j0 + e] - 2101);
                if (j0 == cb) load_x(cb + 16);
#pragma unroll
                for (int e = 0; e < 16; ++e) {
                    const int c = c0 + j0 + e;
                    if (rowin && c < N) Ab[(size_t)c * ld + i] = y[e];
                }
                // exponents of the new columns (scaled by the row shifts) for
                // the next flush's phase A
                int mx[16];
#pragma unroll
                for (int e = 0; e < 16; ++e)
                    mx[e] = __reduce_max_sync(0xffffffffu, (rowin && c0 + j0 + e < N && nz(y[e]))
                                                               ? bexp(y[e]) - ri : 0);
                if (lane == 0) {
#pragma unroll
                    for (int e = 0; e < 16; ++e)
                        if (c0 + j0 + e < N) atomicMax(cex + c0 + j0 + e, mx[e]);
                }
            }
            asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
            __syncthreads();
        }
    }
    return true;
}

// (out of line for the same reason as flush_columns_small_ool)
template <typename T>
__device__ __noinline__ bool flush_oz(const SweepParams<T> &p, int w, int k, int grp, int rank,
                         unsigned char *smem, uint32_t tmem, unsigned *tph, unsigned *flush_ctr,
                         unsigned &n_flush)
{
    const int Gf = p.Gf, tid = threadIdx.x;
    // wall time of the three phases (barrier waits included) as seen by
    // group 0's first CTA, into the profile's phase timers 8..10
    const bool timed = p.phase_ns && grp == 0 && rank == 0 && tid == 0;
    unsigned long long tp = timed ? globaltimer() : 0ull;
    auto tick = [&](int slot) {
        if (timed) {
            const unsigned long long t = globaltimer();
            p.phase_ns[slot] += t - tp;
            tp = t;
        }
    };

    oz_slice_v(p, w, k, grp, rank);
    if (!group_barrier(flush_ctr, (++n_flush) * Gf, p.status, p.budget_ns)) return false;
    if (!oz_phase_a(p, w, k, grp, rank, smem, tmem, tph)) return false;
    if (!group_barrier(flush_ctr, (++n_flush) * Gf, p.status, p.budget_ns)) return false;
    tick(8);
    if (!oz_phase_b(p, w, k, grp, rank, smem, tmem, tph)) return false;
    if (!group_barrier(flush_ctr, (++n_flush) * Gf, p.status, p.budget_ns)) return false;
    tick(9);
    if (!oz_phase_c(p, w, k, grp, rank, smem, tmem, tph)) return false;
    tick(10);
    return true;
}

template <typename T, bool RES, int FM, bool CL>
__device__ void sweep_body(const SweepParams<T> &p, unsigned char *smem, uint32_t tmem)
{
    const int grp = blockIdx.x / p.Gf, rank = blockIdx.x - grp * p.Gf;
    if (grp >= p.ngroups) return;
    unsigned tph[8] = {0, 0, 0, 0, 0, 0, 0, 0};  // phases of the tensor-core flush's mbarriers
    const int N = p.N, K = p.K, ld = p.ld, Gf = p.Gf, Gr = p.Gr;
    const size_t wN = (size_t)N * ld, wK = (size_t)K * ld;
    unsigned *flush_ctr = p.sync + SYNC_STRIDE * grp + 32;
    unsigned *cmd = p.sync + SYNC_STRIDE * grp + 64;
    unsigned n_ratio = 0, n_flush = 0, n_event = 0, bar_phase = 0;
    const int cpc = (N + Gf - 1) / Gf;                 // columns per CTA in the flush
    const int fc0 = min(N, rank * cpc), fc1 = min(N, fc0 + cpc);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

    if (rank >= Gr) {
        // Helper CTA: take part in every flush of every walker of the group.
        for (int t = grp; t < p.nw; t += p.ngroups) {
            const int w = p.wlist ? __ldg(p.wlist + t) : t;
            if (FM == FM_OZ && !oz_colexp_init(p, w, grp, rank, flush_ctr, n_flush, nullptr, 0)) return;
            for (;;) {
                if (!group_wait_for(cmd, 2u * (n_event + 1), p.status, p.budget_ns, 128)) return;
                const bool last = (ld_acquire(cmd) & 1u) != 0;
                ++n_event;
                if (!group_barrier(flush_ctr, (++n_flush) * Gf, p.status, p.budget_ns)) return;
                const int k = __ldcg(p.kglob + w);
                if (FM == FM_OZ) {
                    if (k >= SMALL_K) {
                        if (!flush_oz(p, w, k, grp, rank, smem, tmem, tph, flush_ctr, n_flush)) return;
                    } else if (k > 0) {
                        flush_columns_small_ool(p, w, k, fc0, fc1);
                    }
                } else if (FM == FM_TC) {
                    if (k > 0 && !flush_tc(p, w, k, fc0, fc1, smem, tmem, tph)) return;
                } else if (k > 0 && k < SMALL_K) {
                    flush_columns_small(p, w, k, fc0, fc1);
                } else if (k > 0 && p.block_ok && fc1 - fc0 >= BT) {
                    flush_block(p, w, k, fc0, fc1, smem);
                } else if (k > 0 && !flush_columns(p, w, k, fc0, fc1, smem, bar_phase)) {
                    return;
                }
                if (!group_barrier(flush_ctr, (++n_flush) * Gf, p.status, p.budget_ns)) return;
                if (last) break;
            }
        }
        return;
    }

    // Ratio CTA: rows [i0, i0 + L) of every N-vector.
    T *vs = (T *)(smem + p.off_vs);                    // [2][chunk] change u = v - a_j (working prec.)
    T *as = (T *)(smem + p.off_as);                    // [2][chunk] column j of A^{-1}
    double *vd = (double *)(smem + p.off_vd);          // [2][chunk] proposed row (fp64)
    double *red = (double *)(smem + p.off_red);        // [2K+1] reduced dots
    T *coef = (T *)(smem + p.off_ts);                  // accept: [0,K) c_m, [K,2K) y_m/r, [2K,..) z
    T *Wsm = (T *)(smem + p.off_wsm);                  // RES: [K][LP]
    T *Vsm = (T *)(smem + p.off_vsm);                  // RES: [K][LP]
    __shared__ double rinv_s, u_s[2];
    __shared__ int acc_s, vx_s[2];
    const int chunk = p.chunk, LP = chunk + 1;
    const int i0 = rank * chunk;
    const int L = max(0, min(chunk, N - i0));
    const int nj = 2 * K + 1;
    const int njs = 2 * K + 2;                         // row stride of the partials in global memory

    for (int t = grp; t < p.nw; t += p.ngroups) {
        const int w = p.wlist ? __ldg(p.wlist + t) : t;
        const int orow = t;            // output row: walker w, or list entry t
        double *Aw = p.A + (size_t)w * wN;
        const T *Ainv = p.Ainv + (size_t)w * wN;
        const double *Gw = p.gauss + (size_t)w * wN;
        const double *Uw = p.unif + (size_t)w * N;
        T *Ww = p.W + (size_t)w * wK;
        T *Vw = p.V + (size_t)w * wK;
        if (FM == FM_OZ) {
            if (!oz_colexp_init(p, w, grp, rank, flush_ctr, n_flush, nullptr, 0)) return;
            if (threadIdx.x < 2) vx_s[threadIdx.x] = 0;
        }

        // proposed row of electron jj, v = a_jj + sigma g (fp64, for the new row
        // of A), its change u = v - a_jj (working precision, for the dot
        // products and the queue) and column jj of A^{-1}; with the emulated
        // flush also the largest exponent of the CTA's part of u
        auto stage = [&](int jj, int bb, bool row, bool col) {
            if (row) {
                const double *arow = Aw + (size_t)jj * ld + i0;
                const double *grow = Gw + (size_t)jj * ld + i0;
                for (int t = threadIdx.x; t < L; t += STHREADS) {
                    const double a0 = arow[t];
                    const double v = __dadd_rn(a0, __dmul_rn(p.sigma, __ldcg(grow + t)));
                    const double u = __dsub_rn(v, a0);
                    vs[bb * chunk + t] = (T)u;
                    vd[bb * chunk + t] = v;
                    if (FM == FM_OZ && ozf::nz(u)) atomicMax(&vx_s[bb], ozf::bexp(u));
                }
                if (threadIdx.x == 0) u_s[bb] = __ldcg(Uw + jj);
            }
            if (col) {
                const T *acol = Ainv + (size_t)jj * ld + i0;
                for (int t = threadIdx.x; t < L; t += STHREADS) as[bb * chunk + t] = __ldcg(acol + t);
            }
        };

        int k = 0;
        __syncthreads();
        stage(0, 0, true, true);
        const bool timed = p.phase_ns && grp == 0 && rank == 0 && threadIdx.x == 0;
        unsigned long long tp = timed ? globaltimer() : 0ull, ph[8] = {0, 0, 0, 0, 0, 0, 0, 0};
        auto tick = [&](int slot) {
            if (timed) {
                const unsigned long long t = globaltimer();
                ph[slot] += t - tp;
                tp = t;
            }
        };
        for (int j = 0; j < N; ++j) {
            const int b = j & 1;
            const T *vsb = vs + b * chunk, *asb = as + b * chunk;
            const double *vdb = vd + b * chunk;
            __syncthreads();
            // ---- the next proposal's inputs (row j + 1 of A and its Gaussians,
            // column j + 1 of A^{-1}, u): loaded now, so that their latency
            // overlaps the dot products, and staged after them
            const bool pf = L <= STHREADS && j + 1 < N;
            double pa = 0.0, pg = 0.0, pu = 0.0;
            T pc = 0;
            if (pf) {
                if (threadIdx.x < L) {
                    pa = Aw[(size_t)(j + 1) * ld + i0 + threadIdx.x];
                    pg = __ldcg(Gw + (size_t)(j + 1) * ld + i0 + threadIdx.x);
                    pc = __ldcg(Ainv + (size_t)(j + 1) * ld + i0 + threadIdx.x);
                }
                if (threadIdx.x == 0) pu = __ldcg(Uw + j + 1);
            }
            // ---- partial dot products over the chunk: d = u.a, y_m = W[m].u, c_m = V[m].a
            // (cluster mode: into this CTA's shared memory, for the siblings to read)
            double *clp = (double *)(smem + p.off_cl);
            unsigned *clflag = (unsigned *)(clp + 2 * nj);
            // (partials as double-fp32 pairs; outside cluster mode as tagged
            // words in buffer pbuf of the group's two)
            const unsigned pbuf = n_ratio & 1u, tag = 1u + n_ratio % 3u;
            double *part = CL ? clp + b * nj : p.partial + (((size_t)grp * 2 + pbuf) * Gr + rank) * njs;
            if (RES) {
                // G consecutive lanes per job (a power of two up to 8 that the
                // CTA's threads allow), lane g taking elements g, g + G, ...,
                // then a fixed shuffle tree over the group
                const int njk = 2 * k + 1;
                int G = 1;
                while (G < 8 && 2 * G * njk <= STHREADS) G *= 2;
                for (int t0 = threadIdx.x; t0 < njk * G; t0 += STHREADS) {
                    const int job = t0 / G, g = t0 - job * G;
                    const T *src = job == 0 ? asb : (job <= k ? Wsm + (job - 1) * LP : Vsm + (job - 1 - k) * LP);
                    const T *with = job <= k ? vsb : asb;
                    T acc0 = 0, acc1 = 0;
                    int t = g;
#pragma unroll 4
                    for (; t + G < L; t += 2 * G) {
                        acc0 += src[t] * with[t];
                        acc1 += src[t + G] * with[t + G];
                    }
                    if (t < L) acc0 += src[t] * with[t];
                    double s = (double)acc0 + (double)acc1;
                    const unsigned act = lanes_below(t0, njk * G);
                    for (int o = G / 2; o > 0; o >>= 1) s += __shfl_down_sync(act, s, o, G);
                    if (g == 0) {
                        if (CL) reinterpret_cast<float2 *>(part)[job] = df_split(s);
                        else st_tagged(part + job, df_split(s), tag);
                    }
                }
            } else {
                // queue rows in global memory: four jobs per warp at a time, so that
                // each lane keeps 4 x (unroll) independent loads in flight
                const int nj_k = 2 * k + 1;
                for (int j0 = warp * 4; j0 < nj_k; j0 += SWARPS * 4) {
                    const T *src[4];
                    const T *with[4];
#pragma unroll
                    for (int q = 0; q < 4; ++q) {
                        const int job = min(j0 + q, nj_k - 1);
                        if (job == 0) { src[q] = asb; with[q] = vsb; }
                        else if (job <= k) { src[q] = Ww + (size_t)(job - 1) * ld + i0; with[q] = vsb; }
                        else { src[q] = Vw + (size_t)(job - 1 - k) * ld + i0; with[q] = asb; }
                    }
                    T acc[4] = {0, 0, 0, 0};
#pragma unroll 4
                    for (int t = lane; t < L; t += 32) {
#pragma unroll
                        for (int q = 0; q < 4; ++q) acc[q] += src[q][t] * with[q][t];
                    }
#pragma unroll
                    for (int q = 0; q < 4; ++q) {
                        const T v = warp_allsum(acc[q]);
                        if (lane == 0 && j0 + q < nj_k) {
                            if (CL) reinterpret_cast<float2 *>(part)[j0 + q] = df_split((double)v);
                            else st_tagged(part + j0 + q, df_split((double)v), tag);
                        }
                    }
                }
            }
            if (!CL && threadIdx.x < 4 && 2 * k + 1 + (int)threadIdx.x < nj)
                st_tagged(part + 2 * k + 1 + threadIdx.x, make_float2(0.f, 0.f), tag);
            tick(0);
            // ---- (cluster mode: arrive), stage the next proposal (its column
            // speculatively), wait
            if (CL) {
                __syncthreads();                       // every partial written
                if (threadIdx.x == 0) cl_st_release(clflag, n_ratio + 1);
            }
            if (pf) {
                if (threadIdx.x < L) {
                    const double v = __dadd_rn(pa, __dmul_rn(p.sigma, pg));
                    const double u = __dsub_rn(v, pa);
                    vs[(b ^ 1) * chunk + threadIdx.x] = (T)u;
                    vd[(b ^ 1) * chunk + threadIdx.x] = v;
                    as[(b ^ 1) * chunk + threadIdx.x] = pc;
                    if (FM == FM_OZ && ozf::nz(u)) atomicMax(&vx_s[b ^ 1], ozf::bexp(u));
                }
                if (threadIdx.x == 0) u_s[b ^ 1] = pu;
            } else if (j + 1 < N) {
                stage(j + 1, b ^ 1, true, true);
            }
            tick(1);
            if (CL && !cl_wait_flags(clflag, n_ratio + 1, Gr, p.status, p.budget_ns)) return;
            tick(2);
            // ---- every ratio CTA sums the partials in the same order: G
            // consecutive lanes per job (a power of two up to 8 that the CTA's
            // threads allow), lane g of the group summing the partials of CTAs
            // g, g + G, ..., then a fixed shuffle tree over the group. Outside
            // cluster mode the loads poll the tagged words until every one
            // carries this proposal's tag (the stall option asks for a tag that
            // never comes, to exercise the timeout).
            const double *pb = p.partial + ((size_t)grp * 2 + pbuf) * Gr * njs;
            const unsigned want = (p.stall && n_ratio == 0) ? 4u : tag;
            int late = 0;
            {
                const int njk = 2 * k + 1;
                int G = 1;
                while (G < 8 && 2 * G * njk <= STHREADS) G *= 2;
                for (int t = threadIdx.x; t < njk * G; t += STHREADS) {
                    const int job = t / G, g = t - job * G;
                    // the partials as double-fp32 pairs, summed with two-sums
                    float2 s = make_float2(0.f, 0.f);
                    int q = g;
                    if (CL) {
                        // sibling q's partials in its shared memory, same order
                        const double *mine = clp + b * nj + job;
                        for (; q + 7 * G < Gr; q += 8 * G) {
                            float2 x[8];
#pragma unroll
                            for (int e = 0; e < 8; ++e) x[e] = cl_ld_f2(cl_map(mine, q + e * G));
#pragma unroll
                            for (int e = 0; e < 8; ++e) s = df_add(s, x[e]);
                        }
                        for (; q < Gr; q += G) s = df_add(s, cl_ld_f2(cl_map(mine, q)));
                    } else {
                        const double *pbj = pb + job;
                        unsigned long long deadline = 0;
                        const size_t stp = (size_t)G * njs;
                        constexpr int PL = 16;          // tagged loads in flight per lane and round
                        for (; q < Gr; q += PL * G) {
                            const int cnt = min(PL, (Gr - q + G - 1) / G);
                            const double *pq = pbj + (size_t)q * njs;
                            unsigned long long x[PL];
#pragma unroll
                            for (int e = 0; e < PL; ++e)
                                if (e < cnt) x[e] = ld_tagged(pq + e * stp);
                            for (unsigned spins = 1;; ++spins) {
                                unsigned stale = 0;
#pragma unroll
                                for (int e = 0; e < PL; ++e)
                                    if (e < cnt && tag_of(x[e]) != want) stale |= 1u << e;
                                if (!stale || late) break;
                                if ((spins & 15u) == 0) {
                                    const unsigned long long now = globaltimer();
                                    if (!deadline) deadline = now + (unsigned long long)p.budget_ns;
                                    else if (now > deadline || (*(volatile const int *)p.status & ST_TIMEOUT)) late = 1;
                                }
#pragma unroll
                                for (int e = 0; e < PL; ++e)
                                    if ((stale >> e) & 1u) x[e] = ld_tagged(pq + e * stp);
                            }
#pragma unroll
                            for (int e = 0; e < PL; ++e)
                                if (e < cnt) s = df_add(s, untag(x[e]));
                        }
                    }
                    // groups are whole (njk * G is a multiple of G), so the lanes
                    // of the iteration hold complete groups
                    const unsigned act = lanes_below(t, njk * G);
                    for (int o = G / 2; o > 0; o >>= 1) {
                        float2 t2;
                        t2.x = __shfl_down_sync(act, s.x, o, G);
                        t2.y = __shfl_down_sync(act, s.y, o, G);
                        s = df_add(s, t2);
                    }
                    if (g == 0) red[job] = (double)s.x + (double)s.y;
                }
            }
            ++n_ratio;
            if (__syncthreads_or(late)) {
                if (threadIdx.x == 0) atomicOr(p.status, ST_TIMEOUT);
                return;
            }
            // ---- the ratio and the Metropolis decision in warp 0 (fp64 work on
            // one warp only: the fp64 pipe retires two lanes per clock), then a
            // broadcast through shared memory
            if (warp == 0) {
                double s = 0.0;
                for (int m = lane; m < k; m += 32) s += red[1 + m] * red[1 + k + m];
                s = warp_allsum(s);
                if (lane == 0) {
                    const double r = 1.0 + (red[0] - s);
                    const double u = u_s[b];
                    const double prob = fmin(1.0, r * r);
                    const int ov = p.override_ ? (int)p.override_[(size_t)w * N + j] : -1;
                    int a = ov == 0 ? 0 : (ov == 1 ? 1 : (u < prob ? 1 : 0));
                    const bool bad = a && !(r != 0.0 && isfinite(r));
                    if (bad) a = 0;
                    rinv_s = a ? 1.0 / r : 0.0;      // once, not in every thread
                    acc_s = a;
                    if (rank == 0) {
                        if (bad) atomicOr(p.status, ST_SINGULAR);
                        p.acc_out[(size_t)orow * N + j] = (unsigned char)a;
                        p.ratio_out[(size_t)orow * N + j] = r;
                        if (fabs(prob - u) < 1e-10) p.ties[orow] += 1;
                        if (a || p.fixed_slot) p.idx[(size_t)w * K + k] = j;
                    }
                }
            } else if (RES) {
                // meanwhile warps 1.. compute the accept's z = a - W c (it needs
                // only the reduced dots), discarded if the move is rejected: ZG
                // consecutive lanes per row, lane g taking m = g, g + ZG, ..., then
                // a fixed shuffle tree (fp64: two lanes, since every tree step costs
                // a warp-wide fp64 add)
                constexpr int ZG = sizeof(T) == 8 ? 2 : 8;
                T *zs = coef + 2 * K;
                const int nzt = ((L + 31) / 32) * 32 * ZG;      // whole warps
                for (int t0 = threadIdx.x - 32; t0 < nzt; t0 += STHREADS - 32) {
                    const int t = t0 / ZG, g = t0 - t * ZG;
                    T z0 = 0, z1 = 0;
                    if (t < L) {
                        const double *cr = red + 1 + k;
                        int m = g;
#pragma unroll 2
                        for (; m + ZG < k; m += 2 * ZG) {
                            z0 += (T)cr[m] * Wsm[m * LP + t];
                            z1 += (T)cr[m + ZG] * Wsm[(m + ZG) * LP + t];
                        }
                        if (m < k) z0 += (T)cr[m] * Wsm[m * LP + t];
                    }
                    T z = z0 + z1;
#pragma unroll
                    for (int o = ZG / 2; o > 0; o >>= 1) z += __shfl_down_sync(0xffffffffu, z, o, ZG);
                    if (g == 0 && t < L) zs[t] = asb[t] - z;
                }
            }
            __syncthreads();
            const int a = acc_s;
            tick(3);
            if (a || p.fixed_slot) {
                // ---- accept: z = a - W c, W <- [W - z y'/r, z/r], V[k] = u, A[j] = v.
                // A rejected proposal with fixed slots takes the slot as the zero
                // change: y = W'0 = 0 and the Schur complement is 1, so
                // W <- [W, z], V[k] = 0, and A keeps its row.
                const double rinv = a ? rinv_s : 1.0;
                T *cT = coef, *yT = coef + K, *zs = coef + 2 * K;
                for (int m = threadIdx.x; m < k; m += STHREADS) {
                    cT[m] = (T)red[1 + k + m];
                    yT[m] = a ? (T)(red[1 + m] * rinv) : (T)0;
                }
                double *arow_w = Aw + (size_t)j * ld;
                if (RES) {
                    // (z is in zs already)
                    for (int t = threadIdx.x; t < L; t += STHREADS) {
                        Vsm[k * LP + t] = a ? vsb[t] : (T)0;
                        if (a) arow_w[i0 + t] = vdb[t];
                    }
                    __syncthreads();
                    const T rT = (T)rinv;
                    for (int e = threadIdx.x + (a ? 0 : k * L); e < (k + 1) * L; e += STHREADS) {
                        const int m = e / L, t = e - m * L;
                        if (m < k) Wsm[m * LP + t] -= zs[t] * yT[m];
                        else Wsm[k * LP + t] = zs[t] * rT;
                    }
                } else {
                    __syncthreads();
                    // queue rows in global memory: four rows per thread, m outermost,
                    // so that loads of different (m, row) are independent
                    const T rT = (T)rinv;
                    constexpr int SUB = 4;
                    for (int tb = 0; tb < L; tb += STHREADS * SUB) {
                        T z[SUB];
#pragma unroll
                        for (int q = 0; q < SUB; ++q) {
                            const int t = tb + threadIdx.x + q * STHREADS;
                            z[q] = t < L ? asb[t] : (T)0;
                        }
#pragma unroll 4
                        for (int m = 0; m < k; ++m) {
                            const T cm = cT[m];
                            const T *wr = Ww + (size_t)m * ld + i0;
#pragma unroll
                            for (int q = 0; q < SUB; ++q) {
                                const int t = tb + threadIdx.x + q * STHREADS;
                                if (t < L) z[q] -= cm * wr[t];
                            }
                        }
#pragma unroll 4
                        for (int m = 0; m < (a ? k : 0); ++m) {
                            const T ym = yT[m];
                            T *wr = Ww + (size_t)m * ld + i0;
#pragma unroll
                            for (int q = 0; q < SUB; ++q) {
                                const int t = tb + threadIdx.x + q * STHREADS;
                                if (t < L) wr[t] -= z[q] * ym;
                            }
                        }
#pragma unroll
                        for (int q = 0; q < SUB; ++q) {
                            const int t = tb + threadIdx.x + q * STHREADS;
                            if (t < L) {
                                Ww[(size_t)k * ld + i0 + t] = z[q] * rT;
                                Vw[(size_t)k * ld + i0 + t] = a ? vsb[t] : (T)0;
                                if (a) arow_w[i0 + t] = vdb[t];
                            }
                        }
                    }
                }
                if (FM == FM_OZ && threadIdx.x == 0) atomicMax(oz_vex(p, grp) + k, a ? vx_s[b] : 0);
                ++k;
            }
            // (vx_s[b] is staged again in the next proposal, after its first barrier)
            if (FM == FM_OZ && threadIdx.x == 0) vx_s[b] = 0;
            tick(4);
            const bool last = (j == N - 1);
            if (k < K && !last) continue;
            // ---- flush event: queue full, or end of the walker's sweep
            if (RES && k > 0) {
                __syncthreads();
                for (int e = threadIdx.x; e < k * L; e += STHREADS) {
                    const int m = e / L, t = e - m * L;
                    Ww[(size_t)m * ld + i0 + t] = Wsm[m * LP + t];
                    Vw[(size_t)m * ld + i0 + t] = Vsm[m * LP + t];
                }
            }
            if (rank == 0 && threadIdx.x == 0) {
                p.kglob[w] = k;
                __threadfence();
                atomicExch(cmd, 2u * (n_event + 1) + (last ? 1u : 0u));
            }
            ++n_event;
            if (!group_barrier(flush_ctr, (++n_flush) * Gf, p.status, p.budget_ns)) return;
            tick(5);
            if (FM == FM_OZ) {
                if (k >= SMALL_K) {
                    if (!flush_oz(p, w, k, grp, rank, smem, tmem, tph, flush_ctr, n_flush)) return;
                } else if (k > 0) {
                    flush_columns_small_ool(p, w, k, fc0, fc1);
                    if (rank == 0 && threadIdx.x < 64) oz_vex(p, grp)[threadIdx.x] = 0;
                }
            } else if (FM == FM_TC) {
                if (k > 0 && !flush_tc(p, w, k, fc0, fc1, smem, tmem, tph)) return;
            } else if (k > 0 && k < SMALL_K) {
                flush_columns_small(p, w, k, fc0, fc1);
            } else if (k > 0 && p.block_ok && fc1 - fc0 >= BT) {
                flush_block(p, w, k, fc0, fc1, smem);
            } else if (k > 0 && !flush_columns(p, w, k, fc0, fc1, smem, bar_phase)) {
                return;
            }
            tick(6);
            if (!group_barrier(flush_ctr, (++n_flush) * Gf, p.status, p.budget_ns)) return;
            if (k > 0 && j + 1 < N) stage(j + 1, b ^ 1, false, true);   // the column changed
            k = 0;
            tick(7);
        }
        if (timed)
            for (int q = 0; q < 8; ++q) p.phase_ns[q] += ph[q];
    }
}


// The kernel: tensor memory for the tensor-core flush (256 columns: two of
// these CTAs at most share an SM, 2 x 256 = 512 columns), the mbarriers, the
// sweep, and the release of the tensor memory on every exit path.
template <typename T, bool RES, int FM, bool CL>
__global__ void __launch_bounds__(STHREADS, FM == FM_SIMT ? 2 : 1) sweep_kernel(SweepParams<T> p)
{
    constexpr bool TC = FM != FM_SIMT;
    // tensor-memory columns: the split-bf16 flush's two accumulators fit in 256
    // (two such CTAs could share an SM); the emulated-fp64 flush takes the whole
    // 512, and its shared memory keeps a second CTA off the SM
    constexpr int TCOLS = FM == FM_OZ ? ozf::TMEM_COLS : 256;
    extern __shared__ __align__(128) unsigned char smem[];
    __shared__ uint32_t tmem_s;
    if (TC && threadIdx.x < 32) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
                     ::"r"(tcf::su32(&tmem_s)), "n"(TCOLS) : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (threadIdx.x == 0) {
        mbar_init((unsigned long long *)(smem + p.off_bar));
        if (TC) {
            unsigned long long *bars = (unsigned long long *)(smem + p.off_tcbar);
            for (int q = 0; q < (FM == FM_OZ ? ozf::NBAR : 4); ++q)
                asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;"
                             ::"r"(tcf::su32(&bars[q])), "r"(FM == FM_OZ ? ozf::bar_count(q) : 1u) : "memory");
            asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        }
    }
    if (CL && threadIdx.x == 0) *(unsigned *)(smem + p.off_cl + 2 * (2 * p.K + 1) * sizeof(double)) = 0u;
    if (TC) asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (TC) asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    // cluster mode: every CTA's flag is set before any sibling reads it, and
    // every CTA's shared memory stays in place until no sibling reads it
    // (the only unbounded waits, both at fixed points every CTA reaches)
    if (CL) cl_barrier();
    sweep_body<T, RES, FM, CL>(p, smem, TC ? tmem_s : 0u);
    if (CL) cl_barrier();
    if (TC) asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (TC && threadIdx.x < 32)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem_s), "n"(TCOLS) : "memory");
}

// Gaussians (Box-Muller pairs) and Metropolis uniforms of one sweep for every
// walker, from the Philox counters of qmcdu_sweep.
__global__ void sweep_draw_kernel(int N, int ld, int nw, unsigned long long seed, int sweep,
                                  const unsigned long long *params, int sweep_offset,
                                  const int *wlist, const unsigned long long *wseed,
                                  const int *wsweep, double *gauss, double *unif)
{
    if (params) {   // parameters in device memory (steps replayed from a CUDA graph)
        seed = params[0];
        sweep = (int)params[1] + sweep_offset;
    }
    const int npair = (N + 1) / 2;
    const long long per_w = (long long)N * npair;
    const long long total = per_w * nw;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
         e += (long long)gridDim.x * blockDim.x) {
        const int t = (int)(e / per_w);
        const long long r = e - (long long)t * per_w;
        const int j = (int)(r / npair), q = (int)(r - (long long)j * npair);
        // walker t of the launch, or the listed walker with its own key and sweep
        const int w = wlist ? wlist[t] : t;
        const unsigned long long ws = wseed ? wseed[t] : seed + (unsigned long long)w;
        const int sw = wsweep ? wsweep[t] : sweep;
        const double2 g = proposal_gaussian_pair(ws, j, sw, q);
        double *row = gauss + ((size_t)w * N + j) * ld;
        row[2 * q] = g.x;
        if (2 * q + 1 < N) row[2 * q + 1] = g.y;
        if (q == 0) unif[(size_t)w * N + j] = metropolis_uniform(ws, j, sw);
    }
}

// The draws of one sweep of nw walkers (keys base_seed + w) into caller
// memory: gauss [nw][N][N], unif [nw][N] (the same kernel as the sweep's own
// draws, rows of length N).
cudaError_t launch_proposal_draws(int N, int nw, unsigned long long base_seed, int sweep, double *gauss,
                                  double *unif, cudaStream_t s)
{
    if (N <= 0 || nw <= 0) return cudaSuccess;
    int dev = 0, sms = 148;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    sweep_draw_kernel<<<sms * 8, 256, 0, s>>>(N, N, nw, base_seed, sweep, nullptr, 0, nullptr, nullptr,
                                              nullptr, gauss, unif);
    return cudaGetLastError();
}

// log|det A| and sign after the sweep: one CTA per walker sums log|r| over the
// accepted proposals in a fixed order.
__global__ void sweep_logdet_kernel(int N, const int *wlist, const unsigned char *acc,
                                    const double *ratio, double *logabs, int *sign)
{
    const int t = blockIdx.x;                 // output row
    const int w = wlist ? wlist[t] : t;       // walker
    __shared__ double sred[STHREADS];
    __shared__ int sneg[STHREADS];
    double s = 0.0;
    int neg = 0;
    for (int j = threadIdx.x; j < N; j += STHREADS) {
        if (acc[(size_t)t * N + j]) {
            const double r = ratio[(size_t)t * N + j];
            s += log(fabs(r));
            neg += r < 0.0;
        }
    }
    sred[threadIdx.x] = s;
    sneg[threadIdx.x] = neg;
    __syncthreads();
    for (int o = STHREADS / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) {
            sred[threadIdx.x] += sred[threadIdx.x + o];
            sneg[threadIdx.x] += sneg[threadIdx.x + o];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        logabs[w] += sred[0];
        if (sneg[0] & 1) sign[w] = -sign[w];
    }
}

// ---------------------------------------------------------------- launcher
static size_t align16(size_t x) { return (x + 15) / 16 * 16; }
static const size_t OZ_MIN_SMEM = 118 * 1024;

template <typename T>
static size_t sweep_smem(int ld, int K, int chunk, int cb, bool res, int fm, bool block, int *offs,
                         bool cl = false)
{
    size_t o = 0;
    offs[8] = (int)o; o = align16(o + 16);                                   // mbarrier
    offs[0] = (int)o; o = align16(o + (size_t)2 * chunk * sizeof(T));        // vs
    offs[1] = (int)o; o = align16(o + (size_t)2 * chunk * sizeof(T));        // as
    offs[2] = (int)o; o = align16(o + (size_t)2 * chunk * sizeof(double));   // vd
    offs[3] = (int)o; o = align16(o + (size_t)(2 * K + 1) * sizeof(double)); // red
    offs[4] = (int)o; o = align16(o + (size_t)std::max(K * cb, 2 * K + chunk) * sizeof(T));  // ts
    offs[5] = (int)o;                                                        // xs / tc region
    size_t xs_bytes = (size_t)cb * ld * sizeof(T);
    if (block) xs_bytes = std::max(xs_bytes, (size_t)std::max(2 * BT * BT, 2 * BI1 * SLD) * sizeof(T));
    const int kp = (K + 15) / 16 * 16;
    const size_t region = fm == FM_TC ? tcf::region_bytes(kp) : fm == FM_OZ ? ozf::region_bytes(kp) : xs_bytes;
    offs[9] = (int)(o + (fm == FM_TC ? tcf::region_bytes(kp) - 4 * sizeof(unsigned long long)
                                     : fm == FM_OZ ? ozf::bar_offset(kp) : 0));
    o = align16(o + region);
    offs[6] = (int)o; if (res) o = align16(o + (size_t)K * (chunk + 1) * sizeof(T));  // Wsm
    offs[7] = (int)o; if (res) o = align16(o + (size_t)K * (chunk + 1) * sizeof(T));  // Vsm
    offs[10] = (int)o; if (cl) o = align16(o + (size_t)2 * (2 * K + 1) * sizeof(double) + 16);  // partials, flag
    // the emulated-fp64 flush allocates all 512 tensor-memory columns: more than
    // half of the SM's shared memory keeps a second CTA off the SM
    if (fm == FM_OZ) o = std::max(o, (size_t)OZ_MIN_SMEM);
    return o;
}

static const size_t SMEM_BUDGET = 200 * 1024;
static const size_t RES_BUDGET = 128 * 1024;

// Cluster mode: the Gr = CLS ratio CTAs of a walker are one thread-block
// cluster; every walker group is a whole number of clusters.
constexpr int CLS = 16;
static const size_t CL_SMEM_BUDGET = 216 * 1024;

template <typename T, bool RES, int FM, bool CL>
static cudaError_t launch_shape(Ctx &c, const SweepLaunch &L, int Gf, int Gr, int chunk)
{
    const int K = c.K;
    int offs[11];
    const size_t budget = CL ? CL_SMEM_BUDGET : SMEM_BUDGET;
    int cb = MAX_CB;
    // the wide-block flush (fp64, K <= 64) when its tiles fit beside everything
    // else: fp64 arithmetic hides its staging; in fp32 (one CTA of 8 warps per SM)
    // the staging latency does not hide and the column tiles are as fast
    bool block = FM == FM_SIMT && K <= BT && std::is_same<T, double>::value;
    size_t smem = sweep_smem<T>(c.ld, K, chunk, cb, RES, FM, block, offs, CL);
    while (cb > 1 && smem > budget) {
        cb >>= 1;
        smem = sweep_smem<T>(c.ld, K, chunk, cb, RES, FM, block, offs, CL);
    }
    if (smem > budget && block) {
        block = false;
        cb = MAX_CB;
        smem = sweep_smem<T>(c.ld, K, chunk, cb, RES, FM, block, offs, CL);
        while (cb > 1 && smem > budget) {
            cb >>= 1;
            smem = sweep_smem<T>(c.ld, K, chunk, cb, RES, FM, block, offs, CL);
        }
    }
    if (smem > budget) return cudaErrorInvalidConfiguration;
    cudaError_t e = cudaFuncSetAttribute(sweep_kernel<T, RES, FM, CL>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, sweep_kernel<T, RES, FM, CL>, STHREADS, smem);
    if (e != cudaSuccess) return e;
    const int nw = L.wlist ? L.nlist : c.batch;
    int ngroups = 0;
    cudaLaunchConfig_t cfg = {};
    cudaLaunchAttribute attr[2];
    if (CL) {
        // as many co-resident clusters as fit, split evenly over the walker groups
        e = cudaFuncSetAttribute(sweep_kernel<T, RES, FM, CL>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
        if (e != cudaSuccess) return e;
        attr[0].id = cudaLaunchAttributeClusterDimension;
        attr[0].val.clusterDim.x = CLS;
        attr[0].val.clusterDim.y = 1;
        attr[0].val.clusterDim.z = 1;
        attr[1].id = cudaLaunchAttributeCooperative;
        attr[1].val.cooperative = 1;
        cfg.gridDim = dim3(CLS);
        cfg.blockDim = dim3(STHREADS);
        cfg.dynamicSmemBytes = smem;
        cfg.stream = c.stream;
        cfg.attrs = attr;
        cfg.numAttrs = 1;
        int ncl = 0;
        e = cudaOccupancyMaxActiveClusters(&ncl, (const void *)sweep_kernel<T, RES, FM, CL>, &cfg);
        if (e != cudaSuccess) return e;
        if (c.opt_max_ctas > 0) ncl = std::min(ncl, c.opt_max_ctas / CLS);
        ngroups = std::min(nw, ncl);
        if (FM == FM_OZ) ngroups = std::min(ngroups, c.oz_groups);
        if (ngroups < 1) return cudaErrorInvalidConfiguration;
        Gf = CLS * (ncl / ngroups);
        Gr = CLS;
    } else {
        int capacity = per_sm * c.num_sms;
        if (c.opt_max_ctas > 0) capacity = std::min(capacity, c.opt_max_ctas);
        if (capacity < 1 || Gf > capacity) return cudaErrorCooperativeLaunchTooLarge;
        ngroups = std::min(nw, std::max(1, capacity / Gf));
        if (FM == FM_OZ) ngroups = std::min(ngroups, c.oz_groups);
        if (ngroups < 1) return cudaErrorInvalidConfiguration;
    }
    if (ngroups * SYNC_STRIDE > c.sync_words) return cudaErrorInvalidConfiguration;
    if ((size_t)ngroups * 2 * Gr * (2 * K + 2) > c.sw_partial_len) return cudaErrorInvalidConfiguration;

    SweepParams<T> p;
    p.N = c.N; p.K = K; p.ld = c.ld; p.batch = c.batch;
    p.Gf = Gf; p.Gr = Gr; p.ngroups = ngroups; p.chunk = chunk; p.cb = cb;
    p.A = c.A; p.Ainv = (T *)c.Ainv; p.W = (T *)c.P; p.V = (T *)c.V;
    p.idx = c.idx; p.kglob = c.kcount;
    p.gauss = c.sw_gauss; p.unif = c.sw_unif;
    p.partial = c.sw_partial; p.sync = c.sw_sync; p.status = c.status;
    p.sigma = L.sigma; p.override_ = L.override;
    p.fixed_slot = c.opt_fixed_slot;
    p.acc_out = L.acc_out; p.ratio_out = L.ratio_out; p.ties = L.ties;
    p.budget_ns = c.opt_budget_ns; p.stall = c.opt_stall;
    p.off_vs = offs[0]; p.off_as = offs[1]; p.off_vd = offs[2]; p.off_red = offs[3];
    p.off_ts = offs[4]; p.off_xs = offs[5]; p.off_wsm = offs[6]; p.off_vsm = offs[7];
    p.off_bar = offs[8];
    p.kp = (K + 15) / 16 * 16;
    p.block_ok = block ? 1 : 0;
    p.phase_ns = c.prof ? c.sw_phase : nullptr;
    p.wlist = L.wlist;
    p.nw = nw;
    p.oz = FM == FM_OZ ? c.oz : nullptr;
    p.oz_stride = c.oz_stride;
    p.off_tcbar = offs[9];
    p.off_cl = offs[10];
    e = cudaMemsetAsync(c.sw_sync, 0, (size_t)ngroups * SYNC_STRIDE * sizeof(unsigned), c.stream);
    if (e != cudaSuccess) return e;
    if (!CL) {
        // tag 0 in every partial slot: no word left by an earlier launch can
        // carry the tag that a proposal of this one waits for
        e = cudaMemsetAsync(c.sw_partial, 0, (size_t)ngroups * 2 * Gr * (2 * K + 2) * sizeof(double), c.stream);
        if (e != cudaSuccess) return e;
    }
    if (CL) {
        cfg.gridDim = dim3(ngroups * Gf);
        cfg.numAttrs = 2;
        e = cudaLaunchKernelEx(&cfg, sweep_kernel<T, RES, FM, CL>, p);
    } else {
        void *args[] = {&p};
        e = cudaLaunchCooperativeKernel((const void *)sweep_kernel<T, RES, FM, CL>, dim3(ngroups * Gf),
                                        dim3(STHREADS), args, smem, c.stream);
    }
    c.last_sweep_shape[0] = Gf;
    c.last_sweep_shape[1] = Gr;
    c.last_sweep_shape[2] = ngroups;
    c.last_sweep_shape[3] = chunk;
    c.last_sweep_shape[4] = FM == FM_TC ? 1000 : FM == FM_OZ ? 2000 : (RES ? cb : -cb);
    c.last_cluster = CL ? CLS : 0;
    return e;
}

size_t oz_group_bytes(int N, int K)
{
    (void)K;   // the recompute's rank-32 updates use the scratch at every K
    return ozf::layout(N, 32).bytes;
}

// The emulated-fp64 flush (flush_oz) for this handle and group size: fp64,
// SMALL_K <= K <= 32, a walker group of several CTAs, scratch allocated, not
// switched off. (Queues shorter than SMALL_K still flush with
// flush_columns_small.)
static bool use_oz(const Ctx &c, int Gf)
{
    return c.prec == QMCDU_FP64 && c.K <= 32 && c.K >= SMALL_K && Gf >= 2 && c.oz && c.oz_groups > 0 &&
           c.opt_fp64_flush != 1;
}

template <typename T>
static cudaError_t launch_sweep_t(Ctx &c, const SweepLaunch &L)
{
    const int N = c.N, K = c.K;
    const int nw = L.wlist ? L.nlist : c.batch;
    int Gf, Gr;
    const int sms = c.opt_max_ctas > 0 ? std::min(c.num_sms, c.opt_max_ctas) : c.num_sms;
    const int target_chunk = c.prec == QMCDU_FP64 ? 32 : 128;
    if (c.opt_group_ctas > 0) {
        // fixed walker-group shape: a walker's arithmetic does not depend on how
        // many walkers share the launch
        Gf = std::min(c.opt_group_ctas, sms);
        Gr = c.opt_ratio_ctas > 0 ? c.opt_ratio_ctas : (N + target_chunk - 1) / target_chunk;
        Gr = std::max(1, std::min(Gr, Gf));
    } else if (nw >= sms) {
        Gf = Gr = 1;
    } else {
        Gf = std::max(1, sms / nw);
        Gr = c.opt_ratio_ctas > 0 ? c.opt_ratio_ctas : (N + target_chunk - 1) / target_chunk;
        Gr = std::max(1, std::min(Gr, Gf));
        if (c.opt_flush_ctas > 0) Gf = std::max(Gr, std::min(Gf, c.opt_flush_ctas));
    }
    int chunk = (N + Gr - 1) / Gr;
    chunk = (chunk + 31) / 32 * 32;
    Gr = std::min(Gr, (N + chunk - 1) / chunk);
    Gf = std::max(Gf, Gr);
    const bool res = chunk <= 256 && 2 * (size_t)K * (chunk + 1) * sizeof(T) <= RES_BUDGET;
    if constexpr (std::is_same<T, double>::value) {
        // cluster mode (on request): fp64, a few large walkers with the GPU to
        // themselves and no fixed group shape; the CLS ratio CTAs of a walker
        // form one cluster and exchange their partial dot products through
        // distributed shared memory instead of global memory. The exchange is
        // faster, but 16 CTAs do the fp64 dot products and the queue update of
        // 64, and the flush runs on the 112 CTAs that 16-CTA clusters leave
        // co-resident: at N = 2048, K = 32 a sweep takes 29.5 ms against
        // 21.8 ms. Any refusal before the launch falls through to the
        // global-memory exchange below.
        const int cchunk = ((N + CLS - 1) / CLS + 31) / 32 * 32;
        const bool cres = cchunk <= 256 && 2 * (size_t)K * (cchunk + 1) * sizeof(T) <= RES_BUDGET;
        if (c.prec == QMCDU_FP64 && c.opt_cluster == 2 && c.opt_group_ctas == 0 && c.opt_ratio_ctas == 0 &&
            c.opt_flush_ctas == 0 && !c.opt_stall && N >= 1024 && nw <= 4 && cres) {
            cudaError_t e = cudaErrorInvalidConfiguration;
            if (use_oz(c, 2 * CLS)) e = launch_shape<T, true, FM_OZ, true>(c, L, 0, CLS, cchunk);
            if (e != cudaSuccess) {
                cudaGetLastError();
                e = launch_shape<T, true, FM_SIMT, true>(c, L, 0, CLS, cchunk);
            }
            if (e == cudaSuccess) return e;
            cudaGetLastError();
        }
    }
    // tensor-core flush: split-bf16 precision, flush blocks of >= 128 columns, K <= 64
    const int cpc = (N + Gf - 1) / Gf;
    const bool tc = std::is_same<T, float>::value && c.prec == QMCDU_FP32_BF16X3 && !res &&
                    K <= 64 && cpc >= 128;
    if (tc) return launch_shape<T, false, FM_TC, false>(c, L, Gf, Gr, chunk);
    if constexpr (std::is_same<T, double>::value) {
        // emulated-fp64 flush: fp64 walkers shared by several CTAs, K <= 32;
        // where its shared memory does not fit beside the resident queue rows
        // (launch_shape refuses before launching), the fp64-unit flush
        if (use_oz(c, Gf)) {
            const cudaError_t e = res ? launch_shape<T, true, FM_OZ, false>(c, L, Gf, Gr, chunk)
                                      : launch_shape<T, false, FM_OZ, false>(c, L, Gf, Gr, chunk);
            if (e != cudaErrorInvalidConfiguration) return e;
        }
    }
    return res ? launch_shape<T, true, FM_SIMT, false>(c, L, Gf, Gr, chunk)
               : launch_shape<T, false, FM_SIMT, false>(c, L, Gf, Gr, chunk);
}

// ---------------------------------------------------------------- recompute panel
// Gauss-Jordan elimination of one panel (columns [c0, c0 + nbe)) of the
// transposed copy X of walker b, over P CTAs that split the rows: the
// multi-CTA form of gj_panel_kernel (kernels_recompute.cu) for a few walkers,
// where one CTA per walker would leave the GPU idle and the panel need not fit
// one SM's shared memory. Per pivot column, one group barrier: every CTA
// publishes its best candidate (largest |x| among its rows >= c, first index
// on ties), that row's panel values, and the owner of row c publishes row c;
// after the barrier all CTAs take the same winner (largest, then lowest
// index: partial pivoting as in LU), the owner of the winner's row takes row
// c's old values, the rows c and p of X outside the panel are swapped in
// column shares, and every CTA eliminates its own rows. Candidate buffers
// alternate between two parities, so one barrier per column suffices.
struct GjScratch { double *candv; int *candi; double *candrow; double *rowc; };
__host__ __device__ inline size_t gj_scratch_bytes(int P, int nb)
{
    return (size_t)2 * P * sizeof(double) + (size_t)2 * P * sizeof(int) + (size_t)2 * P * nb * sizeof(double) +
           (size_t)2 * nb * sizeof(double) + 64;
}
__device__ inline GjScratch gj_scratch(unsigned char *base, int P, int nb)
{
    GjScratch s;
    s.candv = (double *)base;
    s.candrow = s.candv + 2 * P;
    s.rowc = s.candrow + (size_t)2 * P * nb;
    s.candi = (int *)(s.rowc + 2 * nb);
    return s;
}

constexpr int GJ_THREADS = 256;
constexpr int GJ_CTR_STRIDE = 32;     // one 128-byte line per walker
constexpr int GJ_NBMAX = 32;          // panel width at most (the cluster form)

__global__ void __launch_bounds__(GJ_THREADS) gj_panel_mc_kernel(int N, int ld, int nb, int c0, int nbe, int P,
                                                                double *work, int *piv, double *Lt, double *R,
                                                                double *lu_logabs, int *lu_sign, int *status,
                                                                unsigned *gj_ctr, unsigned char *scratch,
                                                                size_t scratch_stride, long long budget_ns)
{
    extern __shared__ double S[];              // [nb][Rr]: column q of the CTA's rows at S + q*Rr
    __shared__ double wval[GJ_THREADS / 32], prow[64];
    __shared__ int widx[GJ_THREADS / 32], win_s, wr_s;
    __shared__ double pvs[32], pvs_log[32];
    const int b = blockIdx.x / P, r = blockIdx.x - b * P;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int Rr = (N + P - 1) / P;
    const int i0 = min(N, r * Rr), nr = min(Rr, N - i0);
    double *X = work + (size_t)b * N * ld;
    unsigned *ctr = gj_ctr + GJ_CTR_STRIDE * b;     // this walker's own barrier counter
    unsigned nbar = 0;
    GjScratch g = gj_scratch(scratch + (size_t)b * scratch_stride, P, nb);
    // the CTA's column share of X for row interchanges and R
    const int xs = (N + P - 1) / P, x0 = min(N, r * xs), x1 = min(N, x0 + xs);

    for (int e = tid; e < nr * nbe; e += GJ_THREADS) {
        const int li = e / nbe, q = e - li * nbe;
        S[q * Rr + li] = X[(size_t)(i0 + li) * ld + c0 + q];
    }
    __syncthreads();
    double la = 0.0;
    int sg = 1, singular = 0;
    for (int q = 0; q < nbe; ++q) {
        const int c = c0 + q, par = q & 1;
        // my candidate, by integer keys (gj_key)
        long long best = -1;
        int bi = N;
        for (int li = tid; li < nr; li += GJ_THREADS) {
            const int gi = i0 + li;
            if (gi < c) continue;
            const long long v = gj_key(S[q * Rr + li]);
            if (v > best || (v == best && gi < bi)) { best = v; bi = gi; }
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const long long ov = __shfl_xor_sync(0xffffffffu, best, o);
            const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
            if (ov > best || (ov == best && oi < bi)) { best = ov; bi = oi; }
        }
        if (lane == 0) { wval[warp] = __longlong_as_double(best); widx[warp] = bi; }
        __syncthreads();
        if (warp == 0) {
            best = lane < GJ_THREADS / 32 ? __double_as_longlong(wval[lane]) : -1;
            bi = lane < GJ_THREADS / 32 ? widx[lane] : N;
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                const long long ov = __shfl_xor_sync(0xffffffffu, best, o);
                const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
                if (ov > best || (ov == best && oi < bi)) { best = ov; bi = oi; }
            }
            if (lane == 0) {
                g.candv[par * P + r] = __longlong_as_double(best);
                g.candi[par * P + r] = bi;
                win_s = bi;
            }
        }
        __syncthreads();
        const int mine = win_s;
        if (mine < N)
            for (int t = tid; t < nbe; t += GJ_THREADS) g.candrow[((size_t)par * P + r) * nb + t] = S[t * Rr + (mine - i0)];
        if (c >= i0 && c < i0 + nr)
            for (int t = tid; t < nbe; t += GJ_THREADS) g.rowc[par * nb + t] = S[t * Rr + (c - i0)];
        if (!group_barrier(ctr, (++nbar) * P, status, budget_ns)) return;
        // the winner: largest candidate, lowest row on ties, in a fixed order
        if (warp == 0) {
            long long bv = -1;
            int bidx = N, brk = 0;
            for (int k = lane; k < P; k += 32) {
                const long long v = __double_as_longlong(__ldcg(g.candv + par * P + k));
                const int i = __ldcg(g.candi + par * P + k);
                if (v > bv || (v == bv && i < bidx)) { bv = v; bidx = i; brk = k; }
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                const long long ov = __shfl_xor_sync(0xffffffffu, bv, o);
                const int oi = __shfl_xor_sync(0xffffffffu, bidx, o);
                const int ok_ = __shfl_xor_sync(0xffffffffu, brk, o);
                if (ov > bv || (ov == bv && oi < bidx)) { bv = ov; bidx = oi; brk = ok_; }
            }
            if (lane == 0) {
                win_s = bidx < N ? bidx : c;
                wr_s = bidx < N ? brk : -1;
            }
        }
        __syncthreads();
        const int p = win_s, rp = wr_s;
        const double pv = rp >= 0 ? __ldcg(g.candrow + ((size_t)par * P + rp) * nb + q) : 0.0;
        if (r == 0 && tid == 0) piv[(size_t)b * N + c] = p;
        if (p != c) sg = -sg;
        if (pv == 0.0) {
            singular = 1;
            continue;
        }
        if (tid == 0) pvs[q] = pv;     // its log after the panel, off the pivot chain
        if (pv < 0.0) sg = -sg;
        if (tid < nbe) prow[tid] = (tid == q) ? 1.0 / pv : __ldcg(g.candrow + ((size_t)par * P + rp) * nb + tid) / pv;
        // the owner of row p takes row c's old panel values
        if (p != c && p >= i0 && p < i0 + nr)
            for (int t = tid; t < nbe; t += GJ_THREADS) S[t * Rr + (p - i0)] = __ldcg(g.rowc + par * nb + t);
        __syncthreads();
        if (warp == GJ_THREADS / 32 - 1) {
            // the last warp interchanges rows c and p of X outside the panel
            // (its column share; the same lane takes the same columns at every
            // pivot, so the interchanges stay in order) while the others
            // eliminate: the round trip to memory leaves the pivot's chain
            if (p != c)
                for (int x = x0 + lane; x < x1; x += 32) {
                    if (x >= c0 && x < c0 + nbe) continue;
                    const double s = X[(size_t)c * ld + x];
                    X[(size_t)c * ld + x] = X[(size_t)p * ld + x];
                    X[(size_t)p * ld + x] = s;
                }
        } else {
            for (int li = tid; li < nr; li += GJ_THREADS - 32) {
                const int gi = i0 + li;
                if (gi == c) {
                    for (int t = 0; t < nbe; ++t) S[t * Rr + li] = prow[t];
                } else {
                    const double f = S[q * Rr + li];
                    S[q * Rr + li] = 0.0;
                    for (int t = 0; t < nbe; ++t) S[t * Rr + li] -= f * prow[t];
                }
            }
        }
        __syncthreads();
    }
    // every CTA's interchanges of X are done before the pivot rows are read
    if (!group_barrier(ctr, (++nbar) * P, status, budget_ns)) return;
    double *Ltb = Lt + (size_t)b * nb * ld;
    double *Rb = R + (size_t)b * nb * ld;
    for (int e = tid; e < nr * nbe; e += GJ_THREADS) {
        const int li = e / nbe, q = e - li * nbe, gi = i0 + li;
        const double v = S[q * Rr + li];
        X[(size_t)gi * ld + c0 + q] = v;
        Ltb[(size_t)q * ld + gi] = v - (gi == c0 + q ? 1.0 : 0.0);
    }
    for (int q = 0; q < nbe; ++q)
        for (int x = x0 + tid; x < x1; x += GJ_THREADS)
            Rb[(size_t)q * ld + x] = (x >= c0 && x < c0 + nbe) ? 0.0 : X[(size_t)(c0 + q) * ld + x];
    // log|det| of the panel's pivots, added in pivot order as one thread would
    // (the fp64 log of each pivot, on the slow fp64 pipe, stays off the chain
    // of pivot steps)
    if (r == 0 && warp == 0) {
        pvs_log[lane] = (lane < nbe && !singular) ? log(fabs(pvs[lane])) : 0.0;
        __syncwarp();
    }
    if (r == 0 && tid == 0) {
        for (int q = 0; q < nbe && !singular; ++q) la += pvs_log[q];
        if (singular) {
            atomicOr(status, ST_SINGULAR);
            lu_logabs[b] = -INFINITY;
            lu_sign[b] = 0;
        } else if (lu_sign[b] != 0) {
            lu_logabs[b] += la;
            lu_sign[b] *= sg;
        }
    }
}

// The same panel elimination over one thread-block cluster of GJ_CL CTAs per
// walker. Each pivot column costs one hardware cluster barrier instead of a
// group barrier in global memory. Every CTA writes its candidate (value,
// row, the row's panel values) and, if it owns row c, row c's panel values
// into a buffer of its own shared memory, alternating between two parities.
// After the barrier every CTA reads the GJ_CL candidates, the winner's row and
// row c from its siblings' shared memory. A CTA writes a parity again only
// after the next barrier, which its siblings pass only once they have read
// it. The interchange of rows c and p outside the panel goes to the last warp,
// beside the elimination. Every CTA executes the same sequence of cluster
// barriers (a singular pivot is seen by all), and a last barrier ends every
// read of a sibling's shared memory before any CTA exits.
constexpr int GJ_CL = 16;
__global__ void __launch_bounds__(GJ_THREADS) gj_panel_cl_kernel(int N, int ld, int nb, int c0, int nbe,
                                                                double *work, int *piv, double *Lt, double *R,
                                                                double *lu_logabs, int *lu_sign, int *status)
{
    extern __shared__ double S[];              // [nb][Rr]: column q of the CTA's rows at S + q*Rr
    __shared__ double cand_v[2], cand_row[2][GJ_NBMAX], rowc_b[2][GJ_NBMAX];
    __shared__ int cand_i[2];
    __shared__ double wval[GJ_THREADS / 32], prow[GJ_NBMAX], crow_s[GJ_NBMAX], rowc_s[GJ_NBMAX];
    __shared__ int widx[GJ_THREADS / 32], win_s, wr_s;
    __shared__ double pvs[GJ_NBMAX], pvs_log[32];
    constexpr int P = GJ_CL;
    const int b = blockIdx.x / P, r = blockIdx.x - b * P;       // r: the CTA's rank in its cluster
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int Rr = (N + P - 1) / P;
    const int i0 = min(N, r * Rr), nr = min(Rr, N - i0);
    double *X = work + (size_t)b * N * ld;
    const int xs = (N + P - 1) / P, x0 = min(N, r * xs), x1 = min(N, x0 + xs);

    for (int e = tid; e < nr * nbe; e += GJ_THREADS) {
        const int li = e / nbe, q = e - li * nbe;
        S[q * Rr + li] = X[(size_t)(i0 + li) * ld + c0 + q];
    }
    __syncthreads();
    double la = 0.0;
    int sg = 1, singular = 0;
    for (int q = 0; q < nbe; ++q) {
        const int c = c0 + q, par = q & 1;
        // the largest |x| as an integer key: the bit pattern of |x|, which orders
        // non-negative doubles as their values do (NaN below every candidate,
        // as an fp64 comparison leaves it), so that the search and its trees
        // compare on the integer pipe, not the fp64 one
        long long best = -1;
        int bi = N;
        for (int li = tid; li < nr; li += GJ_THREADS) {
            const int gi = i0 + li;
            if (gi < c) continue;
            const long long v = gj_key(S[q * Rr + li]);
            if (v > best || (v == best && gi < bi)) { best = v; bi = gi; }
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const long long ov = __shfl_xor_sync(0xffffffffu, best, o);
            const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
            if (ov > best || (ov == best && oi < bi)) { best = ov; bi = oi; }
        }
        if (lane == 0) { wval[warp] = __longlong_as_double(best); widx[warp] = bi; }
        __syncthreads();
        if (warp == 0) {
            best = lane < GJ_THREADS / 32 ? __double_as_longlong(wval[lane]) : -1;
            bi = lane < GJ_THREADS / 32 ? widx[lane] : N;
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                const long long ov = __shfl_xor_sync(0xffffffffu, best, o);
                const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
                if (ov > best || (ov == best && oi < bi)) { best = ov; bi = oi; }
            }
            if (lane == 0) {
                cand_v[par] = __longlong_as_double(best);
                cand_i[par] = bi;
                win_s = bi;
            }
        }
        __syncthreads();
        const int mine = win_s;
        if (mine < N && tid < nbe) cand_row[par][tid] = S[tid * Rr + (mine - i0)];
        if (c >= i0 && c < i0 + nr && tid >= 32 && tid < 32 + nbe) rowc_b[par][tid - 32] = S[(tid - 32) * Rr + (c - i0)];
        cl_barrier();
        // the winner: largest candidate, lowest row on ties, in a fixed order
        if (warp == 0) {
            long long bv = -1;
            int bidx = N, brk = 0;
            if (lane < P) {
                bv = __double_as_longlong(cl_ld_f64(cl_map(&cand_v[par], lane)));
                bidx = (int)cl_ld_acquire(cl_map(&cand_i[par], lane));
                brk = lane;
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                const long long ov = __shfl_xor_sync(0xffffffffu, bv, o);
                const int oi = __shfl_xor_sync(0xffffffffu, bidx, o);
                const int ok_ = __shfl_xor_sync(0xffffffffu, brk, o);
                if (ov > bv || (ov == bv && oi < bidx)) { bv = ov; bidx = oi; brk = ok_; }
            }
            if (lane == 0) {
                win_s = bidx < N ? bidx : c;
                wr_s = bidx < N ? brk : -1;
            }
        }
        __syncthreads();
        {
            const int rw = wr_s;
            if (tid < nbe) crow_s[tid] = rw >= 0 ? cl_ld_f64(cl_map(&cand_row[par][tid], rw)) : 0.0;
            else if (tid >= 32 && tid < 32 + nbe) rowc_s[tid - 32] = cl_ld_f64(cl_map(&rowc_b[par][tid - 32], c / Rr));
        }
        __syncthreads();
        const int p = win_s, rp = wr_s;
        const double pv = rp >= 0 ? crow_s[q] : 0.0;
        if (r == 0 && tid == 0) piv[(size_t)b * N + c] = p;
        if (p != c) sg = -sg;
        if (pv == 0.0) {
            singular = 1;
            continue;
        }
        if (tid == 0) pvs[q] = pv;     // its log after the panel, off the pivot chain
        if (pv < 0.0) sg = -sg;
        if (tid < nbe) prow[tid] = (tid == q) ? 1.0 / pv : crow_s[tid] / pv;
        // the owner of row p takes row c's old panel values
        if (p != c && p >= i0 && p < i0 + nr)
            for (int t = tid; t < nbe; t += GJ_THREADS) S[t * Rr + (p - i0)] = rowc_s[t];
        __syncthreads();
        if (warp == GJ_THREADS / 32 - 1) {
            if (p != c)
                for (int x = x0 + lane; x < x1; x += 32) {
                    if (x >= c0 && x < c0 + nbe) continue;
                    const double s = X[(size_t)c * ld + x];
                    X[(size_t)c * ld + x] = X[(size_t)p * ld + x];
                    X[(size_t)p * ld + x] = s;
                }
        } else {
            for (int li = tid; li < nr; li += GJ_THREADS - 32) {
                const int gi = i0 + li;
                if (gi == c) {
                    for (int t = 0; t < nbe; ++t) S[t * Rr + li] = prow[t];
                } else {
                    const double f = S[q * Rr + li];
                    S[q * Rr + li] = 0.0;
                    for (int t = 0; t < nbe; ++t) S[t * Rr + li] -= f * prow[t];
                }
            }
        }
        __syncthreads();
    }
    // every CTA's interchanges of X are done, and every read of a sibling's
    // shared memory, before the pivot rows are read and any CTA exits
    __threadfence();
    cl_barrier();
    double *Ltb = Lt + (size_t)b * nb * ld;
    double *Rb = R + (size_t)b * nb * ld;
    for (int e = tid; e < nr * nbe; e += GJ_THREADS) {
        const int li = e / nbe, q = e - li * nbe, gi = i0 + li;
        const double v = S[q * Rr + li];
        X[(size_t)gi * ld + c0 + q] = v;
        Ltb[(size_t)q * ld + gi] = v - (gi == c0 + q ? 1.0 : 0.0);
    }
    for (int q = 0; q < nbe; ++q)
        for (int x = x0 + tid; x < x1; x += GJ_THREADS)
            Rb[(size_t)q * ld + x] = (x >= c0 && x < c0 + nbe) ? 0.0 : X[(size_t)(c0 + q) * ld + x];
    // log|det| of the panel's pivots, added in pivot order as one thread would
    // (the fp64 log of each pivot, on the slow fp64 pipe, stays off the chain
    // of pivot steps)
    if (r == 0 && warp == 0) {
        pvs_log[lane] = (lane < nbe && !singular) ? log(fabs(pvs[lane])) : 0.0;
        __syncwarp();
    }
    if (r == 0 && tid == 0) {
        for (int q = 0; q < nbe && !singular; ++q) la += pvs_log[q];
        if (singular) {
            atomicOr(status, ST_SINGULAR);
            lu_logabs[b] = -INFINITY;
            lu_sign[b] = 0;
        } else if (lu_sign[b] != 0) {
            lu_logabs[b] += la;
            lu_sign[b] *= sg;
        }
    }
}

size_t gj_mc_scratch_bytes(int P, int nb) { return (gj_scratch_bytes(P, nb) + 255) / 256 * 256; }

// The cluster form of the panel (gj_panel_cl_kernel): one cluster of GJ_CL
// CTAs per walker. cudaErrorNotSupported where it cannot run (its shared
// memory, a panel wider than GJ_NBMAX, no co-resident cluster of that size).
static cudaError_t launch_gj_panel_cl(Ctx &c, int c0, int nbe)
{
    const int N = c.N, Rr = (N + GJ_CL - 1) / GJ_CL;
    const size_t smem = (size_t)c.nb * Rr * sizeof(double);
    if (c.nb > GJ_NBMAX || smem > 160 * 1024) return cudaErrorNotSupported;
    cudaError_t e = cudaFuncSetAttribute(gj_panel_cl_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(gj_panel_cl_kernel, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    if (e != cudaSuccess) return e;
    cudaLaunchConfig_t cfg = {};
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = GJ_CL;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.gridDim = dim3(c.batch * GJ_CL);
    cfg.blockDim = dim3(GJ_THREADS);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = c.stream;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    int ncl = 0;
    e = cudaOccupancyMaxActiveClusters(&ncl, (const void *)gj_panel_cl_kernel, &cfg);
    if (e != cudaSuccess) return e;
    if (ncl < 1) return cudaErrorNotSupported;
    return cudaLaunchKernelEx(&cfg, gj_panel_cl_kernel, N, c.ld, c.nb, c0, nbe, c.work, c.piv, c.Lt, c.R,
                              c.lu_logabs, c.lu_sign, c.status);
}

cudaError_t launch_gj_panel_mc(Ctx &c, int c0, int nbe)
{
    {
        const cudaError_t ec = launch_gj_panel_cl(c, c0, nbe);
        if (ec != cudaErrorNotSupported) return ec;
        cudaGetLastError();
    }
    const int P = c.gj_ctas, N = c.N;
    const int Rr = (N + P - 1) / P;
    const size_t smem = (size_t)c.nb * Rr * sizeof(double);
    cudaError_t e = cudaFuncSetAttribute(gj_panel_mc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    // its own counters: a serving pool recomputes admitted walkers on one
    // stream while its sweep runs on another
    e = cudaMemsetAsync(c.gj_ctr, 0, (size_t)c.batch * GJ_CTR_STRIDE * sizeof(unsigned), c.stream);
    if (e != cudaSuccess) return e;
    int n = N, ld = c.ld, nb = c.nb, cc0 = c0, nn = nbe, PP = P;
    size_t stride = gj_mc_scratch_bytes(P, c.nb);
    long long budget = c.opt_budget_ns;
    void *args[] = {&n, &ld, &nb, &cc0, &nn, &PP, &c.work, &c.piv, &c.Lt, &c.R, &c.lu_logabs, &c.lu_sign,
                    &c.status, &c.gj_ctr, &c.gj_scr, &stride, &budget};
    return cudaLaunchCooperativeKernel((const void *)gj_panel_mc_kernel, dim3(c.batch * P), dim3(GJ_THREADS), args,
                                       smem, c.stream);
}

// ---------------------------------------------------------------- per-call flush
// qmcdu_flush of fp64 walkers (K <= 32): the two N x N x k contractions of
// Eq. 4 emulated on the tensor cores by flush_oz, one walker at a time per
// group of CTAs, for the walkers whose queue holds at least kthresh moves.
// W = P Kinv is already in c.Wbuf. The exponents that the persistent sweep
// keeps up to date are computed here: columns of A^{-1}, rows of V.
__global__ void __launch_bounds__(STHREADS, 1) oz_flush_kernel(SweepParams<double> p, const int *kcount,
                                                              int kthresh)
{
    extern __shared__ __align__(128) unsigned char smem[];
    __shared__ uint32_t tmem_s;
    if (threadIdx.x < 32) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
                     ::"r"(tcf::su32(&tmem_s)), "n"(ozf::TMEM_COLS) : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (threadIdx.x == 0) {
        unsigned long long *bars = (unsigned long long *)(smem + p.off_tcbar);
        for (int q = 0; q < ozf::NBAR; ++q)
            asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;"
                         ::"r"(tcf::su32(&bars[q])), "r"(ozf::bar_count(q)) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    {
        const int grp = blockIdx.x / p.Gf, rank = blockIdx.x - grp * p.Gf;
        unsigned *flush_ctr = p.sync + SYNC_STRIDE * grp + 32;
        unsigned n_flush = 0, tph[8] = {0, 0, 0, 0, 0, 0, 0, 0};
        const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
        for (int w = grp; w < p.batch; w += p.ngroups) {
            const int k = __ldcg(kcount + w);
            if (k < kthresh || k < 1) continue;           // uniform for the group
            if (!oz_colexp_init(p, w, grp, rank, flush_ctr, n_flush,
                                (const double *)p.V + (size_t)w * p.K * p.ld, k)) break;
            if (rank == 0) {
                // exponents of V's scaled rows, max_i (E(V[m][i]) + s_i) (warp m: row m)
                int *vex = oz_vex(p, grp);
                const int *rex = (const int *)(p.oz + (size_t)grp * p.oz_stride + ozf::layout(p.N, p.kp).rex);
                const double *Vb = p.V + (size_t)w * p.K * p.ld;
                for (int m = warp; m < 64; m += SWARPS) {
                    int e = 0;
                    if (m < k)
                        for (int i = lane; i < p.N; i += 32) {
                            const double x = __ldcg(Vb + (size_t)m * p.ld + i);
                            if (ozf::nz(x)) e = max(e, ozf::bexp(x) + __ldcg(rex + i));
                        }
                    e = __reduce_max_sync(0xffffffffu, e);
                    if (lane == 0) vex[m] = e;
                }
            }
            if (!group_barrier(flush_ctr, (++n_flush) * p.Gf, p.status, p.budget_ns)) break;
            if (!flush_oz(p, w, k, grp, rank, smem, tmem_s, tph, flush_ctr, n_flush)) break;
            if (!group_barrier(flush_ctr, (++n_flush) * p.Gf, p.status, p.budget_ns)) break;
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (threadIdx.x < 32)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem_s), "n"(ozf::TMEM_COLS) : "memory");
}

// ---------------------------------------------------------------- recompute update
// The rank-nb update of the Gauss-Jordan recompute, X[c][i] += sum_m Lt[m][c]
// R[m][i] (X = A' row-major, the panel's multipliers Lt and pivot rows R, nb
// <= 32), as the emulated-fp64 contraction of the flush: it is phase C's
// A^{-1}[i][c] -= sum_m W[m][i] T[m][c] with W = R and T = -Lt. The slicing
// takes the place of phase B: queue entry m is balanced by 2^f_m on R's row
// and 2^-f_m on Lt's row, f_m half the difference of the two rows' largest
// exponents (found in a first pass over all CTAs of the group), then Lt's
// columns and R's rows are cut with one exponent each.
template <typename T>
__device__ bool oz_slice_lr(const SweepParams<T> &p, int k, int grp, int rank, const double *Lt,
                            const double *R, unsigned *flush_ctr, unsigned &n_flush)
{
    using namespace tcf;
    using namespace ozf;
    const int N = p.N, ld = p.ld, kp = p.kp, Gf = p.Gf;
    const Layout Ly = layout(N, kp);
    unsigned char *scr = p.oz + (size_t)grp * p.oz_stride;
    int *fex = (int *)(scr + Ly.fex);                // [0, 32) Lt rows, [32, 64) R rows
    __half *wsl = (__half *)(scr + Ly.wsl);
    __half *tsl = (__half *)(scr + Ly.tsl);
    int *wex = (int *)(scr + Ly.wex);
    int *tex = (int *)(scr + Ly.tex);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    // pass 1: the rows' largest exponents (fex cleared before the launch)
    for (int m = warp; m < 2 * k; m += SWARPS) {
        const double *row = (m < k ? Lt + (size_t)m * ld : R + (size_t)(m - k) * ld);
        int e = 0;
        for (int i = rank * 32 + lane; i < N; i += Gf * 32) e = max(e, bexp(__ldcg(row + i)));
        e = __reduce_max_sync(0xffffffffu, e);
        if (lane == 0 && e > 0) atomicMax(fex + (m < k ? m : 32 + m - k), e);
    }
    if (!group_barrier(flush_ctr, (++n_flush) * Gf, p.status, p.budget_ns)) return false;
    __shared__ int fs[32];
    if (tid < 32) fs[tid] = tid < k ? (__ldcg(fex + tid) - __ldcg(fex + 32 + tid)) >> 1 : 0;
    __syncthreads();
    // T = -Lt: eight consecutive m per thread, the kp / 8 threads of a column
    // adjacent in the warp (as phase B)
    const int ng = kp / 8;
    const int totT = N * ng;
    for (int base = rank * STHREADS; base < totT; base += Gf * STHREADS) {
        const int e = base + tid;
        const bool in = e < totT;
        const int c = in ? e / ng : 0, m0 = (e - (e / ng) * ng) * 8;
        double t[8];
#pragma unroll
        for (int q = 0; q < 8; ++q) t[q] = (in && m0 + q < k) ? -__ldcg(Lt + (size_t)(m0 + q) * ld + c) : 0.0;
        int em = 0;
#pragma unroll
        for (int q = 0; q < 8; ++q)
            if (nz(t[q])) em = max(em, bexp(t[q]) - fs[m0 + q]);
        for (int o = 1; o < ng; o <<= 1) em = max(em, __shfl_xor_sync(0xffffffffu, em, o));
        if (in) {
            int emq[8];
#pragma unroll
            for (int q = 0; q < 8; ++q) emq[q] = em + fs[m0 + q];
            uint4 sl[NS];
            slice8(t, emq, sl);
            const int ct = c / CN;
            const uint32_t o = coff(c - ct * CN, m0, kp) >> 1;
#pragma unroll
            for (int j = 0; j < NS; ++j)
                *reinterpret_cast<uint4 *>(tsl + ((size_t)ct * NS + j) * CN * kp + o) = sl[j];
            if (m0 == 0) tex[c] = em;
        }
    }
    // W = R: one thread per row i, all kp values of m
    for (int i = rank * STHREADS + tid; i < N; i += Gf * STHREADS) {
        double x[32];
        int em = 0;
#pragma unroll
        for (int m = 0; m < 32; ++m) {
            x[m] = (m < k) ? __ldcg(R + (size_t)m * ld + i) : 0.0;
            if (nz(x[m])) em = max(em, bexp(x[m]) + fs[m]);
        }
        const int rb = i / CM;
#pragma unroll
        for (int g = 0; g < 4; ++g) {
            if (g * 8 < kp) {
                double y[8];
                int emq[8];
#pragma unroll
                for (int q = 0; q < 8; ++q) {
                    y[q] = x[g * 8 + q];
                    emq[q] = em - fs[g * 8 + q];
                }
                uint4 sl[NS];
                slice8(y, emq, sl);
                const uint32_t o = coff(i - rb * CM, g * 8, kp) >> 1;
#pragma unroll
                for (int j = 0; j < NS; ++j)
                    *reinterpret_cast<uint4 *>(wsl + ((size_t)rb * NS + j) * CM * kp + o) = sl[j];
            }
        }
        wex[i] = em;
    }
    return true;
}

// One update of every walker's X (walker groups as in oz_flush_kernel); k
// the panel's width (<= kp = 32). fex of every group is cleared before the
// launch.
__global__ void __launch_bounds__(STHREADS, 1) oz_gj_update_kernel(SweepParams<double> p, const double *Lt,
                                                                   const double *R, int nb, int k)
{
    extern __shared__ __align__(128) unsigned char smem[];
    __shared__ uint32_t tmem_s;
    if (threadIdx.x < 32) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
                     ::"r"(tcf::su32(&tmem_s)), "n"(ozf::TMEM_COLS) : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (threadIdx.x == 0) {
        unsigned long long *bars = (unsigned long long *)(smem + p.off_tcbar);
        for (int q = 0; q < ozf::NBAR; ++q)
            asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;"
                         ::"r"(tcf::su32(&bars[q])), "r"(ozf::bar_count(q)) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    {
        const int grp = blockIdx.x / p.Gf, rank = blockIdx.x - grp * p.Gf;
        unsigned *flush_ctr = p.sync + SYNC_STRIDE * grp + 32;
        unsigned n_flush = 0, tph[8] = {0, 0, 0, 0, 0, 0, 0, 0};
        for (int w = grp; w < p.batch; w += p.ngroups) {
            const double *Ltw = Lt + (size_t)w * nb * p.ld, *Rw = R + (size_t)w * nb * p.ld;
            if (w != grp) {
                // the group's fex is cleared for each further walker (the first
                // is cleared before the launch)
                if (rank == 0 && threadIdx.x < 64) ((int *)(p.oz + (size_t)grp * p.oz_stride +
                                                            ozf::layout(p.N, p.kp).fex))[threadIdx.x] = 0;
                if (!group_barrier(flush_ctr, (++n_flush) * p.Gf, p.status, p.budget_ns)) break;
            }
            if (!oz_slice_lr(p, k, grp, rank, Ltw, Rw, flush_ctr, n_flush)) break;
            if (!group_barrier(flush_ctr, (++n_flush) * p.Gf, p.status, p.budget_ns)) break;
            if (!oz_phase_c(p, w, k, grp, rank, smem, tmem_s, tph)) break;
            if (!group_barrier(flush_ctr, (++n_flush) * p.Gf, p.status, p.budget_ns)) break;
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (threadIdx.x < 32)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem_s), "n"(ozf::TMEM_COLS) : "memory");
}

// cudaErrorNotSupported when the emulated update does not apply (the caller
// then takes the fp64 tile GEMM).
cudaError_t launch_gj_update_oz(Ctx &c, int nbe)
{
    constexpr int KP = 32;
    // the handle owns the GPU (no group shape or grid cap: a serving pool
    // recomputes admitted walkers on a second stream while its sweep, which
    // shares this scratch, runs)
    if (c.prec != QMCDU_FP64 || !c.oz || c.oz_groups < 1 || c.opt_fp64_flush == 1 || nbe < 1 || nbe > KP ||
        c.nb > KP || c.oz_stride < ozf::layout(c.N, KP).bytes || c.opt_group_ctas != 0 || c.opt_max_ctas != 0)
        return cudaErrorNotSupported;
    const size_t smem = std::max((size_t)OZ_MIN_SMEM, ozf::region_bytes(KP));
    cudaError_t e = cudaFuncSetAttribute(oz_gj_update_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return e;
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, oz_gj_update_kernel, STHREADS, smem);
    if (e != cudaSuccess) return e;
    if (per_sm != 1) return cudaErrorNotSupported;     // the TMEM allocation would wait
    const int ngroups = std::min(c.batch, c.oz_groups);
    const int Gf = c.num_sms / ngroups;
    if (Gf < 2 || ngroups * SYNC_STRIDE > c.sync_words) return cudaErrorNotSupported;
    SweepParams<double> p{};
    p.N = c.N; p.K = KP; p.ld = c.ld; p.batch = c.batch;
    p.Gf = Gf; p.Gr = 1; p.ngroups = ngroups;
    p.Ainv = c.work;                 // X[c][i] at c * ld + i: phase C's column c, row i
    p.sync = c.sw_sync; p.status = c.status;
    p.budget_ns = c.opt_budget_ns;
    p.kp = KP; p.oz = c.oz; p.oz_stride = c.oz_stride;
    p.off_xs = 0;
    p.off_tcbar = (int)ozf::bar_offset(KP);
    p.phase_ns = nullptr;
    e = cudaMemsetAsync(c.sw_sync, 0, (size_t)ngroups * SYNC_STRIDE * sizeof(unsigned), c.stream);
    if (e != cudaSuccess) return e;
    const size_t fex = ozf::layout(c.N, KP).fex;
    for (int g = 0; g < ngroups; ++g) {
        e = cudaMemsetAsync(c.oz + (size_t)g * c.oz_stride + fex, 0, 64 * sizeof(int), c.stream);
        if (e != cudaSuccess) return e;
    }
    const double *Lt = c.Lt, *R = c.R;
    int nb = c.nb, k = nbe;
    void *args[] = {&p, &Lt, &R, &nb, &k};
    return cudaLaunchCooperativeKernel((const void *)oz_gj_update_kernel, dim3(ngroups * Gf), dim3(STHREADS),
                                       args, smem, c.stream);
}

// cudaErrorNotSupported when the emulated flush does not apply (the caller
// then takes the fp64 GEMMs).
cudaError_t launch_flush_oz(Ctx &c, int kthresh)
{
    const int K = c.K;
    if (c.prec != QMCDU_FP64 || K > 32 || K < SMALL_K || !c.oz || c.oz_groups < 1 || c.opt_fp64_flush == 1)
        return cudaErrorNotSupported;
    const int kp = (K + 15) / 16 * 16;
    const size_t smem = std::max((size_t)OZ_MIN_SMEM, ozf::region_bytes(kp));
    cudaError_t e = cudaFuncSetAttribute(oz_flush_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, oz_flush_kernel, STHREADS, smem);
    if (e != cudaSuccess) return e;
    if (per_sm != 1) return cudaErrorNotSupported;     // the TMEM allocation would wait
    const int ngroups = std::min(c.batch, c.oz_groups);
    const int Gf = c.num_sms / ngroups;
    if (Gf < 2 || ngroups * SYNC_STRIDE > c.sync_words) return cudaErrorNotSupported;
    SweepParams<double> p{};
    p.N = c.N; p.K = K; p.ld = c.ld; p.batch = c.batch;
    p.Gf = Gf; p.Gr = 1; p.ngroups = ngroups;
    p.Ainv = (double *)c.Ainv; p.W = (double *)c.Wbuf; p.V = (double *)c.V;
    p.idx = c.idx; p.kglob = c.kcount;
    p.sync = c.sw_sync; p.status = c.status;
    p.budget_ns = c.opt_budget_ns;
    p.kp = kp; p.oz = c.oz; p.oz_stride = c.oz_stride;
    p.off_xs = 0;
    p.off_tcbar = (int)ozf::bar_offset(kp);
    p.phase_ns = nullptr;
    e = cudaMemsetAsync(c.sw_sync, 0, (size_t)ngroups * SYNC_STRIDE * sizeof(unsigned), c.stream);
    if (e != cudaSuccess) return e;
    void *args[] = {&p, &c.kcount, &kthresh};
    return cudaLaunchCooperativeKernel((const void *)oz_flush_kernel, dim3(ngroups * Gf), dim3(STHREADS), args,
                                       smem, c.stream);
}

cudaError_t launch_sweep(Ctx &c, const SweepLaunch &L)
{
    // the sweep's proposal draws, then the sweep, then the running log-det
    const int nw = L.wlist ? L.nlist : c.batch;
    if (nw == 0) return cudaSuccess;
    sweep_draw_kernel<<<c.num_sms * 8, 256, 0, c.stream>>>(c.N, c.ld, nw, L.seed, L.sweep,
                                                           L.params, L.sweep_offset, L.wlist,
                                                           L.wseed, L.wsweep, c.sw_gauss,
                                                           c.sw_unif);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    e = prof_begin(&c, c.ev_sweep);
    if (e != cudaSuccess) return e;
    e = c.prec == QMCDU_FP64 ? launch_sweep_t<double>(c, L) : launch_sweep_t<float>(c, L);
    if (e != cudaSuccess) return e;
    e = prof_end(&c, c.ev_sweep);
    if (e != cudaSuccess) return e;
    sweep_logdet_kernel<<<nw, STHREADS, 0, c.stream>>>(c.N, L.wlist, L.acc_out, L.ratio_out, c.logabs,
                                                            c.sign);
    return cudaGetLastError();
}

}  // namespace qmcdu
