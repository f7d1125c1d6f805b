// kernels_move.cu -- per-proposal kernels of the delayed update.
//
// ratio_stage_kernel, ratio_dots_kernel, ratio_finish_kernel : determinant
//                 ratio of one proposal per walker (Eq. 1 at k = 0, Eq. 3
//                 through the queued panels otherwise). GEMV class: reads
//                 A^{-1}[:, j], the change u = v - a_j, the k queued rows of
//                 P and V (streamed by bulk copies) and the k x k Kinv.
//
// The change form of the paper (Eq. 1-4): a move of electron j to the new row
// v changes A by e_j u' with u = v - a_j, and the ratio is 1 + u . A^{-1}[:, j]
// (Eq. 1). The queue holds the changes of the accepted moves (V row m = u_m),
// the columns P = A^{-1}[:, idx] of the inverse at the last flush and
// Kinv = (I + V'P)^{-1}, the inverse of the k x k matrix of Eq. 3.
// accept_kernel : Metropolis decision (or a given mask), append to the delay
//                 queue with the bordered k x k inverse update, new row of A,
//                 running log|det A|.
// sm_update_kernel : K = 1, Sherman-Morrison (Eq. 2) as one fused pass over
//                 A^{-1}: per column, a dot product with v and a rank-1 axpy.
#include <math.h>

#include <algorithm>
#include <type_traits>

#include "bulk.cuh"
#include "philox.cuh"
#include "qmcdu_internal.cuh"

namespace qmcdu {

constexpr int RTHREADS = 256;  // 8 warps

template <typename T>
struct RatioParams {
    int N, K, ld;
    const double *A;
    const T *Ainv;
    T *P, *V;
    double *vstash;
    const double *Kinv;
    const int *kcount;
    double *rs;
    double *partial;
    int *status;
    const double *v_in;
    const int *elec;
    int uniform_elec;
    int generate;
    unsigned long long seed;
    int sweep;
    double sigma;
    double *ratio_out;
};

__device__ __forceinline__ double warp_sum(double v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}
__device__ __forceinline__ float warp_sum(float v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

__device__ __forceinline__ void fma16(double &acc, double2 x, double2 y)
{
    acc = fma(x.x, y.x, acc);
    acc = fma(x.y, y.y, acc);
}
__device__ __forceinline__ void fma16(float &acc, float4 x, float4 y)
{
    acc = fmaf(x.x, y.x, acc);
    acc = fmaf(x.y, y.y, acc);
    acc = fmaf(x.z, y.z, acc);
    acc = fmaf(x.w, y.w, acc);
}

template <typename T>
struct Vec16;
template <>
struct Vec16<double> {
    using type = double2;
    static __device__ __forceinline__ double2 zero() { return make_double2(0.0, 0.0); }
};
template <>
struct Vec16<float> {
    using type = float4;
    static __device__ __forceinline__ float4 zero() { return make_float4(0.f, 0.f, 0.f, 0.f); }
};

// The ratio of one proposal per walker (Eq. 1 at k = 0, Eq. 3 through the
// queued panels otherwise) in three launches:
//   ratio_stage_kernel   u and A^{-1}[:, j] into slot k of V and P (the slot a
//                        subsequent accept fills; the rows the dots read),
//                        v (fp64) into the stash the accept copies into A
//   ratio_dots_kernel    the 2k+1 full-row dot products of every walker,
//                          d = u . A^{-1}[:, j],  b_m = P[m] . u,  c_m = V[m] . A^{-1}[:, j]:
//                        grid-stride over (walker, row), one warp per row, so
//                        that every warp streams rows from HBM the whole time
//   ratio_finish_kernel  per walker (one CTA): x = Kinv c and y = Kinv' b in
//                        one coalesced pass over Kinv, r = 1 + (d - b' Kinv c)
//                        (the Schur complement of the bordered I + V'P, Eq. 3)
// Rows are padded to ld with zeros (nothing writes past N), so 16-byte vectors
// that reach into the padding add nothing.

template <typename T>
__global__ void __launch_bounds__(RTHREADS) ratio_stage_kernel(RatioParams<T> p)
{
    const int b = blockIdx.y;
    const int N = p.N, K = p.K, ld = p.ld;
    const int k = p.kcount[b];
    const int j = p.elec ? p.elec[b] : p.uniform_elec;
    if (j < 0 || j >= N || k < 0 || k >= K) {
        if (threadIdx.x == 0 && blockIdx.x == 0) atomicOr(p.status, ST_BADARG);
        return;
    }
    const size_t wN = (size_t)N * ld, wK = (size_t)K * ld;
    const T *acol = p.Ainv + b * wN + (size_t)j * ld;
    T *Pk = p.P + b * wK + (size_t)k * ld;
    T *Vk = p.V + b * wK + (size_t)k * ld;
    const int i0 = blockIdx.x * (2 * RTHREADS);
    for (int i = i0 + threadIdx.x; i < min(N, i0 + 2 * RTHREADS); i += RTHREADS) Pk[i] = acol[i];
    const double *arow = p.A + b * wN + (size_t)j * ld;
    double *vst = p.vstash + (size_t)b * ld;
    if (p.generate) {
        // v = a_j + sigma g, g from Philox / Box-Muller in pairs
        const unsigned long long wseed = p.seed + (unsigned long long)b;
        const int i = i0 + 2 * threadIdx.x;
        if (i < N) {
            const double2 g = proposal_gaussian_pair(wseed, j, p.sweep, i >> 1);
            const double v0 = __dadd_rn(arow[i], __dmul_rn(p.sigma, g.x));
            Vk[i] = (T)__dsub_rn(v0, arow[i]);
            vst[i] = v0;
            if (i + 1 < N) {
                const double v1 = __dadd_rn(arow[i + 1], __dmul_rn(p.sigma, g.y));
                Vk[i + 1] = (T)__dsub_rn(v1, arow[i + 1]);
                vst[i + 1] = v1;
            }
        }
    } else {
        for (int i = i0 + threadIdx.x; i < min(N, i0 + 2 * RTHREADS); i += RTHREADS) {
            const double v0 = p.v_in[(size_t)b * N + i];
            Vk[i] = (T)__dsub_rn(v0, arow[i]);
            vst[i] = v0;
        }
    }
}

constexpr int TSEG = 4096;   // bytes of a streamed row segment (one bulk copy)
constexpr int TNS = 16;      // stages of the segment ring
constexpr int TRU = 32;      // rows per CTA of the dots
constexpr int TMAXSEG = 16;  // segments per row at most (rows of <= 64 KB: N <= 8192 in fp64)
constexpr int TTHREADS = 288;  // 8 consumer warps + 1 producer warp

static size_t dots_smem_bytes(size_t rowbytes)
{
    return 512 + (size_t)TRU * TMAXSEG * sizeof(double) + rowbytes + (size_t)TNS * TSEG;
}

// Rows of walker b are the jobs t = 0..2k: t = 0 the A^{-1} column (P row k),
// t = 1..k P row t-1, both against v (V row k); t = k+1..2k V row t-k-1
// against the column (P row k). Grid (U, batch): CTA u takes up to TRU rows
// that share their vector, units 0..U/2-1 the rows against v and U/2..U-1 the
// rows against the column (U = 2 ceil((kmax + 1) / TRU); a walker's units past
// its own k return at once).
//
// The vector goes to shared memory in one bulk copy; the rows stream through a
// ring of TNS segment buffers of 4 KB: the producer warp issues
// cp.async.bulk copies (completion counted in bytes on the stage's "full"
// mbarrier) as soon as the stage's "empty" mbarrier says its last segment was
// read; consumer warp w takes segments w, w + 8, ... and leaves one partial sum
// per (row, segment). Every wait is bounded: on a timeout the CTA stops, flags
// ST_TIMEOUT and waits (bounded) for its copies in flight before it exits.
template <typename T>
__global__ void __launch_bounds__(TTHREADS) ratio_dots_kernel(RatioParams<T> p, int U,
                                                              long long budget_ns)
{
    using V16 = typename Vec16<T>::type;
    extern __shared__ __align__(128) unsigned char tsm[];
    unsigned long long *full = reinterpret_cast<unsigned long long *>(tsm);
    unsigned long long *empty = full + TNS;
    unsigned long long *wbar = empty + TNS;
    double *part = reinterpret_cast<double *>(tsm + 512);                    // [TRU][TMAXSEG]
    unsigned char *wv = tsm + 512 + TRU * TMAXSEG * sizeof(double);          // the shared vector
    const int K = p.K, ld = p.ld;
    const unsigned rowbytes = (unsigned)ld * sizeof(T);                     // a multiple of 128
    unsigned char *ring = wv + rowbytes;                                     // [TNS][TSEG]
    __shared__ int abort_s, issued_s;

    const int b = blockIdx.y, u = blockIdx.x, half = U / 2;
    const int k = p.kcount[b];
    if (k < 0 || k >= K) return;                      // flagged by the stage kernel
    const size_t wK = (size_t)K * ld;
    const T *Pw = p.P + b * wK, *Vw = p.V + b * wK;
    int rb, re;
    const T *with;
    if (u < half) {
        rb = u * TRU;
        re = min(rb + TRU, k + 1);
        with = Vw + (size_t)k * ld;
    } else {
        rb = k + 1 + (u - half) * TRU;
        re = min(rb + TRU, 2 * k + 1);
        with = Pw + (size_t)k * ld;
    }
    if (rb >= re) return;
    const int nrows = re - rb;
    const int nseg = (int)((rowbytes + TSEG - 1) / TSEG);
    const int items = nrows * nseg;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

    if (threadIdx.x == 0) {
        for (int s = 0; s < TNS; ++s) {
            mbar_init_count(&full[s], 1);
            mbar_init_count(&empty[s], 1);
        }
        mbar_init_count(wbar, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        abort_s = 0;
        issued_s = 0;
    }
    __syncthreads();

    if (warp == 8) {
        // producer: one lane issues every copy
        if (lane == 0) {
            mbar_expect(wbar, rowbytes);
            bulk_g2s(wv, with, rowbytes, wbar);
            int i = 0;
            for (; i < items; ++i) {
                const int s = i % TNS;
                if (i >= TNS && !mbar_wait(&empty[s], ((i / TNS) - 1) & 1, p.status, budget_ns)) {
                    abort_s = 1;
                    break;
                }
                if (*(volatile int *)&abort_s) break;
                const int r = i / nseg, sg = i - r * nseg;
                const int t = rb + r;
                const T *row = t == 0 ? Pw + (size_t)k * ld
                                      : (t <= k ? Pw + (size_t)(t - 1) * ld : Vw + (size_t)(t - 1 - k) * ld);
                const unsigned off = (unsigned)sg * TSEG;
                const unsigned bytes = min((unsigned)TSEG, rowbytes - off);
                mbar_expect(&full[s], bytes);
                bulk_g2s(ring + (size_t)s * TSEG, reinterpret_cast<const unsigned char *>(row) + off,
                         bytes, &full[s]);
            }
            issued_s = i;
        }
    } else {
        // consumers
        bool ok = mbar_wait(wbar, 0, p.status, budget_ns);
        for (int i = warp; ok && i < items; i += 8) {
            const int s = i % TNS;
            if (!mbar_wait(&full[s], (i / TNS) & 1, p.status, budget_ns) ||
                *(volatile int *)&abort_s) {
                ok = false;
                break;
            }
            const int r = i / nseg, sg = i - r * nseg;
            const unsigned off = (unsigned)sg * TSEG;
            const int nv = (int)(min((unsigned)TSEG, rowbytes - off) / 16);
            const V16 *x = reinterpret_cast<const V16 *>(ring + (size_t)s * TSEG);
            const V16 *w = reinterpret_cast<const V16 *>(wv + off);
            T acc = 0;
#pragma unroll 4
            for (int v = lane; v < nv; v += 32) fma16(acc, x[v], w[v]);
            acc = warp_sum(acc);
            __syncwarp();
            if (lane == 0) {
                part[r * TMAXSEG + sg] = (double)acc;
                mbar_arrive(&empty[s]);
            }
        }
        if (!ok) abort_s = 1;
    }
    __syncthreads();
    if (abort_s) {
        // copies issued but not waited for may still be landing: wait for the
        // last TNS of them (bounded) before the CTA's shared memory goes away
        if (threadIdx.x == 0) {
            const int n = issued_s;
            for (int i = max(0, n - TNS); i < n; ++i)
                mbar_wait(&full[i % TNS], (i / TNS) & 1, p.status, budget_ns);
            mbar_wait(wbar, 0, p.status, budget_ns);
        }
        __syncthreads();
        return;
    }
    if (threadIdx.x < nrows) {
        double d = 0.0;
        for (int sg = 0; sg < nseg; ++sg) d += part[threadIdx.x * TMAXSEG + sg];
        p.partial[(size_t)b * (2 * K + 1) + rb + threadIdx.x] = d;
    }
}

// The same dot products by persistent CTAs. Items are (walker, 32 consecutive
// rows t of that walker's 2k + 1); CTA x takes items x, x + grid, ... Warp 8
// loads, per item, both of the walker's vectors (u, for rows t <= k, and the
// column, for the rest) into one of two vector buffers. Consumer warp w takes
// rows w, w + 8, ... of each item and streams their segments through a ring
// of SPW slots of its own: its lane 0 issues the bulk copies SPW segments
// ahead of the reads, across item boundaries, and the warp waits for each in
// turn, so that every warp keeps SPW copies in flight with no producer in
// between (one producer lane for all warps issued too slowly: 21% of HBM at
// 128 x N = 512, fp32; per-warp copies drained at each item: 36%). A slot is
// refilled only by the warp that has just read it (after a proxy fence), so a
// wait on a fill's phase parity is never answered by an older fill. When a
// warp is done with an item it releases the item's vector buffer. Waits are
// bounded as in ratio_dots_kernel.
constexpr int PRU = 32;      // rows per item
constexpr int SPW = 4;       // ring slots of each consumer warp
template <typename T>
__global__ void __launch_bounds__(TTHREADS) ratio_dots_persist_kernel(RatioParams<T> p, int U, int nitems,
                                                                      long long budget_ns)
{
    using V16 = typename Vec16<T>::type;
    extern __shared__ __align__(128) unsigned char tsm[];
    unsigned long long *full = reinterpret_cast<unsigned long long *>(tsm);   // [8][SPW]
    unsigned long long *vfull = full + 8 * SPW;                               // [2]
    unsigned long long *vempty = vfull + 2;                                   // [2]
    const int K = p.K, ld = p.ld;
    const unsigned rowbytes = (unsigned)ld * sizeof(T);                      // a multiple of 128
    const unsigned slot = min((unsigned)TSEG, rowbytes);                      // bytes per ring slot
    unsigned char *vec = tsm + 512;                                          // [2][u, column][rowbytes]
    unsigned char *ring = vec + 4 * (size_t)rowbytes;                        // [8][SPW][slot]
    __shared__ int abort_s, nvec_s, issued_cnt[8];
    const int nseg = (int)((rowbytes + slot - 1) / slot);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const size_t wK = (size_t)K * ld;

    if (threadIdx.x == 0) {
        for (int s = 0; s < 8 * SPW; ++s) mbar_init_count(&full[s], 1);
        for (int q = 0; q < 2; ++q) {
            mbar_init_count(&vfull[q], 1);
            mbar_init_count(&vempty[q], 8);
        }
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        abort_s = 0;
        nvec_s = 0;
        for (int w = 0; w < 8; ++w) issued_cnt[w] = 0;
    }
    __syncthreads();

    // item -> walker b, first row rb, rows nrows (0: nothing to do)
    auto item = [&](int it, int &b, int &k, int &rb, int &nrows) {
        b = it / U;
        const int u = it - b * U;
        k = p.kcount[b];
        rb = u * PRU;
        nrows = (k < 0 || k >= K) ? 0 : max(0, min(rb + PRU, 2 * k + 1) - rb);
    };

    if (warp == 8) {
        // the vectors of every item, two buffers ahead
        if (lane == 0) {
            int nv = 0;
            for (int it = blockIdx.x; it < nitems && !*(volatile int *)&abort_s; it += gridDim.x) {
                int b, k, rb, nrows;
                item(it, b, k, rb, nrows);
                if (nrows == 0) continue;
                const int buf = nv & 1;
                if (nv >= 2 && !mbar_wait(&vempty[buf], ((nv >> 1) - 1) & 1, p.status, budget_ns)) {
                    abort_s = 1;
                    break;
                }
                const T *Pw = p.P + b * wK, *Vw = p.V + b * wK;
                mbar_expect(&vfull[buf], 2 * rowbytes);
                bulk_g2s(vec + (size_t)(2 * buf) * rowbytes, Vw + (size_t)k * ld, rowbytes, &vfull[buf]);
                bulk_g2s(vec + (size_t)(2 * buf + 1) * rowbytes, Pw + (size_t)k * ld, rowbytes, &vfull[buf]);
                ++nv;
                nvec_s = nv;
            }
        }
    } else {
        unsigned long long *myfull = full + warp * SPW;
        unsigned char *myring = ring + (size_t)warp * SPW * slot;
        // This warp's segments form one stream over its items: rows r = warp,
        // warp + 8, ... of each item, nseg segments per row. Lane 0 keeps an
        // issue cursor SPW segments ahead of the reads, across item
        // boundaries, so that the warp's copies stay in flight between items.
        struct Cur { int it, j, m, b, k, rb; };
        auto seek = [&](Cur &q, int it) {       // the first item >= it with segments for this warp
            q.j = 0;
            for (q.it = it; q.it < nitems; q.it += gridDim.x) {
                int nrows;
                item(q.it, q.b, q.k, q.rb, nrows);
                const int myrows = nrows > warp ? (nrows - warp + 7) / 8 : 0;
                q.m = myrows * nseg;
                if (q.m > 0) return;
            }
            q.m = 0;
        };
        Cur is = {nitems, 0, 0, 0, 0, 0};         // issue cursor (lane 0)
        int n_issued = 0;
        auto issue_next = [&]() {
            if (is.it >= nitems) return;
            const int r = warp + 8 * (is.j / nseg), sg = is.j - (is.j / nseg) * nseg;
            const int t = is.rb + r, kk = is.k;
            const T *Pw = p.P + is.b * wK, *Vw = p.V + is.b * wK;
            const T *row = t == 0 ? Pw + (size_t)kk * ld
                                  : (t <= kk ? Pw + (size_t)(t - 1) * ld : Vw + (size_t)(t - 1 - kk) * ld);
            const int s = n_issued % SPW;
            const unsigned off = (unsigned)sg * slot;
            const unsigned bytes = min(slot, rowbytes - off);
            mbar_expect(&myfull[s], bytes);
            bulk_g2s(myring + (size_t)s * slot, reinterpret_cast<const unsigned char *>(row) + off, bytes,
                     &myfull[s]);
            ++n_issued;
            issued_cnt[warp] = n_issued;
            if (++is.j == is.m) seek(is, is.it + gridDim.x);
        };
        if (lane == 0) {
            seek(is, blockIdx.x);
            for (int q = 0; q < SPW; ++q) issue_next();
        }
        int nv = 0, c = 0;        // c: segments this warp has read
        bool ok = true;
        for (int it = blockIdx.x; ok && it < nitems; it += gridDim.x) {
            int b, k, rb, nrows;
            item(it, b, k, rb, nrows);
            if (nrows == 0) continue;
            const int buf = nv & 1;
            const int myrows = nrows > warp ? (nrows - warp + 7) / 8 : 0;
            const int m = myrows * nseg;
            if (!mbar_wait(&vfull[buf], (nv >> 1) & 1, p.status, budget_ns) || *(volatile int *)&abort_s) {
                ok = false;
                break;
            }
            T acc = 0;
            for (int j = 0; j < m; ++j) {
                const int n = c + j, s = n % SPW, sg = j - (j / nseg) * nseg;
                if (!mbar_wait(&myfull[s], (n / SPW) & 1, p.status, budget_ns) || *(volatile int *)&abort_s) {
                    ok = false;
                    break;
                }
                const int t = rb + warp + 8 * (j / nseg);
                const V16 *wv = reinterpret_cast<const V16 *>(vec + (size_t)(2 * buf + (t <= k ? 0 : 1)) * rowbytes) +
                                sg * (slot / 16);
                const int nvv = (int)(min(slot, rowbytes - (unsigned)sg * slot) / 16);
                const V16 *x = reinterpret_cast<const V16 *>(myring + (size_t)s * slot);
#pragma unroll 4
                for (int v = lane; v < nvv; v += 32) fma16(acc, x[v], wv[v]);
                if (sg == nseg - 1) {
                    const T tot = warp_sum(acc);
                    if (lane == 0) p.partial[(size_t)b * (2 * K + 1) + t] = (double)tot;
                    acc = 0;
                }
                // every lane's reads of slot s are done before the copy that refills it
                asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                __syncwarp();
                if (lane == 0) issue_next();
            }
            if (!ok) break;
            c += m;
            __syncwarp();
            if (lane == 0) mbar_arrive(&vempty[buf]);
            ++nv;
        }
        if (!ok) abort_s = 1;
    }
    __syncthreads();
    if (abort_s) {
        // copies issued but not waited for may still be landing: wait for each
        // warp's last SPW segments and the last two vector loads (bounded)
        // before the CTA's shared memory goes away
        if (threadIdx.x == 0) {
            for (int w = 0; w < 8; ++w)
                for (int n = max(0, issued_cnt[w] - SPW); n < issued_cnt[w]; ++n)
                    mbar_wait(&full[w * SPW + n % SPW], (n / SPW) & 1, p.status, budget_ns);
            const int nv = nvec_s;
            for (int q = max(0, nv - 2); q < nv; ++q)
                mbar_wait(&vfull[q & 1], (q >> 1) & 1, p.status, budget_ns);
        }
        __syncthreads();
    }
}

// The k x k pass, one CTA per walker (grid = batch), over parts of 32 rows of
// Kinv in turn: in part p, warp w takes rows 32 p + 4 w .. + 3, its lanes the
// columns q = lane, lane + 32, ...; x_m = (Kinv c)_m is a fixed shuffle tree
// over the lanes; each lane's share of y = Kinv' b over the warp's four rows
// and each warp's share of b.x are added over the warps in warp order, and the
// parts in part order: r = 1 + (d - b.x) (the Schur complement of the
// bordered I + V'P, Eq. 3), deterministic, with no cross-CTA hand-off, and in
// the association of the earlier kernel that took one CTA per part (the
// bordered update of Kinv that x and y feed amplifies rounding differences on
// ill-conditioned walks).
template <typename T>
__global__ void __launch_bounds__(RTHREADS) ratio_finish_kernel(RatioParams<T> p)
{
    const int b = blockIdx.x;
    const int N = p.N, K = p.K;
    const int k = p.kcount[b];
    const int j = p.elec ? p.elec[b] : p.uniform_elec;
    if (j < 0 || j >= N || k < 0 || k >= K) return;     // flagged by the stage kernel
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int njobs = 2 * k + 1;
    constexpr int QL = QMCDU_MAX_K / 32;
    __shared__ double red[2 * QMCDU_MAX_K + 1];
    __shared__ double ypart[RTHREADS / 32][QMCDU_MAX_K];
    __shared__ double bxw_s[RTHREADS / 32];
    for (int job = threadIdx.x; job < njobs; job += RTHREADS)
        red[job] = p.partial[(size_t)b * (2 * K + 1) + job];
    __syncthreads();
    const double d = red[0];
    const double *bv = red + 1, *cv = red + 1 + k;
    double *rec = p.rs + (size_t)b * rs_stride(K);
    const double *Kb = p.Kinv + (size_t)b * K * K;
    double cq[QL];
#pragma unroll
    for (int s2 = 0; s2 < QL; ++s2) {
        const int q = lane + 32 * s2;
        cq[s2] = q < k ? cv[q] : 0.0;
    }
    double ysum[QMCDU_MAX_K / RTHREADS + 1];       // thread t: y_q for q = t, t + RTHREADS
#pragma unroll
    for (int e = 0; e < QMCDU_MAX_K / RTHREADS + 1; ++e) ysum[e] = 0.0;
    double bxsum = 0.0;                            // thread 0
    for (int m0p = 0; m0p < k; m0p += 32) {
        const int m0 = m0p + warp * 4;
        double yl[QL];
        double bxw = 0.0;
#pragma unroll
        for (int s2 = 0; s2 < QL; ++s2) yl[s2] = 0.0;
        if (m0 < k) {
            double kv[4][QL];
#pragma unroll
            for (int r = 0; r < 4; ++r)
#pragma unroll
                for (int s2 = 0; s2 < QL; ++s2) {
                    const int q = lane + 32 * s2, m = m0 + r;
                    kv[r][s2] = (q < k && m < k) ? __ldg(Kb + (size_t)m * K + q) : 0.0;
                }
            double xm[4] = {0.0, 0.0, 0.0, 0.0};
#pragma unroll
            for (int s2 = 0; s2 < QL; ++s2) {
                const int q = lane + 32 * s2;
                if (q < k) {
#pragma unroll
                    for (int r = 0; r < 4; ++r) {
                        const int m = m0 + r;
                        if (m < k) {
                            xm[r] += kv[r][s2] * cq[s2];
                            yl[s2] += bv[m] * kv[r][s2];
                        }
                    }
                }
            }
#pragma unroll
            for (int r = 0; r < 4; ++r) {
                const double x = warp_sum(xm[r]);
                if (m0 + r < k) {
                    bxw += bv[m0 + r] * x;
                    if (lane == 0) rec[4 + m0 + r] = x;
                }
            }
        }
#pragma unroll
        for (int s2 = 0; s2 < QL; ++s2) {
            const int q = lane + 32 * s2;
            if (q < k) ypart[warp][q] = yl[s2];
        }
        if (lane == 0) bxw_s[warp] = bxw;
        __syncthreads();
#pragma unroll
        for (int e = 0; e < QMCDU_MAX_K / RTHREADS + 1; ++e) {
            const int q = threadIdx.x + e * RTHREADS;
            if (q < k) {
                double y = 0.0;
#pragma unroll
                for (int w = 0; w < RTHREADS / 32; ++w) y += ypart[w][q];
                ysum[e] += y;
            }
        }
        if (threadIdx.x == 0) {
            double t = 0.0;
            for (int w = 0; w < RTHREADS / 32; ++w) t += bxw_s[w];
            bxsum += t;
        }
        __syncthreads();
    }
#pragma unroll
    for (int e = 0; e < QMCDU_MAX_K / RTHREADS + 1; ++e) {
        const int q = threadIdx.x + e * RTHREADS;
        if (q < k) rec[4 + K + q] = ysum[e];
    }
    if (threadIdx.x == 0) {
        const double r = 1.0 + (d - bxsum);
        rec[0] = d;
        rec[1] = r;
        rec[2] = (double)k;
        rec[3] = (double)j;
        if (p.ratio_out) p.ratio_out[b] = r;
    }
}

template <typename T>
struct AcceptParams {
    int N, K, ld;
    double *A;
    const T *V;
    const double *vstash;
    double *Kinv;
    int *idx;
    int *kcount;
    double *logabs;
    int *sign;
    const double *rs;
    unsigned char *acc;
    int *status;
    int mode;
    const unsigned char *mask;
    unsigned long long seed;
    int sweep;
    const signed char *override_;
    unsigned char *acc_out;
    double *ratio_out;
    long long *ties;
};

constexpr int ATHREADS = 256;
constexpr int ACHUNK = 1024;

// Grid (ceil(N / ACHUNK), batch). Every CTA of a walker takes the same
// decision from the same inputs; CTA 0 owns the small state (bordered
// inverse, queue index, counters, log-det), all CTAs copy a chunk of the new
// row into A.
//
// Bordered inverse (Sec. II, Eq. 3-4 in the row convention): with
// B_k = I + V'P, the proposal borders it as [[B_k, c], [b', 1 + d]] whose
// Schur complement is r, so with x = Kinv c and y = Kinv' b
//   Kinv' = [[Kinv + x y'/r, -x/r], [-y'/r, 1/r]].
template <typename T>
__global__ void __launch_bounds__(ATHREADS) accept_kernel(AcceptParams<T> p)
{
    const int b = blockIdx.y;
    const int N = p.N, K = p.K, ld = p.ld;
    const double *rec = p.rs + (size_t)b * rs_stride(K);
    const double r = rec[1];
    const int k = (int)rec[2];
    const int j = (int)rec[3];
    int a;
    if (p.mode == 0) {
        a = p.mask[b] ? 1 : 0;
    } else {
        const double u = metropolis_uniform(p.seed + (unsigned long long)b, j, p.sweep);
        const double prob = fmin(1.0, r * r);
        const int ov = p.override_ ? (int)p.override_[(size_t)b * N + j] : -1;
        a = ov == 0 ? 0 : (ov == 1 ? 1 : (u < prob ? 1 : 0));
        if (blockIdx.x == 0 && threadIdx.x == 0) {
            if (p.acc_out) p.acc_out[(size_t)b * N + j] = (unsigned char)a;
            if (p.ratio_out) p.ratio_out[(size_t)b * N + j] = r;
            if (p.ties && fabs(prob - u) < 1e-10) p.ties[b] += 1;
        }
    }
    if (a && !(r != 0.0 && isfinite(r))) {
        if (blockIdx.x == 0 && threadIdx.x == 0) atomicOr(p.status, ST_SINGULAR);
        a = 0;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) p.acc[b] = (unsigned char)a;
    if (!a) return;

    // New row of A (fp64, the stash of the proposed row).
    const int i0 = blockIdx.x * ACHUNK, i1 = min(N, i0 + ACHUNK);
    double *arow = p.A + (size_t)b * N * ld + (size_t)j * ld;
    const double *vs = p.vstash + (size_t)b * ld;
    for (int i = i0 + threadIdx.x; i < i1; i += blockDim.x) arow[i] = vs[i];
    if (blockIdx.x != 0) return;

    if (K > 1) {
        double *Kb = p.Kinv + (size_t)b * K * K;
        const double *x = rec + 4, *y = rec + 4 + K;
        const double rinv = 1.0 / r;
        for (int e = threadIdx.x; e < k * k; e += blockDim.x) {
            const int m = e / k, q = e - m * k;
            Kb[(size_t)m * K + q] += x[m] * y[q] * rinv;
        }
        for (int m = threadIdx.x; m < k; m += blockDim.x) {
            Kb[(size_t)m * K + k] = -x[m] * rinv;
            Kb[(size_t)k * K + m] = -y[m] * rinv;
        }
        if (threadIdx.x == 0) {
            Kb[(size_t)k * K + k] = rinv;
            p.idx[(size_t)b * K + k] = j;
            p.kcount[b] = k + 1;
        }
    }
    if (threadIdx.x == 0) {
        p.logabs[b] += log(fabs(r));
        if (r < 0.0) p.sign[b] = -p.sign[b];
    }
}

// K = 1 (Eq. 2 in the row convention): with p = A^{-1}[:, j] (the P slot copy
// taken by the ratio kernel) and w_c = u . A^{-1}[:, c] (u = v - a_j, the V
// slot),
//   A^{-1}[:, c] -= p w_c / r    for every column c.
// One warp per column: a dot product then an axpy over the same column, a
// single pass over A^{-1} (2 N^2 elements moved per accepted move).
constexpr int SMTHREADS = 256;

template <typename T>
__global__ void __launch_bounds__(SMTHREADS) sm_update_kernel(int N, int ld, T *Ainv, const T *P,
                                                             const T *V, const double *rs,
                                                             const unsigned char *acc, int K)
{
    const int b = blockIdx.y;
    if (!acc[b]) return;
    const int c = blockIdx.x * (SMTHREADS / 32) + (threadIdx.x >> 5);
    if (c >= N) return;
    const int lane = threadIdx.x & 31;
    const double *rec = rs + (size_t)b * rs_stride(K);
    const double r = rec[1];
    T *col = Ainv + (size_t)b * N * ld + (size_t)c * ld;
    const T *pcol = P + (size_t)b * K * ld;
    const T *ucol = V + (size_t)b * K * ld;
    T w = 0;
    for (int i = lane; i < N; i += 32) w += __ldg(ucol + i) * col[i];
    w = warp_sum(w);
    const T f = (T)((double)w / r);
    for (int i = lane; i < N; i += 32) col[i] -= __ldg(pcol + i) * f;
}

template <typename T>
static cudaError_t launch_ratio_t(Ctx &c, const RatioLaunch &L)
{
    RatioParams<T> p;
    p.N = c.N; p.K = c.K; p.ld = c.ld;
    p.A = c.A; p.Ainv = (const T *)c.Ainv; p.P = (T *)c.P; p.V = (T *)c.V;
    p.vstash = c.vstash; p.Kinv = c.Kinv; p.kcount = c.kcount; p.rs = c.rs;
    p.partial = c.partial; p.status = c.status;
    p.v_in = L.v_in; p.elec = L.elec; p.uniform_elec = L.uniform_elec;
    p.generate = L.generate; p.seed = L.seed; p.sweep = L.sweep; p.sigma = L.sigma;
    p.ratio_out = L.ratio_out;
    ratio_stage_kernel<T><<<dim3((c.N + 2 * RTHREADS - 1) / (2 * RTHREADS), c.batch), RTHREADS, 0,
                            c.stream>>>(p);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    // units of TRU rows sharing a vector, from the largest queue the host knows of
    const int kmax = L.kmax >= 0 ? std::min(L.kmax, c.K - 1) : c.K - 1;
    const size_t rowbytes = (size_t)c.ld * sizeof(T);
    if (4 * rowbytes <= 64 * 1024) {
        // persistent CTAs streaming items of 32 rows (rows of up to 16 KB, so
        // that two pairs of vector buffers fit beside the ring)
        const int Up = (2 * kmax + 1 + PRU - 1) / PRU;
        const int nitems = Up * c.batch;
        const size_t smem = 512 + 4 * rowbytes + (size_t)8 * SPW * std::min((size_t)TSEG, rowbytes);
        e = cudaFuncSetAttribute(ratio_dots_persist_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)smem);
        if (e != cudaSuccess) return e;
        int per_sm = 0;
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, ratio_dots_persist_kernel<T>, TTHREADS, smem);
        if (e != cudaSuccess) return e;
        const int grid = std::max(1, std::min(nitems, std::max(1, per_sm) * c.num_sms));
        ratio_dots_persist_kernel<T><<<grid, TTHREADS, smem, c.stream>>>(p, Up, nitems, c.opt_budget_ns);
    } else {
        const int U = 2 * ((kmax + 1 + TRU - 1) / TRU);
        const size_t smem = dots_smem_bytes(rowbytes);
        e = cudaFuncSetAttribute(ratio_dots_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)smem);
        if (e != cudaSuccess) return e;
        ratio_dots_kernel<T><<<dim3(U, c.batch), TTHREADS, smem, c.stream>>>(p, U, c.opt_budget_ns);
    }
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    ratio_finish_kernel<T><<<c.batch, RTHREADS, 0, c.stream>>>(p);
    return cudaGetLastError();
}

cudaError_t launch_ratio(Ctx &c, const RatioLaunch &L)
{
    return c.prec == QMCDU_FP64 ? launch_ratio_t<double>(c, L) : launch_ratio_t<float>(c, L);
}

template <typename T>
static cudaError_t launch_accept_t(Ctx &c, const AcceptLaunch &L)
{
    AcceptParams<T> p;
    p.N = c.N; p.K = c.K; p.ld = c.ld;
    p.A = c.A; p.V = (const T *)c.V; p.vstash = c.vstash; p.Kinv = c.Kinv; p.idx = c.idx;
    p.kcount = c.kcount; p.logabs = c.logabs; p.sign = c.sign; p.rs = c.rs; p.acc = c.acc;
    p.status = c.status; p.mode = L.mode; p.mask = L.mask; p.seed = L.seed; p.sweep = L.sweep;
    p.override_ = L.override; p.acc_out = L.acc_out; p.ratio_out = L.ratio_out; p.ties = L.ties;
    dim3 grid((c.N + ACHUNK - 1) / ACHUNK, c.batch);
    accept_kernel<T><<<grid, ATHREADS, 0, c.stream>>>(p);
    return cudaGetLastError();
}

cudaError_t launch_accept(Ctx &c, const AcceptLaunch &L)
{
    return c.prec == QMCDU_FP64 ? launch_accept_t<double>(c, L) : launch_accept_t<float>(c, L);
}

cudaError_t launch_sm_update(Ctx &c)
{
    dim3 grid((c.N + SMTHREADS / 32 - 1) / (SMTHREADS / 32), c.batch);
    if (c.prec == QMCDU_FP64)
        sm_update_kernel<double><<<grid, SMTHREADS, 0, c.stream>>>(
            c.N, c.ld, (double *)c.Ainv, (const double *)c.P, (const double *)c.V, c.rs, c.acc, c.K);
    else
        sm_update_kernel<float><<<grid, SMTHREADS, 0, c.stream>>>(
            c.N, c.ld, (float *)c.Ainv, (const float *)c.P, (const float *)c.V, c.rs, c.acc, c.K);
    return cudaGetLastError();
}

// ---------------------------------------------------------------- utilities
// A walker of two determinants (spin up and spin down): log|det| of the
// product is the sum, its sign the product of the signs.
__global__ void logdet_pair_kernel(int batch, const double *l1, const int *s1, const double *l2,
                                   const int *s2, double *lout, int *sout)
{
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= batch) return;
    lout[b] = l1[b] + l2[b];
    sout[b] = s1[b] * s2[b];
}

cudaError_t launch_logdet_pair(int batch, const double *l1, const int *s1, const double *l2, const int *s2,
                               double *lout, int *sout, cudaStream_t s)
{
    if (batch <= 0) return cudaSuccess;
    logdet_pair_kernel<<<(batch + 255) / 256, 256, 0, s>>>(batch, l1, s1, l2, s2, lout, sout);
    return cudaGetLastError();
}

__global__ void philox_fill_kernel(const unsigned *c0, const unsigned *c1, const unsigned *c2,
                                   const unsigned *c3, int n, unsigned long long seed,
                                   unsigned *out)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    u32x4 o = philox4x32_10(u32x4{c0[i], c1[i], c2[i], c3[i]}, (uint32_t)seed,
                            (uint32_t)(seed >> 32));
    out[4 * (size_t)i + 0] = o.x0;
    out[4 * (size_t)i + 1] = o.x1;
    out[4 * (size_t)i + 2] = o.x2;
    out[4 * (size_t)i + 3] = o.x3;
}

cudaError_t launch_philox_fill(const unsigned *c0, const unsigned *c1, const unsigned *c2,
                               const unsigned *c3, int n, unsigned long long seed,
                               unsigned *out, cudaStream_t s)
{
    if (n <= 0) return cudaSuccess;
    philox_fill_kernel<<<(n + 255) / 256, 256, 0, s>>>(c0, c1, c2, c3, n, seed, out);
    return cudaGetLastError();
}

// Dense fp64 copy of A^{-1} (column-major, no padding) for export.
template <typename T>
__global__ void inverse_export_kernel(int N, int ld, const T *Ainv, double *dst)
{
    const int b = blockIdx.z;
    const int c = blockIdx.y;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < N; i += gridDim.x * blockDim.x)
        dst[((size_t)b * N + c) * N + i] = (double)Ainv[((size_t)b * N + c) * ld + i];
}

cudaError_t launch_inverse_export(Ctx &c, double *dst)
{
    dim3 grid((c.N + 255) / 256, c.N, c.batch);
    if (c.prec == QMCDU_FP64)
        inverse_export_kernel<double><<<grid, 256, 0, c.stream>>>(c.N, c.ld, (const double *)c.Ainv, dst);
    else
        inverse_export_kernel<float><<<grid, 256, 0, c.stream>>>(c.N, c.ld, (const float *)c.Ainv, dst);
    return cudaGetLastError();
}

}  // namespace qmcdu
