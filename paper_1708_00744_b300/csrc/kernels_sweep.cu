// kernels_sweep.cu -- one Metropolis sweep per walker in a single persistent,
// cooperative kernel launch (proposal, ratio, decision, accept and flush fused).
//
// Each walker is served by a group of Gf CTAs. The first Gr of them (the ratio
// CTAs) each own a chunk of rows of the N-vectors and advance the proposals in
// lock step, one group barrier per proposal; all Gf CTAs (ratio CTAs and
// helpers) apply the flush of Eq. 4, each to its own block of columns of
// A^{-1}. Groups never wait on one another.
//
// Delay queue. Instead of the k x k inverse Kinv = (V'P)^{-1} the kernel keeps
// its product with the panel, W = P Kinv (N x k), which is the operand the
// flush needs. The bordered-inverse algebra of Eq. 3-4 carries over: with
// a = A^{-1}[:, j], d = v.a, y = W'v, c = V'a,
//   r  = d - y.c                            (ratio of the proposal, Eq. 3)
//   z  = a - W c,   W <- [W - z y'/r, z/r]   (append on accept)
// so every step is an N-parallel dot product or axpy over the row chunks, with
// no k x k work on the critical path.
//
// Flush (column c of the column-major A^{-1}, T = V'A^{-1} - E'):
//   t_m = V[m] . A^{-1}[:, c] - [idx_m == c],   A^{-1}[:, c] -= sum_m t_m W[m].
//
// Every spin-wait has a time budget (globaltimer); on expiry the kernel sets
// ST_TIMEOUT in the status word and returns. Data written by other CTAs is read
// with ld.global.cg (L2, not the SM's L1).
#include <math.h>

#include <algorithm>
#include <type_traits>

#include "philox.cuh"
#include "qmcdu_internal.cuh"

namespace qmcdu {

constexpr int STHREADS = 256;
constexpr int SWARPS = STHREADS / 32;
constexpr int MAX_CB = 8;

template <typename T>
struct SweepParams {
    int N, K, ld, batch;
    int Gf, Gr, ngroups, chunk, cb;
    double *A;
    T *Ainv, *W, *V;
    int *idx, *kglob;
    double *logabs;
    int *sign;
    double *partial;        // [ngroups][2][Gr][2K+1]
    unsigned *sync;         // [ngroups][4]: ratio barrier, flush barrier, flush command
    int *status;
    unsigned long long seed;
    int sweep;
    double sigma;
    const signed char *override_;
    unsigned char *acc_out;
    double *ratio_out;
    long long *ties;
    long long budget_ns;    // per wait
    int stall;              // test hook: the first ratio barrier waits for one CTA too many
    int off_vs, off_as, off_vd, off_red, off_ts, off_xs, off_wsm, off_vsm;   // shared memory (bytes)
};

__device__ __forceinline__ unsigned ld_acquire(const unsigned *p)
{
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ unsigned long long globaltimer()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Arrive (optionally) on a group counter, then wait until it reaches `target`.
// Returns false, uniformly for the CTA, when the budget runs out or another
// CTA has reported a timeout.
__device__ bool group_wait(unsigned *ctr, unsigned target, bool arrive, int *status,
                           long long budget_ns)
{
    __shared__ int ok_s;
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        if (arrive) atomicAdd(ctr, 1u);
        int ok = 1;
        const unsigned long long t0 = globaltimer();
        unsigned spins = 0;
        while (ld_acquire(ctr) < target) {
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
        __threadfence();
        ok_s = ok;
    }
    __syncthreads();
    return ok_s != 0;
}

template <typename T>
__device__ __forceinline__ T warp_allsum(T v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Flush of walker w on columns [c_begin, c_end): tiles of cb columns staged in
// shared memory; V and W rows streamed from L2 once per tile.
template <typename T>
__device__ void flush_columns(const SweepParams<T> &p, int w, int k, int c_begin, int c_end,
                              unsigned char *smem)
{
    const int N = p.N, ld = p.ld, K = p.K, cb = p.cb;
    T *xs = (T *)(smem + p.off_xs);
    T *ts = (T *)(smem + p.off_ts);
    const size_t wN = (size_t)N * ld, wK = (size_t)K * ld;
    T *Ab = p.Ainv + (size_t)w * wN;
    const T *Vb = p.V + (size_t)w * wK;
    const T *Wb = p.W + (size_t)w * wK;
    const int *idxw = p.idx + (size_t)w * K;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int c0 = c_begin; c0 < c_end; c0 += cb) {
        const int nc = min(cb, c_end - c0);
        __syncthreads();
        for (int e = threadIdx.x; e < nc * N; e += STHREADS) {
            const int cc = e / N, i = e - cc * N;
            xs[(size_t)cc * N + i] = __ldcg(Ab + (size_t)(c0 + cc) * ld + i);
        }
        __syncthreads();
        for (int pr = warp; pr < k * nc; pr += SWARPS) {
            const int m = pr / nc, cc = pr - m * nc;
            const T *vr = Vb + (size_t)m * ld;
            const T *xc = xs + (size_t)cc * N;
            T acc = 0;
            for (int i = lane; i < N; i += 32) acc += __ldcg(vr + i) * xc[i];
            acc = warp_allsum(acc);
            if (lane == 0) ts[m * cb + cc] = acc - (__ldcg(idxw + m) == c0 + cc ? (T)1 : (T)0);
        }
        __syncthreads();
        for (int i = threadIdx.x; i < N; i += STHREADS) {
            T acc[MAX_CB];
#pragma unroll
            for (int cc = 0; cc < MAX_CB; ++cc) acc[cc] = 0;
            for (int m = 0; m < k; ++m) {
                const T wv = __ldcg(Wb + (size_t)m * ld + i);
#pragma unroll
                for (int cc = 0; cc < MAX_CB; ++cc)
                    if (cc < nc) acc[cc] += ts[m * cb + cc] * wv;
            }
#pragma unroll
            for (int cc = 0; cc < MAX_CB; ++cc)
                if (cc < nc) Ab[(size_t)(c0 + cc) * ld + i] = xs[(size_t)cc * N + i] - acc[cc];
        }
    }
    __syncthreads();
}

template <typename T, bool RES>
__global__ void __launch_bounds__(STHREADS) sweep_kernel(SweepParams<T> p)
{
    extern __shared__ __align__(16) unsigned char smem[];
    const int grp = blockIdx.x / p.Gf, rank = blockIdx.x - grp * p.Gf;
    if (grp >= p.ngroups) return;
    const int N = p.N, K = p.K, ld = p.ld, Gf = p.Gf, Gr = p.Gr;
    const size_t wN = (size_t)N * ld, wK = (size_t)K * ld;
    unsigned *ratio_ctr = p.sync + 4 * grp + 0;
    unsigned *flush_ctr = p.sync + 4 * grp + 1;
    unsigned *cmd = p.sync + 4 * grp + 2;
    unsigned n_ratio = 0, n_flush = 0, n_event = 0;
    const int cpc = (N + Gf - 1) / Gf;                 // columns per CTA in the flush
    const int fc0 = min(N, rank * cpc), fc1 = min(N, fc0 + cpc);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

    if (rank >= Gr) {
        // Helper CTA: take part in every flush of every walker of the group.
        for (int w = grp; w < p.batch; w += p.ngroups) {
            for (;;) {
                if (!group_wait(cmd, 2u * (n_event + 1), false, p.status, p.budget_ns)) return;
                const bool last = (ld_acquire(cmd) & 1u) != 0;
                ++n_event;
                if (!group_wait(flush_ctr, (++n_flush) * Gf, true, p.status, p.budget_ns)) return;
                const int k = __ldcg(p.kglob + w);
                if (k > 0) flush_columns(p, w, k, fc0, fc1, smem);
                if (!group_wait(flush_ctr, (++n_flush) * Gf, true, p.status, p.budget_ns)) return;
                if (last) break;
            }
        }
        return;
    }

    // Ratio CTA: rows [i0, i0 + L) of every N-vector. RES: this CTA's rows of
    // the queue panels W and V stay in shared memory for the whole sweep and
    // are written to global memory only for a flush.
    T *vs = (T *)(smem + p.off_vs);                    // [2][chunk] proposed row (working prec.)
    T *as = (T *)(smem + p.off_as);                    // [2][chunk] column j of A^{-1}
    double *vd = (double *)(smem + p.off_vd);          // [2][chunk] proposed row (fp64)
    double *red = (double *)(smem + p.off_red);        // [2K+1] reduced dots
    T *Wsm = (T *)(smem + p.off_wsm);                  // RES: [K][LP]
    T *Vsm = (T *)(smem + p.off_vsm);                  // RES: [K][LP]
    __shared__ double rr_s;
    __shared__ int acc_s;
    const int chunk = p.chunk, LP = chunk + 1;
    const int i0 = rank * chunk;
    const int L = max(0, min(chunk, N - i0));
    const int nj = 2 * K + 1;

    for (int w = grp; w < p.batch; w += p.ngroups) {
        const unsigned long long wseed = p.seed + (unsigned long long)w;
        double *Aw = p.A + (size_t)w * wN;
        const T *Ainv = p.Ainv + (size_t)w * wN;
        T *Ww = p.W + (size_t)w * wK;
        T *Vw = p.V + (size_t)w * wK;

        // proposal row of electron jj into buffer bb; column jj of A^{-1} too
        auto stage = [&](int jj, int bb, bool row, bool col) {
            if (row) {
                const double *arow = Aw + (size_t)jj * ld;
                for (int q = threadIdx.x; 2 * q < L; q += STHREADS) {
                    const int i = i0 + 2 * q;
                    const double2 g = proposal_gaussian_pair(wseed, jj, p.sweep, i >> 1);
                    const double v0 = arow[i] + p.sigma * g.x;
                    vs[bb * chunk + 2 * q] = (T)v0;
                    vd[bb * chunk + 2 * q] = v0;
                    if (2 * q + 1 < L) {
                        const double v1 = arow[i + 1] + p.sigma * g.y;
                        vs[bb * chunk + 2 * q + 1] = (T)v1;
                        vd[bb * chunk + 2 * q + 1] = v1;
                    }
                }
            }
            if (col) {
                const T *acol = Ainv + (size_t)jj * ld + i0;
                for (int t = threadIdx.x; t < L; t += STHREADS) as[bb * chunk + t] = __ldcg(acol + t);
            }
        };

        int k = 0;
        __syncthreads();
        stage(0, 0, true, true);
        for (int j = 0; j < N; ++j) {
            const int b = j & 1;
            const T *vsb = vs + b * chunk, *asb = as + b * chunk;
            const double *vdb = vd + b * chunk;
            __syncthreads();
            // ---- partial dot products over the chunk: d, y_m = W[m].v, c_m = V[m].a
            double *part = p.partial + (((size_t)grp * 2 + b) * Gr + rank) * nj;
            if (RES) {
                for (int job = threadIdx.x; job < 2 * k + 1; job += STHREADS) {
                    const T *src = job == 0 ? asb : (job <= k ? Wsm + (job - 1) * LP : Vsm + (job - 1 - k) * LP);
                    const T *with = (job >= 1 && job <= k) ? vsb : (job == 0 ? vsb : asb);
                    T acc = 0;
#pragma unroll 8
                    for (int t = 0; t < L; ++t) acc += src[t] * with[t];
                    part[job] = (double)acc;
                }
            } else {
                for (int job = warp; job < 2 * k + 1; job += SWARPS) {
                    const T *src, *with;
                    if (job == 0) { src = asb; with = vsb; }
                    else if (job <= k) { src = Ww + (size_t)(job - 1) * ld + i0; with = vsb; }
                    else { src = Vw + (size_t)(job - 1 - k) * ld + i0; with = asb; }
                    T acc = 0;
#pragma unroll 4
                    for (int t = lane; t < L; t += 32) acc += src[t] * with[t];
                    acc = warp_allsum(acc);
                    if (lane == 0) part[job] = (double)acc;
                }
            }
            // ---- next proposal's row, and (speculatively) its column of A^{-1}
            if (j + 1 < N) stage(j + 1, b ^ 1, true, true);
            // ---- group barrier, then every ratio CTA sums the partials in order
            const unsigned extra = (p.stall && n_ratio == 0) ? 1u : 0u;
            if (!group_wait(ratio_ctr, (++n_ratio) * Gr + extra, true, p.status, p.budget_ns)) return;
            const double *pb = p.partial + ((size_t)grp * 2 + b) * Gr * nj;
            for (int job = threadIdx.x; job < 2 * k + 1; job += STHREADS) {
                double s = 0.0;
#pragma unroll 8
                for (int q = 0; q < Gr; ++q) s += __ldcg(pb + (size_t)q * nj + job);
                red[job] = s;
            }
            __syncthreads();
            if (warp == 0) {
                double s = 0.0;
                for (int m = lane; m < k; m += 32) s += red[1 + m] * red[1 + k + m];
                s = warp_allsum(s);
                if (lane == 0) {
                    const double r = red[0] - s;
                    const double u = metropolis_uniform(wseed, j, p.sweep);
                    const double prob = fmin(1.0, r * r);
                    const int ov = p.override_ ? (int)p.override_[(size_t)w * N + j] : -1;
                    int a = ov == 0 ? 0 : (ov == 1 ? 1 : (u < prob ? 1 : 0));
                    if (a && !(r != 0.0 && isfinite(r))) {
                        a = 0;
                        if (rank == 0) atomicOr(p.status, ST_SINGULAR);
                    }
                    rr_s = r;
                    acc_s = a;
                    if (rank == 0) {
                        if (p.acc_out) p.acc_out[(size_t)w * N + j] = (unsigned char)a;
                        if (p.ratio_out) p.ratio_out[(size_t)w * N + j] = r;
                        if (p.ties && fabs(prob - u) < 1e-10) p.ties[w] += 1;
                        if (a) {
                            p.logabs[w] += log(fabs(r));
                            if (r < 0.0) p.sign[w] = -p.sign[w];
                            p.idx[(size_t)w * K + k] = j;
                        }
                    }
                }
            }
            __syncthreads();
            if (acc_s) {
                // ---- accept: z = a - W c, W <- [W - z y'/r, z/r], V[k] = v, A[j] = v
                const double rinv = 1.0 / rr_s;
                const double *yv = red + 1, *cv = red + 1 + k;
                double *arow_w = Aw + (size_t)j * ld;
                if (RES) {
                    T *zs = (T *)(smem + p.off_ts);        // the flush tile is idle here
                    for (int t = threadIdx.x; t < L; t += STHREADS) {
                        T z = asb[t];
#pragma unroll 8
                        for (int m = 0; m < k; ++m) z -= (T)cv[m] * Wsm[m * LP + t];
                        zs[t] = z;
                        Vsm[k * LP + t] = vsb[t];
                        arow_w[i0 + t] = vdb[t];
                    }
                    __syncthreads();
                    for (int e = threadIdx.x; e < (k + 1) * L; e += STHREADS) {
                        const int m = e / L, t = e - m * L;
                        if (m < k) Wsm[m * LP + t] -= zs[t] * (T)(yv[m] * rinv);
                        else Wsm[k * LP + t] = zs[t] * (T)rinv;
                    }
                } else {
                    for (int t = threadIdx.x; t < L; t += STHREADS) {
                        const int i = i0 + t;
                        T z = asb[t];
                        for (int m = 0; m < k; ++m) z -= (T)cv[m] * Ww[(size_t)m * ld + i];
                        for (int m = 0; m < k; ++m) Ww[(size_t)m * ld + i] -= z * (T)(yv[m] * rinv);
                        Ww[(size_t)k * ld + i] = z * (T)rinv;
                        Vw[(size_t)k * ld + i] = vsb[t];
                        arow_w[i] = vdb[t];
                    }
                }
                ++k;
            }
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
            if (!group_wait(flush_ctr, (++n_flush) * Gf, true, p.status, p.budget_ns)) return;
            if (k > 0) flush_columns(p, w, k, fc0, fc1, smem);
            if (!group_wait(flush_ctr, (++n_flush) * Gf, true, p.status, p.budget_ns)) return;
            if (k > 0 && j + 1 < N) stage(j + 1, b ^ 1, false, true);   // the column changed
            k = 0;
        }
    }
}

// ---------------------------------------------------------------- launcher
static size_t align16(size_t x) { return (x + 15) / 16 * 16; }

template <typename T>
static size_t sweep_smem(int N, int K, int chunk, int cb, bool res, int *offs)
{
    size_t o = 0;
    offs[0] = (int)o; o = align16(o + (size_t)2 * chunk * sizeof(T));        // vs
    offs[1] = (int)o; o = align16(o + (size_t)2 * chunk * sizeof(T));        // as
    offs[2] = (int)o; o = align16(o + (size_t)2 * chunk * sizeof(double));   // vd
    offs[3] = (int)o; o = align16(o + (size_t)(2 * K + 1) * sizeof(double)); // red
    offs[4] = (int)o; o = align16(o + (size_t)std::max(K * cb, chunk) * sizeof(T));  // ts / z
    offs[5] = (int)o; o = align16(o + (size_t)cb * N * sizeof(T));           // xs
    offs[6] = (int)o; if (res) o = align16(o + (size_t)K * (chunk + 1) * sizeof(T));  // Wsm
    offs[7] = (int)o; if (res) o = align16(o + (size_t)K * (chunk + 1) * sizeof(T));  // Vsm
    return o;
}

static const size_t SMEM_BUDGET = 200 * 1024;
static const size_t RES_BUDGET = 128 * 1024;

template <typename T, bool RES>
static cudaError_t launch_shape(Ctx &c, const SweepLaunch &L, int Gf, int Gr, int chunk)
{
    const int N = c.N, K = c.K;
    int offs[8];
    int cb = MAX_CB;
    size_t smem = sweep_smem<T>(N, K, chunk, cb, RES, offs);
    while (cb > 1 && smem > SMEM_BUDGET) {
        cb >>= 1;
        smem = sweep_smem<T>(N, K, chunk, cb, RES, offs);
    }
    if (smem > SMEM_BUDGET) return cudaErrorInvalidConfiguration;
    cudaError_t e = cudaFuncSetAttribute(sweep_kernel<T, RES>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, sweep_kernel<T, RES>, STHREADS, smem);
    if (e != cudaSuccess) return e;
    const int capacity = per_sm * c.num_sms;
    if (capacity < 1 || Gf > capacity) return cudaErrorCooperativeLaunchTooLarge;
    const int ngroups = std::min(c.batch, std::max(1, capacity / Gf));
    if (ngroups * 4 > c.sync_words) return cudaErrorInvalidConfiguration;
    if ((size_t)ngroups * 2 * Gr * (2 * K + 1) > c.sw_partial_len) return cudaErrorInvalidConfiguration;

    SweepParams<T> p;
    p.N = N; p.K = K; p.ld = c.ld; p.batch = c.batch;
    p.Gf = Gf; p.Gr = Gr; p.ngroups = ngroups; p.chunk = chunk; p.cb = cb;
    p.A = c.A; p.Ainv = (T *)c.Ainv; p.W = (T *)c.P; p.V = (T *)c.V;
    p.idx = c.idx; p.kglob = c.kcount; p.logabs = c.logabs; p.sign = c.sign;
    p.partial = c.sw_partial; p.sync = c.sw_sync; p.status = c.status;
    p.seed = L.seed; p.sweep = L.sweep; p.sigma = L.sigma; p.override_ = L.override;
    p.acc_out = L.acc_out; p.ratio_out = L.ratio_out; p.ties = L.ties;
    p.budget_ns = c.opt_budget_ns; p.stall = c.opt_stall;
    p.off_vs = offs[0]; p.off_as = offs[1]; p.off_vd = offs[2]; p.off_red = offs[3];
    p.off_ts = offs[4]; p.off_xs = offs[5]; p.off_wsm = offs[6]; p.off_vsm = offs[7];
    e = cudaMemsetAsync(c.sw_sync, 0, (size_t)ngroups * 4 * sizeof(unsigned), c.stream);
    if (e != cudaSuccess) return e;
    void *args[] = {&p};
    e = cudaLaunchCooperativeKernel((const void *)sweep_kernel<T, RES>, dim3(ngroups * Gf),
                                    dim3(STHREADS), args, smem, c.stream);
    c.last_sweep_shape[0] = Gf;
    c.last_sweep_shape[1] = Gr;
    c.last_sweep_shape[2] = ngroups;
    c.last_sweep_shape[3] = chunk;
    c.last_sweep_shape[4] = RES ? cb : -cb;
    return e;
}

template <typename T>
static cudaError_t launch_sweep_t(Ctx &c, const SweepLaunch &L)
{
    const int N = c.N, K = c.K;
    int Gf, Gr;
    if (c.batch >= c.num_sms) {
        Gf = Gr = 1;
    } else {
        Gf = std::max(1, c.num_sms / c.batch);
        const int target_chunk = c.prec == QMCDU_FP64 ? 32 : 128;
        Gr = c.opt_ratio_ctas > 0 ? c.opt_ratio_ctas : (N + target_chunk - 1) / target_chunk;
        Gr = std::max(1, std::min(Gr, Gf));
        if (c.opt_flush_ctas > 0) Gf = std::max(Gr, std::min(Gf, c.opt_flush_ctas));
    }
    int chunk = (N + Gr - 1) / Gr;
    chunk = (chunk + 31) / 32 * 32;
    Gr = std::min(Gr, (N + chunk - 1) / chunk);
    Gf = std::max(Gf, Gr);
    const bool res = chunk <= 256 && 2 * (size_t)K * (chunk + 1) * sizeof(T) <= RES_BUDGET;
    return res ? launch_shape<T, true>(c, L, Gf, Gr, chunk) : launch_shape<T, false>(c, L, Gf, Gr, chunk);
}

cudaError_t launch_sweep(Ctx &c, const SweepLaunch &L)
{
    return c.prec == QMCDU_FP64 ? launch_sweep_t<double>(c, L) : launch_sweep_t<float>(c, L);
}

}  // namespace qmcdu
