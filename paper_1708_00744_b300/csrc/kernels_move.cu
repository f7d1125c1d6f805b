// kernels_move.cu -- per-proposal kernels of the delayed update.
//
// ratio_kernel  : determinant ratio of one proposal per walker (Eq. 1 at k = 0,
//                 Eq. 3 through the queued panels otherwise). HBM-bound GEMV
//                 class: reads A^{-1}[:, j], v, and the k queued rows of P and V.
// accept_kernel : Metropolis decision (or a given mask), append to the delay
//                 queue with the bordered k x k inverse update, new row of A,
//                 running log|det A|.
// sm_update_kernel : K = 1, Sherman-Morrison (Eq. 2) as one fused pass over
//                 A^{-1}: per column, a dot product with v and a rank-1 axpy.
#include <math.h>

#include <type_traits>

#include "philox.cuh"
#include "qmcdu_internal.cuh"

namespace qmcdu {

constexpr int RCHUNK = 256;    // elements of N handled by one CTA of the ratio kernel
constexpr int RTHREADS = 256;  // 8 warps

template <typename T>
struct RatioParams {
    int N, K, ld, nsplit;
    const double *A;
    const T *Ainv;
    T *P, *V;
    double *vstash;
    const double *Kinv;
    const int *kcount;
    double *rs;
    double *partial;
    unsigned *arrive;
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

// Grid (nsplit, batch). CTA `split` owns elements [split*RCHUNK, +RCHUNK) of N
// for walker blockIdx.y. Each CTA stages v and A^{-1}[:, j] for its chunk in
// shared memory, writes them speculatively into slot k of V and P (the slot a
// subsequent accept would fill), and computes 2k+1 partial dot products:
//   d = v . A^{-1}[:, j],  b_m = P[m] . v,  c_m = V[m] . A^{-1}[:, j].
// The last CTA to arrive for the walker sums the partials in split order
// (deterministic), forms x = Kinv c and y = Kinv' b, and the ratio
//   r = d - b' Kinv c   (the Schur complement of the bordered V'P, Eq. 3).
template <typename T>
__global__ void __launch_bounds__(RTHREADS) ratio_kernel(RatioParams<T> p)
{
    using Acc = T;
    const int b = blockIdx.y, split = blockIdx.x;
    const int N = p.N, K = p.K, ld = p.ld;
    const int i0 = split * RCHUNK;
    const int n = min(RCHUNK, N - i0);
    const int k = p.kcount[b];
    const int j = p.elec ? p.elec[b] : p.uniform_elec;
    if (j < 0 || j >= N || k < 0 || k >= K) {
        if (threadIdx.x == 0 && split == 0) atomicOr(p.status, ST_BADARG);
        return;  // every CTA of this walker returns: the arrival count stays 0
    }
    __shared__ T vs[RCHUNK];
    __shared__ T as[RCHUNK];
    const size_t wN = (size_t)N * ld, wK = (size_t)K * ld;
    const T *acol = p.Ainv + b * wN + (size_t)j * ld;
    T *Pk = p.P + b * wK + (size_t)k * ld;
    T *Vk = p.V + b * wK + (size_t)k * ld;

    if (p.generate) {
        // v = a_j + sigma g, g from Philox / Box-Muller in pairs (i0 is even).
        const double *arow = p.A + b * wN + (size_t)j * ld;
        const unsigned long long wseed = p.seed + (unsigned long long)b;
        for (int q = threadIdx.x; 2 * q < n; q += blockDim.x) {
            const int i = i0 + 2 * q;
            const double2 g = proposal_gaussian_pair(wseed, j, p.sweep, i >> 1);
            const double v0 = arow[i] + p.sigma * g.x;
            vs[2 * q] = (T)v0;
            Vk[i] = (T)v0;
            if (!std::is_same<T, double>::value) p.vstash[(size_t)b * ld + i] = v0;
            if (i + 1 < N) {
                const double v1 = arow[i + 1] + p.sigma * g.y;
                vs[2 * q + 1] = (T)v1;
                Vk[i + 1] = (T)v1;
                if (!std::is_same<T, double>::value) p.vstash[(size_t)b * ld + i + 1] = v1;
            }
        }
    } else {
        for (int t = threadIdx.x; t < n; t += blockDim.x) {
            const double v0 = p.v_in[(size_t)b * N + i0 + t];
            vs[t] = (T)v0;
            Vk[i0 + t] = (T)v0;
            if (!std::is_same<T, double>::value) p.vstash[(size_t)b * ld + i0 + t] = v0;
        }
    }
    for (int t = threadIdx.x; t < n; t += blockDim.x) {
        const T a = acol[i0 + t];
        as[t] = a;
        Pk[i0 + t] = a;
    }
    __syncthreads();

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int njobs = 2 * k + 1;
    double *part = p.partial + ((size_t)b * p.nsplit + split) * (2 * K + 1);
    for (int job = warp; job < njobs; job += RTHREADS / 32) {
        const T *src;
        const T *with;
        if (job == 0) {
            src = as;
            with = vs;
        } else if (job <= k) {
            src = p.P + b * wK + (size_t)(job - 1) * ld + i0;
            with = vs;
        } else {
            src = p.V + b * wK + (size_t)(job - 1 - k) * ld + i0;
            with = as;
        }
        Acc acc = 0;
        for (int t = lane; t < n; t += 32) acc += src[t] * with[t];
        acc = warp_sum(acc);
        if (lane == 0) part[job] = (double)acc;
    }

    // Last-arriving CTA of this walker reduces.
    __threadfence();
    __syncthreads();
    __shared__ unsigned ticket;
    if (threadIdx.x == 0) ticket = atomicAdd(&p.arrive[b], 1u);
    __syncthreads();
    if (ticket != (unsigned)(p.nsplit - 1)) return;
    __threadfence();

    __shared__ double red[2 * QMCDU_MAX_K + 1];
    __shared__ double xs[QMCDU_MAX_K];
    for (int job = threadIdx.x; job < njobs; job += blockDim.x) {
        double s = 0.0;
        for (int q = 0; q < p.nsplit; ++q)
            s += __ldcg(p.partial + ((size_t)b * p.nsplit + q) * (2 * K + 1) + job);
        red[job] = s;
    }
    __syncthreads();
    const double d = red[0];
    const double *bv = red + 1, *cv = red + 1 + k;
    double *rec = p.rs + (size_t)b * rs_stride(K);
    const double *Kb = p.Kinv + (size_t)b * K * K;
    for (int m = threadIdx.x; m < k; m += blockDim.x) {
        double x = 0.0, y = 0.0;
        for (int q = 0; q < k; ++q) {
            x += Kb[(size_t)m * K + q] * cv[q];
            y += bv[q] * Kb[(size_t)q * K + m];
        }
        xs[m] = x;
        rec[4 + m] = x;
        rec[4 + K + m] = y;
    }
    __syncthreads();
    if (warp == 0) {
        double s = 0.0;
        for (int m = lane; m < k; m += 32) s += bv[m] * xs[m];
        s = warp_sum(s);
        if (lane == 0) {
            const double r = d - s;
            rec[0] = d;
            rec[1] = r;
            rec[2] = (double)k;
            rec[3] = (double)j;
            if (p.ratio_out) p.ratio_out[b] = r;
            p.arrive[b] = 0u;
        }
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
// B_k = V'P, the proposal borders it as [[B_k, c], [b', d]] whose Schur
// complement is r, so with x = Kinv c and y = Kinv' b
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

    // New row of A (fp64).
    const int i0 = blockIdx.x * ACHUNK, i1 = min(N, i0 + ACHUNK);
    double *arow = p.A + (size_t)b * N * ld + (size_t)j * ld;
    if (std::is_same<T, double>::value) {
        const T *vk = p.V + ((size_t)b * K + k) * ld;
        for (int i = i0 + threadIdx.x; i < i1; i += blockDim.x) arow[i] = (double)vk[i];
    } else {
        const double *vs = p.vstash + (size_t)b * ld;
        for (int i = i0 + threadIdx.x; i < i1; i += blockDim.x) arow[i] = vs[i];
    }
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

// K = 1 (Eq. 2 in the row convention): with u = A^{-1}[:, j] (the P slot copy
// taken by the ratio kernel) and w_c = v . A^{-1}[:, c],
//   A^{-1}[:, c] -= u (w_c - [c == j]) / r    for every column c.
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
    const int j = (int)rec[3];
    T *col = Ainv + (size_t)b * N * ld + (size_t)c * ld;
    const T *u = P + (size_t)b * K * ld;
    const T *v = V + (size_t)b * K * ld;
    T w = 0;
    for (int i = lane; i < N; i += 32) w += __ldg(v + i) * col[i];
    w = warp_sum(w);
    const T f = (T)(((double)w - (c == j ? 1.0 : 0.0)) / r);
    for (int i = lane; i < N; i += 32) col[i] -= __ldg(u + i) * f;
}

template <typename T>
static cudaError_t launch_ratio_t(Ctx &c, const RatioLaunch &L)
{
    RatioParams<T> p;
    p.N = c.N; p.K = c.K; p.ld = c.ld; p.nsplit = c.nsplit;
    p.A = c.A; p.Ainv = (const T *)c.Ainv; p.P = (T *)c.P; p.V = (T *)c.V;
    p.vstash = c.vstash; p.Kinv = c.Kinv; p.kcount = c.kcount; p.rs = c.rs;
    p.partial = c.partial; p.arrive = c.arrive; p.status = c.status;
    p.v_in = L.v_in; p.elec = L.elec; p.uniform_elec = L.uniform_elec;
    p.generate = L.generate; p.seed = L.seed; p.sweep = L.sweep; p.sigma = L.sigma;
    p.ratio_out = L.ratio_out;
    dim3 grid(c.nsplit, c.batch);
    ratio_kernel<T><<<grid, RTHREADS, 0, c.stream>>>(p);
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
