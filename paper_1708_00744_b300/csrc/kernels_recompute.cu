// kernels_recompute.cu -- fp64 recompute of A^{-1} and log|det A| from A.
//
// The paper checks the running determinants against direct calculation after
// a sweep (Sec. III). Here the direct calculation is blocked Gauss-Jordan
// elimination with partial pivoting on X = A' (the transposed copy, so that the
// result lands in the column-major layout of A^{-1} without a transpose):
//   * the pivots are the diagonal of U in P X = L U, so
//     log|det A| = sum log|pivot| and sign = prod sign(pivot) * (-1)^swaps;
//   * eliminating above and below every pivot leaves (S X)^{-1} = X^{-1} S^{-1}
//     in place (S the row interchanges), and X^{-1} = (S X)^{-1} S is a column
//     permutation of it; X^{-1} = A^{-T} stored row-major is A^{-1} stored
//     column-major.
// Equilibration: A' = D_r A D_c with power-of-two scales (each row's largest
// element into [1, 2), then each column's), so that X = A'' has no rows or
// columns many binades apart (which the emulated-fp64 rank-nb update, and
// partial pivoting, handle poorly); A^{-1} = D_c A'^{-1} D_r and
// log|det A| = log|det A'| - log|det D_r D_c| are exact.
// Blocking: for a panel of nb columns, one CTA per walker eliminates the panel
// (all N rows, panel staged in shared memory) -- or, for a few walkers, P CTAs
// per walker split the rows (gj_panel_mc_kernel, kernels_sweep.cu) -- then every
// other column gets the panel's transformation as one rank-nb update,
// X += (Mp - E) X_p, with Mp the eliminated panel and X_p the panel's pivot
// rows: for fp64 handles on the tensor cores, emulated in fp64 by the flush's
// slice products (kernels_sweep.cu, oz_gj_update_kernel), otherwise a SIMT
// tile GEMM. 2 N^3 flops in all.
#include <math.h>

#include <algorithm>

#include "qmcdu_internal.cuh"
#include "philox.cuh"
#include "bulk.cuh"

namespace qmcdu {

cudaError_t launch_gj_update(Ctx &c, int nbe);

constexpr int PTHREADS = 1024;

int choose_panel_width(int N)
{
    const size_t budget = 192 * 1024;
    int nb = 16;
    while (nb > 1 && (size_t)N * nb * sizeof(double) > budget) nb >>= 1;
    return nb;
}

void configure_recompute(Ctx &c)
{
    // a few walkers: each walker's panels over P CTAs (rows split), 32 columns
    // wide; otherwise, and for handles whose grid is shared out (a serving
    // pool sets a group shape), one CTA per walker with the panel in its
    // shared memory (nb1 columns, inside the same Lt / R rows)
    c.nb1 = choose_panel_width(c.N);
    if (c.batch <= 4 && c.N >= 256) {
        c.gj_ctas = std::min(64, std::max(8, c.num_sms / c.batch));
        c.nb = 32;
    } else {
        c.gj_ctas = 0;
        c.nb = c.nb1;
    }
}

// The multi-CTA panels for this launch: configured, and the handle owns the
// GPU (no group shape, no grid cap: a cooperative panel grid beside other
// persistent kernels could not be guaranteed co-resident).
static bool use_gj_mc(const Ctx &c)
{
    return c.gj_ctas > 0 && c.opt_group_ctas == 0 && c.opt_max_ctas == 0;
}

__device__ __forceinline__ int rc_bexp(double x) { return (int)((__double_as_longlong(x) >> 52) & 0x7FF); }

constexpr int EQ_NONE = -(1 << 30);

// Row scales: sr[x] = 1023 - (largest biased exponent of row x) (0 for a zero
// row), one warp per row; the column maxima start empty.
__global__ void eq_rows_kernel(int N, int ld, const double *A, int *eqs)
{
    const int b = blockIdx.y;
    const int x = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5), lane = threadIdx.x & 31;
    if (x >= N) return;
    const double *row = A + ((size_t)b * N + x) * ld;
    unsigned e = 0;
    for (int i = lane; i < N; i += 32) e = max(e, (unsigned)rc_bexp(row[i]));
    e = __reduce_max_sync(0xffffffffu, e);
    if (lane == 0) {
        eqs[(size_t)b * 2 * N + x] = e ? 1023 - (int)e : 0;
        eqs[(size_t)b * 2 * N + N + x] = EQ_NONE;
    }
}

// Column maxima of the row-scaled matrix, max_x (E(A[x][i]) + sr[x]) over the
// nonzero elements: CTA (cx, rx) takes columns [128 cx, +128) of rows
// [64 rx, +64).
__global__ void eq_cols_kernel(int N, int ld, const double *A, int *eqs)
{
    const int b = blockIdx.z;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int x0 = blockIdx.y * 64, x1 = min(N, x0 + 64);
    const int *sr = eqs + (size_t)b * 2 * N;
    int *cm = eqs + (size_t)b * 2 * N + N;
    if (i >= N) return;
    const double *Ab = A + (size_t)b * N * ld;
    int e = EQ_NONE;
    for (int x = x0; x < x1; ++x) {
        const int be = rc_bexp(Ab[(size_t)x * ld + i]);
        if (be) e = max(e, be + sr[x]);
    }
    if (e > EQ_NONE) atomicMax(cm + i, e);
}

// Column scales sc[i] = 1023 - (the column maximum) (0 for a zero column) and
// the log-det correction -ln 2 (sum sr + sum sc), added to the recompute's
// pivot sum; one CTA per walker, fixed summation order.
__global__ void eq_logdet_kernel(int N, int *eqs, double *lu_logabs)
{
    const int b = blockIdx.x;
    __shared__ long long part[256];
    int *sc = eqs + (size_t)b * 2 * N + N;
    for (int t = threadIdx.x; t < N; t += blockDim.x) sc[t] = sc[t] == EQ_NONE ? 0 : 1023 - sc[t];
    __syncthreads();
    long long s = 0;
    for (int t = threadIdx.x; t < 2 * N; t += blockDim.x) s += eqs[(size_t)b * 2 * N + t];
    part[threadIdx.x] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        long long tot = 0;
        for (int q = 0; q < (int)blockDim.x; ++q) tot += part[q];
        lu_logabs[b] -= 0.69314718055994530942 * (double)tot;
    }
}

// work[b][i][x] = A'[b][x][i] = A[b][x][i] 2^(sr[x] + sc[i])  (X = A''); padding stays zero.
__global__ void transpose_kernel(int N, int ld, const double *A, const int *eqs, double *work)
{
    __shared__ double tile[32][33];
    const int b = blockIdx.z;
    const int x0 = blockIdx.x * 32, i0 = blockIdx.y * 32;
    const double *Ab = A + (size_t)b * N * ld;
    double *Wb = work + (size_t)b * N * ld;
    const int *sr = eqs + (size_t)b * 2 * N, *sc = sr + N;
    for (int r = threadIdx.y; r < 32; r += blockDim.y) {
        const int row = i0 + r, col = x0 + threadIdx.x;   // read A[row][col]
        if (row < N && col < N) tile[r][threadIdx.x] = ldexp(ldexp(Ab[(size_t)row * ld + col], sr[row]), sc[col]);
    }
    __syncthreads();
    for (int r = threadIdx.y; r < 32; r += blockDim.y) {
        const int row = x0 + r, col = i0 + threadIdx.x;   // write work[row][col] = A[col][row]
        if (row < N && col < N) Wb[(size_t)row * ld + col] = tile[threadIdx.x][r];
    }
}

__global__ void lu_init_kernel(int batch, double *lu_logabs, int *lu_sign, double *drift)
{
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= batch) return;
    lu_logabs[b] = 0.0;
    lu_sign[b] = 1;
    drift[4 * b + 0] = drift[4 * b + 1] = drift[4 * b + 2] = drift[4 * b + 3] = 0.0;
}

// One CTA per walker: Gauss-Jordan on columns [c0, c0 + nbe) of X over all
// rows, pivot among rows >= c (largest |x|, first index on ties, as LU with
// partial pivoting), whole-row interchanges applied to X in global memory
// at once. Outputs: the eliminated panel written back into X, Lt = (Mp - E)'
// and R = X_p with the panel columns zeroed (the operands of the rank-nb
// update of all other columns).
__global__ void __launch_bounds__(PTHREADS) gj_panel_kernel(int N, int ld, int nb, int c0, int nbe,
                                                            double *work, int *piv, double *Lt,
                                                            double *R, double *lu_logabs,
                                                            int *lu_sign, int *status)
{
    extern __shared__ double S[];          // N x nb, column q at S + q*N (the elimination's
                                           // threads, one row each, hit consecutive banks)
    __shared__ double wval[32];
    __shared__ int widx[32];
    __shared__ double prow[16];
    __shared__ int pivot_row;
    __shared__ int singular;
    const int b = blockIdx.x;
    double *X = work + (size_t)b * N * ld;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    for (int e = tid; e < N * nbe; e += blockDim.x) {
        const int i = e / nbe, q = e - i * nbe;
        S[q * N + i] = X[(size_t)i * ld + c0 + q];
    }
    if (tid == 0) singular = 0;
    __syncthreads();
    double la = 0.0;
    int sg = 1;
    for (int q = 0; q < nbe; ++q) {
        const int c = c0 + q;
        // pivot search, by integer keys (gj_key)
        long long best = -1;
        int bi = N;
        for (int i = c + tid; i < N; i += blockDim.x) {
            const long long v = gj_key(S[q * N + i]);
            if (v > best) { best = v; bi = i; }
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
            best = lane < (blockDim.x >> 5) ? __double_as_longlong(wval[lane]) : -1;
            bi = lane < (blockDim.x >> 5) ? widx[lane] : N;
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                const long long ov = __shfl_xor_sync(0xffffffffu, best, o);
                const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
                if (ov > best || (ov == best && oi < bi)) { best = ov; bi = oi; }
            }
            if (lane == 0) {
                pivot_row = bi < N ? bi : c;
                piv[(size_t)b * N + c] = pivot_row;
            }
        }
        __syncthreads();
        const int p = pivot_row;
        if (p != c) {
            for (int t = tid; t < nbe; t += blockDim.x) {
                const double s = S[t * N + c];
                S[t * N + c] = S[t * N + p];
                S[t * N + p] = s;
            }
            for (int x = tid; x < N; x += blockDim.x) {
                if (x >= c0 && x < c0 + nbe) continue;
                const double s = X[(size_t)c * ld + x];
                X[(size_t)c * ld + x] = X[(size_t)p * ld + x];
                X[(size_t)p * ld + x] = s;
            }
            sg = -sg;
        }
        __syncthreads();
        const double pv = S[q * N + c];
        if (pv == 0.0) {
            if (tid == 0) singular = 1;
            __syncthreads();
            continue;
        }
        if (tid == 0) la += log(fabs(pv));   // one thread: fp64 log is costly on this part
        if (pv < 0.0) sg = -sg;
        if (tid < nbe) prow[tid] = (tid == q) ? 1.0 / pv : S[tid * N + c] / pv;
        __syncthreads();
        for (int i = tid; i < N; i += blockDim.x) {
            if (i == c) {
                for (int t = 0; t < nbe; ++t) S[t * N + i] = prow[t];
            } else {
                const double f = S[q * N + i];
                S[q * N + i] = 0.0;
                for (int t = 0; t < nbe; ++t) S[t * N + i] -= f * prow[t];
            }
        }
        __syncthreads();
    }
    // write back the panel, and the rank-nb update operands
    double *Ltb = Lt + (size_t)b * nb * ld;
    double *Rb = R + (size_t)b * nb * ld;
    for (int e = tid; e < N * nbe; e += blockDim.x) {
        const int i = e / nbe, q = e - i * nbe;
        const double v = S[q * N + i];
        X[(size_t)i * ld + c0 + q] = v;
        Ltb[(size_t)q * ld + i] = v - (i == c0 + q ? 1.0 : 0.0);
    }
    for (int q = 0; q < nbe; ++q)
        for (int x = tid; x < N; x += blockDim.x)
            Rb[(size_t)q * ld + x] = (x >= c0 && x < c0 + nbe) ? 0.0 : X[(size_t)(c0 + q) * ld + x];
    if (tid == 0) {
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

// Column permutation of the result: X^{-1} = M S, i.e. column x of X^{-1} is
// column colperm[x] of M, with the interchanges undone in reverse order.
__global__ void colperm_kernel(int N, int batch, const int *piv, int *colperm)
{
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= batch) return;
    int *cp = colperm + (size_t)b * N;
    const int *pv = piv + (size_t)b * N;
    for (int x = 0; x < N; ++x) cp[x] = x;
    for (int c = N - 1; c >= 0; --c) {
        const int p = pv[c];
        const int t = cp[c];
        cp[c] = cp[p];
        cp[p] = t;
    }
}

// A^{-1} (working precision) from the eliminated matrix, with drift sums:
// column r of A^{-1} is row r of X^{-1} = A'^{-T}, element x scaled back by
// 2^(sc[x] + sr[r]) (A^{-1} = D_c A'^{-1} D_r).
template <typename T>
__global__ void gather_kernel(int N, int ld, const double *work, const int *colperm, const int *eqs, T *Ainv,
                              double *drift, int have_old)
{
    const int b = blockIdx.z, r = blockIdx.y;
    const double *src = work + ((size_t)b * N + r) * ld;
    const int *cp = colperm + (size_t)b * N;
    const int *sr = eqs + (size_t)b * 2 * N, *sc = sr + N;
    T *dst = Ainv + ((size_t)b * N + r) * ld;
    double dsq = 0.0, nsq = 0.0;
    for (int x = blockIdx.x * blockDim.x + threadIdx.x; x < N; x += gridDim.x * blockDim.x) {
        const double v = ldexp(ldexp(src[cp[x]], sc[x]), sr[r]);
        if (have_old) {
            const double o = (double)dst[x];
            dsq += (o - v) * (o - v);
        }
        nsq += v * v;
        dst[x] = (T)v;
    }
    if (!have_old) return;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        dsq += __shfl_xor_sync(0xffffffffu, dsq, o);
        nsq += __shfl_xor_sync(0xffffffffu, nsq, o);
    }
    if ((threadIdx.x & 31) == 0) {
        atomicAdd(drift + 4 * b + 0, dsq);
        atomicAdd(drift + 4 * b + 1, nsq);
    }
}

// Replace the running log-det by the recomputed one; keep the drift report.
__global__ void lu_finish_kernel(int batch, double *logabs, int *sign, const double *lu_logabs,
                                 const int *lu_sign, double *drift, int have_old)
{
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= batch) return;
    drift[4 * b + 2] = have_old ? fabs(logabs[b] - lu_logabs[b]) : 0.0;
    drift[4 * b + 3] = have_old ? sqrt(drift[4 * b + 0] / fmax(drift[4 * b + 1], 1e-300)) : 0.0;
    logabs[b] = lu_logabs[b];
    sign[b] = lu_sign[b];
}

// Initial matrices of walkers [w0, w0 + n) from their keys seeds[0..n): row i
// of walker w0 + t holds the Gaussian pairs at Philox counters (i, 0, 2, q).
__global__ void init_matrix_kernel(int N, int ld, int n, const unsigned long long *seeds, double *A)
{
    const int npair = (N + 1) / 2;
    const long long per_w = (long long)N * npair, total = per_w * n;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
         e += (long long)gridDim.x * blockDim.x) {
        const int t = (int)(e / per_w);
        const long long r = e - (long long)t * per_w;
        const int i = (int)(r / npair), q = (int)(r - (long long)i * npair);
        const double2 g = matrix_gaussian_pair(seeds[t], i, q);
        double *row = A + ((size_t)t * N + i) * ld;
        row[2 * q] = g.x;
        if (2 * q + 1 < N) row[2 * q + 1] = g.y;
    }
}

cudaError_t launch_init_matrix(Ctx &c, int w0, int n, const unsigned long long *seeds)
{
    if (n <= 0) return cudaSuccess;
    init_matrix_kernel<<<c.num_sms * 8, 256, 0, c.stream>>>(c.N, c.ld, n, seeds,
                                                           c.A + (size_t)w0 * c.N * c.ld);
    return cudaGetLastError();
}

cudaError_t launch_recompute(Ctx &c, int have_old)
{
    const int N = c.N, ld = c.ld;
    lu_init_kernel<<<(c.batch + 255) / 256, 256, 0, c.stream>>>(c.batch, c.lu_logabs, c.lu_sign, c.drift);
    eq_rows_kernel<<<dim3((N + 7) / 8, c.batch), 256, 0, c.stream>>>(N, ld, c.A, c.eqs);
    eq_cols_kernel<<<dim3((N + 127) / 128, (N + 63) / 64, c.batch), 128, 0, c.stream>>>(N, ld, c.A, c.eqs);
    eq_logdet_kernel<<<c.batch, 256, 0, c.stream>>>(N, c.eqs, c.lu_logabs);
    {
        dim3 grid((N + 31) / 32, (N + 31) / 32, c.batch);
        transpose_kernel<<<grid, dim3(32, 8), 0, c.stream>>>(N, ld, c.A, c.eqs, c.work);
    }
    const bool mc = use_gj_mc(c);
    const int pw = mc ? c.nb : c.nb1;                       // panel width of this launch
    const size_t smem = (size_t)N * c.nb1 * sizeof(double);
    {
        cudaError_t e = cudaFuncSetAttribute(gj_panel_kernel,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             200 * 1024);
        if (e != cudaSuccess) return e;
    }
    for (int c0 = 0; c0 < N; c0 += pw) {
        const int nbe = N - c0 < pw ? N - c0 : pw;
        cudaError_t e;
        if (mc) {
            e = launch_gj_panel_mc(c, c0, nbe);
        } else {
            gj_panel_kernel<<<c.batch, PTHREADS, smem, c.stream>>>(N, ld, c.nb, c0, nbe, c.work, c.piv,
                                                                  c.Lt, c.R, c.lu_logabs, c.lu_sign,
                                                                  c.status);
            e = cudaGetLastError();
        }
        if (e != cudaSuccess) return e;
        e = launch_gj_update_oz(c, nbe);
        if (e == cudaErrorNotSupported) e = launch_gj_update(c, nbe);
        if (e != cudaSuccess) return e;
    }
    colperm_kernel<<<(c.batch + 127) / 128, 128, 0, c.stream>>>(N, c.batch, c.piv, c.colperm);
    {
        dim3 grid((N + 255) / 256, N, c.batch);
        if (c.prec == QMCDU_FP64)
            gather_kernel<double><<<grid, 256, 0, c.stream>>>(N, ld, c.work, c.colperm, c.eqs,
                                                             (double *)c.Ainv, c.drift, have_old);
        else
            gather_kernel<float><<<grid, 256, 0, c.stream>>>(N, ld, c.work, c.colperm, c.eqs,
                                                            (float *)c.Ainv, c.drift, have_old);
    }
    lu_finish_kernel<<<(c.batch + 255) / 256, 256, 0, c.stream>>>(c.batch, c.logabs, c.sign,
                                                                  c.lu_logabs, c.lu_sign, c.drift,
                                                                  have_old);
    return cudaGetLastError();
}

}  // namespace qmcdu
