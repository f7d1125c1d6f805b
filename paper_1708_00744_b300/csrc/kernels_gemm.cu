// kernels_gemm.cu -- the rank-k flush of the delayed update (Sec. II, Eq. 4)
// on SIMT cores, and the tile GEMM it shares with the recompute.
//
// Row-convention form of Eq. 4: with P = A^{-1}[:, idx] (N x k), V the queued
// changes u_m = v_m - a_idx_m (N x k) and Kinv = (I + V'P)^{-1},
//   A^{-1} <- A^{-1} - (P Kinv) (V' A^{-1}).
// Three launches per flush, each a batched tile GEMM:
//   T = V' A^{-1}          (k x N, inner dimension N)
//   W = P Kinv             (N x k, inner dimension k)
//   A^{-1} -= W T          (N x N, inner dimension k)
// 4 N^2 k flops per flush of k moves (the same 4 N^2 per accepted move as
// Sherman-Morrison, now as matrix-matrix products).
#include <type_traits>

#include "qmcdu_internal.cuh"

namespace qmcdu {

template <typename TA, typename TB, typename TC>
struct GemmArgs {
    const TA *A; long long sAb, sAm, sAl;   // A(m, l) = A[b*sAb + m*sAm + l*sAl]
    const TB *B; long long sBb, sBl, sBn;   // B(l, n)
    TC *C; long long sCb, sCm, sCn;         // C(m, n)
    int M, Nn, Kd;
    const int *kdyn;    // per-walker k (device) or null
    int dyn;            // bit 1: M = k_b, bit 2: Kd = k_b
    int kthresh;        // walkers with k_b < kthresh are skipped (when kdyn)
    double alpha;
    int accumulate;     // C = alpha AB + (accumulate ? C : 0)
};

constexpr int GTHREADS = 256;

// C tile BM x BN per CTA, 256 threads in a 16 x 16 grid, each thread
// (BM/16) x (BN/16) outputs spaced 16 apart. Operand tiles staged in shared
// memory in the accumulation type; A_L_CONTIG / B_N_CONTIG pick which operand
// dimension is contiguous so that global loads are coalesced.
template <typename TA, typename TB, typename TC, typename Acc, int BM, int BN, bool A_L_CONTIG,
          bool B_N_CONTIG, int GBK = 16>
__global__ void __launch_bounds__(GTHREADS) gemm_tile_kernel(GemmArgs<TA, TB, TC> g)
{
    constexpr int TM = BM / 16, TN = BN / 16;
    const int b = blockIdx.z;
    int M = g.M, Kd = g.Kd;
    if (g.kdyn) {
        const int kb = g.kdyn[b];
        if (kb < g.kthresh || kb <= 0) return;
        if (g.dyn & 1) M = kb;
        if (g.dyn & 2) Kd = kb;
    }
    const int m0 = blockIdx.y * BM, n0 = blockIdx.x * BN;
    if (m0 >= M || n0 >= g.Nn) return;

    __shared__ Acc As[GBK][BM + 1];
    __shared__ Acc Bs[GBK][BN + 1];
    const TA *Ab = g.A + b * g.sAb;
    const TB *Bb = g.B + b * g.sBb;
    const int tid = threadIdx.x, ty = tid >> 4, tx = tid & 15;
    Acc acc[TM][TN];
#pragma unroll
    for (int a = 0; a < TM; ++a)
#pragma unroll
        for (int c = 0; c < TN; ++c) acc[a][c] = 0;

    for (int l0 = 0; l0 < Kd; l0 += GBK) {
#pragma unroll
        for (int e = tid; e < BM * GBK; e += GTHREADS) {
            int m, l;
            if (A_L_CONTIG) { l = e % GBK; m = e / GBK; } else { m = e % BM; l = e / BM; }
            const int gm = m0 + m, gl = l0 + l;
            As[l][m] = (gm < M && gl < Kd) ? (Acc)Ab[gm * g.sAm + gl * g.sAl] : (Acc)0;
        }
#pragma unroll
        for (int e = tid; e < BN * GBK; e += GTHREADS) {
            int nn, l;
            if (B_N_CONTIG) { nn = e % BN; l = e / BN; } else { l = e % GBK; nn = e / GBK; }
            const int gn = n0 + nn, gl = l0 + l;
            Bs[l][nn] = (gn < g.Nn && gl < Kd) ? (Acc)Bb[gl * g.sBl + gn * g.sBn] : (Acc)0;
        }
        __syncthreads();
#pragma unroll
        for (int l = 0; l < GBK; ++l) {
            Acc ra[TM], rb[TN];
#pragma unroll
            for (int a = 0; a < TM; ++a) ra[a] = As[l][ty + 16 * a];
#pragma unroll
            for (int c = 0; c < TN; ++c) rb[c] = Bs[l][tx + 16 * c];
#pragma unroll
            for (int a = 0; a < TM; ++a)
#pragma unroll
                for (int c = 0; c < TN; ++c) acc[a][c] += ra[a] * rb[c];
        }
        __syncthreads();
    }

    TC *Cb = g.C + b * g.sCb;
#pragma unroll
    for (int a = 0; a < TM; ++a) {
        const int gm = m0 + ty + 16 * a;
        if (gm >= M) continue;
#pragma unroll
        for (int c = 0; c < TN; ++c) {
            const int gn = n0 + tx + 16 * c;
            if (gn >= g.Nn) continue;
            TC *dst = Cb + gm * g.sCm + gn * g.sCn;
            Acc v = (Acc)g.alpha * acc[a][c];
            if (g.accumulate) v += (Acc)*dst;
            *dst = (TC)v;
        }
    }
}

__global__ void flush_reset_kernel(int batch, int *kcount, int kthresh)
{
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b < batch && kcount[b] >= kthresh && kcount[b] > 0) kcount[b] = 0;
}

template <typename T>
static cudaError_t launch_flush_t(Ctx &c, int kthresh)
{
    const int N = c.N, K = c.K, ld = c.ld;
    const long long wN = (long long)N * ld, wK = (long long)K * ld;
    T *Ainv = (T *)c.Ainv;
    T *Tb = (T *)c.Tbuf;
    T *Wb = (T *)c.Wbuf;
    // W = P Kinv:  W(m, i) = sum_q Kinv[q][m] P[q][i]   (stored W[m][i])
    {
        GemmArgs<double, T, T> g{};
        g.A = c.Kinv; g.sAb = (long long)K * K; g.sAm = 1; g.sAl = K;
        g.B = (const T *)c.P; g.sBb = wK; g.sBl = ld; g.sBn = 1;
        g.C = Wb; g.sCb = wK; g.sCm = ld; g.sCn = 1;
        g.M = K; g.Nn = N; g.Kd = K;
        g.kdyn = c.kcount; g.dyn = 3; g.kthresh = kthresh;
        g.alpha = 1.0; g.accumulate = 0;
        dim3 grid((N + 31) / 32, (K + 31) / 32, c.batch);
        gemm_tile_kernel<double, T, T, T, 32, 32, false, true><<<grid, GTHREADS, 0, c.stream>>>(g);
    }
    if (std::is_same<T, double>::value) {
        // fp64 walkers, K <= 32: the two N x N x k contractions on the tensor
        // cores (emulated fp64, kernels_sweep.cu)
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
        e = launch_flush_oz(c, kthresh);
        if (e == cudaSuccess) {
            flush_reset_kernel<<<(c.batch + 255) / 256, 256, 0, c.stream>>>(c.batch, c.kcount, kthresh);
            return cudaGetLastError();
        }
        if (e != cudaErrorNotSupported) return e;
        cudaGetLastError();
    }
    // T = V' A^{-1}:  T(m, n) = sum_i V[m][i] A^{-1}[i][n]
    {
        GemmArgs<T, T, T> g{};
        g.A = (const T *)c.V; g.sAb = wK; g.sAm = ld; g.sAl = 1;
        g.B = Ainv; g.sBb = wN; g.sBl = 1; g.sBn = ld;       // B(l=i, n=c) = Ainv[c*ld + i]
        g.C = Tb; g.sCb = wK; g.sCm = ld; g.sCn = 1;
        g.M = K; g.Nn = N; g.Kd = N;
        g.kdyn = c.kcount; g.dyn = 1; g.kthresh = kthresh;
        g.alpha = 1.0; g.accumulate = 0;
        dim3 grid((N + 31) / 32, (K + 31) / 32, c.batch);
        gemm_tile_kernel<T, T, T, T, 32, 32, true, false><<<grid, GTHREADS, 0, c.stream>>>(g);
    }
    // A^{-1} -= W T:  stored Ainv[c][i] (column c) -= sum_m T[m][c] W[m][i]
    {
        GemmArgs<T, T, T> g{};
        g.A = Tb; g.sAb = wK; g.sAm = 1; g.sAl = ld;          // A(row=c, l=m) = T[m][c]
        g.B = Wb; g.sBb = wK; g.sBl = ld; g.sBn = 1;          // B(l=m, n=i) = W[m][i]
        g.C = Ainv; g.sCb = wN; g.sCm = ld; g.sCn = 1;
        g.M = N; g.Nn = N; g.Kd = K;
        g.kdyn = c.kcount; g.dyn = 2; g.kthresh = kthresh;
        g.alpha = -1.0; g.accumulate = 1;
        dim3 grid((N + 63) / 64, (N + 63) / 64, c.batch);
        gemm_tile_kernel<T, T, T, T, 64, 64, false, true><<<grid, GTHREADS, 0, c.stream>>>(g);
    }
    flush_reset_kernel<<<(c.batch + 255) / 256, 256, 0, c.stream>>>(c.batch, c.kcount, kthresh);
    return cudaGetLastError();
}

// Tensor-core flush (precision QMCDU_FP32_BF16X3): the two N x N x k
// contractions run in split-bf16 x3 on tcgen05 (kernels_tc.cu); the small
// W = P Kinv stays on SIMT cores.
static cudaError_t launch_flush_tc(Ctx &c, int kthresh)
{
    const int N = c.N, K = c.K, ld = c.ld;
    const long long wN = (long long)N * ld, wK = (long long)K * ld;
    float *Ainv = (float *)c.Ainv;
    float *Tt = (float *)c.Tbuf;     // T' stored [c][m] (N x K, row length K)
    float *Wb = (float *)c.Wbuf;
    // T'(c, m) = A^{-1}[:, c] . V[m]
    cudaError_t e = launch_gemm_bf16x3(N, K, N, Ainv, ld, wN, (const float *)c.V, ld, wK, 0, Tt, K,
                                       wK, 1.f, 0.f, c.batch, c.kcount, 1, kthresh,
                                       c.status, c.opt_budget_ns, c.stream);
    if (e != cudaSuccess) return e;
    {
        GemmArgs<double, float, float> g{};
        g.A = c.Kinv; g.sAb = (long long)K * K; g.sAm = 1; g.sAl = K;
        g.B = (const float *)c.P; g.sBb = wK; g.sBl = ld; g.sBn = 1;
        g.C = Wb; g.sCb = wK; g.sCm = ld; g.sCn = 1;
        g.M = K; g.Nn = N; g.Kd = K;
        g.kdyn = c.kcount; g.dyn = 3; g.kthresh = kthresh;
        g.alpha = 1.0; g.accumulate = 0;
        dim3 grid((N + 31) / 32, (K + 31) / 32, c.batch);
        gemm_tile_kernel<double, float, float, float, 32, 32, false, true>
            <<<grid, GTHREADS, 0, c.stream>>>(g);
        e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    // A^{-1}[:, c] -= sum_m T'(c, m) W[m]   (B operand W read as K x N)
    e = launch_gemm_bf16x3(N, N, K, Tt, K, wK, Wb, ld, wK, 1, Ainv, ld, wN, -1.f, 1.f, c.batch,
                           c.kcount, 0, kthresh, c.status, c.opt_budget_ns, c.stream);
    if (e != cudaSuccess) return e;
    flush_reset_kernel<<<(c.batch + 255) / 256, 256, 0, c.stream>>>(c.batch, c.kcount, kthresh);
    return cudaGetLastError();
}

cudaError_t launch_flush(Ctx &c, int kthresh)
{
    if (c.K <= 1) return cudaSuccess;
    if (c.prec == QMCDU_FP32_BF16X3) return launch_flush_tc(c, kthresh);
    return c.prec == QMCDU_FP64 ? launch_flush_t<double>(c, kthresh) : launch_flush_t<float>(c, kthresh);
}

// Rank-nb update of the Gauss-Jordan recompute: X += Lt' R (all fp64).
cudaError_t launch_gj_update(Ctx &c, int nbe)
{
    const int N = c.N, ld = c.ld;
    GemmArgs<double, double, double> g{};
    g.A = c.Lt; g.sAb = (long long)c.nb * ld; g.sAm = 1; g.sAl = ld;
    g.B = c.R; g.sBb = (long long)c.nb * ld; g.sBl = ld; g.sBn = 1;
    g.C = c.work; g.sCb = (long long)N * ld; g.sCm = ld; g.sCn = 1;
    g.M = N; g.Nn = N; g.Kd = nbe;
    g.alpha = 1.0; g.accumulate = 1;
    dim3 grid((N + 63) / 64, (N + 63) / 64, c.batch);
    if (nbe <= 8)   // the inner dimension is the panel width: no zero padding to 16
        gemm_tile_kernel<double, double, double, double, 64, 64, false, true, 8>
            <<<grid, GTHREADS, 0, c.stream>>>(g);
    else
        gemm_tile_kernel<double, double, double, double, 64, 64, false, true, 16>
            <<<grid, GTHREADS, 0, c.stream>>>(g);
    return cudaGetLastError();
}

}  // namespace qmcdu
