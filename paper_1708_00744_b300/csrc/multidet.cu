// multidet.cu -- multideterminant walkers on top of the delayed update: the
// table method of Clark et al. combined with the rank-K delay queue (the
// combination Sec. II of the paper points to).
//
// Psi = sum_I c_I det(A_I): A_I is the walker's Slater matrix A (electron
// rows, occupied orbital columns) with up to two occupied columns o_p replaced
// by columns a_p of B, the virtual orbitals at the electrons (N x nv). With the
// table T = A^{-1} B (orbitals x virtuals), det(A_I) / det(A) = det(T_I), the
// block of T on rows o_p and columns a_p (Cramer's rule), so
// Psi / det(A) = S = sum_I c_I det(T_I).
//
// A move of electron j changes row j of A by u = v - a_j (the handle's queue
// takes it, Eq. 1-4) and row j of B by w - b_j. With z = A_c^{-1} e_j, the
// column of the CURRENT inverse (A_c: the queued moves applied; the delayed
// queue gives it as a - P Kinv c from the inverse of the last flush), and
// d = (w - b_j) - T'u, the table after the move is T + z d' / r (Sherman-
// Morrison), r the reference ratio. The matrix determinant lemma gives
// r det(T_I + z_I d_I' / r) = r det(T_I) + d_I' adj(T_I) z_I, so the ratio
// R = Psi_new / Psi = sum_I c_I (r det(T_I) + d_I' adj(T_I) z_I) / S needs no
// division by r. The table is kept current at every accepted move (a rank-1
// update of N x nv), while A^{-1} itself waits for the flush: the table
// method's per-move cost is O(N nv), the delayed update's BLAS-3 flush is
// untouched.
//
// Per-call API (qmcdu_md_*), fp64 handles; kernels one grid per step.
#include <math.h>

#include <string>
#include <vector>

#include "qmcdu_internal.cuh"

namespace qmcdu {

constexpr int MTHREADS = 256;

struct MdCtx {
    Ctx *c = nullptr;
    qmcdu_t h = nullptr;
    int nv = 0, ndet = 0;
    int *exc = nullptr;        // device [ndet][4]
    double *coef = nullptr;    // device [ndet]
    double *T = nullptr;       // device [batch][nv][N]: T[a][o] = (A^{-1} B)_{o a}
    double *B = nullptr;       // device [batch][N][nv]
    double *z = nullptr;       // device [batch][N]: column j of the current inverse
    double *d = nullptr;       // device [batch][nv]
    double *w = nullptr;       // device [batch][nv]: the proposed virtual row
    double *r = nullptr;       // device [batch]: reference ratios of the pending proposal
    double *num = nullptr;     // device [batch]: r S_new
    double *R = nullptr;       // device [batch]: Psi ratios
    double *S = nullptr;       // device [batch]
    double *logpsi = nullptr;  // device [batch]
    int *sgn = nullptr;        // device [batch]
    std::vector<int> elec;     // host: the pending proposal's electrons
    bool pending = false, ready = false;
    std::string err;
};

// T[b][a][o] = sum_e A^{-1}[o][e] B[b][e][a]; A^{-1} column-major (column e
// contiguous in o), so the threads of a CTA read consecutive o.
__global__ void md_table_kernel(int N, int ld, int nv, const double *Ainv, const double *B, double *T)
{
    const int b = blockIdx.z, a = blockIdx.y;
    const int o = blockIdx.x * blockDim.x + threadIdx.x;
    if (o >= N) return;
    const double *Ab = Ainv + (size_t)b * N * ld;
    const double *Bb = B + (size_t)b * N * nv;
    double t = 0.0;
    for (int e = 0; e < N; ++e) t += Ab[(size_t)e * ld + o] * Bb[(size_t)e * nv + a];
    T[((size_t)b * nv + a) * N + o] = t;
}

__device__ __forceinline__ double md_block_sum(double v, double *red)
{
    for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    __syncthreads();
    if (lane == 0) red[warp] = v;
    __syncthreads();
    double s = 0.0;
    if (threadIdx.x == 0)
        for (int q = 0; q < (int)(blockDim.x >> 5); ++q) s += red[q];   // fixed order
    return s;
}

// det of determinant I's table block with the rank-1 correction, times r:
// r det(T_I) + d_I' adj(T_I) z_I (r alone for the reference).
__device__ __forceinline__ double md_term(int I, const int *exc, int nv, int N, const double *Tb,
                                          const double *zb, const double *db, double r)
{
    const int o1 = exc[4 * I], a1 = exc[4 * I + 1], o2 = exc[4 * I + 2], a2 = exc[4 * I + 3];
    if (o1 < 0 || a1 < 0) return r;
    const double t11 = Tb[(size_t)a1 * N + o1];
    if (o2 < 0 || a2 < 0) return r * t11 + zb[o1] * db[a1];
    const double t12 = Tb[(size_t)a2 * N + o1], t21 = Tb[(size_t)a1 * N + o2], t22 = Tb[(size_t)a2 * N + o2];
    return r * (t11 * t22 - t12 * t21) + db[a1] * (t22 * zb[o1] - t12 * zb[o2]) +
           db[a2] * (t11 * zb[o2] - t21 * zb[o1]);
}

// S = sum_I c_I det(T_I) and log|Psi| = log|det A| + log|S| (one CTA per walker).
__global__ void md_init_kernel(int N, int nv, int ndet, const int *exc, const double *coef, const double *T,
                               const double *logdet, const int *sign, double *S, double *logpsi, int *sgn)
{
    __shared__ double red[MTHREADS / 32];
    const int b = blockIdx.x;
    const double *Tb = T + (size_t)b * nv * N;
    double s = 0.0;
    for (int I = threadIdx.x; I < ndet; I += blockDim.x) {
        const int o1 = exc[4 * I], a1 = exc[4 * I + 1], o2 = exc[4 * I + 2], a2 = exc[4 * I + 3];
        double t;
        if (o1 < 0 || a1 < 0) t = 1.0;
        else if (o2 < 0 || a2 < 0) t = Tb[(size_t)a1 * N + o1];
        else t = Tb[(size_t)a1 * N + o1] * Tb[(size_t)a2 * N + o2] - Tb[(size_t)a2 * N + o1] * Tb[(size_t)a1 * N + o2];
        s += coef[I] * t;
    }
    s = md_block_sum(s, red);
    if (threadIdx.x == 0) {
        S[b] = s;
        logpsi[b] = logdet[b] + log(fabs(s));
        sgn[b] = (s < 0.0 ? -1 : 1) * sign[b];
    }
}

// z = A_c^{-1} e_j = a - sum_{m<k} P[m] x_m (a in P slot k, x = Kinv c in the
// proposal record), and r from the record.
__global__ void md_z_kernel(int N, int K, int ld, const double *P, const double *rs, double *z, double *r)
{
    const int b = blockIdx.y;
    const double *rec = rs + (size_t)b * rs_stride(K);
    const int k = (int)rec[2];
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (blockIdx.x == 0 && threadIdx.x == 0) r[b] = rec[1];
    if (i >= N) return;
    const double *Pb = P + (size_t)b * K * ld;
    double t = Pb[(size_t)k * ld + i];
    for (int m = 0; m < k; ++m) t -= Pb[(size_t)m * ld + i] * rec[4 + m];
    z[(size_t)b * N + i] = t;
}

// d_a = (w_a - B[j][a]) - sum_o u_o T[a][o], u the move's change (V slot k).
__global__ void md_delta_kernel(int N, int K, int ld, int nv, const double *V, const double *rs,
                                const double *T, const double *B, const double *w, const int *elec, double *d)
{
    __shared__ double red[MTHREADS / 32];
    const int a = blockIdx.x, b = blockIdx.y;
    const double *rec = rs + (size_t)b * rs_stride(K);
    const int k = (int)rec[2];
    const double *u = V + ((size_t)b * K + k) * ld;
    const double *Ta = T + ((size_t)b * nv + a) * N;
    double s = 0.0;
    for (int o = threadIdx.x; o < N; o += blockDim.x) s += u[o] * Ta[o];
    s = md_block_sum(s, red);
    if (threadIdx.x == 0) {
        const int j = elec[b];
        d[(size_t)b * nv + a] = (w[(size_t)b * nv + a] - B[((size_t)b * N + j) * nv + a]) - s;
    }
}

// R = sum_I c_I (r det(T_I) + d_I' adj(T_I) z_I) / S (one CTA per walker).
__global__ void md_ratio_kernel(int N, int nv, int ndet, const int *exc, const double *coef, const double *T,
                                const double *z, const double *d, const double *r, const double *S, double *num,
                                double *R, double *ratio_out)
{
    __shared__ double red[MTHREADS / 32];
    const int b = blockIdx.x;
    const double *Tb = T + (size_t)b * nv * N, *zb = z + (size_t)b * N, *db = d + (size_t)b * nv;
    const double rb = r[b];
    double s = 0.0;
    for (int I = threadIdx.x; I < ndet; I += blockDim.x) s += coef[I] * md_term(I, exc, nv, N, Tb, zb, db, rb);
    s = md_block_sum(s, red);
    if (threadIdx.x == 0) {
        num[b] = s;
        const double x = s / S[b];
        R[b] = x;
        ratio_out[b] = x;
    }
}

// After the handle's accept: for the accepted walkers, T += z d' / r, row j of
// B = w, S = r S_new / r, log|Psi| += log|R|.
__global__ void md_update_kernel(int N, int nv, const unsigned char *acc, const int *elec, const double *z,
                                 const double *d, const double *r, const double *num, const double *R,
                                 const double *w, double *T, double *B, double *S, double *logpsi, int *sgn)
{
    const int b = blockIdx.y;
    if (!acc[b]) return;
    const int o = blockIdx.x * blockDim.x + threadIdx.x;
    const double rinv = 1.0 / r[b];
    if (o < N) {
        const double zo = z[(size_t)b * N + o] * rinv;
        for (int a = 0; a < nv; ++a) T[((size_t)b * nv + a) * N + o] += zo * d[(size_t)b * nv + a];
    }
    if (blockIdx.x == 0) {
        const int j = elec[b];
        for (int a = threadIdx.x; a < nv; a += blockDim.x)
            B[((size_t)b * N + j) * nv + a] = w[(size_t)b * nv + a];
        if (threadIdx.x == 0) {
            S[b] = num[b] * rinv;
            logpsi[b] += log(fabs(R[b]));
            if (R[b] < 0.0) sgn[b] = -sgn[b];
        }
    }
}

}  // namespace qmcdu

using namespace qmcdu;

namespace {

int md_fail(MdCtx *m, int code, const std::string &msg)
{
    if (m) m->err = msg;
    else set_handleless_error(msg);
    return code;
}

int md_cuda(MdCtx *m, cudaError_t e, const char *where)
{
    if (e == cudaSuccess) return QMCDU_OK;
    return md_fail(m, QMCDU_ERR_CUDA, std::string(where) + ": " + cudaGetErrorString(e));
}

#define MDCK(m, call)                                          \
    do {                                                       \
        const int st_ = md_cuda((m), (call), #call);           \
        if (st_) return st_;                                   \
    } while (0)

void md_release(MdCtx *m)
{
    void *p[] = {m->exc, m->coef, m->T, m->B, m->z, m->d, m->w, m->r, m->num, m->R, m->S, m->logpsi, m->sgn};
    for (void *x : p)
        if (x) cudaFree(x);
}

}  // namespace

extern "C" int qmcdu_md_create(qmcdu_t h, int nv, int ndet, const int *exc, const double *coef, qmcdu_md_t *out)
{
    if (!h || !out || nv < 1 || ndet < 1 || !exc || !coef)
        return md_fail(nullptr, QMCDU_ERR_ARG, "qmcdu_md_create: null argument or empty expansion");
    Ctx *c = reinterpret_cast<Ctx *>(h);
    if (c->prec != QMCDU_FP64)
        return md_fail(nullptr, QMCDU_ERR_ARG, "qmcdu_md_create: multideterminant walkers need an fp64 handle");
    for (int I = 0; I < ndet; ++I)
        for (int p = 0; p < 2; ++p) {
            const int o = exc[4 * I + 2 * p], a = exc[4 * I + 2 * p + 1];
            if ((o >= 0) != (a >= 0) || o >= c->N || a >= nv)
                return md_fail(nullptr, QMCDU_ERR_ARG, "qmcdu_md_create: excitation " + std::to_string(I) +
                                                           " outside the orbitals");
        }
    MdCtx *m = new MdCtx();
    m->c = c;
    m->h = h;
    m->nv = nv;
    m->ndet = ndet;
    const size_t B = c->batch, N = c->N;
    cudaError_t e = cudaSuccess;
    auto al = [&](void **p, size_t bytes) {
        if (e == cudaSuccess) e = cudaMalloc(p, bytes);
        if (e == cudaSuccess) e = cudaMemsetAsync(*p, 0, bytes, c->stream);
    };
    al((void **)&m->exc, (size_t)ndet * 4 * sizeof(int));
    al((void **)&m->coef, (size_t)ndet * sizeof(double));
    al((void **)&m->T, B * nv * N * sizeof(double));
    al((void **)&m->B, B * N * nv * sizeof(double));
    al((void **)&m->z, B * N * sizeof(double));
    al((void **)&m->d, B * nv * sizeof(double));
    al((void **)&m->w, B * nv * sizeof(double));
    for (double **p : {&m->r, &m->num, &m->R, &m->S, &m->logpsi}) al((void **)p, B * sizeof(double));
    al((void **)&m->sgn, B * sizeof(int));
    if (e == cudaSuccess) e = cudaMemcpyAsync(m->exc, exc, (size_t)ndet * 4 * sizeof(int), cudaMemcpyDefault, c->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(m->coef, coef, (size_t)ndet * sizeof(double), cudaMemcpyDefault, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) {
        md_release(m);
        delete m;
        return md_fail(nullptr, e == cudaErrorMemoryAllocation ? QMCDU_ERR_OOM : QMCDU_ERR_CUDA,
                       std::string("qmcdu_md_create: ") + cudaGetErrorString(e));
    }
    m->elec.assign(B, 0);
    *out = reinterpret_cast<qmcdu_md_t>(m);
    return QMCDU_OK;
}

extern "C" int qmcdu_md_destroy(qmcdu_md_t mh)
{
    if (!mh) return QMCDU_ERR_ARG;
    MdCtx *m = reinterpret_cast<MdCtx *>(mh);
    cudaStreamSynchronize(m->c->stream);
    md_release(m);
    delete m;
    return QMCDU_OK;
}

extern "C" int qmcdu_md_set_virtuals(qmcdu_md_t mh, const double *B)
{
    if (!mh || !B) return QMCDU_ERR_ARG;
    MdCtx *m = reinterpret_cast<MdCtx *>(mh);
    Ctx *c = m->c;
    int st = qmcdu_flush(m->h);                 // the table starts from the current inverse
    if (st) return st;
    const int N = c->N, nv = m->nv;
    MDCK(m, cudaMemcpyAsync(m->B, B, (size_t)c->batch * N * nv * sizeof(double), cudaMemcpyDefault, c->stream));
    md_table_kernel<<<dim3((N + 127) / 128, nv, c->batch), 128, 0, c->stream>>>(N, c->ld, nv, (const double *)c->Ainv,
                                                                                m->B, m->T);
    MDCK(m, cudaGetLastError());
    md_init_kernel<<<c->batch, MTHREADS, 0, c->stream>>>(N, nv, m->ndet, m->exc, m->coef, m->T, c->logabs, c->sign,
                                                          m->S, m->logpsi, m->sgn);
    MDCK(m, cudaGetLastError());
    m->pending = false;
    m->ready = true;
    return qmcdu_sync(m->h);
}

extern "C" int qmcdu_md_ratio(qmcdu_md_t mh, const int *elec, const double *v, const double *w,
                              double *ratio_out, double *ref_ratio_out)
{
    if (!mh || !elec || !v || !w || !ratio_out) return QMCDU_ERR_ARG;
    MdCtx *m = reinterpret_cast<MdCtx *>(mh);
    if (!m->ready) return md_fail(m, QMCDU_ERR_STATE, "qmcdu_md_ratio: qmcdu_md_set_virtuals first");
    Ctx *c = m->c;
    int st = qmcdu_ratio(m->h, elec, v, ref_ratio_out ? ref_ratio_out : m->r);
    if (st) return st;
    const int N = c->N, nv = m->nv;
    std::copy(elec, elec + c->batch, m->elec.begin());
    MDCK(m, cudaMemcpyAsync(m->w, w, (size_t)c->batch * nv * sizeof(double), cudaMemcpyDefault, c->stream));
    md_z_kernel<<<dim3((N + MTHREADS - 1) / MTHREADS, c->batch), MTHREADS, 0, c->stream>>>(
        N, c->K, c->ld, (const double *)c->P, c->rs, m->z, m->r);
    MDCK(m, cudaGetLastError());
    md_delta_kernel<<<dim3(nv, c->batch), MTHREADS, 0, c->stream>>>(N, c->K, c->ld, nv, (const double *)c->V, c->rs,
                                                                    m->T, m->B, m->w, c->elec_d, m->d);
    MDCK(m, cudaGetLastError());
    md_ratio_kernel<<<c->batch, MTHREADS, 0, c->stream>>>(N, nv, m->ndet, m->exc, m->coef, m->T, m->z, m->d, m->r,
                                                          m->S, m->num, m->R, ratio_out);
    MDCK(m, cudaGetLastError());
    m->pending = true;
    return QMCDU_OK;
}

extern "C" int qmcdu_md_accept(qmcdu_md_t mh, const unsigned char *mask)
{
    if (!mh || !mask) return QMCDU_ERR_ARG;
    MdCtx *m = reinterpret_cast<MdCtx *>(mh);
    if (!m->pending) return md_fail(m, QMCDU_ERR_STATE, "qmcdu_md_accept: no pending qmcdu_md_ratio");
    Ctx *c = m->c;
    int st = qmcdu_accept(m->h, mask);          // reference: queue, bordered Kinv, A's row, log|det A|
    if (st) return st;
    const int N = c->N;
    md_update_kernel<<<dim3((N + MTHREADS - 1) / MTHREADS, c->batch), MTHREADS, 0, c->stream>>>(
        N, m->nv, c->acc, c->elec_d, m->z, m->d, m->r, m->num, m->R, m->w, m->T, m->B, m->S, m->logpsi, m->sgn);
    MDCK(m, cudaGetLastError());
    m->pending = false;
    return QMCDU_OK;
}

extern "C" int qmcdu_md_logpsi(qmcdu_md_t mh, double *logabs, int *sign)
{
    if (!mh) return QMCDU_ERR_ARG;
    MdCtx *m = reinterpret_cast<MdCtx *>(mh);
    Ctx *c = m->c;
    if (logabs) MDCK(m, cudaMemcpyAsync(logabs, m->logpsi, c->batch * sizeof(double), cudaMemcpyDefault, c->stream));
    if (sign) MDCK(m, cudaMemcpyAsync(sign, m->sgn, c->batch * sizeof(int), cudaMemcpyDefault, c->stream));
    return qmcdu_sync(m->h);
}

extern "C" const char *qmcdu_md_last_error(qmcdu_md_t mh)
{
    if (!mh) return "";
    return reinterpret_cast<MdCtx *>(mh)->err.c_str();
}
