// qmcdu_api.cu -- the extern "C" entry points of libqmcdu (declared in
// include/qmcdu.h): handle life cycle, argument checks, host-side delay-queue
// bookkeeping, and the order of kernel launches.
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <initializer_list>
#include <new>
#include <vector>

#include "qmcdu_internal.cuh"

using qmcdu::Ctx;

namespace qmcdu {

size_t elem_size(int prec) { return prec == QMCDU_FP64 ? sizeof(double) : sizeof(float); }

static thread_local std::string handleless_error;

void set_handleless_error(const std::string &msg) { handleless_error = msg; }

static int fail(Ctx *c, int code, const char *fmt, const char *detail = "")
{
    if (c) {
        char buf[512];
        snprintf(buf, sizeof buf, fmt, detail);
        c->err = buf;
    }
    return code;
}

static int cuda_fail(Ctx *c, cudaError_t e, const char *where)
{
    if (c) c->err = std::string(where) + ": " + cudaGetErrorString(e);
    return e == cudaErrorMemoryAllocation ? QMCDU_ERR_OOM : QMCDU_ERR_CUDA;
}

#define CK(call)                                                   \
    do {                                                           \
        cudaError_t e_ = (call);                                   \
        if (e_ != cudaSuccess) return cuda_fail(c, e_, #call);     \
    } while (0)

// Allocate and zero on the handle's stream (a plain cudaMemset runs on the
// legacy default stream, which work on non-blocking streams does not wait for).
template <typename P>
static cudaError_t dalloc(P **p, size_t bytes, cudaStream_t s)
{
    if (bytes == 0) bytes = 16;
    cudaError_t e = cudaMalloc((void **)p, bytes);
    if (e == cudaSuccess) e = cudaMemsetAsync(*p, 0, bytes, s);
    return e;
}

// Every device allocation of a handle, in one list: with do_alloc false only
// the bytes are summed (qmcdu_footprint), each rounded up to cudaMalloc's
// 512-byte granule.
static cudaError_t alloc_state(Ctx *c, bool do_alloc, size_t *total)
{
    const int N = c->N, K = c->K;
    const size_t es = elem_size(c->prec);
    const size_t B = c->batch, ld = c->ld, NN = (size_t)N * ld, KN = (size_t)K * ld;
    cudaError_t e = cudaSuccess;
    *total = 0;
#define AL(ptr, bytes)                                                  \
    do {                                                                \
        const size_t b_ = (bytes);                                      \
        *total += (std::max<size_t>(b_, 16) + 511) / 512 * 512;         \
        if (do_alloc && e == cudaSuccess) e = dalloc(&(ptr), b_, c->stream); \
    } while (0)
    AL(c->A, B * NN * sizeof(double));
    AL(c->Ainv, B * NN * es);
    AL(c->P, B * KN * es);
    AL(c->V, B * KN * es);
    AL(c->vstash, B * ld * sizeof(double));
    AL(c->Kinv, B * K * K * sizeof(double));
    AL(c->idx, B * K * sizeof(int));
    AL(c->kcount, B * sizeof(int));
    AL(c->logabs, B * sizeof(double));
    AL(c->sign, B * sizeof(int));
    AL(c->rs, B * rs_stride(K) * sizeof(double));
    AL(c->partial, B * c->nsplit * (2 * K + 1) * sizeof(double));
    AL(c->acc, B);
    AL(c->elec_d, B * sizeof(int));
    AL(c->mask_d, B);
    AL(c->status, sizeof(int));
    if (K > 1) {
        AL(c->Tbuf, B * KN * es);
        AL(c->Wbuf, B * KN * es);
    }
    AL(c->work, B * NN * sizeof(double));
    AL(c->piv, B * N * sizeof(int));
    AL(c->colperm, B * N * sizeof(int));
    AL(c->Lt, B * c->nb * ld * sizeof(double));
    AL(c->R, B * c->nb * ld * sizeof(double));
    AL(c->eqs, B * 2 * N * sizeof(int));
    AL(c->lu_logabs, B * sizeof(double));
    AL(c->lu_sign, B * sizeof(int));
    AL(c->drift, B * 4 * sizeof(double));
    AL(c->pair_logabs, B * sizeof(double));
    AL(c->pair_sign, B * sizeof(int));
    if (c->gj_ctas > 0) {
        AL(c->gj_scr, B * gj_mc_scratch_bytes(c->gj_ctas, c->nb));
        AL(c->gj_ctr, B * 32 * sizeof(unsigned));
    }
    AL(c->sw_acc, B * N);
    AL(c->sw_ratio, B * N * sizeof(double));
    AL(c->sw_ties, B * sizeof(long long));
    AL(c->sw_override, B * N);
    {
        const size_t cap = (size_t)c->num_sms * 8;   // 256-thread CTAs resident per GPU, at most
        c->sw_partial_len = cap * 2 * (2 * K + 2);
        c->sync_words = (int)(cap * 96);
        AL(c->sw_partial, c->sw_partial_len * sizeof(double));
        AL(c->sw_sync, cap * 96 * sizeof(unsigned));
        AL(c->sw_phase, 11 * sizeof(unsigned long long));
        AL(c->sw_gauss, B * NN * sizeof(double));
        AL(c->sw_unif, B * N * sizeof(double));
        AL(c->d_params, 2 * sizeof(unsigned long long));
        AL(c->d_wlist, B * sizeof(int));
        AL(c->d_wseed, B * sizeof(unsigned long long));
        AL(c->d_wsweep, B * sizeof(int));
        AL(c->d_lseed, B * sizeof(unsigned long long));
        // emulated-fp64 flush: one scratch block per walker group of >= 2 CTAs
        if (c->prec == QMCDU_FP64 && oz_group_bytes(N, K) > 0) {
            c->oz_stride = oz_group_bytes(N, K);
            c->oz_groups = (int)std::min<size_t>(B, (size_t)std::max(1, c->num_sms / 2));
            AL(c->oz, (size_t)c->oz_groups * c->oz_stride);
        }
    }
#undef AL
    return e;
}

static void release(Ctx *c)
{
    void *ptrs[] = {c->A, c->Ainv, c->P, c->V, c->vstash, c->Kinv, c->idx, c->kcount, c->logabs,
                    c->sign, c->rs, c->partial, c->acc, c->elec_d, c->mask_d,
                    c->status, c->Tbuf, c->Wbuf, c->work, c->piv, c->colperm, c->Lt, c->R,
                    c->lu_logabs, c->lu_sign, c->drift, c->sw_acc, c->sw_ratio, c->sw_ties,
                    c->sw_override, c->sw_partial, c->sw_sync, c->sw_phase, c->sw_gauss,
                    c->sw_unif};
    for (void *p : ptrs)
        if (p) cudaFree(p);
    void *more[] = {c->d_params, c->step_acc, c->step_ratio, c->step_ties, c->d_wlist,
                    c->d_wseed, c->d_wsweep, c->d_lseed, c->oz, c->gj_scr, c->gj_ctr,
                    c->pair_logabs, c->pair_sign, c->eqs};
    for (void *p : more)
        if (p) cudaFree(p);
    if (c->graph_exec) cudaGraphExecDestroy(c->graph_exec);
    if (c->pin_buf) cudaFreeHost(c->pin_buf);
    for (cudaEvent_t e : c->pin_ev)
        if (e) cudaEventDestroy(e);
}

// Small host-to-device argument copies through a ring of pinned slots: each
// part is copied into the next slot on the host, then asynchronously to the
// device; the slot's event marks when the device has read it, and the host
// waits on it only when the ring wraps.
struct H2D {
    void *dst;
    const void *src;
    size_t bytes;
};

static int stage_h2d(Ctx *c, std::initializer_list<H2D> parts)
{
    size_t total = 0;
    for (const H2D &x : parts) total += (x.bytes + 15) / 16 * 16;
    if (total > c->pin_cap) {
        CK(cudaStreamSynchronize(c->stream));
        if (c->pin_buf) cudaFreeHost(c->pin_buf);
        c->pin_buf = nullptr;
        const size_t cap = std::max<size_t>(total, (size_t)16 * c->batch + 64);
        CK(cudaMallocHost(&c->pin_buf, cap * Ctx::NPIN));
        c->pin_cap = cap;
        for (int i = 0; i < Ctx::NPIN; ++i) {
            if (!c->pin_ev[i]) CK(cudaEventCreateWithFlags(&c->pin_ev[i], cudaEventDisableTiming));
            c->pin_used[i] = false;
        }
    }
    const int slot = c->pin_next;
    c->pin_next = (slot + 1) % Ctx::NPIN;
    if (c->pin_used[slot]) CK(cudaEventSynchronize(c->pin_ev[slot]));
    char *h = c->pin_buf + (size_t)slot * c->pin_cap;
    size_t off = 0;
    for (const H2D &x : parts) {
        if (x.bytes == 0) continue;
        memcpy(h + off, x.src, x.bytes);
        CK(cudaMemcpyAsync(x.dst, h + off, x.bytes, cudaMemcpyHostToDevice, c->stream));
        off += (x.bytes + 15) / 16 * 16;
    }
    CK(cudaEventRecord(c->pin_ev[slot], c->stream));
    c->pin_used[slot] = true;
    return QMCDU_OK;
}

static bool is_device_ptr(const void *p)
{
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

// Read the latched device status (after a stream sync).
static int read_status(Ctx *c)
{
    int st = 0;
    CK(cudaMemcpyAsync(&st, c->status, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    if (st & ST_TIMEOUT) return fail(c, QMCDU_ERR_TIMEOUT, "device spin-wait budget exceeded%s");
    if (st & ST_SINGULAR)
        return fail(c, QMCDU_ERR_SINGULAR, "singular or non-finite ratio / zero pivot%s");
    if (st & ST_BADARG) return fail(c, QMCDU_ERR_ARG, "electron index out of range on device%s");
    return QMCDU_OK;
}

static void clear_queues(Ctx *c)
{
    for (int b = 0; b < c->batch; ++b) {
        c->h_k[b] = 0;
        std::fill(c->h_inq[b].begin(), c->h_inq[b].end(), 0);
    }
}

cudaError_t prof_begin(Ctx *c, std::vector<std::pair<cudaEvent_t, cudaEvent_t>> &v)
{
    if (!c->prof) return cudaSuccess;
    cudaEvent_t a, b;
    cudaError_t e = cudaEventCreate(&a);
    if (e == cudaSuccess) e = cudaEventCreate(&b);
    if (e == cudaSuccess) e = cudaEventRecord(a, c->stream);
    if (e == cudaSuccess) v.emplace_back(a, b);
    return e;
}

cudaError_t prof_end(Ctx *c, std::vector<std::pair<cudaEvent_t, cudaEvent_t>> &v)
{
    if (!c->prof || v.empty()) return cudaSuccess;
    return cudaEventRecord(v.back().second, c->stream);
}

// Flush every walker with k_b >= kthresh (Eq. 4): four kernel launches.
static int do_flush(Ctx *c, int kthresh)
{
    CK(prof_begin(c, c->ev_flush));
    CK(launch_flush(*c, kthresh));
    CK(prof_end(c, c->ev_flush));
    c->n_launch += 4;
    c->n_flush += 1;
    return QMCDU_OK;
}

static int do_recompute(Ctx *c, int have_old)
{
    CK(prof_begin(c, c->ev_recompute));
    CK(launch_recompute(*c, have_old));
    CK(prof_end(c, c->ev_recompute));
    c->n_launch += 8 + 2 * ((c->N + c->nb - 1) / c->nb);
    c->n_recompute += 1;
    return QMCDU_OK;
}

static int do_ratio(Ctx *c, const RatioLaunch &L)
{
    CK(launch_ratio(*c, L));
    c->n_launch += 3;          // stage, dots, finish
    c->n_ratio += 1;
    return QMCDU_OK;
}

static int do_accept(Ctx *c, const AcceptLaunch &L)
{
    CK(launch_accept(*c, L));
    c->n_launch += 1;
    c->n_accept += 1;
    if (c->K == 1) {
        CK(launch_sm_update(*c));
        c->n_launch += 1;
    }
    return QMCDU_OK;
}

static void drop_events(Ctx *c)
{
    for (auto *v : {&c->ev_flush, &c->ev_recompute, &c->ev_sweep}) {
        for (auto &p : *v) {
            cudaEventDestroy(p.first);
            cudaEventDestroy(p.second);
        }
        v->clear();
    }
}

int copy_sweep_outputs(Ctx *c, unsigned char *accepted_out, double *ratios_out,
                       long long *near_ties_out, int rows = -1);

static int flush_all(Ctx *c)
{
    if (c->K > 1) {
        bool any = false;
        for (int b = 0; b < c->batch; ++b) any |= c->h_k[b] > 0;
        if (any) {
            int st = do_flush(c, 1);
            if (st) return st;
        }
    }
    clear_queues(c);
    return QMCDU_OK;
}

}  // namespace qmcdu

using namespace qmcdu;

extern "C" {

const char *qmcdu_version(void) { return "qmcdu 0.1 (sm_103a)"; }

const char *qmcdu_last_error(qmcdu_t h)
{
    return h ? reinterpret_cast<Ctx *>(h)->err.c_str() : handleless_error.c_str();
}

int qmcdu_create(int N, int K, int precision, int batch, void *stream, qmcdu_t *out)
{
    if (!out) return QMCDU_ERR_ARG;
    *out = nullptr;
    if (N < 1 || N > QMCDU_MAX_N || K < 1 || K > QMCDU_MAX_K || K > N || batch < 1 ||
        batch > 65535 || precision < QMCDU_FP64 || precision > QMCDU_FP32_BF16X3)
        return QMCDU_ERR_ARG;
    Ctx *c = new (std::nothrow) Ctx();
    if (!c) return QMCDU_ERR_OOM;
    c->N = N; c->K = K; c->prec = precision; c->batch = batch; c->ld = padded_ld(N);
    c->stream = (cudaStream_t)stream;
    cudaGetDevice(&c->device);
    if (cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, c->device) != cudaSuccess)
        c->num_sms = 148;
    c->nsplit = (N + 255) / 256;
    configure_recompute(*c);
    size_t total = 0;
    cudaError_t e = alloc_state(c, true, &total);
    // the zeroing is complete when create returns: any stream may use the handle
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) {
        cudaGetLastError();
        release(c);
        delete c;
        return e == cudaErrorMemoryAllocation ? QMCDU_ERR_OOM : QMCDU_ERR_CUDA;
    }
    c->h_k.assign(batch, 0);
    c->h_inq.assign(batch, std::vector<unsigned char>(N, 0));
    c->h_elec.assign(batch, 0);
    *out = reinterpret_cast<qmcdu_t>(c);
    return QMCDU_OK;
}

int qmcdu_destroy(qmcdu_t h)
{
    if (!h) return QMCDU_ERR_ARG;
    Ctx *c = reinterpret_cast<Ctx *>(h);
    cudaStreamSynchronize(c->stream);
    drop_events(c);
    release(c);
    delete c;
    return QMCDU_OK;
}

int qmcdu_set_matrix(qmcdu_t h, const double *A)
{
    if (!h || !A) return QMCDU_ERR_ARG;
    Ctx *c = reinterpret_cast<Ctx *>(h);
    const size_t N = c->N;
    CK(cudaMemcpy2DAsync(c->A, c->ld * sizeof(double), A, N * sizeof(double), N * sizeof(double),
                         N * c->batch, cudaMemcpyDefault, c->stream));
    CK(cudaMemsetAsync(c->status, 0, sizeof(int), c->stream));
    CK(cudaMemsetAsync(c->kcount, 0, c->batch * sizeof(int), c->stream));
    clear_queues(c);
    c->pending = false;
    return do_recompute(c, 0);
}

int qmcdu_get_matrix(qmcdu_t h, double *A_out)
{
    if (!h || !A_out) return QMCDU_ERR_ARG;
    Ctx *c = reinterpret_cast<Ctx *>(h);
    const size_t N = c->N;
    CK(cudaMemcpy2DAsync(A_out, N * sizeof(double), c->A, c->ld * sizeof(double),
                         N * sizeof(double), N * c->batch, cudaMemcpyDefault, c->stream));
    return read_status(c);
}

int qmcdu_get_inverse(qmcdu_t h, double *Ainv_out)
{
    if (!h || !Ainv_out) return QMCDU_ERR_ARG;
    Ctx *c = reinterpret_cast<Ctx *>(h);
    int st = flush_all(c);
    if (st) return st;
    const size_t N = c->N;
    if (c->prec == QMCDU_FP64) {
        CK(cudaMemcpy2DAsync(Ainv_out, N * sizeof(double), c->Ainv, c->ld * sizeof(double),
                             N * sizeof(double), N * c->batch, cudaMemcpyDefault, c->stream));
    } else {
        double *tmp = nullptr;
        CK(cudaMalloc(&tmp, (size_t)c->batch * N * N * sizeof(double)));
        cudaError_t e = launch_inverse_export(*c, tmp);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(Ainv_out, tmp, (size_t)c->batch * N * N * sizeof(double),
                                cudaMemcpyDefault, c->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
        cudaFree(tmp);
        if (e != cudaSuccess) return cuda_fail(c, e, "get_inverse");
    }
    return read_status(c);
}

int qmcdu_ratio(qmcdu_t h, const int *elec, const double *v, double *ratio_out)
{
    if (!h || !elec || !v || !ratio_out) return QMCDU_ERR_ARG;
    Ctx *c = reinterpret_cast<Ctx *>(h);
    bool need_flush = false;
    for (int b = 0; b < c->batch; ++b) {
        if (elec[b] < 0 || elec[b] >= c->N)
            return fail(c, QMCDU_ERR_ARG, "electron index out of range%s");
        need_flush |= c->h_inq[b][elec[b]] != 0;
    }
    if (need_flush) {
        int st = flush_all(c);
        if (st) return st;
    }
    int st0 = stage_h2d(c, {{c->elec_d, elec, c->batch * sizeof(int)}});
    if (st0) return st0;
    RatioLaunch L{};
    L.v_in = v;
    L.elec = c->elec_d;
    L.ratio_out = ratio_out;
    L.kmax = *std::max_element(c->h_k.begin(), c->h_k.end());
    int st = do_ratio(c, L);
    if (st) return st;
    std::copy(elec, elec + c->batch, c->h_elec.begin());
    c->pending = true;
    return QMCDU_OK;
}

int qmcdu_accept(qmcdu_t h, const unsigned char *mask)
{
    if (!h || !mask) return QMCDU_ERR_ARG;
    Ctx *c = reinterpret_cast<Ctx *>(h);
    if (!c->pending) return fail(c, QMCDU_ERR_STATE, "accept without a pending ratio%s");
    int st0 = stage_h2d(c, {{c->mask_d, mask, (size_t)c->batch}});
    if (st0) return st0;
    AcceptLaunch L{};
    L.mode = 0;
    L.mask = c->mask_d;
    int st = do_accept(c, L);
    if (st) return st;
    c->pending = false;
    if (c->K == 1) return QMCDU_OK;
    bool full = false;
    for (int b = 0; b < c->batch; ++b) {
        if (!mask[b]) continue;
        c->h_k[b] += 1;
        c->h_inq[b][c->h_elec[b]] = 1;
        full |= c->h_k[b] == c->K;
    }
    if (full) {
        st = do_flush(c, c->K);
        if (st) return st;
        for (int b = 0; b < c->batch; ++b)
            if (c->h_k[b] == c->K) {
                c->h_k[b] = 0;
                std::fill(c->h_inq[b].begin(), c->h_inq[b].end(), 0);
            }
    }
    return QMCDU_OK;
}

int qmcdu_flush(qmcdu_t h)
{
    if (!h) return QMCDU_ERR_ARG;
    return flush_all(reinterpret_cast<Ctx *>(h));
}

int qmcdu_recompute(qmcdu_t h, double *drift_out)
{
    if (!h) return QMCDU_ERR_ARG;
    Ctx *c = reinterpret_cast<Ctx *>(h);
    int st = flush_all(c);
    if (st) return st;
    c->pending = false;
    st = do_recompute(c, 1);
    if (st) return st;
    if (drift_out) {
        // drift sums are [b][4]: report entries 2 (log-det) and 3 (inverse)
        CK(cudaMemcpy2DAsync(drift_out, 2 * sizeof(double), c->drift + 2, 4 * sizeof(double),
                             2 * sizeof(double), c->batch, cudaMemcpyDefault, c->stream));
        if (!is_device_ptr(drift_out)) return read_status(c);
    }
    return QMCDU_OK;
}

int qmcdu_logdet(qmcdu_t h, double *logabs, int *sign)
{
    if (!h) return QMCDU_ERR_ARG;
    Ctx *c = reinterpret_cast<Ctx *>(h);
    if (logabs)
        CK(cudaMemcpyAsync(logabs, c->logabs, c->batch * sizeof(double), cudaMemcpyDefault, c->stream));
    if (sign)
        CK(cudaMemcpyAsync(sign, c->sign, c->batch * sizeof(int), cudaMemcpyDefault, c->stream));
    return read_status(c);
}

int qmcdu_logdet_product(qmcdu_t h1, qmcdu_t h2, double *logabs, int *sign)
{
    if (!h1 || !h2 || h1 == h2) return QMCDU_ERR_ARG;
    Ctx *c1 = reinterpret_cast<Ctx *>(h1), *c2 = reinterpret_cast<Ctx *>(h2);
    if (c1->batch != c2->batch || c1->device != c2->device) {
        c1->err = "qmcdu_logdet_product: the handles differ in batch or device";
        return QMCDU_ERR_ARG;
    }
    // h2's running values as of now, then the combination on h1's stream
    Ctx *c = c1;        // (errors are reported on h1)
    cudaEvent_t ev;
    CK(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
    cudaError_t e = cudaEventRecord(ev, c2->stream);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(c1->stream, ev, 0);
    cudaEventDestroy(ev);
    CK(e);
    CK(launch_logdet_pair(c1->batch, c1->logabs, c1->sign, c2->logabs, c2->sign, c1->pair_logabs,
                          c1->pair_sign, c1->stream));
    if (logabs)
        CK(cudaMemcpyAsync(logabs, c1->pair_logabs, c1->batch * sizeof(double), cudaMemcpyDefault,
                           c1->stream));
    if (sign)
        CK(cudaMemcpyAsync(sign, c1->pair_sign, c1->batch * sizeof(int), cudaMemcpyDefault, c1->stream));
    const int st = read_status(c2);
    return st ? st : read_status(c1);
}

int qmcdu_sync(qmcdu_t h)
{
    if (!h) return QMCDU_ERR_ARG;
    return read_status(reinterpret_cast<Ctx *>(h));
}

int qmcdu_sweep(qmcdu_t h, unsigned long long base_seed, int sweep_index, double sigma,
                const signed char *override, unsigned char *accepted_out, double *ratios_out,
                long long *near_ties_out)
{
    if (!h || sweep_index < 0) return QMCDU_ERR_ARG;
    Ctx *c = reinterpret_cast<Ctx *>(h);
    int st = flush_all(c);
    if (st) return st;
    c->pending = false;
    const int N = c->N, K = c->K;
    const signed char *ov = nullptr;
    if (override) {
        CK(cudaMemcpyAsync(c->sw_override, override, (size_t)c->batch * N, cudaMemcpyDefault,
                           c->stream));
        ov = c->sw_override;
    }
    CK(cudaMemsetAsync(c->sw_ties, 0, c->batch * sizeof(long long), c->stream));
    if (c->opt_persistent) {
        SweepLaunch S{};
        S.seed = base_seed;
        S.sweep = sweep_index;
        S.sigma = sigma;
        S.override = ov;
        S.acc_out = c->sw_acc;
        S.ratio_out = c->sw_ratio;
        S.ties = c->sw_ties;
        CK(launch_sweep(*c, S));
        c->n_launch += 3;
        c->opt_stall = 0;
        CK(cudaMemsetAsync(c->kcount, 0, c->batch * sizeof(int), c->stream));
        return copy_sweep_outputs(c, accepted_out, ratios_out, near_ties_out);
    }
    if (c->opt_fixed_slot)
        return fail(c, QMCDU_ERR_STATE, "fixed slots need the persistent sweep%s");
    int kub = 0;                      // upper bound on max_b k_b
    std::vector<int> hk(c->batch);
    for (int j = 0; j < N; ++j) {
        RatioLaunch R{};
        R.uniform_elec = j;
        R.kmax = K == 1 ? 0 : std::min(kub, K - 1);
        R.generate = 1;
        R.seed = base_seed;
        R.sweep = sweep_index;
        R.sigma = sigma;
        st = do_ratio(c, R);
        if (st) return st;
        AcceptLaunch L{};
        L.mode = 1;
        L.seed = base_seed;
        L.sweep = sweep_index;
        L.override = ov;
        L.acc_out = c->sw_acc;
        L.ratio_out = c->sw_ratio;
        L.ties = c->sw_ties;
        st = do_accept(c, L);
        if (st) return st;
        if (K == 1) continue;
        if (++kub < K) continue;
        // Some walker may have reached K: look, and flush every non-empty
        // queue if one has (a grouped flush keeps all walkers in step).
        CK(cudaMemcpyAsync(hk.data(), c->kcount, c->batch * sizeof(int), cudaMemcpyDeviceToHost,
                           c->stream));
        CK(cudaStreamSynchronize(c->stream));
        c->n_sync += 1;
        const int kmax = *std::max_element(hk.begin(), hk.end());
        if (kmax >= K) {
            st = do_flush(c, 1);
            if (st) return st;
            kub = 0;
        } else {
            kub = kmax;
        }
    }
    if (K > 1) {
        st = do_flush(c, 1);
        if (st) return st;
    }
    clear_queues(c);
    return copy_sweep_outputs(c, accepted_out, ratios_out, near_ties_out);
}

}  // extern "C"

namespace qmcdu {

// Step buffers for `nsweeps` sweeps (outside any capture).
static int ensure_step_buffers(Ctx *c, int nsweeps)
{
    if (nsweeps <= c->step_cap) return QMCDU_OK;
    if (c->graph_exec) {
        cudaGraphExecDestroy(c->graph_exec);
        c->graph_exec = nullptr;
    }
    CK(cudaStreamSynchronize(c->stream));
    cudaFree(c->step_acc);
    cudaFree(c->step_ratio);
    cudaFree(c->step_ties);
    c->step_acc = nullptr; c->step_ratio = nullptr; c->step_ties = nullptr;
    c->step_cap = 0;
    const size_t BN = (size_t)c->batch * c->N;
    CK(dalloc(&c->step_acc, (size_t)nsweeps * BN, c->stream));
    CK(dalloc(&c->step_ratio, (size_t)nsweeps * BN * sizeof(double), c->stream));
    CK(dalloc(&c->step_ties, (size_t)nsweeps * c->batch * sizeof(long long), c->stream));
    c->step_cap = nsweeps;
    return QMCDU_OK;
}

// The kernels of one step on the handle's stream: nsweeps persistent sweeps
// (proposal draws read their seed and sweep index from c->d_params), then the
// recompute. No host synchronisation, so the sequence can be captured.
static int enqueue_step(Ctx *c, int nsweeps, double sigma, int recompute)
{
    const size_t BN = (size_t)c->batch * c->N;
    for (int i = 0; i < nsweeps; ++i) {
        CK(cudaMemsetAsync(c->step_ties + (size_t)i * c->batch, 0, c->batch * sizeof(long long),
                           c->stream));
        SweepLaunch S{};
        S.params = c->d_params;
        S.sweep_offset = i;
        S.sigma = sigma;
        S.acc_out = c->step_acc + i * BN;
        S.ratio_out = c->step_ratio + i * BN;
        S.ties = c->step_ties + (size_t)i * c->batch;
        CK(launch_sweep(*c, S));
        CK(cudaMemsetAsync(c->kcount, 0, c->batch * sizeof(int), c->stream));
        c->n_launch += 3;
    }
    if (recompute) return do_recompute(c, 1);
    return QMCDU_OK;
}

static bool step_graph_ready(const Ctx *c, int nsweeps, int recompute, double sigma)
{
    return c->graph_exec && c->graph_key[0] == nsweeps && c->graph_key[1] == recompute &&
           c->graph_sigma == sigma;
}

static int capture_step(Ctx *c, int nsweeps, double sigma, int recompute)
{
    if (c->graph_exec) {
        cudaGraphExecDestroy(c->graph_exec);
        c->graph_exec = nullptr;
    }
    const bool prof = c->prof;
    c->prof = false;
    cudaGraph_t graph = nullptr;
    CK(cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeRelaxed));
    const long long launches = c->n_launch;
    int st = enqueue_step(c, nsweeps, sigma, recompute);
    c->n_launch = launches;
    cudaError_t e = cudaStreamEndCapture(c->stream, &graph);
    c->prof = prof;
    if (st) {
        if (graph) cudaGraphDestroy(graph);
        return st;
    }
    if (e != cudaSuccess) return cuda_fail(c, e, "cudaStreamEndCapture");
    e = cudaGraphInstantiate(&c->graph_exec, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) {
        c->graph_exec = nullptr;
        return cuda_fail(c, e, "cudaGraphInstantiate");
    }
    c->graph_key[0] = nsweeps;
    c->graph_key[1] = recompute;
    c->graph_sigma = sigma;
    return QMCDU_OK;
}

static int step_outputs(Ctx *c, int nsweeps, unsigned char *accepted_out, double *drift_out,
                        int recompute)
{
    bool host_out = false;
    if (accepted_out) {
        CK(cudaMemcpyAsync(accepted_out, c->step_acc, (size_t)nsweeps * c->batch * c->N,
                           cudaMemcpyDefault, c->stream));
        host_out |= !is_device_ptr(accepted_out);
    }
    if (drift_out && recompute) {
        CK(cudaMemcpy2DAsync(drift_out, 2 * sizeof(double), c->drift + 2, 4 * sizeof(double),
                             2 * sizeof(double), c->batch, cudaMemcpyDefault, c->stream));
        host_out |= !is_device_ptr(drift_out);
    }
    return host_out ? read_status(c) : QMCDU_OK;
}

struct GroupCtx {
    std::vector<Ctx *> hs;
    std::vector<cudaEvent_t> done;
    cudaEvent_t fork = nullptr;
    cudaGraphExec_t exec = nullptr;
    int key[2] = {-1, -1};
    double sigma = 0.0;
    std::string err;
};

// The fork/join body of a group step on the first handle's stream.
static int group_body(GroupCtx *g, int nsweeps, double sigma, int recompute)
{
    Ctx *c0 = g->hs[0];
    cudaStream_t s0 = c0->stream;
    if (cudaError_t e = cudaEventRecord(g->fork, s0)) return cuda_fail(c0, e, "cudaEventRecord");
    for (size_t i = 0; i < g->hs.size(); ++i) {
        Ctx *c = g->hs[i];
        CK(cudaStreamWaitEvent(c->stream, g->fork, 0));
        int st = enqueue_step(c, nsweeps, sigma, recompute);
        if (st) return st;
        CK(cudaEventRecord(g->done[i], c->stream));
        CK(cudaStreamWaitEvent(s0, g->done[i], 0));
    }
    return QMCDU_OK;
}

}  // namespace qmcdu

extern "C" {

int qmcdu_step(qmcdu_t h, unsigned long long base_seed, int first_sweep, int nsweeps, double sigma,
               int recompute, int use_graph, unsigned char *accepted_out, double *drift_out)
{
    if (!h || first_sweep < 0 || nsweeps < 0) return QMCDU_ERR_ARG;
    Ctx *c = reinterpret_cast<Ctx *>(h);
    int st = flush_all(c);
    if (st) return st;
    c->pending = false;
    const size_t BN = (size_t)c->batch * c->N;
    if (!c->opt_persistent) {
        // per-proposal launches: run the sweeps one call at a time (no graph)
        for (int i = 0; i < nsweeps; ++i) {
            st = qmcdu_sweep(h, base_seed, first_sweep + i, sigma, nullptr,
                             accepted_out ? accepted_out + i * BN : nullptr, nullptr, nullptr);
            if (st) return st;
        }
        if (recompute) return qmcdu_recompute(h, drift_out);
        return QMCDU_OK;
    }
    if (use_graph && c->stream == nullptr)
        return fail(c, QMCDU_ERR_ARG, "graph capture needs a handle on a non-default stream%s");
    st = ensure_step_buffers(c, nsweeps);
    if (st) return st;
    const unsigned long long hp[2] = {base_seed, (unsigned long long)first_sweep};
    CK(cudaMemcpyAsync(c->d_params, hp, sizeof hp, cudaMemcpyHostToDevice, c->stream));
    if (use_graph && step_graph_ready(c, nsweeps, recompute, sigma)) {
        CK(cudaGraphLaunch(c->graph_exec, c->stream));
        c->n_launch += 3 * nsweeps + (recompute ? 8 + 2 * ((c->N + c->nb - 1) / c->nb) : 0);
    } else {
        st = enqueue_step(c, nsweeps, sigma, recompute);
        if (st) return st;
        if (use_graph) {
            st = capture_step(c, nsweeps, sigma, recompute);
            if (st) return st;
        }
    }
    return step_outputs(c, nsweeps, accepted_out, drift_out, recompute);
}

int qmcdu_step_results(qmcdu_t h, int nsweeps, unsigned char *accepted_out, double *ratios_out,
                       long long *near_ties_out)
{
    if (!h || nsweeps < 0) return QMCDU_ERR_ARG;
    Ctx *c = reinterpret_cast<Ctx *>(h);
    if (nsweeps > c->step_cap) return fail(c, QMCDU_ERR_STATE, "no step of that many sweeps%s");
    const size_t BN = (size_t)c->batch * c->N;
    if (accepted_out)
        CK(cudaMemcpyAsync(accepted_out, c->step_acc, nsweeps * BN, cudaMemcpyDefault, c->stream));
    if (ratios_out)
        CK(cudaMemcpyAsync(ratios_out, c->step_ratio, nsweeps * BN * sizeof(double), cudaMemcpyDefault,
                           c->stream));
    if (near_ties_out)
        CK(cudaMemcpyAsync(near_ties_out, c->step_ties, (size_t)nsweeps * c->batch * sizeof(long long),
                           cudaMemcpyDefault, c->stream));
    return read_status(c);
}

int qmcdu_group_create(qmcdu_t *hs, int n, qmcdu_group_t *out)
{
    if (!hs || n < 1 || !out) return QMCDU_ERR_ARG;
    *out = nullptr;
    GroupCtx *g = new (std::nothrow) GroupCtx();
    if (!g) return QMCDU_ERR_OOM;
    double total = 0.0;
    for (int i = 0; i < n; ++i) {
        if (!hs[i]) { delete g; return QMCDU_ERR_ARG; }
        Ctx *c = reinterpret_cast<Ctx *>(hs[i]);
        if (!c->opt_persistent) { delete g; return QMCDU_ERR_ARG; }
        g->hs.push_back(c);
        total += (double)c->batch * c->N * c->N * c->N;
    }
    // share of the SMs per size class, in proportion to its flush work (batch N^3)
    const int sms = g->hs[0]->num_sms;
    int used = 0;
    for (int i = 0; i < n; ++i) {
        Ctx *c = g->hs[i];
        int share = (int)((double)sms * c->batch * c->N * c->N * (double)c->N / total);
        share = std::max(1, std::min(share, sms - (n - 1 - i) - used));
        if (i == n - 1) share = std::max(1, sms - used);
        used += share;
        c->opt_max_ctas = 2 * share;   // at most two sweep CTAs fit on one SM
    }
    cudaError_t e = cudaEventCreateWithFlags(&g->fork, cudaEventDisableTiming);
    g->done.assign(n, nullptr);
    for (int i = 0; i < n && e == cudaSuccess; ++i)
        e = cudaEventCreateWithFlags(&g->done[i], cudaEventDisableTiming);
    if (e != cudaSuccess) {
        if (g->fork) cudaEventDestroy(g->fork);
        for (auto ev : g->done)
            if (ev) cudaEventDestroy(ev);
        delete g;
        return QMCDU_ERR_CUDA;
    }
    *out = reinterpret_cast<qmcdu_group_t>(g);
    return QMCDU_OK;
}

int qmcdu_group_step(qmcdu_group_t gh, const unsigned long long *seeds, int first_sweep, int nsweeps,
                     double sigma, int recompute, int use_graph)
{
    if (!gh || !seeds || first_sweep < 0 || nsweeps < 0) return QMCDU_ERR_ARG;
    GroupCtx *g = reinterpret_cast<GroupCtx *>(gh);
    Ctx *c0 = g->hs[0];
    if (use_graph && c0->stream == nullptr)
        return fail(c0, QMCDU_ERR_ARG, "graph capture needs a non-default stream%s");
    bool rebuilt = false;
    for (size_t i = 0; i < g->hs.size(); ++i) {
        Ctx *c = g->hs[i];
        int st = flush_all(c);
        if (st) return st;
        c->pending = false;
        const int had = c->step_cap;
        st = ensure_step_buffers(c, nsweeps);
        if (st) return st;
        rebuilt |= c->step_cap != had;
        // every parameter block is written on the first handle's stream, ahead of the fork
        const unsigned long long hp[2] = {seeds[i], (unsigned long long)first_sweep};
        CK(cudaMemcpyAsync(c->d_params, hp, sizeof hp, cudaMemcpyHostToDevice, c0->stream));
    }
    Ctx *c = c0;   // error reports of the group go to its first handle
    if (rebuilt && g->exec) {
        cudaGraphExecDestroy(g->exec);
        g->exec = nullptr;
    }
    if (use_graph && g->exec && g->key[0] == nsweeps && g->key[1] == recompute && g->sigma == sigma) {
        CK(cudaGraphLaunch(g->exec, c0->stream));
        return QMCDU_OK;
    }
    int st = group_body(g, nsweeps, sigma, recompute);
    if (st) return st;
    if (!use_graph) return QMCDU_OK;
    if (g->exec) {
        cudaGraphExecDestroy(g->exec);
        g->exec = nullptr;
    }
    std::vector<bool> prof(g->hs.size());
    for (size_t i = 0; i < g->hs.size(); ++i) { prof[i] = g->hs[i]->prof; g->hs[i]->prof = false; }
    cudaGraph_t graph = nullptr;
    CK(cudaStreamBeginCapture(c0->stream, cudaStreamCaptureModeRelaxed));
    st = group_body(g, nsweeps, sigma, recompute);
    cudaError_t e = cudaStreamEndCapture(c0->stream, &graph);
    for (size_t i = 0; i < g->hs.size(); ++i) g->hs[i]->prof = prof[i];
    if (st) {
        if (graph) cudaGraphDestroy(graph);
        return st;
    }
    if (e != cudaSuccess) return cuda_fail(c0, e, "cudaStreamEndCapture (group)");
    e = cudaGraphInstantiate(&g->exec, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) {
        g->exec = nullptr;
        return cuda_fail(c0, e, "cudaGraphInstantiate (group)");
    }
    g->key[0] = nsweeps;
    g->key[1] = recompute;
    g->sigma = sigma;
    return QMCDU_OK;
}

int qmcdu_group_destroy(qmcdu_group_t gh)
{
    if (!gh) return QMCDU_ERR_ARG;
    GroupCtx *g = reinterpret_cast<GroupCtx *>(gh);
    for (Ctx *c : g->hs) cudaStreamSynchronize(c->stream);
    if (g->exec) cudaGraphExecDestroy(g->exec);
    if (g->fork) cudaEventDestroy(g->fork);
    for (auto ev : g->done)
        if (ev) cudaEventDestroy(ev);
    delete g;
    return QMCDU_OK;
}

int qmcdu_set_option(qmcdu_t h, int option, long long value)
{
    if (!h || value < 0) return QMCDU_ERR_ARG;
    Ctx *c = reinterpret_cast<Ctx *>(h);
    switch (option) {
    case QMCDU_OPT_SWEEP_PERSISTENT: c->opt_persistent = value ? 1 : 0; break;
    case QMCDU_OPT_RATIO_CTAS: c->opt_ratio_ctas = (int)std::min(value, 1LL << 20); break;
    case QMCDU_OPT_FLUSH_CTAS: c->opt_flush_ctas = (int)std::min(value, 1LL << 20); break;
    case QMCDU_OPT_WAIT_BUDGET_NS: c->opt_budget_ns = value ? value : 2000000000LL; break;
    case QMCDU_OPT_TEST_STALL: c->opt_stall = value ? 1 : 0; break;
    case QMCDU_OPT_MAX_CTAS: c->opt_max_ctas = (int)std::min(value, 1LL << 20); break;
    case QMCDU_OPT_GROUP_CTAS: c->opt_group_ctas = (int)std::min(value, 1LL << 20); break;
    case QMCDU_OPT_CLUSTER:
        if (value < 0 || value > 2) return QMCDU_ERR_ARG;
        c->opt_cluster = (int)value;
        break;
    case QMCDU_OPT_FP64_FLUSH:
        if (value < 0 || value > 2) return QMCDU_ERR_ARG;
        c->opt_fp64_flush = (int)value;
        break;
    case QMCDU_OPT_FIXED_SLOT:
        if (value > 1) return QMCDU_ERR_ARG;
        c->opt_fixed_slot = (int)value;
        break;
    default: return fail(c, QMCDU_ERR_ARG, "unknown option%s");
    }
    return QMCDU_OK;
}

// ---- walker subsets (serving: walkers join and leave between sweeps)

int qmcdu_footprint(int N, int K, int precision, int batch, unsigned long long *bytes)
{
    if (!bytes || N < 1 || N > QMCDU_MAX_N || K < 1 || K > QMCDU_MAX_K || K > N || batch < 1 ||
        batch > 65535 || precision < QMCDU_FP64 || precision > QMCDU_FP32_BF16X3)
        return QMCDU_ERR_ARG;
    Ctx c;
    c.N = N; c.K = K; c.prec = precision; c.batch = batch; c.ld = padded_ld(N);
    c.nsplit = (N + 255) / 256;
    configure_recompute(c);
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) == cudaSuccess &&
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) == cudaSuccess && sms > 0)
        c.num_sms = sms;
    else
        cudaGetLastError();      // no device: size the sweep scratch for 148 SMs
    size_t total = 0;
    alloc_state(&c, false, &total);
    *bytes = total;
    return QMCDU_OK;
}

// The handle restricted to walkers [w0, w0 + n) for the recompute kernels:
// device pointers offset, no host state.
static void range_view(const Ctx &c, int w0, int n, Ctx &v)
{
    const size_t wN = (size_t)c.N * c.ld, w = (size_t)w0;
    v.N = c.N; v.K = c.K; v.prec = c.prec; v.batch = n; v.ld = c.ld;
    v.stream = c.stream; v.device = c.device; v.num_sms = c.num_sms;
    v.nb = c.nb; v.nsplit = c.nsplit; v.status = c.status;
    v.gj_ctas = c.gj_ctas;
    v.gj_scr = c.gj_scr ? c.gj_scr + w * gj_mc_scratch_bytes(c.gj_ctas, c.nb) : nullptr;
    v.gj_ctr = c.gj_ctr ? c.gj_ctr + w * 32 : nullptr;
    v.opt_budget_ns = c.opt_budget_ns; v.nb1 = c.nb1;
    v.opt_group_ctas = c.opt_group_ctas; v.opt_max_ctas = c.opt_max_ctas;
    v.A = c.A + w * wN;
    v.Ainv = (char *)c.Ainv + w * wN * elem_size(c.prec);
    v.work = c.work + w * wN;
    v.piv = c.piv + w * c.N;
    v.colperm = c.colperm + w * c.N;
    v.Lt = c.Lt + w * c.nb * c.ld;
    v.R = c.R + w * c.nb * c.ld;
    v.lu_logabs = c.lu_logabs + w;
    v.lu_sign = c.lu_sign + w;
    v.eqs = c.eqs + (size_t)2 * c.N * w;
    v.drift = c.drift + 4 * w;
    v.logabs = c.logabs + w;
    v.sign = c.sign + w;
}

static int recompute_range(Ctx *c, int first, int count, int have_old)
{
    Ctx v;
    range_view(*c, first, count, v);
    CK(prof_begin(c, c->ev_recompute));
    CK(launch_recompute(v, have_old));
    CK(prof_end(c, c->ev_recompute));
    c->n_launch += 8 + 2 * ((c->N + c->nb - 1) / c->nb);
    c->n_recompute += 1;
    return QMCDU_OK;
}

int qmcdu_load_walkers(qmcdu_t h, int first, int count, const double *A,
                       const unsigned long long *seeds)
{
    if (!h || first < 0 || count < 0) return QMCDU_ERR_ARG;
    Ctx *c = reinterpret_cast<Ctx *>(h);
    if ((long long)first + count > c->batch) return fail(c, QMCDU_ERR_ARG, "walker range out of bounds%s");
    if (count == 0) return QMCDU_OK;
    if (!A && !seeds) return fail(c, QMCDU_ERR_ARG, "need matrices or seeds%s");
    int st = flush_all(c);
    if (st) return st;
    c->pending = false;
    const size_t N = c->N, ld = c->ld;
    if (A) {
        CK(cudaMemcpy2DAsync(c->A + (size_t)first * N * ld, ld * sizeof(double), A,
                             N * sizeof(double), N * sizeof(double), N * count, cudaMemcpyDefault,
                             c->stream));
    } else {
        st = stage_h2d(c, {{c->d_lseed, seeds, count * sizeof(unsigned long long)}});
        if (st) return st;
        CK(launch_init_matrix(*c, first, count, c->d_lseed));
        c->n_launch += 1;
    }
    CK(cudaMemsetAsync(c->kcount + first, 0, count * sizeof(int), c->stream));
    return recompute_range(c, first, count, 0);
}

int qmcdu_recompute_walkers(qmcdu_t h, int first, int count, double *drift_out)
{
    if (!h || first < 0 || count < 0) return QMCDU_ERR_ARG;
    Ctx *c = reinterpret_cast<Ctx *>(h);
    if ((long long)first + count > c->batch) return fail(c, QMCDU_ERR_ARG, "walker range out of bounds%s");
    if (count == 0) return QMCDU_OK;
    int st = flush_all(c);
    if (st) return st;
    c->pending = false;
    st = recompute_range(c, first, count, 1);
    if (st) return st;
    if (drift_out) {
        CK(cudaMemcpy2DAsync(drift_out, 2 * sizeof(double), c->drift + 4 * (size_t)first + 2,
                             4 * sizeof(double), 2 * sizeof(double), count, cudaMemcpyDefault,
                             c->stream));
        if (!is_device_ptr(drift_out)) return read_status(c);
    }
    return QMCDU_OK;
}

int qmcdu_sweep_walkers(qmcdu_t h, int count, const int *walkers, const unsigned long long *seeds,
                        const int *sweeps, double sigma, unsigned char *accepted_out,
                        double *ratios_out, long long *near_ties_out)
{
    if (!h || count < 0 || (count > 0 && (!walkers || !seeds || !sweeps))) return QMCDU_ERR_ARG;
    Ctx *c = reinterpret_cast<Ctx *>(h);
    if (!c->opt_persistent)
        return fail(c, QMCDU_ERR_STATE, "walker subsets need the persistent sweep%s");
    if (count > c->batch) return fail(c, QMCDU_ERR_ARG, "more walkers listed than the handle holds%s");
    std::vector<unsigned char> seen(c->batch, 0);
    for (int t = 0; t < count; ++t) {
        if (walkers[t] < 0 || walkers[t] >= c->batch || seen[walkers[t]])
            return fail(c, QMCDU_ERR_ARG, "walker list has an index out of range or twice%s");
        if (sweeps[t] < 0) return fail(c, QMCDU_ERR_ARG, "negative sweep number%s");
        seen[walkers[t]] = 1;
    }
    if (count == 0) return QMCDU_OK;
    int st = flush_all(c);
    if (st) return st;
    c->pending = false;
    // copied into pinned staging before the call returns: the caller's arrays may change
    st = stage_h2d(c, {{c->d_wlist, walkers, count * sizeof(int)},
                       {c->d_wseed, seeds, count * sizeof(unsigned long long)},
                       {c->d_wsweep, sweeps, count * sizeof(int)}});
    if (st) return st;
    CK(cudaMemsetAsync(c->sw_ties, 0, count * sizeof(long long), c->stream));
    SweepLaunch S{};
    S.sigma = sigma;
    S.acc_out = c->sw_acc;
    S.ratio_out = c->sw_ratio;
    S.ties = c->sw_ties;
    S.wlist = c->d_wlist;
    S.nlist = count;
    S.wseed = c->d_wseed;
    S.wsweep = c->d_wsweep;
    CK(launch_sweep(*c, S));
    c->n_launch += 3;
    c->opt_stall = 0;
    CK(cudaMemsetAsync(c->kcount, 0, c->batch * sizeof(int), c->stream));
    return copy_sweep_outputs(c, accepted_out, ratios_out, near_ties_out, count);
}

int qmcdu_sweep_shape(qmcdu_t h, int *shape5)
{
    if (!h || !shape5) return QMCDU_ERR_ARG;
    Ctx *c = reinterpret_cast<Ctx *>(h);
    for (int i = 0; i < 5; ++i) shape5[i] = c->last_sweep_shape[i];
    return QMCDU_OK;
}

}  // extern "C"

namespace qmcdu {
int copy_sweep_outputs(Ctx *c, unsigned char *accepted_out, double *ratios_out,
                       long long *near_ties_out, int rows)
{
    const int N = c->N;
    const size_t R = rows < 0 ? (size_t)c->batch : (size_t)rows;
    bool host_out = false;
    if (accepted_out) {
        CK(cudaMemcpyAsync(accepted_out, c->sw_acc, R * N, cudaMemcpyDefault, c->stream));
        host_out |= !is_device_ptr(accepted_out);
    }
    if (ratios_out) {
        CK(cudaMemcpyAsync(ratios_out, c->sw_ratio, R * N * sizeof(double), cudaMemcpyDefault,
                           c->stream));
        host_out |= !is_device_ptr(ratios_out);
    }
    if (near_ties_out) {
        CK(cudaMemcpyAsync(near_ties_out, c->sw_ties, R * sizeof(long long), cudaMemcpyDefault,
                           c->stream));
        host_out |= !is_device_ptr(near_ties_out);
    }
    if (host_out) return read_status(c);
    return QMCDU_OK;
}
}  // namespace qmcdu

extern "C" {

int qmcdu_gemm_bf16x3(int M, int N, int K, const float *A, int lda, const float *B, int ldb,
                      int b_trans, float *C, int ldc, float alpha, float beta, void *stream)
{
    if (M < 0 || N < 0 || K < 0 || (M && N && (!C || (K && (!A || !B)))) || lda < K ||
        ldb < (b_trans ? N : K) || ldc < N) {
        set_handleless_error("qmcdu_gemm_bf16x3: invalid sizes, strides or null pointer");
        return QMCDU_ERR_ARG;
    }
    cudaError_t e = launch_gemm_bf16x3(M, N, K, A, lda, 0, B, ldb, 0, b_trans, C, ldc, 0, alpha,
                                       beta, 1, nullptr, 0, 0, nullptr, 2000000000LL,
                                       (cudaStream_t)stream);
    if (e != cudaSuccess) {
        set_handleless_error(std::string("qmcdu_gemm_bf16x3: ") + cudaGetErrorString(e));
        return QMCDU_ERR_CUDA;
    }
    return QMCDU_OK;
}

int qmcdu_profile_enable(qmcdu_t h, int enable)
{
    if (!h) return QMCDU_ERR_ARG;
    Ctx *c = reinterpret_cast<Ctx *>(h);
    CK(cudaStreamSynchronize(c->stream));
    drop_events(c);
    c->prof = enable != 0;
    c->n_launch = c->n_flush = c->n_recompute = c->n_sync = c->n_ratio = c->n_accept = 0;
    CK(cudaMemsetAsync(c->sw_phase, 0, 11 * sizeof(unsigned long long), c->stream));
    CK(cudaStreamSynchronize(c->stream));
    return QMCDU_OK;
}

int qmcdu_profile_read(qmcdu_t h, double *out, int n)
{
    if (!h || !out || n < 0) return QMCDU_ERR_ARG;
    Ctx *c = reinterpret_cast<Ctx *>(h);
    CK(cudaStreamSynchronize(c->stream));
    double ms_flush = 0.0, ms_rec = 0.0, ms_sweep = 0.0;
    for (auto &p : c->ev_sweep) {
        float ms = 0.f;
        CK(cudaEventElapsedTime(&ms, p.first, p.second));
        ms_sweep += ms;
    }
    for (auto &p : c->ev_flush) {
        float ms = 0.f;
        CK(cudaEventElapsedTime(&ms, p.first, p.second));
        ms_flush += ms;
    }
    for (auto &p : c->ev_recompute) {
        float ms = 0.f;
        CK(cudaEventElapsedTime(&ms, p.first, p.second));
        ms_rec += ms;
    }
    unsigned long long ph[11];
    CK(cudaMemcpyAsync(ph, c->sw_phase, sizeof ph, cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    const double vals[21] = {(double)c->n_launch, (double)c->n_flush, ms_flush,
                             (double)c->n_recompute, ms_rec, (double)c->n_sync,
                             (double)c->n_ratio, (double)c->n_accept,
                             ph[0] * 1e-6, ph[1] * 1e-6, ph[2] * 1e-6, ph[3] * 1e-6,
                             ph[4] * 1e-6, ph[5] * 1e-6, ph[6] * 1e-6, ph[7] * 1e-6,
                             (double)c->ev_sweep.size(), ms_sweep,
                             ph[8] * 1e-6, ph[9] * 1e-6, ph[10] * 1e-6};
    for (int i = 0; i < n && i < 21; ++i) out[i] = vals[i];
    return QMCDU_OK;
}

int qmcdu_profile_sweep_times(qmcdu_t h, double *ms_out, int max_n, int *n_out)
{
    if (!h || max_n < 0 || (max_n > 0 && !ms_out) || !n_out) return QMCDU_ERR_ARG;
    Ctx *c = reinterpret_cast<Ctx *>(h);
    CK(cudaStreamSynchronize(c->stream));
    int n = 0;
    for (auto &p : c->ev_sweep) {
        if (n >= max_n) break;
        float ms = 0.f;
        CK(cudaEventElapsedTime(&ms, p.first, p.second));
        ms_out[n++] = ms;
    }
    *n_out = n;
    return QMCDU_OK;
}

int qmcdu_philox4x32_10(const unsigned *c0, const unsigned *c1, const unsigned *c2,
                        const unsigned *c3, int n, unsigned long long seed, unsigned *out,
                        void *stream)
{
    if (n < 0 || (n > 0 && (!c0 || !c1 || !c2 || !c3 || !out))) return QMCDU_ERR_ARG;
    cudaError_t e = launch_philox_fill(c0, c1, c2, c3, n, seed, out, (cudaStream_t)stream);
    return e == cudaSuccess ? QMCDU_OK : QMCDU_ERR_CUDA;
}

int qmcdu_proposal_draws(int N, int nwalkers, unsigned long long base_seed, int sweep, double *gauss_out,
                         double *unif_out, void *stream)
{
    if (N < 1 || N > QMCDU_MAX_N || nwalkers < 0 || sweep < 0 ||
        (nwalkers > 0 && (!gauss_out || !unif_out))) {
        set_handleless_error("qmcdu_proposal_draws: invalid sizes or null pointer");
        return QMCDU_ERR_ARG;
    }
    cudaError_t e = launch_proposal_draws(N, nwalkers, base_seed, sweep, gauss_out, unif_out,
                                          (cudaStream_t)stream);
    if (e != cudaSuccess) {
        set_handleless_error(std::string("qmcdu_proposal_draws: ") + cudaGetErrorString(e));
        return QMCDU_ERR_CUDA;
    }
    return QMCDU_OK;
}

}  // extern "C"

namespace qmcdu {
// qmcdu_load_walkers on another stream than the handle's (the serving loop's
// admission stream): the loaded walkers' kernels touch only their own slots
// and the seed buffer of loads, so they may overlap sweeps of other walkers.
int load_walkers_on(qmcdu_t h, cudaStream_t s, int first, int count,
                    const unsigned long long *seeds)
{
    Ctx *c = reinterpret_cast<Ctx *>(h);
    cudaStream_t keep = c->stream;
    c->stream = s;
    const int st = qmcdu_load_walkers(h, first, count, nullptr, seeds);
    c->stream = keep;
    return st;
}
}  // namespace qmcdu
