// qmcdu_internal.cuh -- shared definitions of libqmcdu's translation units.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/qmcdu.h"

namespace qmcdu {

// Leading dimension of every per-walker N-vector and N x N matrix: rows start
// on 128-byte boundaries for fp64 (16 elements) so vector loads stay aligned.
__host__ __device__ static inline int padded_ld(int N) { return (N + 15) / 16 * 16; }

// Device status word bits (latched; cleared by set_matrix).
enum : int {
    ST_SINGULAR = 1,   // zero / non-finite ratio accepted, or zero pivot
    ST_TIMEOUT = 2,    // spin-wait budget exceeded
    ST_BADARG = 4,     // electron index out of range seen on the device
};

// Per-proposal scratch record (fp64) for walker b at rs + b * rs_stride:
//   [0] d = v . A^{-1}[:, j]     [1] r (the ratio)       [2] k at proposal
//   [3] electron j               [4..4+K) x = Kinv c     [4+K..4+2K) y = Kinv' b
__host__ __device__ static inline int rs_stride(int K) { return 4 + 2 * K; }

struct Ctx {
    int N, K, prec, batch, ld;
    cudaStream_t stream;
    int device;
    // walker state
    double *A = nullptr;        // batch x N x ld, row-major
    void *Ainv = nullptr;       // batch x N x ld, column-major (working precision)
    void *P = nullptr;          // batch x K x ld  (P[m] = A^{-1}[:, idx_m])
    void *V = nullptr;          // batch x K x ld  (V[m] = change u_m = v_m - a_idx_m of move m)
    double *vstash = nullptr;   // batch x ld fp64 copy of the pending proposed row
    double *Kinv = nullptr;     // batch x K x K, row-major
    int *idx = nullptr;         // batch x K
    int *kcount = nullptr;      // batch
    double *logabs = nullptr;   // batch
    int *sign = nullptr;        // batch
    double *rs = nullptr;       // batch x rs_stride(K)
    double *partial = nullptr;  // batch x nsplit x (2K+1)
    unsigned char *acc = nullptr; // batch: decision of the last resolved proposal
    int *elec_d = nullptr;      // batch
    unsigned char *mask_d = nullptr; // batch
    int *status = nullptr;      // 1 int
    // flush workspace
    void *Tbuf = nullptr;       // batch x K x ld  (T = V^t A^{-1}, row m)
    void *Wbuf = nullptr;       // batch x K x ld  (W = P Kinv, column m)
    // recompute workspace
    double *work = nullptr;     // batch x N x ld fp64
    int *piv = nullptr;         // batch x N
    int *colperm = nullptr;     // batch x N
    double *Lt = nullptr;       // batch x nb x ld
    double *R = nullptr;        // batch x nb x ld
    int *eqs = nullptr;         // batch x 2 x N: the recompute's power-of-two row and column scales
    double *lu_logabs = nullptr; // batch
    int *lu_sign = nullptr;     // batch
    double *drift = nullptr;    // batch x 4 (sums for the drift report)
    double *pair_logabs = nullptr; // batch: log|det| of this handle's walkers and another's, summed
    int *pair_sign = nullptr;      // batch: the product of their signs
    // sweep outputs (device staging)
    unsigned char *sw_acc = nullptr; // batch x N
    double *sw_ratio = nullptr;      // batch x N
    long long *sw_ties = nullptr;    // batch
    signed char *sw_override = nullptr; // batch x N
    // host mirror of the delay queues (exact for the per-call API)
    std::vector<int> h_k;
    std::vector<std::vector<unsigned char>> h_inq;  // batch x N membership
    std::vector<int> h_elec;
    bool pending = false;
    int nsplit = 1;
    int nb = 16;                     // recompute: Lt / R rows per walker, the multi-CTA panel width
    int nb1 = 16;                    // recompute: the one-CTA panel width (<= nb)
    int gj_ctas = 0;                 // > 0: each walker's recompute panels over this many CTAs
    unsigned char *gj_scr = nullptr; // their pivot-candidate buffers (batch x gj_mc_scratch_bytes)
    unsigned *gj_ctr = nullptr;      // their barrier counters (batch x 32 words)
    std::string err;
    // profiling (qmcdu_profile_*)
    bool prof = false;
    long long n_launch = 0, n_flush = 0, n_recompute = 0, n_sync = 0, n_ratio = 0, n_accept = 0;
    std::vector<std::pair<cudaEvent_t, cudaEvent_t>> ev_flush, ev_recompute, ev_sweep;
    // persistent sweep (kernels_sweep.cu)
    int num_sms = 148;
    double *sw_partial = nullptr;   // capacity x 2 x (2K+2)
    size_t sw_partial_len = 0;
    unsigned *sw_sync = nullptr;    // capacity x 4
    unsigned long long *sw_phase = nullptr;  // 11 phase timers of the persistent sweep
    double *sw_gauss = nullptr;     // batch x N x ld proposal Gaussians of the current sweep
    double *sw_unif = nullptr;      // batch x N Metropolis uniforms of the current sweep
    int sync_words = 0;
    int last_sweep_shape[5] = {0, 0, 0, 0, 0};   // Gf, Gr, groups, chunk, cb
    // options (qmcdu_set_option)
    int opt_persistent = 1;
    int opt_ratio_ctas = 0;
    int opt_flush_ctas = 0;
    long long opt_budget_ns = 2000000000LL;
    int opt_stall = 0;
    int opt_max_ctas = 0;            // cap on the persistent sweep's grid (0: whole GPU)
    int opt_group_ctas = 0;          // fixed CTAs per walker group (0: from the batch)
    int opt_fp64_flush = 0;          // 0: auto, 1: fp64 arithmetic only, 2: emulated on the tensor cores
    int opt_fixed_slot = 0;          // 1: rejected proposals take queue slots (Sec. II)
    int opt_cluster = 0;             // 0, 1: global-memory exchange; 2: cluster mode where it applies
    int last_cluster = 0;            // cluster size of the last persistent sweep (0: none)
    // emulated-fp64 flush of the persistent sweep (kernels_sweep.cu): scratch of
    // oz_groups walker groups, oz_stride bytes each
    unsigned char *oz = nullptr;
    size_t oz_stride = 0;
    int oz_groups = 0;
    // walker subsets (qmcdu_sweep_walkers): list, keys and sweep numbers
    int *d_wlist = nullptr;
    unsigned long long *d_wseed = nullptr;
    int *d_wsweep = nullptr;
    unsigned long long *d_lseed = nullptr;   // keys of qmcdu_load_walkers' draws
    // pinned staging ring for small host-to-device argument copies (a copy
    // from pageable memory would make the host wait for the stream first)
    static constexpr int NPIN = 16;
    char *pin_buf = nullptr;
    size_t pin_cap = 0;                      // bytes per slot
    int pin_next = 0;
    cudaEvent_t pin_ev[NPIN] = {};
    bool pin_used[NPIN] = {};
    // qmcdu_step: device parameter block and per-sweep outputs, graph cache
    unsigned long long *d_params = nullptr;   // [0] base seed, [1] first sweep index
    unsigned char *step_acc = nullptr;        // nsweeps x batch x N
    double *step_ratio = nullptr;             // nsweeps x batch x N
    long long *step_ties = nullptr;           // nsweeps x batch
    int step_cap = 0;                         // sweeps the step buffers hold
    cudaGraphExec_t graph_exec = nullptr;
    int graph_key[3] = {-1, -1, -1};          // nsweeps, recompute, sigma bits (hashed)
    double graph_sigma = 0.0;
};

struct SweepLaunch {
    unsigned long long seed;
    int sweep;
    const unsigned long long *params;   // device [seed, first sweep] (then seed/sweep unused)
    int sweep_offset;                   // added to params[1]
    double sigma;
    const signed char *override;
    unsigned char *acc_out;
    double *ratio_out;
    long long *ties;
    // optional subset of walkers (device arrays of nlist entries): walker
    // wlist[t] draws from key wseed[t] and sweep number wsweep[t]
    const int *wlist;
    int nlist;
    const unsigned long long *wseed;
    const int *wsweep;
};
cudaError_t launch_sweep(Ctx &c, const SweepLaunch &L);
// Scratch bytes of one walker group of the emulated-fp64 flush (0: not used for N, K).
size_t oz_group_bytes(int N, int K);
// qmcdu_flush of fp64 walkers on the tensor cores (W = P Kinv in c.Wbuf); cudaErrorNotSupported
// where it does not apply.
cudaError_t launch_flush_oz(Ctx &c, int kthresh);
cudaError_t prof_begin(Ctx *c, std::vector<std::pair<cudaEvent_t, cudaEvent_t>> &v);
cudaError_t prof_end(Ctx *c, std::vector<std::pair<cudaEvent_t, cudaEvent_t>> &v);

size_t elem_size(int prec);

// Error text of the last failed call that has no handle (qmcdu_last_error(NULL)).
void set_handleless_error(const std::string &msg);

// ---- launchers (kernels_move.cu) ----
struct RatioLaunch {
    const double *v_in;         // [batch][N] or null when generating
    const int *elec;            // device [batch] or null (uniform electron)
    int uniform_elec;
    int generate;               // 1: v = a_j + sigma g (Philox)
    unsigned long long seed;
    int sweep;
    double sigma;
    double *ratio_out;          // device [batch] or null
    int kmax = -1;              // largest queue length of any walker (-1: K - 1)
};
cudaError_t launch_ratio(Ctx &c, const RatioLaunch &L);

struct AcceptLaunch {
    int mode;                   // 0: mask (device), 1: Metropolis with Philox u
    const unsigned char *mask;  // mode 0
    unsigned long long seed;    // mode 1
    int sweep;
    const signed char *override; // mode 1, [batch][N] or null
    unsigned char *acc_out;     // [batch][N] or null (mode 1)
    double *ratio_out;          // [batch][N] or null (mode 1)
    long long *ties;            // [batch] or null (mode 1)
};
cudaError_t launch_accept(Ctx &c, const AcceptLaunch &L);
cudaError_t launch_sm_update(Ctx &c);

// ---- flush (kernels_gemm.cu) ----
cudaError_t launch_flush(Ctx &c, int kthresh);

// ---- recompute (kernels_recompute.cu) ----
cudaError_t launch_recompute(Ctx &c, int have_old_inverse);
cudaError_t launch_init_matrix(Ctx &c, int w0, int n, const unsigned long long *seeds);
// Recompute panels over several CTAs per walker (kernels_sweep.cu).
cudaError_t launch_gj_panel_mc(Ctx &c, int c0, int nbe);
size_t gj_mc_scratch_bytes(int P, int nb);
// Recompute shape of a handle: the panel width and, for a few walkers, the CTAs per walker.
void configure_recompute(Ctx &c);
cudaError_t launch_gj_update(Ctx &c, int nbe);
// the same update as the emulated-fp64 tensor-core contraction of the flush
// (fp64 handles with its scratch); cudaErrorNotSupported where it does not apply
cudaError_t launch_gj_update_oz(Ctx &c, int nbe);
int choose_panel_width(int N);

// ---- tensor-core contraction (kernels_tc.cu) ----
cudaError_t launch_gemm_bf16x3(int M, int N, int K, const float *A, long long lda, long long sA,
                               const float *B, long long ldb, long long sB, int b_trans, float *C,
                               long long ldc, long long sC, float alpha, float beta, int batch,
                               const int *kdyn, int kdyn_is_n, int kthresh, int *status,
                               long long budget_ns, cudaStream_t s);

// ---- utilities (kernels_move.cu) ----
cudaError_t launch_logdet_pair(int batch, const double *l1, const int *s1, const double *l2, const int *s2,
                               double *lout, int *sout, cudaStream_t s);
cudaError_t launch_proposal_draws(int N, int nw, unsigned long long base_seed, int sweep, double *gauss,
                                  double *unif, cudaStream_t s);
cudaError_t launch_philox_fill(const unsigned *c0, const unsigned *c1, const unsigned *c2,
                               const unsigned *c3, int n, unsigned long long seed,
                               unsigned *out, cudaStream_t s);
cudaError_t launch_inverse_export(Ctx &c, double *dst);

// qmcdu_load_walkers (drawn matrices) on stream s instead of the handle's.
int load_walkers_on(qmcdu_t h, cudaStream_t s, int first, int count,
                    const unsigned long long *seeds);

}  // namespace qmcdu
