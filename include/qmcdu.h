/*
 * qmcdu.h -- C ABI of libqmcdu: rank-K delayed Slater-determinant updates for
 * quantum Monte Carlo on one NVIDIA B300 (sm_103a).
 *
 * Method: McDaniel, D'Azevedo, Li, Wong, Kent, "Delayed Slater determinant
 * update algorithms for high efficiency quantum Monte Carlo".
 *   - A single-electron move changes one row of the Slater matrix; its
 *     acceptance probability is the squared determinant ratio, which the
 *     matrix determinant lemma gives from the explicit inverse (Sec. I, Eq. 1).
 *   - K = 1 applies every accepted move at once by Sherman-Morrison (Eq. 2).
 *   - K > 1 delays accepted moves: ratios come from the generalised lemma
 *     (Eq. 3) through N x k panels and a k x k inverse, and the queued moves
 *     are applied en bloc by Sherman-Morrison-Woodbury (Eq. 4) when k reaches
 *     K or the sweep ends (Sec. II). Rejected moves change nothing.
 *   - Every formula is taken in the paper's change form: a move of electron j
 *     to the new row v is the rank-1 change e_j u' with u = v - a_j, its
 *     ratio is 1 + u . A^{-1}[:, j] (Eq. 1), and the queue holds the changes of
 *     the accepted moves (Eq. 3-4). The change is small next to the row, so
 *     the error of the running inverse enters the ratio only through u.
 *   - The determinant is checked against direct calculation after a sweep
 *     (Sec. III): qmcdu_recompute.
 *
 * Conventions (row form; the paper's matrix transposed, same determinant):
 *   A       batch x N x N fp64, row-major; row j holds electron j's orbitals.
 *   A^{-1}  kept in the working precision, COLUMN-major: column j of A^{-1}
 *           is contiguous (it is the vector the ratio of electron j needs).
 *   Every call is asynchronous on the handle's stream. A handle is bound to
 *   one stream and one thread; it is not thread-safe.
 *   "host or device" pointers: any pointer the CUDA runtime can copy from or
 *   to with cudaMemcpyDefault (pinned or pageable host memory, device
 *   memory). "device" pointers: device memory the caller owns, to be read or
 *   written in stream order.
 *   Errors found on the device (a singular or non-finite ratio on accept, a
 *   zero pivot in the recompute, an exceeded spin-wait budget) are latched in a
 *   device status word and returned by the next synchronising call
 *   (qmcdu_sync, qmcdu_logdet, qmcdu_get_*); the handle must then be reloaded
 *   with qmcdu_set_matrix.
 */
#ifndef QMCDU_H
#define QMCDU_H

#ifdef __cplusplus
extern "C" {
#endif

typedef struct qmcdu_ctx *qmcdu_t;
typedef struct qmcdu_group_ctx *qmcdu_group_t;
typedef struct qmcdu_md_ctx *qmcdu_md_t;

/* Working precision of A^{-1}, the panels and the flush. */
enum {
    QMCDU_FP64 = 0,        /* everything fp64                                     */
    QMCDU_FP32 = 1,        /* A^{-1}, panels, flush fp32; k x k inverse, ratios,  */
                           /* log-det and the recompute fp64                      */
    QMCDU_FP32_BF16X3 = 2  /* as FP32, flush on tensor cores with split-bf16 x3   */
                           /* (tcgen05) wherever a flush block is >= 128       */
                           /* columns and K <= 64; fp32 SIMT flush otherwise.  */
                           /* Small moves (DMC-like, sigma ~ 0.1) only: at     */
                           /* sigma = 1 its ratio errors reach 0.02-0.16 and   */
                           /* most decisions fall within them of a tie, which  */
                           /* no tolerance of the method accepts; use FP32     */
};

enum {
    QMCDU_OK = 0,
    QMCDU_ERR_ARG = 1,      /* invalid argument; nothing was launched             */
    QMCDU_ERR_STATE = 2,    /* call out of order (accept without ratio, ...)      */
    QMCDU_ERR_SINGULAR = 3, /* zero / non-finite ratio accepted, or zero pivot    */
    QMCDU_ERR_OOM = 4,      /* device allocation failed                           */
    QMCDU_ERR_CUDA = 5,     /* CUDA runtime error (text in qmcdu_last_error)      */
    QMCDU_ERR_TIMEOUT = 6   /* a device spin-wait exceeded its budget             */
};

/* Limits of one handle. */
#define QMCDU_MAX_N 8192
#define QMCDU_MAX_K 256

/*
 * Create a handle for `batch` independent walkers of N electrons with delay K
 * (K = 1: Sherman-Morrison, Eq. 2; 1 < K <= min(N, QMCDU_MAX_K): delayed,
 * Eq. 3-4). `stream` is a cudaStream_t (NULL: the legacy default stream).
 * The library allocates and owns all walker state on the current device:
 * A, A^{-1}, the N x K panels, the K x K inverse, the recompute workspace.
 * On success *out receives the handle. Errors: ERR_ARG, ERR_OOM, ERR_CUDA.
 */
int qmcdu_create(int N, int K, int precision, int batch, void *stream, qmcdu_t *out);

/* Release the handle and its device memory (synchronises its stream). */
int qmcdu_destroy(qmcdu_t h);

/*
 * Load the Slater matrices (host or device, batch x N x N fp64 row-major) and
 * compute A^{-1} and log|det A| by the fp64 recompute (see qmcdu_recompute).
 * Clears pending moves and the error latch. ERR_SINGULAR (at the next sync)
 * if a matrix is singular.
 */
int qmcdu_set_matrix(qmcdu_t h, const double *A);

/* Copy the current A (host or device, batch x N x N fp64 row-major). */
int qmcdu_get_matrix(qmcdu_t h, double *A_out);

/*
 * Copy the current A^{-1} (host or device, batch x N x N fp64, column-major:
 * element (i, c) of A^{-1} at [b][c][i]). Pending delayed moves are flushed
 * first (Eq. 4), so this is the inverse of the current A. Synchronises.
 */
int qmcdu_get_inverse(qmcdu_t h, double *Ainv_out);

/*
 * Determinant ratio of one proposed move per walker (Eq. 1 for k = 0; the
 * generalised lemma, Eq. 3, through the queued panels otherwise):
 *   r_b = det(A_b with row elec[b] replaced by v_b) / det(A_b).
 *   elec       host, [batch] electron indices in [0, N)
 *   v          device, [batch][N] fp64 proposed rows (read during the call's
 *              stream order; may be reused afterwards)
 *   ratio_out  device, [batch] fp64
 * If a walker's electron is already in its delay queue, that walker's queue is
 * flushed first (the paper's queue holds distinct moves). Leaves one pending
 * proposal per walker for qmcdu_accept.
 */
int qmcdu_ratio(qmcdu_t h, const int *elec, const double *v, double *ratio_out);

/*
 * Resolve the pending proposals: mask (host, [batch], 1 = accept, 0 = reject).
 * Accepted moves are queued (K > 1: panel append and bordered k x k inverse
 * update; a full queue is flushed at once, Eq. 4) or applied (K = 1, Eq. 2);
 * A's row and the running log|det A| and sign are updated. Rejected moves
 * leave the state untouched. ERR_STATE without a pending proposal.
 */
int qmcdu_accept(qmcdu_t h, const unsigned char *mask);

/* Apply all queued moves now (Eq. 4). A no-op when the queues are empty. */
int qmcdu_flush(qmcdu_t h);

/*
 * Recompute A^{-1} and log|det A| from A in fp64 (Sec. III's direct
 * calculation): Gauss-Jordan elimination with partial pivoting, whose pivots
 * are the diagonal of U in P A' = L U. Queued moves are flushed first.
 * drift_out (host or device, [batch][2] fp64, or NULL): per walker
 * |log|det|_running - log|det|_recomputed| and
 * ||A^{-1}_running - A^{-1}_recomputed||_F / ||A^{-1}_recomputed||_F.
 */
int qmcdu_recompute(qmcdu_t h, double *drift_out);

/* Running log|det A| (host or device, [batch] fp64) and sign (host or device,
 * [batch] int, +1/-1). Synchronises. */
int qmcdu_logdet(qmcdu_t h, double *logabs, int *sign);

/*
 * A walker of two determinants, one per spin (the paper sizes its solid-state
 * walkers by both spins, Sec. III): walker b's up determinant in handle h1
 * and its down determinant in handle h2 (same batch, same device). Writes
 * log|det A_up det A_down| = log|det A_up| + log|det A_down| (host or device,
 * [batch] fp64) and the product of the signs (host or device, [batch] int),
 * formed on the device on h1's stream after h2's work so far. Synchronises
 * both handles. ERR_ARG for a null or repeated handle, or handles that differ
 * in batch or device.
 */
int qmcdu_logdet_product(qmcdu_t h1, qmcdu_t h2, double *logabs, int *sign);

/*
 * One Metropolis sweep per walker, entirely on the device: electrons
 * j = 0..N-1 in order; proposal v = a_j + sigma * g (a_j the current row j,
 * g ~ N(0,1)^N); accept iff u < min(1, r^2) (Sec. I); queued moves flushed at
 * k = K and at the end of the sweep (Sec. II). g and u come from the
 * Philox4x32-10 counter generator (Salmon et al., SC'11) with key
 * base_seed + walker and counters (j, sweep_index, 1, block) for g and
 * (j, sweep_index, 0, 0) for u; g pairs by Box-Muller.
 *   override      host or device [batch][N] int8 (-1 decide, 0 reject,
 *                 1 accept), or NULL
 *   accepted_out  host or device [batch][N] uint8, or NULL
 *   ratios_out    host or device [batch][N] fp64, or NULL
 *   near_ties_out host or device [batch] int64 (count of
 *                 |min(1, r^2) - u| < 1e-10), or NULL
 * Outputs written to host memory are valid when the call returns; to device
 * memory, in stream order.
 */
int qmcdu_sweep(qmcdu_t h, unsigned long long base_seed, int sweep_index, double sigma,
                const signed char *override, unsigned char *accepted_out,
                double *ratios_out, long long *near_ties_out);

/*
 * A step of the benchmark's and the paper's measurement protocol (Sec. III:
 * complete sweeps, then the determinant checked against direct calculation):
 * `nsweeps` sweeps numbered first_sweep.. (as qmcdu_sweep, no override), then,
 * if `recompute`, the fp64 recompute (qmcdu_recompute). With use_graph = 1 the
 * kernels of the step are captured into a CUDA graph on first use and replayed
 * by later calls with the same (nsweeps, recompute, sigma); the seed and first
 * sweep index are read from device memory, so they may change between calls.
 * Graph capture needs a handle on a non-default stream (ERR_ARG otherwise).
 *   accepted_out  host or device [nsweeps][batch][N] uint8, or NULL
 *   drift_out     host or device [batch][2] (as qmcdu_recompute), or NULL
 * Handles with persistent sweeps switched off run the sweeps call by call
 * without a graph.
 */
int qmcdu_step(qmcdu_t h, unsigned long long base_seed, int first_sweep, int nsweeps, double sigma,
               int recompute, int use_graph, unsigned char *accepted_out, double *drift_out);

/* Results of the last qmcdu_step / qmcdu_group_step of this handle for its
 * first `nsweeps` sweeps (host or device buffers, each may be NULL): accept
 * masks [nsweeps][batch][N] uint8, ratios [nsweeps][batch][N] fp64, near-tie
 * counts [nsweeps][batch] int64. Synchronises. */
int qmcdu_step_results(qmcdu_t h, int nsweeps, unsigned char *accepted_out, double *ratios_out,
                       long long *near_ties_out);

/*
 * Walkers of uneven N: one handle per size class, stepped together. The group
 * gives each handle a share of the SMs in proportion to its flush work
 * (batch N^3; QMCDU_OPT_MAX_CTAS) so that the classes' persistent sweeps run
 * side by side, forks every handle's stream from the first handle's stream
 * and joins them back, and (use_graph) captures the whole fork/join step in
 * one CUDA graph. seeds[i] is handle i's base seed. Handles without
 * persistent sweeps are refused (ERR_ARG). The group does not own the
 * handles; destroy it before them.
 */
int qmcdu_group_create(qmcdu_t *handles, int n, qmcdu_group_t *out);
int qmcdu_group_step(qmcdu_group_t g, const unsigned long long *seeds, int first_sweep,
                     int nsweeps, double sigma, int recompute, int use_graph);
int qmcdu_group_destroy(qmcdu_group_t g);

/* Wait for the handle's stream and return the latched device status. */
int qmcdu_sync(qmcdu_t h);

/* Text of the last error on this handle ("" if none). Valid until the next call.
 * With h == NULL: the last error of a call without a handle on this thread. */
const char *qmcdu_last_error(qmcdu_t h);

/*
 * Philox4x32-10 on the device (Salmon et al., SC'11): out[4 i + w] = word w of
 * the generator at counter (c0[i], c1[i], c2[i], c3[i]) and key
 * (seed & 0xffffffff, seed >> 32). All pointers device, n entries per counter
 * word, 4 n outputs. Runs on `stream` (cudaStream_t, NULL = default).
 */
int qmcdu_philox4x32_10(const unsigned *c0, const unsigned *c1, const unsigned *c2,
                        const unsigned *c3, int n, unsigned long long seed,
                        unsigned *out, void *stream);

/*
 * The random draws of one sweep (the a_j + sigma g proposals and the
 * Metropolis uniforms of Sec. I), exactly as qmcdu_sweep / qmcdu_step draw
 * them on the device for walkers 0..nwalkers-1 of base seed `base_seed`
 * (walker w's key base_seed + w) and sweep number `sweep`:
 *   gauss_out  device [nwalkers][N][N] fp64: row j = the Gaussians g of
 *              electron j's proposal (Philox4x32-10, Box-Muller pairs)
 *   unif_out   device [nwalkers][N] fp64: u of electron j
 * Lets a caller replay a sweep elsewhere (a checkpoint, a reference
 * implementation) from the very proposals the device used. Allocates nothing;
 * asynchronous on `stream`. ERR_ARG for N outside 1..QMCDU_MAX_N, a negative
 * count or sweep, null pointers (text at qmcdu_last_error(NULL)).
 */
int qmcdu_proposal_draws(int N, int nwalkers, unsigned long long base_seed, int sweep,
                         double *gauss_out, double *unif_out, void *stream);

/*
 * Profiling. While enabled, the library records CUDA events on the handle's
 * stream around every flush (Eq. 4) and every recompute, and counts its
 * kernel launches. qmcdu_profile_enable(h, 1) resets the counters; 0 stops.
 * qmcdu_profile_read synchronises and writes n <= 21 values to out (host):
 *   [0] kernel launches  [1] flushes   [2] flush time (ms)
 *   [3] recomputes       [4] recompute time (ms)   [5] stream syncs inside
 *   sweeps  [6] ratio launches  [7] accept launches
 *   [8..15] persistent sweeps, walker 0's lead CTA, time (ms) in: partial
 *   dot products, staging the next proposal, the cluster-mode exchange wait
 *   (near zero otherwise), waiting for and summing the other CTAs' partials
 *   plus the decision, accept, the flush's first barrier, the flush
 *   arithmetic, the flush's second barrier (host-driven sweeps time [2]
 *   instead)
 *   [16] persistent sweep kernel launches  [17] their total time (ms)
 *   [18..20] the emulated-fp64 flush's phases (walker 0's lead CTA, barrier
 *   waits included), time (ms): T' = V'A^{-1} over row chunks; the reduction
 *   and slicing of T and W; the update of A^{-1}
 */
int qmcdu_profile_enable(qmcdu_t h, int enable);
int qmcdu_profile_read(qmcdu_t h, double *out, int n);

/* While profiling is enabled: the device time (ms, CUDA events on the
 * handle's stream) of each persistent sweep launch since the last enable, in
 * launch order, into ms_out (host, up to max_n values); *n_out receives the
 * count written. One launch sweeps every walker of the handle once, so these
 * are per-sweep latencies. Synchronises. */
int qmcdu_profile_sweep_times(qmcdu_t h, double *ms_out, int max_n, int *n_out);

/*
 * Options of a handle (value semantics in brackets; 0 restores the default):
 *   QMCDU_OPT_SWEEP_PERSISTENT  [1] qmcdu_sweep runs as one persistent
 *       cooperative kernel per sweep; 0 drives the per-proposal kernels from
 *       the host (same results, for comparison and debugging)
 *   QMCDU_OPT_RATIO_CTAS   [auto] CTAs per walker that compute the ratios
 *   QMCDU_OPT_FLUSH_CTAS   [auto] CTAs per walker that apply the flush
 *   QMCDU_OPT_WAIT_BUDGET_NS [2e9] time budget of every device spin-wait;
 *       on expiry the call fails with ERR_TIMEOUT at the next sync
 *   QMCDU_OPT_TEST_STALL   [0] test hook: the next persistent sweep's first
 *       proposal waits for partial sums that never come, so that its wait runs
 *       out of budget
 *   QMCDU_OPT_MAX_CTAS     [whole GPU] cap on the persistent sweep's grid, so
 *       that several handles' sweeps can run side by side (qmcdu_group_*)
 *   QMCDU_OPT_GROUP_CTAS   [from the batch] fixed CTAs per walker group (at
 *       most the grid cap). Every walker then gets the same arithmetic, in the
 *       same order, whatever the number of walkers in the launch: its results
 *       are bit-identical alone and in a batch (qmcdu_sweep_walkers, serving)
 *   QMCDU_OPT_FP64_FLUSH   [0: auto] the flush (Eq. 4) of fp64 walkers: 1 =
 *       fp64 arithmetic units only; 2 (and auto) = the contraction emulated on
 *       the tensor cores (operands cut into seven 8-bit slices relative to
 *       shared exponents after a power-of-two rescaling of every contraction
 *       index, exact fp32 accumulation of slice products, exact integer
 *       recombination; the error of fp64 arithmetic, also on matrices whose
 *       rows and columns span many binades) where it applies: 4 <= K <= 32
 *       and walker groups of two or more CTAs; also the recompute's rank-32
 *       updates (on the equilibrated matrix: the recompute scales A's rows
 *       and columns by powers of two first) where the handle owns the GPU
 *   QMCDU_OPT_CLUSTER      [0: off] persistent sweeps of fp64 walkers (at
 *       most 4 walkers, N >= 1024, no fixed group shape, ratio or flush CTA
 *       counts left automatic): 2 = the 16 ratio CTAs of a walker form one
 *       thread-block cluster and exchange the partial dot products of every
 *       proposal through distributed shared memory (sweep_shape then reports
 *       16 ratio CTAs); results agree with the global-memory exchange to
 *       rounding (other sums of the same terms). Slower than the default at
 *       N = 2048 (fp64 work on 16 CTAs instead of 64); 0 and 1 = off
 *   QMCDU_OPT_FIXED_SLOT   [0: off] 1 = Sec. II's fixed slots in the
 *       persistent sweep: a rejected proposal also takes a queue slot, as
 *       an unchanged row (a zero change, which leaves the ratios of later
 *       proposals and the determinant as they are), so that every walker's
 *       queue is flushed every K proposals whatever its acceptance. The
 *       results are those of the default policy (rejected moves take no slot)
 *       up to rounding. qmcdu_sweep with QMCDU_OPT_SWEEP_PERSISTENT = 0
 *       returns ERR_STATE while it is set.
 * Returns ERR_ARG for an unknown option or a negative value.
 */
enum {
    QMCDU_OPT_SWEEP_PERSISTENT = 1,
    QMCDU_OPT_RATIO_CTAS = 2,
    QMCDU_OPT_FLUSH_CTAS = 3,
    QMCDU_OPT_WAIT_BUDGET_NS = 4,
    QMCDU_OPT_TEST_STALL = 5,
    QMCDU_OPT_MAX_CTAS = 6,
    QMCDU_OPT_GROUP_CTAS = 7,
    QMCDU_OPT_FP64_FLUSH = 8,
    QMCDU_OPT_CLUSTER = 9,
    QMCDU_OPT_FIXED_SLOT = 10
};
int qmcdu_set_option(qmcdu_t h, int option, long long value);

/*
 * Shape of the last persistent sweep launch (host, 5 ints): CTAs per walker
 * group (flush), ratio CTAs per group, walker groups, rows per ratio CTA,
 * flush kind: columns per shared-memory tile (> 0 with the queue rows
 * resident in the ratio CTAs, < 0 without), 1000 for the split-bf16
 * tensor-core flush, 2000 for the emulated-fp64 tensor-core flush.
 */
int qmcdu_sweep_shape(qmcdu_t h, int *shape5);

/*
 * Walker subsets: walkers that join and leave a handle between sweeps
 * (continuous batching in a serving loop). The paper runs one walker per
 * process; these calls let one handle hold `batch` walker slots whose walkers
 * advance at their own pace.
 *
 * qmcdu_footprint: device bytes a handle of these sizes allocates (every
 * cudaMalloc of qmcdu_create, each rounded up to 512 bytes). Host only; needs
 * no GPU. ERR_ARG for sizes qmcdu_create would refuse.
 *
 * qmcdu_load_walkers: walkers first..first+count-1 get new matrices and
 * start afresh (empty delay queues), then A^{-1} and log|det A| are computed
 * from them by the fp64 LU of qmcdu_recompute. A: host or device
 * [count][N][N] fp64 row-major, copied; or NULL to draw each walker's matrix
 * on the device from its key seeds[t] (host [count]): A_ij ~ N(0,1), Box-
 * Muller pairs at Philox counters (i, 0, 2, pair), the draws of qmcdu_create's
 * conventions above. Pending queues of the other walkers are flushed first.
 * Asynchronous. ERR_ARG: range outside 0..batch, both A and seeds NULL.
 *
 * qmcdu_recompute_walkers: qmcdu_recompute for walkers first..first+count-1
 * only; drift_out host or device [count][2] (log-det, inverse) or NULL.
 *
 * qmcdu_sweep_walkers: one Metropolis sweep (as qmcdu_sweep) of the `count`
 * listed walkers only. walkers[t] (distinct slots in 0..batch-1) draws its
 * proposals and uniforms from key seeds[t] and sweep number sweeps[t] (host
 * arrays, read before the call returns); unlisted walkers are untouched.
 * Outputs (host or device, each may be NULL) are compact, in list order:
 * accepted_out [count][N] uint8, ratios_out [count][N] fp64, near_ties_out
 * [count] int64; host outputs make the call synchronise. Needs persistent
 * sweeps (ERR_STATE otherwise). ERR_ARG: bad or repeated index, negative
 * sweep number, null arrays with count > 0.
 */
int qmcdu_footprint(int N, int K, int precision, int batch, unsigned long long *bytes);
int qmcdu_load_walkers(qmcdu_t h, int first, int count, const double *A,
                       const unsigned long long *seeds);
int qmcdu_recompute_walkers(qmcdu_t h, int first, int count, double *drift_out);
int qmcdu_sweep_walkers(qmcdu_t h, int count, const int *walkers, const unsigned long long *seeds,
                        const int *sweeps, double sigma, unsigned char *accepted_out,
                        double *ratios_out, long long *near_ties_out);

/*
 * Determinant ratio of one proposed move for callers that cannot allocate
 * device memory. The paper has no counterpart to this entry point; it serves
 * callers for whom cudaMalloc is not an option: code that must not
 * synchronise the device (cudaMalloc can), or code running where another
 * allocator (a framework's caching allocator, a pool reserved up front) owns
 * the device's memory. It computes what qmcdu_ratio computes for one walker
 * (the change form of Eq. 1-3), from a delay queue the caller holds, and
 * allocates nothing: its
 * scratch (the CTAs' partial sums and their arrival counter, 131,584 bytes) is
 * a fixed array in the library's device memory, which every GPU that loads
 * the library holds until the process exits.
 *   N          1..8192 electrons;  k  0..min(N, 256) queued moves
 *   ainv_col   device [N]     column j of A^{-1} as of the last flush (j is
 *                             the moving electron, not among the queued ones)
 *   u          device [N]     the move's change of row j: u = v - a_j (proposed
 *                             row minus the current row)
 *   P          device [k][N]  row m: column idx_m of A^{-1} as of the last flush
 *   V          device [k][N]  row m: the change u_m of queued move m
 *   Kinv       device [k][k]  (I + V P')^{-1}, row-major (P, V, Kinv may be NULL
 *                             if k = 0)
 *   ratio_out  device [1]     r = 1 + (u.a - (P u)' Kinv (V a)), a = ainv_col
 *   stream     cudaStream_t (NULL: the legacy default stream)
 * Asynchronous on `stream`. Every call on a device shares the one scratch
 * array, which keeps the last call's contents; each call clears what must
 * start at zero. Calls whose executions overlap on the GPU (concurrent
 * streams, or several host threads) race on the scratch and give wrong
 * results: serialise them. The first call on a device looks up the scratch's
 * device address (once per device, with that device current); under CUDA's
 * lazy module loading that look-up also loads this library's device code,
 * which places the scratch array in device memory and may synchronise the
 * device. Make that first call during the caller's own set-up, before any
 * stream capture; later calls neither allocate nor synchronise. Errors: ERR_ARG for sizes beyond the limits
 * above or null pointers, ERR_CUDA; the text is at qmcdu_last_error(NULL).
 * No cudaMalloc, cudaFree or allocating library routine is called.
 */
int qmcdu_ratio_noalloc(int N, int k, const double *ainv_col, const double *u, const double *P,
                        const double *V, const double *Kinv, double *ratio_out, void *stream);

/*
 * Multideterminant walkers: the delayed update combined with the table method
 * of Clark et al. for Psi = sum_I c_I det(A_I) (the extension Sec. II names).
 * det(A_I) replaces up to two occupied orbital columns o_p of A by virtual
 * orbital columns a_p; B (N x nv) holds the nv virtual orbitals at the
 * electrons. The context keeps the table T = A^{-1} B of the CURRENT matrix
 * (queued moves included) by a rank-1 update per accepted move, from the
 * current inverse column the delay queue yields, while A^{-1} itself is
 * updated only at the handle's flushes (Eq. 4). A move's ratio is
 * R = Psi_new / Psi = sum_I c_I (r det T_I + d_I' adj(T_I) z_I) / S, with r
 * the reference ratio (Eq. 1/3), z = A_c^{-1} e_j, d = (w - b_j) - T'u and
 * S = sum_I c_I det(T_I) (no division by r). The table is relative to the
 * reference determinant: accepting a move with r = 0 is ERR_SINGULAR.
 * Per-call, on fp64 handles; one context per handle, which it uses through
 * qmcdu_ratio / qmcdu_accept (call those only through the context while it
 * exists).
 *   qmcdu_md_create   exc host [ndet][4] ints (o1, a1, o2, a2; -1 = unused
 *                     pair, all -1 = the reference), coef host [ndet]
 *   qmcdu_md_set_virtuals  B host or device [batch][N][nv] fp64: flushes the
 *                     queue, builds T from the current A^{-1} and S, log|Psi|
 *                     (recall after a recompute or qmcdu_set_matrix)
 *   qmcdu_md_ratio    as qmcdu_ratio, plus w device [batch][nv] (the proposed
 *                     virtual orbital values); ratio_out device [batch]: R;
 *                     ref_ratio_out device [batch] or NULL: r
 *   qmcdu_md_accept   as qmcdu_accept, then the table update
 *   qmcdu_md_logpsi   running log|Psi| and sign (host or device); synchronises
 * Errors: ERR_ARG (null pointers, excitations outside the orbitals, a
 * non-fp64 handle), ERR_STATE (ratio before set_virtuals, accept without a
 * pending ratio), and those of the handle's calls; text at qmcdu_md_last_error.
 */
int qmcdu_md_create(qmcdu_t h, int nv, int ndet, const int *exc, const double *coef, qmcdu_md_t *out);
int qmcdu_md_destroy(qmcdu_md_t m);
int qmcdu_md_set_virtuals(qmcdu_md_t m, const double *B);
int qmcdu_md_ratio(qmcdu_md_t m, const int *elec, const double *v, const double *w, double *ratio_out,
                   double *ref_ratio_out);
int qmcdu_md_accept(qmcdu_md_t m, const unsigned char *mask);
int qmcdu_md_logpsi(qmcdu_md_t m, double *logabs, int *sign);
const char *qmcdu_md_last_error(qmcdu_md_t m);

/*
 * The tensor-core contraction of the fp32 flush (Eq. 4), exposed for direct use
 * and testing: C = alpha * A B' + beta * C with fp32 operands split as
 * x = hi + lo (hi = bf16(x), lo = bf16(x - hi)) and hi*hi + hi*lo + lo*hi
 * accumulated in fp32 tensor memory by tcgen05.mma (relative error about
 * 2^-16 of sum |a||b|, coarser than fp32 arithmetic).
 *   A  device, M x K, A(m, k) at A[m*lda + k]
 *   B  device, N x K with B(n, k) at B[n*ldb + k]; or, b_trans = 1, K x N with
 *      B(n, k) at B[k*ldb + n]
 *   C  device, M x N, C(m, n) at C[m*ldc + n]
 * Asynchronous on `stream`. For N > 128 and K > 0 the operands are first split
 * once into bf16 planes laid out as tensor-core tiles (a workspace of
 * 4 (M + N) K bytes, rounded up to whole 128 x 32 / 256 x 32 tiles, from a
 * memory pool the library keeps per device and never shrinks), then streamed
 * by bulk copies through a 4-stage pipeline; narrower products split on the
 * fly. ERR_ARG for negative sizes, short leading dimensions or null pointers
 * (text at qmcdu_last_error(NULL)).
 */
int qmcdu_gemm_bf16x3(int M, int N, int K, const float *A, int lda, const float *B, int ldb,
                      int b_trans, float *C, int ldc, float alpha, float beta, void *stream);

/*
 * Serving loop (native, in the library). Requests for walkers of different
 * electron counts arrive over time. Each is admitted, when a walker slot,
 * device memory and the GPU's compute allow (the resident walkers' CTAs within
 * `sm_oversubscription` times the SM count), into a size-class handle (a "pool" of `class_slots`
 * slots, created while the pools held stay within `hbm_budget`; idle pools of
 * other classes are destroyed to make room). Admission draws the walker's
 * matrix from its key and computes A^{-1} and log|det A| by the fp64 LU on a
 * second stream of the pool. Every pool sweeps the walkers it holds, one
 * sweep each per round (qmcdu_sweep_walkers), on its own stream, several pools
 * at once with their CTA shares summing to at most the SM count; walkers join
 * between rounds (continuous batching) and leave after `nsweeps` sweeps and a
 * final fp64 recompute. A walker's sweep s uses Philox key `seed` and sweep
 * number s, and every pool of a class has the same walker-group shape, so a
 * request's results are bit-identical alone and in any mix.
 *
 * The paper runs one walker per process and has no serving layer; this is the
 * continuous-batching pattern applied to its delayed-update sweep.
 */
#define QMCDU_SERVER_MAX_CLASSES 16
typedef struct qmcdu_server *qmcdu_server_t;

typedef struct {
    int precision;                  /* working precision of every walker */
    int recompute_every;            /* fp64 recompute every R sweeps of a walker (0: only at the end) */
    double sigma;                   /* proposal width: v = a_j + sigma g */
    unsigned long long hbm_budget;  /* device bytes the pools may hold (qmcdu_footprint + outputs) */
    int num_classes;                /* 1..QMCDU_SERVER_MAX_CLASSES */
    int class_N[QMCDU_SERVER_MAX_CLASSES];      /* electrons of each class (requests match one) */
    int class_K[QMCDU_SERVER_MAX_CLASSES];      /* delay K (0: min(N, 32)) */
    int class_slots[QMCDU_SERVER_MAX_CLASSES];  /* walker slots per pool (0: 8) */
    int class_group_ctas[QMCDU_SERVER_MAX_CLASSES]; /* CTAs per walker group (0: max(1, min(32, N/128))) */
    int max_inflight;               /* pools sweeping at once (0: no cap but the SMs) */
    int max_walkers;                /* walkers resident at once (0: no cap but slots and budget) */
    int keep_traces;                /* 1: keep each request's accept masks and ratios (qmcdu_server_trace) */
    int simulate;                   /* 1: no GPU work; a cost model on a virtual clock (tests of the scheduler) */
    double sim_flops;               /* simulate: flush flop/s of the whole GPU (working precision) */
    double sim_fp64_flops;          /* simulate: LU flop/s */
    double sim_proposal_s;          /* simulate: latency of one proposal of a sweep */
    double sm_oversubscription;     /* admission stops while the resident walkers' group CTAs,
                                       summed, would pass this multiple of the SM count (0: 2;
                                       < 0: no cap but slots and budget) */
} qmcdu_server_config;

typedef struct {
    unsigned long long id;          /* caller's tag, returned in the result */
    unsigned long long seed;        /* Philox key of the walker: its matrix and every draw */
    int N;                          /* electrons; must be one of class_N */
    int nsweeps;                    /* >= 1 */
    double arrival_s;               /* arrival time on the server clock (s) */
} qmcdu_request;

typedef struct {
    unsigned long long id;
    int N, nsweeps;
    int status;                     /* QMCDU_OK, ERR_OOM (can never fit the budget), or the pool's error */
    int pool;                       /* pool that served it (-1 if none) */
    double arrival_s, admit_s, done_s;
    long long accepted, near_ties;
    int recomputes;
    int sign;                       /* of det A after the final recompute */
    double logabs;                  /* log|det A| after the final recompute */
    double drift_logdet, drift_inverse; /* largest drift of the running values at a recompute */
    double sweep_ms_mean, sweep_ms_max; /* device time of the rounds that swept it */
    long long first_round, last_round;  /* the pool's round numbers of its first and last sweep */
} qmcdu_result;

/*
 * create: copies the configuration (validated: ERR_ARG). The server uses the
 * current device. submit: queues requests (any arrival order; each is held
 * until the clock passes its arrival_s); ERR_ARG for an N that is no class,
 * nsweeps < 1. run: runs the loop until every submitted request has
 * finished, or the server clock passes until_s (< 0: no limit); the clock
 * starts at the first run (wall clock; virtual under `simulate`). Returns the
 * first fatal CUDA error (ERR_CUDA, ERR_OOM), else QMCDU_OK. results: copies
 * out up to `max` finished requests not returned before, in order of
 * completion. trace (keep_traces): accept masks [nsweeps][N] and ratios
 * [nsweeps][N] of a finished request (host; either may be NULL); ERR_ARG for
 * an unknown id. stats: QMCDU_SERVER_STATS doubles, in order: clock (s),
 * submitted, finished, failed, walker-sweeps, accepted updates, proposals,
 * per-sweep latency p50 and p99 (ms, device time of the round per walker-
 * sweep), request latency p50 and p99 (s, arrival to done), admission wait p50
 * and p99 (s), peak bytes held, budget, pools created, pools destroyed,
 * rounds, most walkers resident at once, most pools in flight at once,
 * walker-sweeps in rounds that held walkers admitted at different times, clock
 * at the last finished round (s). destroy: waits for the device work of the
 * pools and frees them. Not thread-safe: one host thread drives a server.
 */
#define QMCDU_SERVER_STATS 22
/*
 * Per size class (index into class_N): QMCDU_SERVER_CLASS_STATS doubles, in
 * order: walker-sweeps, per-sweep latency p50 and p99 (ms), requests finished,
 * request latency p50 and p99 (s), accepted updates of finished requests.
 * ERR_ARG for a class index out of range.
 */
#define QMCDU_SERVER_CLASS_STATS 7
int qmcdu_server_create(const qmcdu_server_config *cfg, qmcdu_server_t *out);
int qmcdu_server_submit(qmcdu_server_t s, const qmcdu_request *reqs, int n);
int qmcdu_server_run(qmcdu_server_t s, double until_s);
int qmcdu_server_results(qmcdu_server_t s, qmcdu_result *out, int max, int *count);
int qmcdu_server_trace(qmcdu_server_t s, unsigned long long id, unsigned char *accepted,
                       double *ratios);
int qmcdu_server_stats(qmcdu_server_t s, double *out, int n);
int qmcdu_server_class_stats(qmcdu_server_t s, int cls, double *out, int n);
const char *qmcdu_server_error(qmcdu_server_t s);
int qmcdu_server_destroy(qmcdu_server_t s);

/* Library version string. */
const char *qmcdu_version(void);

#ifdef __cplusplus
}
#endif

#endif /* QMCDU_H */
