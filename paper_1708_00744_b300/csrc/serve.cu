// serve.cu -- the serving loop of libqmcdu (qmcdu_server_*, declared in
// include/qmcdu.h). Requests for walkers of different electron counts arrive
// over time; each is admitted into a walker slot of a size-class handle (a
// "pool") while the pools held fit a device-memory budget; every pool sweeps
// the walkers it holds, one sweep each per round, on its own stream, with
// walkers joining and leaving between rounds (continuous batching). Host code
// only: every step of a walker runs in the library's kernels.
//
// A walker's state machine: queued -> loaded (matrix drawn from its key, fp64
// LU for A^{-1} and log|det A|, on the pool's admission stream) -> swept once
// per round -> every R sweeps an fp64 recompute before its next sweep -> after
// its last sweep a final recompute and the read-back of log|det A| -> done.
//
// Under `simulate` no GPU work is issued: a cost model advances a virtual
// clock, so that the policy (admission against the budget, eviction of idle
// pools, SM shares, round membership) can be tested without a GPU.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <deque>
#include <memory>
#include <string>
#include <thread>
#include <vector>

#include "qmcdu_internal.cuh"

namespace qmcdu {
namespace {

enum Need { NEED_SWEEP = 0, NEED_RECOMPUTE = 1, NEED_FINAL = 2 };

struct Req {
    qmcdu_request r{};
    int cls = -1;
    int pool = -1, slot = -1;
    int need = NEED_SWEEP;
    int done_sweeps = 0, recomputes = 0;
    int status = QMCDU_OK;
    bool finished = false;
    double admit_s = -1.0, done_s = -1.0;
    long long accepted = 0, ties = 0;
    double drift_ld = 0.0, drift_inv = 0.0, lat_sum = 0.0, lat_max = 0.0;
    double logabs = 0.0;
    int sign = 0;
    long long first_round = -1, last_round = -1;
    std::vector<unsigned char> tacc;
    std::vector<double> trat;
};

struct Pool {
    int id = -1, cls = -1, N = 0, K = 0, slots = 0, gf = 1;
    unsigned long long bytes = 0;
    qmcdu_t h = nullptr;
    cudaStream_t s = nullptr, ls = nullptr;      // sweeps; admissions (loads)
    std::vector<int> slot_req;                   // request per slot, -1 if free
    std::vector<char> load_wait;                 // next round waits for the slot's load
    std::vector<double> ready_at;                // simulate: load finished
    cudaEvent_t ev_load = nullptr, ev0 = nullptr, ev1 = nullptr, ev_done = nullptr;
    bool inflight = false;
    int share = 0;
    long long rounds = 0;
    double sim_end = 0.0, sim_lat = 0.0, last_used = 0.0;
    bool mixed = false;                          // round holds walkers admitted at different times
    std::vector<int> r_sweep, r_recomp, r_final; // slots of the round in flight
    unsigned char *d_acc = nullptr, *h_acc = nullptr;
    double *d_rat = nullptr, *h_rat = nullptr;
    long long *d_ties = nullptr, *h_ties = nullptr;
    double *d_drift = nullptr, *h_drift = nullptr;   // [slots][2]
    double *h_logabs = nullptr;
    int *h_sign = nullptr, *h_status = nullptr;

    int occupied() const
    {
        int n = 0;
        for (int r : slot_req) n += r >= 0;
        return n;
    }
};

double percentile(std::vector<double> v, double q)
{
    if (v.empty()) return 0.0;
    std::sort(v.begin(), v.end());
    const double pos = q * (double)(v.size() - 1);
    const size_t i = (size_t)pos;
    const double f = pos - (double)i;
    return i + 1 < v.size() ? v[i] * (1.0 - f) + v[i + 1] * f : v[i];
}

}  // namespace

struct Server {
    qmcdu_server_config cfg{};
    std::vector<Req> reqs;
    std::vector<int> pending;                     // not yet arrived, latest arrival first
    std::deque<int> queue[QMCDU_SERVER_MAX_CLASSES];
    std::vector<std::unique_ptr<Pool>> pools;
    std::deque<int> completed;                    // finished, not yet returned
    unsigned long long held = 0, peak_held = 0;
    bool started = false;
    std::chrono::steady_clock::time_point t0;
    double vclock = 0.0;
    int num_sms = 148;
    int next_pool_id = 0;
    int error = QMCDU_OK;
    std::string err;
    std::vector<double> sweep_lat_ms;
    std::vector<double> class_lat_ms[QMCDU_SERVER_MAX_CLASSES];   // per size class
    long long walker_sweeps = 0, accepted_total = 0, proposals_total = 0;
    long long pools_created = 0, pools_destroyed = 0, rounds = 0, mixed_walker_sweeps = 0;
    int max_resident = 0, max_inflight_seen = 0;
    int finished_n = 0, failed_n = 0;
    double last_round_end = 0.0;

    double now() const
    {
        if (cfg.simulate) return vclock;
        if (!started) return 0.0;
        return std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    }

    int class_of(int N) const
    {
        for (int c = 0; c < cfg.num_classes; ++c)
            if (cfg.class_N[c] == N) return c;
        return -1;
    }

    int resident() const
    {
        int n = 0;
        for (auto &p : pools) n += p->occupied();
        return n;
    }

    // walker-group CTAs the resident walkers need to be swept at once
    long long resident_ctas() const
    {
        long long n = 0;
        for (auto &p : pools) n += (long long)p->occupied() * p->gf;
        return n;
    }

    int fail_cuda(cudaError_t e, const char *where)
    {
        if (error == QMCDU_OK) {
            error = e == cudaErrorMemoryAllocation ? QMCDU_ERR_OOM : QMCDU_ERR_CUDA;
            err = std::string(where) + ": " + cudaGetErrorString(e);
        }
        return error;
    }

    int fail_api(int st, qmcdu_t h, const char *where)
    {
        if (error == QMCDU_OK) {
            error = st;
            err = std::string(where) + ": " + qmcdu_last_error(h);
        }
        return error;
    }

    // bytes of one pool of class c: the handle plus the server's outputs
    unsigned long long pool_bytes(int c) const
    {
        unsigned long long b = 0;
        const int N = cfg.class_N[c], S = cfg.class_slots[c];
        qmcdu_footprint(N, cfg.class_K[c], cfg.precision, S, &b);
        b += (unsigned long long)S * N + (unsigned long long)S * 8 * 3;
        if (cfg.keep_traces) b += (unsigned long long)S * N * 8;
        return b;
    }

    void finish(int ri, int status)
    {
        Req &q = reqs[ri];
        q.status = status;
        q.finished = true;
        q.done_s = now();
        completed.push_back(ri);
        if (status == QMCDU_OK) ++finished_n;
        else ++failed_n;
    }

    // ---- pools
    void free_pool_resources(Pool &p)
    {
        if (cfg.simulate) return;
        if (p.h) {
            cudaStreamSynchronize(p.s);
            cudaStreamSynchronize(p.ls);
            qmcdu_destroy(p.h);
        }
        cudaEvent_t evs[] = {p.ev_load, p.ev0, p.ev1, p.ev_done};
        for (cudaEvent_t e : evs)
            if (e) cudaEventDestroy(e);
        if (p.s) cudaStreamDestroy(p.s);
        if (p.ls) cudaStreamDestroy(p.ls);
        void *dev[] = {p.d_acc, p.d_rat, p.d_ties, p.d_drift};
        for (void *d : dev)
            if (d) cudaFree(d);
        void *host[] = {p.h_acc, p.h_rat, p.h_ties, p.h_drift, p.h_logabs, p.h_sign, p.h_status};
        for (void *x : host)
            if (x) cudaFreeHost(x);
    }

    Pool *make_pool(int c)
    {
        auto p = std::make_unique<Pool>();
        p->id = next_pool_id++;
        p->cls = c;
        p->N = cfg.class_N[c];
        p->K = cfg.class_K[c];
        p->slots = cfg.class_slots[c];
        p->gf = cfg.class_group_ctas[c];
        p->bytes = pool_bytes(c);
        p->slot_req.assign(p->slots, -1);
        p->load_wait.assign(p->slots, 0);
        p->ready_at.assign(p->slots, 0.0);
        if (!cfg.simulate) {
            const int S = p->slots, N = p->N;
            cudaError_t e = cudaStreamCreateWithFlags(&p->s, cudaStreamNonBlocking);
            if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&p->ls, cudaStreamNonBlocking);
            cudaEvent_t *evs[] = {&p->ev_load, &p->ev0, &p->ev1, &p->ev_done};
            for (cudaEvent_t *ev : evs)
                if (e == cudaSuccess)
                    e = cudaEventCreateWithFlags(ev, ev == &p->ev0 || ev == &p->ev1
                                                         ? cudaEventDefault
                                                         : cudaEventDisableTiming);
            if (e == cudaSuccess) e = cudaMalloc(&p->d_acc, (size_t)S * N);
            if (e == cudaSuccess) e = cudaMalloc(&p->d_ties, (size_t)S * sizeof(long long));
            if (e == cudaSuccess) e = cudaMalloc(&p->d_drift, (size_t)S * 2 * sizeof(double));
            if (e == cudaSuccess && cfg.keep_traces)
                e = cudaMalloc(&p->d_rat, (size_t)S * N * sizeof(double));
            if (e == cudaSuccess) e = cudaMallocHost(&p->h_acc, (size_t)S * N);
            if (e == cudaSuccess) e = cudaMallocHost(&p->h_ties, (size_t)S * sizeof(long long));
            if (e == cudaSuccess) e = cudaMallocHost(&p->h_drift, (size_t)S * 2 * sizeof(double));
            if (e == cudaSuccess) e = cudaMallocHost(&p->h_logabs, (size_t)S * sizeof(double));
            if (e == cudaSuccess) e = cudaMallocHost(&p->h_sign, (size_t)S * sizeof(int));
            if (e == cudaSuccess) e = cudaMallocHost(&p->h_status, sizeof(int));
            if (e == cudaSuccess && cfg.keep_traces)
                e = cudaMallocHost(&p->h_rat, (size_t)S * N * sizeof(double));
            if (e != cudaSuccess) {
                free_pool_resources(*p);
                fail_cuda(e, "server pool buffers");
                return nullptr;
            }
            int st = qmcdu_create(p->N, p->K, cfg.precision, S, p->s, &p->h);
            if (st == QMCDU_OK) st = qmcdu_set_option(p->h, QMCDU_OPT_GROUP_CTAS, p->gf);
            if (st != QMCDU_OK) {
                if (error == QMCDU_OK) {
                    error = st;
                    err = "server pool: qmcdu_create failed";
                }
                free_pool_resources(*p);
                return nullptr;
            }
        }
        held += p->bytes;
        peak_held = std::max(peak_held, held);
        ++pools_created;
        pools.push_back(std::move(p));
        return pools.back().get();
    }

    void destroy_pool(size_t i)
    {
        Pool &p = *pools[i];
        free_pool_resources(p);
        held -= p.bytes;
        ++pools_destroyed;
        pools.erase(pools.begin() + i);
    }

    // Room for `bytes` more: destroy idle pools of other classes, least
    // recently used first, while that helps.
    bool make_room(unsigned long long bytes, int for_cls)
    {
        if (bytes > cfg.hbm_budget) return false;
        while (held + bytes > cfg.hbm_budget) {
            int best = -1;
            for (size_t i = 0; i < pools.size(); ++i) {
                const Pool &p = *pools[i];
                if (p.inflight || p.occupied() > 0 || p.cls == for_cls) continue;
                if (best < 0 || p.last_used < pools[best]->last_used) best = (int)i;
            }
            if (best < 0) return false;
            destroy_pool((size_t)best);
        }
        return true;
    }

    // ---- arrivals and admission
    bool move_arrivals(double t)
    {
        bool any = false;
        while (!pending.empty() && reqs[pending.back()].r.arrival_s <= t) {
            const int ri = pending.back();
            pending.pop_back();
            queue[reqs[ri].cls].push_back(ri);
            any = true;
        }
        return any;
    }

    bool admit(double t)
    {
        bool any = false;
        bool blocked[QMCDU_SERVER_MAX_CLASSES] = {};
        for (;;) {
            if (cfg.max_walkers > 0 && resident() >= cfg.max_walkers) break;
            // the earliest arrival at the head of a class queue that is not blocked
            int c = -1;
            for (int k = 0; k < cfg.num_classes; ++k)
                if (!blocked[k] && !queue[k].empty() &&
                    (c < 0 || reqs[queue[k].front()].r.arrival_s < reqs[queue[c].front()].r.arrival_s))
                    c = k;
            if (c < 0) break;
            // compute: more resident walkers than the SMs can sweep in a few
            // waves only lengthen every round (and their admission LUs crowd
            // the sweeps out); the first walker is always admitted
            if (cfg.sm_oversubscription > 0.0 && resident() > 0 &&
                (double)(resident_ctas() + cfg.class_group_ctas[c]) >
                    cfg.sm_oversubscription * num_sms) {
                blocked[c] = true;
                continue;
            }
            // a free slot: in the fullest pool of the class that has one
            Pool *best = nullptr;
            for (auto &pp : pools) {
                Pool &p = *pp;
                if (p.cls != c) continue;
                const int occ = p.occupied();
                if (occ == p.slots) continue;
                if (!best || occ > best->occupied()) best = &p;
            }
            if (!best) {
                const unsigned long long b = pool_bytes(c);
                if (b > cfg.hbm_budget) {     // can never be admitted
                    const int ri = queue[c].front();
                    queue[c].pop_front();
                    finish(ri, QMCDU_ERR_OOM);
                    any = true;
                    continue;
                }
                if (!make_room(b, c)) {
                    blocked[c] = true;
                    continue;
                }
                // slots chosen earlier in this pass stay marked (load_wait 2) in
                // their pools, which make_room does not destroy (they are occupied)
                best = make_pool(c);
                if (!best) return any;
            }
            int slot = -1;
            for (int s = 0; s < best->slots; ++s)
                if (best->slot_req[s] < 0) {
                    slot = s;
                    break;
                }
            const int ri = queue[c].front();
            queue[c].pop_front();
            Req &q = reqs[ri];
            q.pool = best->id;
            q.slot = slot;
            q.admit_s = t;
            q.need = NEED_SWEEP;
            best->slot_req[slot] = ri;
            best->load_wait[slot] = 2;     // 2: load to issue; 1: issued, round must wait
            best->last_used = t;
            any = true;
            if (cfg.keep_traces) {
                q.tacc.reserve((size_t)q.r.nsweeps * q.r.N);
                q.trat.reserve((size_t)q.r.nsweeps * q.r.N);
            }
        }
        max_resident = std::max(max_resident, resident());
        // issue the loads: contiguous runs of new slots per pool
        for (auto &pp : pools) {
            Pool &p = *pp;
            int s = 0;
            bool issued = false;
            while (s < p.slots) {
                if (p.load_wait[s] != 2) {
                    ++s;
                    continue;
                }
                int e = s;
                std::vector<unsigned long long> seeds;
                while (e < p.slots && p.load_wait[e] == 2) {
                    seeds.push_back(reqs[p.slot_req[e]].r.seed);
                    p.load_wait[e] = 1;
                    ++e;
                }
                if (cfg.simulate) {
                    const double n3 = (double)p.N * p.N * p.N;
                    const double done = t + (double)(e - s) * 2.0 * n3 / cfg.sim_fp64_flops;
                    for (int k = s; k < e; ++k) p.ready_at[k] = done;
                } else {
                    const int st = load_walkers_on(p.h, p.ls, s, e - s, seeds.data());
                    if (st != QMCDU_OK) return fail_api(st, p.h, "load_walkers"), any;
                    issued = true;
                }
                s = e;
            }
            if (issued) {
                cudaError_t e = cudaEventRecord(p.ev_load, p.ls);
                if (e != cudaSuccess) return fail_cuda(e, "record load"), any;
            }
        }
        return any;
    }

    // ---- rounds
    double work_of(const Pool &p) const
    {
        const double n3 = (double)p.N * p.N * p.N;
        return n3 * p.occupied();
    }

    bool launch_ready(double t)
    {
        if (error) return false;
        int inflight = 0, used = 0;
        double wsum = 0.0;
        for (auto &p : pools) {
            if (p->inflight) {
                ++inflight;
                used += p->share;
            }
            if (p->occupied() > 0) wsum += work_of(*p);
        }
        // ready pools, the one with the earliest-arrived walker first
        std::vector<Pool *> ready;
        for (auto &p : pools)
            if (!p->inflight && p->occupied() > 0) ready.push_back(p.get());
        auto first_arrival = [&](const Pool *p) {
            double a = 1e300;
            for (int r : p->slot_req)
                if (r >= 0) a = std::min(a, reqs[r].r.arrival_s);
            return a;
        };
        std::sort(ready.begin(), ready.end(),
                  [&](const Pool *a, const Pool *b) { return first_arrival(a) < first_arrival(b); });
        bool any = false;
        for (Pool *p : ready) {
            if (cfg.max_inflight > 0 && inflight >= cfg.max_inflight) break;
            const int free_sms = num_sms - used;
            if (free_sms < p->gf) continue;
            int want = (int)std::ceil((double)num_sms * work_of(*p) / std::max(wsum, 1.0));
            // whole walker groups, at least one, at most one group per walker
            want = std::max(p->gf, std::min(want, p->gf * p->occupied()));
            int share = std::min(want, free_sms);
            share = std::max(p->gf, share / p->gf * p->gf);
            if (!launch_round(*p, share, t)) return any;
            used += share;
            ++inflight;
            any = true;
        }
        max_inflight_seen = std::max(max_inflight_seen, inflight);
        return any;
    }

    bool launch_round(Pool &p, int share, double t)
    {
        p.r_sweep.clear();
        p.r_recomp.clear();
        p.r_final.clear();
        double admit_min = 1e300, admit_max = -1e300;
        for (int s = 0; s < p.slots; ++s) {
            const int ri = p.slot_req[s];
            if (ri < 0) continue;
            const Req &q = reqs[ri];
            if (q.need == NEED_FINAL) {
                p.r_recomp.push_back(s);
                p.r_final.push_back(s);
                continue;
            }
            if (q.need == NEED_RECOMPUTE) p.r_recomp.push_back(s);
            p.r_sweep.push_back(s);
            admit_min = std::min(admit_min, q.admit_s);
            admit_max = std::max(admit_max, q.admit_s);
        }
        p.mixed = p.r_sweep.size() > 1 && admit_max > admit_min;
        const int n = (int)p.r_sweep.size();
        p.share = share;
        p.inflight = true;
        p.last_used = t;
        ++p.rounds;
        ++rounds;
        if (cfg.simulate) {
            const double n3 = (double)p.N * p.N * p.N;
            double start = t;
            for (int s = 0; s < p.slots; ++s)
                if (p.slot_req[s] >= 0 && p.load_wait[s]) start = std::max(start, p.ready_at[s]);
            std::fill(p.load_wait.begin(), p.load_wait.end(), 0);
            const double trec = (double)p.r_recomp.size() * 2.0 * n3 / cfg.sim_fp64_flops;
            const int groups = std::max(1, share / p.gf);
            const double waves = std::ceil((double)n / groups);
            const double frac = (double)share / num_sms;
            const double tsw = n == 0 ? 0.0
                                      : waves * p.N * cfg.sim_proposal_s +
                                            (double)n * 4.0 * n3 / (cfg.sim_flops * frac);
            p.sim_lat = tsw;
            p.sim_end = start + trec + tsw;
            return true;
        }
        Ctx *c = reinterpret_cast<Ctx *>(p.h);
        cudaError_t e = cudaSuccess;
        bool wait_load = false;
        for (int s = 0; s < p.slots; ++s) {
            wait_load |= p.slot_req[s] >= 0 && p.load_wait[s] == 1;
            if (p.slot_req[s] >= 0) p.load_wait[s] = 0;
        }
        if (wait_load) e = cudaStreamWaitEvent(p.s, p.ev_load, 0);
        if (e != cudaSuccess) return fail_cuda(e, "wait for loads"), false;
        int st = qmcdu_set_option(p.h, QMCDU_OPT_MAX_CTAS, share);
        if (st != QMCDU_OK) return fail_api(st, p.h, "set_option"), false;
        // recomputes, by runs of consecutive slots
        for (size_t i = 0; i < p.r_recomp.size();) {
            size_t j = i + 1;
            while (j < p.r_recomp.size() && p.r_recomp[j] == p.r_recomp[j - 1] + 1) ++j;
            const int first = p.r_recomp[i], count = (int)(j - i);
            st = qmcdu_recompute_walkers(p.h, first, count, p.d_drift + 2 * first);
            if (st != QMCDU_OK) return fail_api(st, p.h, "recompute_walkers"), false;
            i = j;
        }
        if (!p.r_recomp.empty()) {
            e = cudaMemcpyAsync(p.h_drift, p.d_drift, (size_t)p.slots * 2 * sizeof(double),
                                cudaMemcpyDeviceToHost, p.s);
            if (e == cudaSuccess)
                e = cudaMemcpyAsync(p.h_logabs, c->logabs, (size_t)p.slots * sizeof(double),
                                    cudaMemcpyDeviceToHost, p.s);
            if (e == cudaSuccess)
                e = cudaMemcpyAsync(p.h_sign, c->sign, (size_t)p.slots * sizeof(int),
                                    cudaMemcpyDeviceToHost, p.s);
            if (e != cudaSuccess) return fail_cuda(e, "recompute read-back"), false;
        }
        e = cudaEventRecord(p.ev0, p.s);
        if (e != cudaSuccess) return fail_cuda(e, "record"), false;
        if (n > 0) {
            std::vector<unsigned long long> seeds(n);
            std::vector<int> sweeps(n);
            for (int k = 0; k < n; ++k) {
                const Req &q = reqs[p.slot_req[p.r_sweep[k]]];
                seeds[k] = q.r.seed;
                sweeps[k] = q.done_sweeps;
            }
            st = qmcdu_sweep_walkers(p.h, n, p.r_sweep.data(), seeds.data(), sweeps.data(),
                                     cfg.sigma, p.d_acc, cfg.keep_traces ? p.d_rat : nullptr,
                                     p.d_ties);
            if (st != QMCDU_OK) return fail_api(st, p.h, "sweep_walkers"), false;
        }
        e = cudaEventRecord(p.ev1, p.s);
        if (e == cudaSuccess && n > 0)
            e = cudaMemcpyAsync(p.h_acc, p.d_acc, (size_t)n * p.N, cudaMemcpyDeviceToHost, p.s);
        if (e == cudaSuccess && n > 0)
            e = cudaMemcpyAsync(p.h_ties, p.d_ties, (size_t)n * sizeof(long long),
                                cudaMemcpyDeviceToHost, p.s);
        if (e == cudaSuccess && n > 0 && cfg.keep_traces)
            e = cudaMemcpyAsync(p.h_rat, p.d_rat, (size_t)n * p.N * sizeof(double),
                                cudaMemcpyDeviceToHost, p.s);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(p.h_status, c->status, sizeof(int), cudaMemcpyDeviceToHost, p.s);
        if (e == cudaSuccess) e = cudaEventRecord(p.ev_done, p.s);
        if (e != cudaSuccess) return fail_cuda(e, "round read-back"), false;
        return true;
    }

    bool round_done(Pool &p)
    {
        if (cfg.simulate) return vclock >= p.sim_end;
        const cudaError_t e = cudaEventQuery(p.ev_done);
        if (e == cudaErrorNotReady) return false;
        if (e != cudaSuccess) {
            fail_cuda(e, "round");
            return false;
        }
        return true;
    }

    void complete_round(Pool &p, double t)
    {
        p.inflight = false;
        p.share = 0;
        last_round_end = t;
        int dev_status = 0;
        float lat_ms = 0.0f;
        if (cfg.simulate) {
            lat_ms = (float)(p.sim_lat * 1e3);
        } else {
            dev_status = *p.h_status;
            cudaEventElapsedTime(&lat_ms, p.ev0, p.ev1);
        }
        if (dev_status != 0) {
            // the pool's walkers fail; the pool is retired (its status is latched)
            const int code = (dev_status & ST_TIMEOUT) ? QMCDU_ERR_TIMEOUT : QMCDU_ERR_SINGULAR;
            for (int s = 0; s < p.slots; ++s)
                if (p.slot_req[s] >= 0) {
                    finish(p.slot_req[s], code);
                    p.slot_req[s] = -1;
                }
            return;
        }
        const int n = (int)p.r_sweep.size();
        const int N = p.N;
        for (int k = 0; k < n; ++k) {
            Req &q = reqs[p.slot_req[p.r_sweep[k]]];
            long long acc = 0;
            if (cfg.simulate) {
                acc = N;
            } else {
                const unsigned char *row = p.h_acc + (size_t)k * N;
                for (int j = 0; j < N; ++j) acc += row[j];
                q.ties += p.h_ties[k];
            }
            if (cfg.keep_traces) {
                if (cfg.simulate) {
                    q.tacc.insert(q.tacc.end(), (size_t)N, (unsigned char)1);
                    q.trat.insert(q.trat.end(), (size_t)N, 1.0);
                } else {
                    q.tacc.insert(q.tacc.end(), p.h_acc + (size_t)k * N, p.h_acc + (size_t)(k + 1) * N);
                    q.trat.insert(q.trat.end(), p.h_rat + (size_t)k * N, p.h_rat + (size_t)(k + 1) * N);
                }
            }
            q.accepted += acc;
            accepted_total += acc;
            proposals_total += N;
            ++walker_sweeps;
            if (p.mixed) ++mixed_walker_sweeps;
            sweep_lat_ms.push_back(lat_ms);
            class_lat_ms[p.cls].push_back(lat_ms);
            q.lat_sum += lat_ms;
            q.lat_max = std::max(q.lat_max, (double)lat_ms);
            if (q.first_round < 0) q.first_round = p.rounds;
            q.last_round = p.rounds;
            ++q.done_sweeps;
        }
        for (int s : p.r_recomp) {
            Req &q = reqs[p.slot_req[s]];
            ++q.recomputes;
            if (!cfg.simulate) {
                q.drift_ld = std::max(q.drift_ld, p.h_drift[2 * s]);
                q.drift_inv = std::max(q.drift_inv, p.h_drift[2 * s + 1]);
            }
        }
        for (int s : p.r_final) {
            const int ri = p.slot_req[s];
            Req &q = reqs[ri];
            if (!cfg.simulate) {
                q.logabs = p.h_logabs[s];
                q.sign = p.h_sign[s];
            }
            finish(ri, QMCDU_OK);
            p.slot_req[s] = -1;
        }
        // what each remaining walker needs next
        for (int s : p.r_sweep) {
            const int ri = p.slot_req[s];
            if (ri < 0) continue;
            Req &q = reqs[ri];
            if (q.done_sweeps >= q.r.nsweeps) q.need = NEED_FINAL;
            else if (cfg.recompute_every > 0 && q.done_sweeps % cfg.recompute_every == 0)
                q.need = NEED_RECOMPUTE;
            else q.need = NEED_SWEEP;
        }
    }

    bool poll(double t)
    {
        bool any = false;
        for (auto &pp : pools) {
            Pool &p = *pp;
            if (p.inflight && round_done(p)) {
                complete_round(p, t);
                any = true;
            }
        }
        // pools whose device status latched an error hold no walkers any more
        for (size_t i = 0; i < pools.size();) {
            Pool &p = *pools[i];
            if (!cfg.simulate && !p.inflight && p.occupied() == 0 && *p.h_status != 0) {
                destroy_pool(i);
                continue;
            }
            ++i;
        }
        return any;
    }

    bool all_done() const { return finished_n + failed_n == (int)reqs.size(); }

    // nothing could progress: wait for the next arrival or round end
    void idle(double until)
    {
        if (cfg.simulate) {
            double next = 1e300;
            if (!pending.empty()) next = reqs[pending.back()].r.arrival_s;
            for (auto &p : pools)
                if (p->inflight) next = std::min(next, p->sim_end);
            if (until >= 0.0) next = std::min(next, until);
            if (next < 1e300) vclock = std::max(vclock, next);
            return;
        }
        std::this_thread::sleep_for(std::chrono::microseconds(20));
    }

    int run(double until)
    {
        if (!started) {
            started = true;
            t0 = std::chrono::steady_clock::now();
        }
        if (!cfg.simulate) {
            int dev = 0;
            if (cudaGetDevice(&dev) == cudaSuccess)
                cudaDeviceGetAttribute(&num_sms, cudaDevAttrMultiProcessorCount, dev);
        }
        for (;;) {
            if (error) return error;
            const double t = now();
            bool progress = poll(t);
            if (error) return error;
            progress |= move_arrivals(t);
            progress |= admit(t);
            if (error) return error;
            progress |= launch_ready(t);
            if (error) return error;
            if (all_done()) return QMCDU_OK;
            if (until >= 0.0 && t >= until) return QMCDU_OK;
            if (!progress) {
                bool inflight = false;
                for (auto &p : pools) inflight |= p->inflight;
                if (cfg.simulate && !inflight && pending.empty()) {
                    // nothing in flight, nothing to arrive: the rest can never run
                    bool queued = false;
                    for (int c = 0; c < cfg.num_classes; ++c) queued |= !queue[c].empty();
                    if (queued) {
                        error = QMCDU_ERR_STATE;
                        err = "queued requests cannot be admitted";
                        return error;
                    }
                }
                idle(until);
            }
        }
    }
};

}  // namespace qmcdu

using qmcdu::Server;

extern "C" {

int qmcdu_server_create(const qmcdu_server_config *cfg, qmcdu_server_t *out)
{
    if (!cfg || !out) return QMCDU_ERR_ARG;
    *out = nullptr;
    if (cfg->num_classes < 1 || cfg->num_classes > QMCDU_SERVER_MAX_CLASSES ||
        cfg->precision < QMCDU_FP64 || cfg->precision > QMCDU_FP32_BF16X3 ||
        cfg->recompute_every < 0 || cfg->max_inflight < 0 || cfg->max_walkers < 0 ||
        !(cfg->sigma >= 0.0))
        return QMCDU_ERR_ARG;
    if (cfg->simulate && !(cfg->sim_flops > 0 && cfg->sim_fp64_flops > 0 && cfg->sim_proposal_s >= 0))
        return QMCDU_ERR_ARG;
    Server *s = new (std::nothrow) Server();
    if (!s) return QMCDU_ERR_OOM;
    s->cfg = *cfg;
    if (s->cfg.sm_oversubscription == 0.0) s->cfg.sm_oversubscription = 2.0;
    for (int c = 0; c < cfg->num_classes; ++c) {
        const int N = cfg->class_N[c];
        int &K = s->cfg.class_K[c], &S = s->cfg.class_slots[c], &G = s->cfg.class_group_ctas[c];
        if (K == 0) K = std::min(N, 32);
        if (S == 0) S = 8;
        if (G == 0) G = std::max(1, std::min(32, N / 128));
        unsigned long long b = 0;
        bool dup = false;
        for (int d = 0; d < c; ++d) dup |= cfg->class_N[d] == N;
        if (dup || G < 1 || G > 148 || qmcdu_footprint(N, K, cfg->precision, S, &b) != QMCDU_OK) {
            delete s;
            return QMCDU_ERR_ARG;
        }
    }
    *out = reinterpret_cast<qmcdu_server_t>(s);
    return QMCDU_OK;
}

int qmcdu_server_submit(qmcdu_server_t h, const qmcdu_request *reqs, int n)
{
    if (!h || n < 0 || (n > 0 && !reqs)) return QMCDU_ERR_ARG;
    Server *s = reinterpret_cast<Server *>(h);
    for (int i = 0; i < n; ++i)
        if (s->class_of(reqs[i].N) < 0 || reqs[i].nsweeps < 1 || !(reqs[i].arrival_s >= 0.0)) {
            s->err = "request with an N of no class, nsweeps < 1 or a negative arrival";
            return QMCDU_ERR_ARG;
        }
    for (int i = 0; i < n; ++i) {
        qmcdu::Req q;
        q.r = reqs[i];
        q.cls = s->class_of(reqs[i].N);
        s->reqs.push_back(std::move(q));
        s->pending.push_back((int)s->reqs.size() - 1);
    }
    // latest arrival first (pop_back takes the earliest); ties by submission order
    std::stable_sort(s->pending.begin(), s->pending.end(), [&](int a, int b) {
        const double ta = s->reqs[a].r.arrival_s, tb = s->reqs[b].r.arrival_s;
        return ta != tb ? ta > tb : a > b;
    });
    return QMCDU_OK;
}

int qmcdu_server_run(qmcdu_server_t h, double until_s)
{
    if (!h) return QMCDU_ERR_ARG;
    return reinterpret_cast<Server *>(h)->run(until_s);
}

int qmcdu_server_results(qmcdu_server_t h, qmcdu_result *out, int max, int *count)
{
    if (!h || !count || max < 0 || (max > 0 && !out)) return QMCDU_ERR_ARG;
    Server *s = reinterpret_cast<Server *>(h);
    int n = 0;
    while (n < max && !s->completed.empty()) {
        const qmcdu::Req &q = s->reqs[s->completed.front()];
        s->completed.pop_front();
        qmcdu_result &r = out[n++];
        r.id = q.r.id;
        r.N = q.r.N;
        r.nsweeps = q.r.nsweeps;
        r.status = q.status;
        r.pool = q.pool;
        r.arrival_s = q.r.arrival_s;
        r.admit_s = q.admit_s;
        r.done_s = q.done_s;
        r.accepted = q.accepted;
        r.near_ties = q.ties;
        r.recomputes = q.recomputes;
        r.sign = q.sign;
        r.logabs = q.logabs;
        r.drift_logdet = q.drift_ld;
        r.drift_inverse = q.drift_inv;
        r.sweep_ms_mean = q.done_sweeps ? q.lat_sum / q.done_sweeps : 0.0;
        r.sweep_ms_max = q.lat_max;
        r.first_round = q.first_round;
        r.last_round = q.last_round;
    }
    *count = n;
    return QMCDU_OK;
}

int qmcdu_server_trace(qmcdu_server_t h, unsigned long long id, unsigned char *accepted,
                       double *ratios)
{
    if (!h) return QMCDU_ERR_ARG;
    Server *s = reinterpret_cast<Server *>(h);
    for (const qmcdu::Req &q : s->reqs) {
        if (q.r.id != id || !q.finished) continue;
        if (!s->cfg.keep_traces || q.status != QMCDU_OK) return QMCDU_ERR_STATE;
        if (accepted) std::copy(q.tacc.begin(), q.tacc.end(), accepted);
        if (ratios) std::copy(q.trat.begin(), q.trat.end(), ratios);
        return QMCDU_OK;
    }
    return QMCDU_ERR_ARG;
}

int qmcdu_server_stats(qmcdu_server_t h, double *out, int n)
{
    if (!h || !out || n < 0) return QMCDU_ERR_ARG;
    Server *s = reinterpret_cast<Server *>(h);
    std::vector<double> lat_req, wait;
    for (const qmcdu::Req &q : s->reqs) {
        if (q.finished && q.status == QMCDU_OK) lat_req.push_back(q.done_s - q.r.arrival_s);
        if (q.admit_s >= 0.0) wait.push_back(q.admit_s - q.r.arrival_s);
    }
    const double v[QMCDU_SERVER_STATS] = {
        s->now(),
        (double)s->reqs.size(),
        (double)s->finished_n,
        (double)s->failed_n,
        (double)s->walker_sweeps,
        (double)s->accepted_total,
        (double)s->proposals_total,
        qmcdu::percentile(s->sweep_lat_ms, 0.50),
        qmcdu::percentile(s->sweep_lat_ms, 0.99),
        qmcdu::percentile(lat_req, 0.50),
        qmcdu::percentile(lat_req, 0.99),
        qmcdu::percentile(wait, 0.50),
        qmcdu::percentile(wait, 0.99),
        (double)s->peak_held,
        (double)s->cfg.hbm_budget,
        (double)s->pools_created,
        (double)s->pools_destroyed,
        (double)s->rounds,
        (double)s->max_resident,
        (double)s->max_inflight_seen,
        (double)s->mixed_walker_sweeps,
        s->last_round_end,
    };
    for (int i = 0; i < n && i < QMCDU_SERVER_STATS; ++i) out[i] = v[i];
    return QMCDU_OK;
}

int qmcdu_server_class_stats(qmcdu_server_t h, int cls, double *out, int n)
{
    if (!h || !out || n < 0) return QMCDU_ERR_ARG;
    Server *s = reinterpret_cast<Server *>(h);
    if (cls < 0 || cls >= s->cfg.num_classes) return QMCDU_ERR_ARG;
    std::vector<double> lat_req;
    long long fin = 0, acc = 0;
    for (const qmcdu::Req &q : s->reqs)
        if (q.cls == cls && q.finished && q.status == QMCDU_OK) {
            ++fin;
            acc += q.accepted;
            lat_req.push_back(q.done_s - q.r.arrival_s);
        }
    const std::vector<double> &l = s->class_lat_ms[cls];
    const double v[QMCDU_SERVER_CLASS_STATS] = {
        (double)l.size(), qmcdu::percentile(l, 0.50), qmcdu::percentile(l, 0.99), (double)fin,
        qmcdu::percentile(lat_req, 0.50), qmcdu::percentile(lat_req, 0.99), (double)acc};
    for (int i = 0; i < n && i < QMCDU_SERVER_CLASS_STATS; ++i) out[i] = v[i];
    return QMCDU_OK;
}

const char *qmcdu_server_error(qmcdu_server_t h)
{
    return h ? reinterpret_cast<Server *>(h)->err.c_str() : "";
}

int qmcdu_server_destroy(qmcdu_server_t h)
{
    if (!h) return QMCDU_ERR_ARG;
    Server *s = reinterpret_cast<Server *>(h);
    while (!s->pools.empty()) s->destroy_pool(s->pools.size() - 1);
    delete s;
    return QMCDU_OK;
}

}  // extern "C"
