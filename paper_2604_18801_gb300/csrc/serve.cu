// Request loop: pc_server_* and pc_serve_* (include/pc.h).  Not part of the paper.
//
// One worker thread per server.  Jobs are admitted in FIFO order into cohorts; a cohort
// gathers its jobs' inputs into one block set (one block per job), runs the count pass
// of the selection, waits until the memory its counts call for fits the budget, selects
// its constraints and builds a PgdSolver whose iterations replay a CUDA graph on the
// cohort's own stream.  The worker interleaves: admitting and setting up new cohorts,
// launching iteration chunks of the running ones, and finishing each job as soon as its
// block has stopped (output rows of that block, copy-out, optional edit stream).
// Blocks of a set never interact, so a job's result does not depend on its cohort.
#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <functional>
#include <map>
#include <memory>
#include <mutex>
#include <thread>

#include "pipeline.cuh"

namespace pc {
namespace {

constexpr int GRAPH_LAUNCHES = 8;     // iteration launches per captured graph
constexpr int MAX_CHUNK = 64;         // launches between two status polls

int64_t now_ns() {
    return std::chrono::duration_cast<std::chrono::nanoseconds>(std::chrono::steady_clock::now().time_since_epoch())
        .count();
}

struct Job {
    uint64_t ticket = 0;
    pc_job spec{};
    pc_job_result res{};
};

enum CohortState { C_COUNTED, C_RUNNING };

struct Cohort {
    std::vector<Job *> jobs;
    cudaStream_t s = nullptr;
    CohortState state = C_COUNTED;
    int64_t n = 0;
    int64_t bytes1 = 0, bytes2 = 0;      // estimates: count pass, the rest
    DBuf<float> orig, recon, corr;       // gathered inputs and the corrected coordinates
    std::unique_ptr<Selection> sel;
    std::unique_ptr<PgdSolver> sol;
    std::vector<char> finished;
    int chunk = GRAPH_LAUNCHES;
    int64_t launched = 0;
    ~Cohort() {
        // release device memory on the cohort's stream before the stream goes away
        sol.reset();
        sel.reset();
        orig.release();
        recon.release();
        corr.release();
        if (s) {
            cudaStreamSynchronize(s);
            cudaStreamDestroy(s);
        }
    }
};

}  // namespace
}  // namespace pc

struct pc_server {
    int device = 0;
    int64_t budget = 0;
    int max_slots = 0;
    int64_t max_cohort_n = 0;
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    bool stopping = false;
    uint64_t next_ticket = 1;
    std::map<uint64_t, std::unique_ptr<pc::Job>> jobs;   // every job ever submitted
    std::deque<pc::Job *> pending;                         // FIFO, under mu
    // worker-only state
    std::vector<std::unique_ptr<pc::Cohort>> cohorts;
    pc::HostScratch hs;
    int64_t used = 0, peak = 0, resident_jobs = 0;
    int64_t n_submitted = 0, n_finished = 0, n_cohorts = 0;
    std::thread worker;
};

namespace pc {
namespace {

void publish(pc_server *srv, Job *j, int32_t state, int32_t status, const char *msg) {
    std::lock_guard<std::mutex> lk(srv->mu);
    j->res.state = state;
    j->res.status = status;
    if (msg) {
        std::strncpy(j->res.error, msg, sizeof(j->res.error) - 1);
        j->res.error[sizeof(j->res.error) - 1] = 0;
    }
    if (state == PC_JOB_DONE || state == PC_JOB_ERROR) {
        j->res.done_ns = now_ns();
        ++srv->n_finished;
    }
    srv->cv_done.notify_all();
}

// Device bytes of the count pass for n particles (gathered inputs, binning, labels).
int64_t count_pass_bytes(int64_t n) { return 176 * n + (int64_t)(1 << 20); }

// Validates one job alone (finiteness, |recon - orig| <= xi, periodic box); throws Fail.
void validate(Job *j, cudaStream_t s, HostScratch &hs) {
    BlockSet V;
    V.nb = 1;
    V.n = j->spec.n;
    V.prm.assign(1, j->spec.params);
    V.off = {0, j->spec.n};
    inspect_blocks(j->spec.orig_dev, j->spec.recon_dev, V, s, hs);
    check_inspect(V.ins[0]);
    const Consts c = make_consts(&j->spec.params, V.ins[0], j->spec.n, true);
    if (!(c.xi_box_d > 0.0)) fail(PC_EINVAL, "xi too small for float32 coordinates of this magnitude");
}

void fail_cohort(pc_server *srv, Cohort &c, pc_status st, const char *msg) {
    for (size_t k = 0; k < c.jobs.size(); ++k)
        if (!c.finished.size() || !c.finished[k]) publish(srv, c.jobs[k], PC_JOB_ERROR, st, msg);
    if (c.finished.size()) std::fill(c.finished.begin(), c.finished.end(), 1);
}

// Gathers the jobs' inputs and runs the count pass.
void setup_count(pc_server *srv, Cohort &c) {
    const int nb = (int)c.jobs.size();
    PC_CUDA(cudaStreamCreateWithFlags(&c.s, cudaStreamNonBlocking));
    c.orig.alloc(3 * c.n, c.s);
    c.recon.alloc(3 * c.n, c.s);
    c.corr.alloc(3 * c.n, c.s);
    c.sel.reset(new Selection());
    BlockSet &S = c.sel->S;
    S.nb = nb;
    S.n = c.n;
    S.prm.resize(nb);
    S.off.resize(nb + 1);
    int64_t at = 0;
    for (int b = 0; b < nb; ++b) {
        const pc_job &sp = c.jobs[b]->spec;
        S.prm[b] = sp.params;
        S.off[b] = at;
        PC_CUDA(cudaMemcpyAsync(c.orig.p + 3 * at, sp.orig_dev, 12 * sp.n, cudaMemcpyDeviceToDevice, c.s));
        PC_CUDA(cudaMemcpyAsync(c.recon.p + 3 * at, sp.recon_dev, 12 * sp.n, cudaMemcpyDeviceToDevice, c.s));
        at += sp.n;
    }
    S.off[nb] = at;
    PC_CUDA(cudaMemcpyAsync(c.corr.p, c.recon.p, 12 * c.n, cudaMemcpyDeviceToDevice, c.s));
    select_count(srv->hs, c.orig.p, c.s, *c.sel);
    c.bytes2 = select_more_bytes(*c.sel);
}

// Selection, PGD state and the captured graph; the first chunk is launched.
void setup_run(pc_server *srv, Cohort &c) {
    select_emit(srv->hs, c.s, *c.sel);
    BlockSet &S = c.sel->S;
    // PGD constants need M over orig and recon of each block
    BlockSet V;
    V.nb = S.nb;
    V.n = S.n;
    V.prm = S.prm;
    V.off = S.off;
    inspect_blocks(c.orig.p, c.recon.p, V, c.s, srv->hs);
    std::vector<Consts> cp(V.nb);
    for (int b = 0; b < V.nb; ++b) cp[b] = make_consts(&V.prm[b], V.ins[b], V.off[b + 1] - V.off[b], true);
    c.sol.reset(new PgdSolver(c.sel->B, S, cp, c.orig.p, c.recon.p, c.sel->A.p, c.sel->nA, c.s, srv->hs));
    // the solver keeps what it needs: cell lists and pairs go back to the pool
    c.sel->A.release();
    c.sel->B.keys.release();
    c.sel->B.order.release();
    c.sel->B.P4.release();
    c.sel->B.cell_start.release();
    c.finished.assign(c.jobs.size(), 0);
    const int64_t t0 = now_ns();
    {
        std::lock_guard<std::mutex> lk(srv->mu);
        for (Job *j : c.jobs) {
            j->res.state = PC_JOB_RUNNING;
            j->res.start_ns = t0;
            j->res.cohort_jobs = (int32_t)c.jobs.size();
        }
    }
    if (!c.sol->empty()) {
        c.sol->capture(GRAPH_LAUNCHES);
        c.launched += c.sol->launch(c.chunk);
    }
    c.sol->post_status();
    c.state = C_RUNNING;
}

// Finishes job b of the cohort (its block has stopped).
void finish_job(pc_server *srv, Cohort &c, int b) {
    Job *j = c.jobs[b];
    const pc_job &sp = j->spec;
    const int64_t off = c.sel->S.off[b];
    c.sol->output(c.corr.p, b);
    PC_CUDA(cudaMemcpyAsync(sp.corrected_dev, c.corr.p + 3 * off, 12 * sp.n, cudaMemcpyDeviceToDevice, c.s));
    PgdResult r;
    c.sol->block_result(b, r);
    pc_correct_stats &st = j->res.stats;
    memset(&st, 0, sizeof(st));
    st.iters = r.iters;
    st.loss_evals = r.loss_evals;
    st.viol0 = r.viol0;
    st.viol_final = r.viol_final;
    st.loss0 = r.loss0;
    st.loss_final = r.loss_final;
    st.n_vulnerable = c.sel->stats[b].n_vulnerable;
    st.n_active = c.sel->stats[b].n_active;
    st.n_editable = r.n_editable;
    st.converged = r.converged ? 1 : 0;
    st.pgd_launches = c.launched;
    if (sp.stream_dev) {
        j->res.stream_bytes = encode_edits(sp.recon_dev, sp.corrected_dev, sp.n, &sp.params, sp.stream_dev,
                                           sp.stream_cap, c.s, srv->hs);
    } else {
        PC_CUDA(cudaStreamSynchronize(c.s));
    }
    c.finished[b] = 1;
    publish(srv, j, PC_JOB_DONE, r.converged ? PC_OK : PC_WARN_NOT_CONVERGED, nullptr);
}

// One look at a running cohort; returns true if anything happened.
bool progress(pc_server *srv, Cohort &c) {
    if (!c.sol->empty() && !c.sol->status_ready()) return false;
    if (c.sol->empty()) c.sol->wait_status();
    for (size_t b = 0; b < c.jobs.size(); ++b) {
        if (c.finished[b] || !c.sol->block_stopped((int)b)) continue;
        try {
            finish_job(srv, c, (int)b);
        } catch (const Fail &f) {
            c.finished[b] = 1;
            publish(srv, c.jobs[b], PC_JOB_ERROR, f.st, pc_last_error());
        }
    }
    bool all = true;
    for (char f : c.finished) all &= f != 0;
    if (all) return true;
    if (c.launched >= c.sol->max_launches()) {
        fail_cohort(srv, c, PC_ETIMEOUT, "PGD loop did not reach its stop decision");
        return true;
    }
    c.launched += c.sol->launch(c.chunk);
    c.sol->post_status();
    c.chunk = std::min(c.chunk * 2, MAX_CHUNK);
    return true;
}

bool cohort_done(const Cohort &c) {
    if (c.finished.empty()) return false;
    for (char f : c.finished)
        if (!f) return false;
    return true;
}

// Forms and counts one cohort from the head of the queue; returns true if it did.
bool admit(pc_server *srv) {
    std::vector<Job *> take;
    int64_t n = 0;
    {
        std::lock_guard<std::mutex> lk(srv->mu);
        while (!srv->pending.empty()) {
            Job *j = srv->pending.front();
            if (srv->resident_jobs + (int64_t)take.size() >= srv->max_slots) break;
            const int64_t nn = n + j->spec.n;
            if (!take.empty() && nn > srv->max_cohort_n) break;
            if (!take.empty() && srv->used + count_pass_bytes(nn) > srv->budget) break;
            if (take.empty() && srv->used + count_pass_bytes(j->spec.n) > srv->budget) {
                if (count_pass_bytes(j->spec.n) > srv->budget) {
                    // can never fit
                    srv->pending.pop_front();
                    j->res.state = PC_JOB_ERROR;
                    j->res.status = PC_ENOMEM;
                    std::strncpy(j->res.error, "job does not fit the server's memory budget", sizeof(j->res.error) - 1);
                    j->res.done_ns = now_ns();
                    ++srv->n_finished;
                    srv->cv_done.notify_all();
                    continue;
                }
                break;   // wait for memory
            }
            srv->pending.pop_front();
            take.push_back(j);
            n = nn;
        }
    }
    if (take.empty()) return false;
    // validate each job alone; failures end here
    std::vector<Job *> ok;
    cudaStream_t vs = nullptr;
    PC_CUDA(cudaStreamCreateWithFlags(&vs, cudaStreamNonBlocking));
    for (Job *j : take) {
        try {
            validate(j, vs, srv->hs);
            ok.push_back(j);
        } catch (const Fail &f) {
            publish(srv, j, PC_JOB_ERROR, f.st, pc_last_error());
        }
    }
    cudaStreamSynchronize(vs);
    cudaStreamDestroy(vs);
    if (ok.empty()) return true;
    std::unique_ptr<Cohort> c(new Cohort());
    c->jobs = ok;
    c->n = 0;
    for (Job *j : ok) c->n += j->spec.n;
    c->bytes1 = count_pass_bytes(c->n);
    srv->used += c->bytes1;
    srv->resident_jobs += (int64_t)ok.size();
    ++srv->n_cohorts;
    try {
        setup_count(srv, *c);
    } catch (const Fail &f) {
        c->finished.assign(c->jobs.size(), 0);
        fail_cohort(srv, *c, f.st, pc_last_error());
    }
    srv->peak = std::max(srv->peak, srv->used);
    srv->cohorts.push_back(std::move(c));
    return true;
}

void retire_finished(pc_server *srv) {
    for (size_t k = 0; k < srv->cohorts.size();) {
        Cohort &c = *srv->cohorts[k];
        if (cohort_done(c)) {
            srv->used -= c.bytes1 + (c.state == C_RUNNING ? c.bytes2 : 0);
            srv->resident_jobs -= (int64_t)c.jobs.size();
            srv->cohorts.erase(srv->cohorts.begin() + k);
        } else {
            ++k;
        }
    }
}

void worker_main(pc_server *srv) {
    cudaSetDevice(srv->device);
    for (;;) {
        {
            std::unique_lock<std::mutex> lk(srv->mu);
            if (srv->stopping && srv->pending.empty() && srv->cohorts.empty()) break;
        }
        bool did = false;
        // counted cohorts move on when their estimate fits (or fail if it never can)
        for (auto &cp : srv->cohorts) {
            Cohort &c = *cp;
            if (c.state != C_COUNTED || cohort_done(c)) continue;
            bool others = false;
            for (auto &o : srv->cohorts)
                if (o.get() != &c && o->state == C_RUNNING && !cohort_done(*o)) others = true;
            if (srv->used + c.bytes2 > srv->budget) {
                if (!others) {
                    c.finished.assign(c.jobs.size(), 0);
                    fail_cohort(srv, c, PC_ENOMEM, "cohort does not fit the server's memory budget");
                    did = true;
                }
                continue;
            }
            srv->used += c.bytes2;
            srv->peak = std::max(srv->peak, srv->used);
            try {
                setup_run(srv, c);
            } catch (const Fail &f) {
                c.state = C_RUNNING;
                if (c.finished.empty()) c.finished.assign(c.jobs.size(), 0);
                fail_cohort(srv, c, f.st, pc_last_error());
            }
            did = true;
        }
        for (auto &cp : srv->cohorts) {
            Cohort &c = *cp;
            if (c.state != C_RUNNING || cohort_done(c)) continue;
            try {
                did |= progress(srv, c);
            } catch (const Fail &f) {
                fail_cohort(srv, c, f.st, pc_last_error());
                did = true;
            }
        }
        retire_finished(srv);
        did |= admit(srv);
        if (!did) {
            std::unique_lock<std::mutex> lk(srv->mu);
            srv->cv_work.wait_for(lk, std::chrono::microseconds(50));
        }
    }
}

pc_status server_guard(const std::function<pc_status()> &f) {
    try {
        return f();
    } catch (const Fail &e) {
        return e.st;
    } catch (const std::bad_alloc &) {
        set_error("host allocation failed");
        return PC_ENOMEM;
    } catch (...) {
        set_error("unknown failure");
        return PC_ECUDA;
    }
}

}  // namespace
}  // namespace pc

using namespace pc;

extern "C" {

pc_status pc_server_create(pc_ctx *ctx, size_t mem_budget, int32_t max_slots, int64_t max_cohort_particles,
                           pc_server **out) {
    return server_guard([&]() -> pc_status {
        if (!ctx || !out) fail(PC_EINVAL, "NULL argument");
        *out = nullptr;
        const int dev = ctx_device(ctx);
        PC_CUDA(cudaSetDevice(dev));
        if (max_slots < 0 || max_cohort_particles < 0) fail(PC_EINVAL, "negative limit");
        pc_server *s = new pc_server();
        s->device = dev;
        s->budget = mem_budget ? (int64_t)mem_budget : ((int64_t)40 << 30);
        s->max_slots = max_slots ? max_slots : 256;
        s->max_cohort_n = max_cohort_particles ? max_cohort_particles : ((int64_t)1 << 24);
        s->worker = std::thread(worker_main, s);
        *out = s;
        return PC_OK;
    });
}

void pc_server_destroy(pc_server *srv) {
    if (!srv) return;
    {
        std::lock_guard<std::mutex> lk(srv->mu);
        srv->stopping = true;
    }
    srv->cv_work.notify_all();
    if (srv->worker.joinable()) srv->worker.join();
    if (srv->hs.p) cudaFreeHost(srv->hs.p);
    delete srv;
}

pc_status pc_serve_submit(pc_server *srv, const pc_job *job, uint64_t *ticket) {
    return server_guard([&]() -> pc_status {
        if (!srv || !job || !ticket) fail(PC_EINVAL, "NULL argument");
        check_params(&job->params, job->n, true);
        if (!job->orig_dev || !job->recon_dev || !job->corrected_dev) fail(PC_EINVAL, "NULL buffer");
        if (job->stream_dev && (!(job->params.xi > 0.0)))
            fail(PC_EINVAL, "xi must be > 0 to encode edits");
        std::unique_ptr<Job> j(new Job());
        j->spec = *job;
        j->res.state = PC_JOB_PENDING;
        j->res.submit_ns = now_ns();
        {
            std::lock_guard<std::mutex> lk(srv->mu);
            if (srv->stopping) fail(PC_EBUSY, "server is stopping");
            j->ticket = srv->next_ticket++;
            *ticket = j->ticket;
            srv->pending.push_back(j.get());
            srv->jobs[j->ticket] = std::move(j);
            ++srv->n_submitted;
        }
        srv->cv_work.notify_all();
        return PC_OK;
    });
}

pc_status pc_serve_poll(pc_server *srv, uint64_t ticket, pc_job_result *res) {
    if (!srv || !res) return PC_EINVAL;
    std::lock_guard<std::mutex> lk(srv->mu);
    auto it = srv->jobs.find(ticket);
    if (it == srv->jobs.end()) {
        set_error("unknown ticket");
        return PC_EBUSY;
    }
    *res = it->second->res;
    return PC_OK;
}

pc_status pc_serve_wait(pc_server *srv, uint64_t ticket, int64_t timeout_ms, pc_job_result *res) {
    if (!srv || !res) return PC_EINVAL;
    std::unique_lock<std::mutex> lk(srv->mu);
    auto it = srv->jobs.find(ticket);
    if (it == srv->jobs.end()) {
        set_error("unknown ticket");
        return PC_EBUSY;
    }
    Job *j = it->second.get();
    auto done = [&]() { return j->res.state == PC_JOB_DONE || j->res.state == PC_JOB_ERROR; };
    if (timeout_ms < 0) {
        srv->cv_done.wait(lk, done);
    } else if (!srv->cv_done.wait_for(lk, std::chrono::milliseconds(timeout_ms), done)) {
        *res = j->res;
        set_error("wait timed out");
        return PC_ETIMEOUT;
    }
    *res = j->res;
    return PC_OK;
}

pc_status pc_serve_counters(pc_server *srv, int64_t out[4]) {
    if (!srv || !out) return PC_EINVAL;
    std::lock_guard<std::mutex> lk(srv->mu);
    out[0] = srv->n_submitted;
    out[1] = srv->n_finished;
    out[2] = srv->n_cohorts;
    out[3] = srv->peak;
    return PC_OK;
}

}  // extern "C"
