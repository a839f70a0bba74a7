// Request loop: pc_server_* and pc_serve_* (include/pc.h).  Not part of the paper.
//
// Two threads per server.  The setup thread admits jobs in FIFO order into cohorts: a
// cohort gathers its jobs' inputs into one block set (one block per job), runs the
// count pass of the selection, waits until the memory its counts call for fits the
// budget, selects its constraints, builds a PgdSolver whose iterations replay a CUDA
// graph on the cohort's own stream, and hands the cohort to the run thread.  The run
// thread launches iteration chunks and finishes each job as soon as its block has
// stopped (output rows of that block, copy-out, optional edit stream).  Chunks go to
// the oldest cohorts first: a younger cohort waits while the cohorts ahead of it keep
// enough rows in flight to fill the GPU, so large early jobs are not starved by the
// stream of later ones.  Blocks of a set never interact, so a job's result does not
// depend on its cohort.
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
constexpr int64_t SATURATE_ROWS = int64_t(1) << 21;   // rows in flight that fill the GPU

int64_t now_ns() {
    return std::chrono::duration_cast<std::chrono::nanoseconds>(std::chrono::steady_clock::now().time_since_epoch())
        .count();
}

struct Job {
    uint64_t ticket = 0;
    pc_job spec{};
    pc_job_result res{};
    bool alone = false;   // admit in a cohort of its own (its cohort did not fit the budget)
};

enum CohortState { C_COUNTED, C_RUNNING };

struct Cohort {
    std::vector<Job *> jobs;
    cudaStream_t s = nullptr;            // high priority: PGD state, iterations, finishing jobs
    cudaStream_t s_setup = nullptr;      // low priority: gathering, binning, pair search, selection
    CohortState state = C_COUNTED;
    int64_t n = 0;
    int64_t bytes1 = 0, bytes2 = 0;      // estimates: count pass, the rest
    DBuf<float> orig, recon, corr;       // gathered inputs and the corrected coordinates
    std::unique_ptr<Selection> sel;
    std::unique_ptr<PgdSolver> sol;
    std::vector<char> finished;
    int64_t slots_back = 0;              // finished jobs whose slots went back to the server
    int chunk = GRAPH_LAUNCHES;
    int64_t launched = 0;
    bool in_flight = false;              // a chunk and its status copy are queued
    int64_t rows = 0;                    // rows of the blocks still iterating (last status)
    ~Cohort() {
        // everything queued on the run stream finishes before the setup stream's buffers go
        if (s) cudaStreamSynchronize(s);
        sol.reset();
        sel.reset();
        orig.release();
        recon.release();
        corr.release();
        if (s_setup) {
            cudaStreamSynchronize(s_setup);
            cudaStreamDestroy(s_setup);
        }
        if (s) cudaStreamDestroy(s);
    }
};

}  // namespace
}  // namespace pc

struct pc_server {
    int device = 0;
    int64_t budget = 0;
    int max_slots = 0;
    int64_t max_cohort_n = 0;
    std::mutex mu;                                         // everything below up to the threads
    std::condition_variable cv_setup, cv_run, cv_done;
    bool stopping = false, setup_exited = false;
    uint64_t next_ticket = 1;
    std::map<uint64_t, std::unique_ptr<pc::Job>> jobs;   // every job ever submitted
    std::deque<pc::Job *> pending;                         // FIFO
    std::vector<std::unique_ptr<pc::Cohort>> ready;       // set up, not yet taken by the run thread
    int64_t used = 0, peak = 0, resident_jobs = 0;         // memory estimate; unfinished jobs of live cohorts
    int64_t live_cohorts = 0;                              // admitted and not yet retired
    int64_t n_submitted = 0, n_finished = 0, n_cohorts = 0;
    // thread-owned
    std::vector<std::unique_ptr<pc::Cohort>> running;     // run thread, oldest first
    pc::HostScratch hs_setup, hs_run;
    std::thread setup_thr, run_thr;
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

// Device bytes of a job's count pass: gathered inputs, binning, labels, the cell table
// (4 B per cell, at most cell_factor cells per particle) and the vulnerable-pair buffer.
int64_t count_pass_bytes(const pc_job &sp) {
    const int64_t f = sp.params.cell_factor > 0 ? sp.params.cell_factor : 8;
    const int64_t cells = sp.params.cell_cap_log2 > 0 ? ((int64_t)1 << std::min(sp.params.cell_cap_log2, 30))
                                                      : std::min<int64_t>((int64_t)1 << 28, f * sp.n);
    return 176 * sp.n + 4 * std::max<int64_t>(cells, 1 << 16) + 8 * vulnerable_guess(sp.n) + (int64_t)(1 << 20);
}

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
    // iterations of running cohorts take precedence over the setup of new ones
    int least = 0, greatest = 0;
    PC_CUDA(cudaDeviceGetStreamPriorityRange(&least, &greatest));
    PC_CUDA(cudaStreamCreateWithPriority(&c.s, cudaStreamNonBlocking, greatest));
    PC_CUDA(cudaStreamCreateWithPriority(&c.s_setup, cudaStreamNonBlocking, least));
    const cudaStream_t ss = c.s_setup;
    c.orig.alloc(3 * c.n, ss);
    c.recon.alloc(3 * c.n, ss);
    c.corr.alloc(3 * c.n, ss);
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
        PC_CUDA(cudaMemcpyAsync(c.orig.p + 3 * at, sp.orig_dev, 12 * sp.n, cudaMemcpyDeviceToDevice, ss));
        PC_CUDA(cudaMemcpyAsync(c.recon.p + 3 * at, sp.recon_dev, 12 * sp.n, cudaMemcpyDeviceToDevice, ss));
        at += sp.n;
    }
    S.off[nb] = at;
    PC_CUDA(cudaMemcpyAsync(c.corr.p, c.recon.p, 12 * c.n, cudaMemcpyDeviceToDevice, ss));
    select_count(srv->hs_setup, c.orig.p, ss, *c.sel);
    c.bytes2 = select_more_bytes(*c.sel);
}

// Selection, PGD state and the captured graph; the first chunk is launched.
void setup_run(pc_server *srv, Cohort &c) {
    const cudaStream_t ss = c.s_setup;
    select_emit(srv->hs_setup, ss, *c.sel);
    BlockSet &S = c.sel->S;
    // PGD constants need M over orig and recon of each block
    BlockSet V;
    V.nb = S.nb;
    V.n = S.n;
    V.prm = S.prm;
    V.off = S.off;
    inspect_blocks(c.orig.p, c.recon.p, V, ss, srv->hs_setup);
    std::vector<Consts> cp(V.nb);
    for (int b = 0; b < V.nb; ++b) cp[b] = make_consts(&V.prm[b], V.ins[b], V.off[b + 1] - V.off[b], true);
    // the run stream starts after the setup stream's work, and the setup stream frees the
    // selection's buffers only after the solver has read them
    cudaEvent_t ev = nullptr;
    PC_CUDA(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
    PC_CUDA(cudaEventRecord(ev, ss));
    PC_CUDA(cudaStreamWaitEvent(c.s, ev, 0));
    try {
        c.sol.reset(new PgdSolver(c.sel->B, S, cp, c.orig.p, c.recon.p, c.sel->A.p, c.sel->nA, c.s, srv->hs_setup));
    } catch (...) {
        cudaEventDestroy(ev);
        throw;
    }
    PC_CUDA(cudaEventRecord(ev, c.s));
    PC_CUDA(cudaStreamWaitEvent(ss, ev, 0));
    cudaEventDestroy(ev);
    // the solver keeps what it needs: cell lists and pairs go back to the pool
    c.sel->A.release();
    c.sel->B.keys.release();
    c.sel->B.order.release();
    c.sel->B.P4.release();
    c.sel->B.cell_start.release();
    c.sel->B.occ.release();
    c.sel->B.dense.release();
    c.sel->B.chunks.release();
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
    c.in_flight = true;
    c.rows = c.sol->rows();
    c.state = C_RUNNING;
}

// A finished job's slot goes back to the server at once (its device memory stays with
// the cohort's buffers until the cohort retires).
void give_back_slot(pc_server *srv, Cohort &c) {
    std::lock_guard<std::mutex> lk(srv->mu);
    --srv->resident_jobs;
    ++c.slots_back;
    srv->cv_setup.notify_all();
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
    st.resets = r.resets;
    st.row_updates = r.row_updates;
    st.pair_evals = r.pair_evals;
    if (sp.stream_dev) {
        j->res.stream_bytes = encode_edits(sp.recon_dev, sp.corrected_dev, sp.n, &sp.params, sp.stream_dev,
                                           sp.stream_cap, c.s, srv->hs_run);
    } else {
        PC_CUDA(cudaStreamSynchronize(c.s));
    }
    c.finished[b] = 1;
    publish(srv, j, PC_JOB_DONE, r.converged ? PC_OK : PC_WARN_NOT_CONVERGED, nullptr);
    give_back_slot(srv, c);
}

// Finishes the jobs whose blocks have stopped, from the landed status copy.
void finish_stopped(pc_server *srv, Cohort &c) {
    for (size_t b = 0; b < c.jobs.size(); ++b) {
        if (c.finished[b] || !c.sol->block_stopped((int)b)) continue;
        try {
            finish_job(srv, c, (int)b);
        } catch (const Fail &f) {
            c.finished[b] = 1;
            publish(srv, c.jobs[b], PC_JOB_ERROR, f.st, pc_last_error());
            give_back_slot(srv, c);
        }
    }
    c.rows = c.sol->active_rows();
}

bool cohort_done(const Cohort &c) {
    if (c.finished.empty()) return false;
    for (char f : c.finished)
        if (!f) return false;
    return true;
}

void release(pc_server *srv, const Cohort &c) {
    std::lock_guard<std::mutex> lk(srv->mu);
    srv->used -= c.bytes1 + (c.state == C_RUNNING ? c.bytes2 : 0);
    srv->resident_jobs -= (int64_t)c.jobs.size() - c.slots_back;
    --srv->live_cohorts;
    srv->cv_setup.notify_all();
}

// ----------------------------------------------------------------------------- setup thread
// Takes the next cohort's jobs from the head of the queue (under srv->mu); empty when
// the queue is empty or memory and slots are short.
std::vector<Job *> take_jobs(pc_server *srv, int64_t &n, int64_t &bytes) {
    std::vector<Job *> take;
    n = 0;
    bytes = 0;
    while (!srv->pending.empty()) {
        Job *j = srv->pending.front();
        if (srv->resident_jobs + (int64_t)take.size() >= srv->max_slots) break;
        if (j->alone && !take.empty()) break;     // it goes in a cohort of its own
        const int64_t nn = n + j->spec.n, bj = count_pass_bytes(j->spec);
        if (!take.empty() && nn > srv->max_cohort_n) break;
        if (srv->used + bytes + bj > srv->budget) {
            if (take.empty() && bj > srv->budget) {
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
        bytes += bj;
        if (j->alone) break;
    }
    if (!take.empty()) {
        srv->used += bytes;
        srv->resident_jobs += (int64_t)take.size();
        ++srv->live_cohorts;
        ++srv->n_cohorts;
        srv->peak = std::max(srv->peak, srv->used);
    }
    return take;
}

void setup_main(pc_server *srv) {
    cudaSetDevice(srv->device);
    cudaStream_t vs = nullptr;
    cudaStreamCreateWithFlags(&vs, cudaStreamNonBlocking);
    for (;;) {
        std::vector<Job *> take;
        int64_t n = 0, bytes1 = 0;
        {
            std::unique_lock<std::mutex> lk(srv->mu);
            for (;;) {
                take = take_jobs(srv, n, bytes1);
                if (!take.empty()) break;
                if (srv->stopping && srv->pending.empty()) break;
                srv->cv_setup.wait_for(lk, std::chrono::milliseconds(1));
            }
            if (take.empty()) break;
        }
        // validate each job alone; failures end here
        std::vector<Job *> ok;
        for (Job *j : take) {
            try {
                validate(j, vs, srv->hs_setup);
                ok.push_back(j);
            } catch (const Fail &f) {
                publish(srv, j, PC_JOB_ERROR, f.st, pc_last_error());
            }
        }
        std::unique_ptr<Cohort> c(new Cohort());
        c->jobs = ok;
        c->bytes1 = bytes1;
        for (Job *j : ok) c->n += j->spec.n;
        if (ok.size() < take.size()) {
            // the failed jobs give back their slots (their bytes stay with the cohort's estimate)
            std::lock_guard<std::mutex> lk(srv->mu);
            srv->resident_jobs -= (int64_t)(take.size() - ok.size());
        }
        if (ok.empty()) {
            release(srv, *c);
            continue;
        }
        c->finished.assign(c->jobs.size(), 0);
        try {
            setup_count(srv, *c);
        } catch (const Fail &f) {
            fail_cohort(srv, *c, f.st, pc_last_error());
            release(srv, *c);
            continue;
        }
        // the rest of the cohort's memory, once it fits
        bool fits = true;
        {
            std::unique_lock<std::mutex> lk(srv->mu);
            while (srv->used + c->bytes2 > srv->budget) {
                if (srv->live_cohorts == 1) {   // this is the only cohort: nothing else will free memory
                    fits = false;
                    break;
                }
                srv->cv_setup.wait_for(lk, std::chrono::milliseconds(1));
            }
            if (fits) {
                srv->used += c->bytes2;
                srv->peak = std::max(srv->peak, srv->used);
            }
        }
        if (!fits && c->jobs.size() > 1) {
            // together they do not fit: back to the head of the queue, each in a cohort of its own
            release(srv, *c);
            {
                std::lock_guard<std::mutex> lk(srv->mu);
                for (auto it = c->jobs.rbegin(); it != c->jobs.rend(); ++it) {
                    (*it)->alone = true;
                    srv->pending.push_front(*it);
                }
            }
            c->jobs.clear();
            continue;
        }
        if (!fits) {
            fail_cohort(srv, *c, PC_ENOMEM, "cohort does not fit the server's memory budget");
            release(srv, *c);
            continue;
        }
        try {
            setup_run(srv, *c);
        } catch (const Fail &f) {
            c->state = C_RUNNING;
            fail_cohort(srv, *c, f.st, pc_last_error());
            release(srv, *c);
            continue;
        }
        {
            std::lock_guard<std::mutex> lk(srv->mu);
            srv->ready.push_back(std::move(c));
        }
        srv->cv_run.notify_all();
    }
    cudaStreamDestroy(vs);
    std::lock_guard<std::mutex> lk(srv->mu);
    srv->setup_exited = true;
    srv->cv_run.notify_all();
}

// ----------------------------------------------------------------------------- run thread
void run_main(pc_server *srv) {
    cudaSetDevice(srv->device);
    for (;;) {
        {
            std::unique_lock<std::mutex> lk(srv->mu);
            for (auto &c : srv->ready) srv->running.push_back(std::move(c));
            srv->ready.clear();
            if (srv->setup_exited && srv->running.empty()) break;
        }
        bool did = false;
        // land status copies and finish stopped jobs
        for (auto &cp : srv->running) {
            Cohort &c = *cp;
            if (!c.in_flight) continue;
            try {
                if (!c.sol->empty() && !c.sol->status_ready()) continue;
                if (c.sol->empty()) c.sol->wait_status();
                c.in_flight = false;
                finish_stopped(srv, c);
            } catch (const Fail &f) {
                fail_cohort(srv, c, f.st, pc_last_error());
            }
            did = true;
        }
        // oldest first: launch while the rows in flight do not fill the GPU
        int64_t rows = 0;
        for (auto &cp : srv->running)
            if (cp->in_flight) rows += cp->rows;
        bool first = true;
        for (auto &cp : srv->running) {
            Cohort &c = *cp;
            if (cohort_done(c)) continue;
            const bool oldest = first;
            first = false;
            if (c.in_flight) continue;
            if (!oldest && rows + c.rows > SATURATE_ROWS) continue;
            try {
                if (c.launched >= c.sol->max_launches()) {
                    fail_cohort(srv, c, PC_ETIMEOUT, "PGD loop did not reach its stop decision");
                    continue;
                }
                c.launched += c.sol->launch(c.chunk);
                c.sol->post_status();
                c.in_flight = true;
                c.chunk = std::min(c.chunk * 2, MAX_CHUNK);
                rows += c.rows;
            } catch (const Fail &f) {
                fail_cohort(srv, c, f.st, pc_last_error());
            }
            did = true;
        }
        // retire finished cohorts (their memory goes back to the pool and the budget)
        for (size_t k = 0; k < srv->running.size();) {
            if (cohort_done(*srv->running[k]) && !srv->running[k]->in_flight) {
                release(srv, *srv->running[k]);
                srv->running.erase(srv->running.begin() + k);
                did = true;
            } else {
                ++k;
            }
        }
        if (!did) {
            std::unique_lock<std::mutex> lk(srv->mu);
            srv->cv_run.wait_for(lk, std::chrono::microseconds(50));
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
        s->setup_thr = std::thread(setup_main, s);
        s->run_thr = std::thread(run_main, s);
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
    srv->cv_setup.notify_all();
    srv->cv_run.notify_all();
    if (srv->setup_thr.joinable()) srv->setup_thr.join();
    if (srv->run_thr.joinable()) srv->run_thr.join();
    if (srv->hs_setup.p) cudaFreeHost(srv->hs_setup.p);
    if (srv->hs_run.p) cudaFreeHost(srv->hs_run.p);
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
        srv->cv_setup.notify_all();
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
