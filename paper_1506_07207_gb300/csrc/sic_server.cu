// sic_server.cu -- request server with continuous batching.
//
// Requests (a simulation and a step count) wait in a first-come queue.  Each
// tick admits queued requests while an active slot is free and their device
// memory fits the budget, advances every active simulation by one chunk of
// steps -- every step is one launch of the step kernel over all of them, so
// their work shares the GPU -- and retires the ones that are done.  The plain
// mode is the one-simulation-per-launch baseline: one request at a time, run
// to completion with sic_step.  A simulation gives the same bits alone and in
// any batch, because every per-simulation result is an integer sum or a
// fixed-order reduction.  The batched mode overlaps its host work with the
// GPU: a tick collects the chunk in flight, launches the next one, and only
// then retires finished requests and creates newly admitted ones, on a side
// stream; those join the launches from the next tick on.  A request with a
// refinement length (Sec. 2.6) holds
// after the step that leaves a particle longer than it; the server then
// refines it (its device memory grows) and it goes on in the next chunk, so it
// is refined at the same steps alone and in the mix.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>
#include <deque>
#include <new>
#include <vector>

#include "sic.h"
#include "sic_host.h"

namespace {

using Clock = std::chrono::steady_clock;

struct Request {
    int64_t id = 0;
    bool horizontal = false;
    int32_t n_steps = 0;
    int32_t keep = 0;
    sic_config cfg{};
    std::vector<int32_t> counts;
    std::vector<uint8_t> closed;
    std::vector<int32_t> winding;
    std::vector<double> a, b, c;  // horizontal: x_template, v_sheet, w_sheet; else x, v, w
    int32_t n_template = 0;
    size_t bytes = 0;
    int64_t segments = 0;
    double t_submit = 0;
};

struct Active {
    Request req;
    sic_sim *sim = nullptr;
    int32_t left = 0;
    double t_admit = 0;
    int64_t steps_seen = 0;       // the simulation's step count at the last look
    int64_t segment_updates = 0;  // segments x steps, with the segments refinement added
};

}  // namespace

struct sic_server {
    sic_server_config cfg{};
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    cudaStream_t side = nullptr;            // creation and retirement, beside the steps
    std::deque<Request> queue;
    std::vector<Active> active;
    std::vector<Active> fresh;              // created on the side stream, stepping from the next tick
    bool inflight = false;                  // a chunk of steps is launched and not yet collected
    int launch_rc = SIC_OK;                 // a launch of that chunk failed
    std::vector<sic_result> done;
    int64_t next_id = 1;
    size_t used = 0, peak = 0;
    sic_host::Plan plan[2];
    bool plan_valid = false;
    Clock::time_point t0;
    int64_t completed = 0, segment_updates = 0, ticks = 0;
    int64_t waits_slots = 0, waits_memory = 0, refinements = 0;
    cudaEvent_t ev[2] = {nullptr, nullptr};  // around each tick's steps
    double busy_s = 0;
    SimScalars *scal = nullptr;             // pinned: the active simulations' scalars
    int scal_cap = 0;

    double now() const { return std::chrono::duration<double>(Clock::now() - t0).count(); }
};

namespace {

void drop_plans(sic_server *s)
{
    for (auto &p : s->plan)
        sic_host::free_plan(p, s->stream);
    s->plan_valid = false;
}

// Device memory one request will hold once admitted.
size_t request_bytes(const sic_config &cfg, const int32_t *counts, int M, bool per_q)
{
    const int64_t n_alloc = sic_host::padded_tracers(counts, M);
    const int64_t n_items = sic_host::work_items(counts, M);
    return sic_host::sim_layout(cfg.nx, n_alloc, n_items, per_q, std::max(1, cfg.history_len), cfg.deposit,
                               cfg.mode_k).total;
}

int make_sim(Request &r, cudaStream_t stream, sic_sim **out)
{
    sic_config cfg = r.cfg;
    cfg.stream = stream;
    cfg.history_len = std::max(1, cfg.history_len);
    if (r.horizontal)
        return sic_create_horizontal(&cfg, r.n_template, r.a.data(), r.b.data(), r.c.data(), out);
    cfg.tracers_per_sheet = r.counts.data();
    cfg.sheet_closed = r.closed.data();
    cfg.sheet_winding = r.winding.data();
    return sic_create(&cfg, r.a.data(), r.b.data(), r.c.data(), out);
}

void finish(sic_server *s, Active &a, int status, double t_done)
{
    sic_result res{};
    res.id = a.req.id;
    res.status = status;
    res.t_submit = a.req.t_submit;
    res.t_admit = a.t_admit;
    res.t_done = t_done;
    if (a.sim) {
        sic_diag d{};
        const int rc = sic_diagnostics(a.sim, &d);
        if (status == SIC_OK)
            res.status = rc;
        res.steps = d.step;
        res.segment_updates = a.segment_updates;
        res.field_energy = d.field_energy;
        res.kinetic_energy = d.kinetic_energy;
        res.momentum = d.momentum;
        res.charge_fixed = d.charge_fixed;
        s->used -= a.sim->dbytes;
        if (a.req.keep && (res.status == SIC_OK || res.status == SIC_ELIMIT)) {
            // the caller owns it now: it gets a stream of its own, since the
            // server's may be destroyed with the server
            cudaStream_t own = nullptr;
            if (cudaStreamSynchronize(a.sim->stream) == cudaSuccess &&
                cudaStreamCreateWithFlags(&own, cudaStreamNonBlocking) == cudaSuccess) {
                a.sim->stream = own;
                a.sim->own_stream = true;
                res.sim = a.sim;
            } else {
                res.status = SIC_ECUDA;
                sic_destroy(a.sim);
            }
        } else {
            sic_destroy(a.sim);
        }
        a.sim = nullptr;
    }
    s->completed += 1;
    s->segment_updates += res.segment_updates;
    s->done.push_back(res);
}

// Account a simulation's steps since the last look (at its segments before any
// refinement that follows) and refine it if it holds for that; its device
// memory may grow.  sc: its scalars, read after its steps.  Returns a SIC_E*
// code.
// With `defer` set, a simulation that holds for refinement is not refined:
// *defer is left true for it (false otherwise) and the caller refines it.
int look(sic_server *srv, Active &a, const SimScalars &sc, bool *defer = nullptr)
{
    int st = sic_host::scalars_status(sc);
    a.segment_updates += (sc.step - a.steps_seen) * sic_host::segments(a.sim);
    a.steps_seen = sc.step;
    a.left = a.req.n_steps - (int32_t)sc.step;
    const bool wants = st == SIC_OK && (sc.hold & SIC_HOLD_REFINE) && a.left > 0;
    if (defer) {
        *defer = wants;
        return st;
    }
    if (wants) {
        srv->refinements += 1;
        const size_t before = a.sim->dbytes;
        st = sic_host::refine_held(a.sim, nullptr);
        srv->used += a.sim->dbytes - before;
        srv->peak = std::max(srv->peak, srv->used);
        srv->plan_valid = false;
    }
    return st;
}

// Read every active simulation's scalars with one synchronisation (they all
// run on the server's stream) into srv->scal.
int read_all(sic_server *srv)
{
    const int n = (int)srv->active.size();
    if (n > srv->scal_cap) {
        if (srv->scal)
            cudaFreeHost(srv->scal);
        srv->scal = nullptr;
        srv->scal_cap = 0;
        if (cudaMallocHost(&srv->scal, sizeof(SimScalars) * (size_t)std::max(n, 64)) != cudaSuccess)
            return SIC_ENOMEM;
        srv->scal_cap = std::max(n, 64);
    }
    for (int i = 0; i < n; ++i)
        if (cudaMemcpyAsync(&srv->scal[i], srv->active[i].sim->h.sc, sizeof(SimScalars), cudaMemcpyDeviceToHost,
                            srv->stream) != cudaSuccess)
            return SIC_ECUDA;
    return cudaStreamSynchronize(srv->stream) == cudaSuccess ? SIC_OK : SIC_ECUDA;
}

// Admit queued requests in arrival order while a slot is free and the memory
// fits, creating each on `stream` into `into`.
void admit(sic_server *srv, cudaStream_t stream, std::vector<Active> &into)
{
    while (!srv->queue.empty()) {
        Request &r = srv->queue.front();
        if ((int64_t)r.bytes > srv->cfg.hbm_budget) {
            Active a;
            a.req = std::move(r);
            srv->queue.pop_front();
            finish(srv, a, SIC_EBUSY, srv->now());
            continue;
        }
        if ((int)(srv->active.size() + srv->fresh.size()) >= srv->cfg.max_active) {
            srv->waits_slots += 1;
            break;
        }
        if ((int64_t)(srv->used + r.bytes) > srv->cfg.hbm_budget) {
            srv->waits_memory += 1;
            break;
        }
        Active a;
        a.t_admit = srv->now();
        const int rc = make_sim(r, stream, &a.sim);
        if (rc == SIC_ENOMEM && !(srv->active.empty() && srv->fresh.empty()))
            break;  // wait for memory to come free
        a.req = std::move(r);
        srv->queue.pop_front();
        if (rc != SIC_OK) {
            a.sim = nullptr;
            finish(srv, a, rc, srv->now());
            continue;
        }
        a.left = a.req.n_steps;
        srv->used += a.sim->dbytes;
        srv->peak = std::max(srv->peak, srv->used);
        into.push_back(std::move(a));
        srv->plan_valid = false;
    }
}

// One tick of the batched mode: collect the chunk in flight, let the newly
// created simulations join, launch the next chunk, and while it runs retire
// the finished requests and create the newly admitted ones on the side
// stream.
int tick_batched(sic_server *srv)
{
    int rc = SIC_OK;
    std::vector<Active> retired, to_refine;
    std::vector<int> rstatus;
    if (srv->inflight) {
        srv->inflight = false;
        rc = srv->launch_rc;
        srv->launch_rc = SIC_OK;
        if (cudaStreamSynchronize(srv->stream) != cudaSuccess)
            rc = SIC_ECUDA;
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, srv->ev[0], srv->ev[1]) == cudaSuccess)
            srv->busy_s += 1e-3 * ms;
        // each simulation's own step count (a held one took fewer than the
        // chunk); one that holds for refinement (Sec. 2.6) sits out the next
        // chunk, is refined beside it (its device memory growing) and steps
        // again from the tick after
        std::vector<int> status(srv->active.size(), SIC_OK);
        std::vector<char> held(srv->active.size(), 0);
        if (rc == SIC_OK) {
            rc = read_all(srv);
            if (rc == SIC_OK)
                for (size_t i = 0; i < srv->active.size(); ++i) {
                    bool h = false;
                    status[i] = look(srv, srv->active[i], srv->scal[i], &h);
                    held[i] = h;
                }
        }
        std::vector<Active> keep;
        for (size_t i = 0; i < srv->active.size(); ++i) {
            Active &a = srv->active[i];
            const int st = rc != SIC_OK ? rc : status[i];
            if (a.left <= 0 || st != SIC_OK) {
                retired.push_back(std::move(a));
                rstatus.push_back(st);
            } else if (held[i]) {
                to_refine.push_back(std::move(a));  // refined beside the next chunk
            } else {
                keep.push_back(std::move(a));
            }
        }
        if (keep.size() != srv->active.size())
            srv->plan_valid = false;
        srv->active.swap(keep);
        if (rc != SIC_OK)
            drop_plans(srv);
    }
    // the simulations created while the last chunk ran join it
    if (!srv->fresh.empty()) {
        const bool ok = cudaStreamSynchronize(srv->side) == cudaSuccess;
        for (Active &a : srv->fresh) {
            if (ok) {
                a.sim->stream = srv->stream;
                srv->active.push_back(std::move(a));
            } else {
                retired.push_back(std::move(a));
                rstatus.push_back(SIC_ECUDA);
            }
        }
        srv->fresh.clear();
        srv->plan_valid = false;
    }
    // a request with no steps to take (none asked) is done as it stands
    {
        std::vector<Active> keep;
        for (Active &a : srv->active) {
            if (a.left <= 0) {
                retired.push_back(std::move(a));
                rstatus.push_back(SIC_OK);
            } else {
                keep.push_back(std::move(a));
            }
        }
        if (keep.size() != srv->active.size()) {
            srv->active.swap(keep);
            srv->plan_valid = false;
        }
    }
    // the next chunk: k = min(chunk_steps, steps left of any active request)
    if (!srv->active.empty()) {
        int32_t k = srv->cfg.chunk_steps;
        for (const Active &a : srv->active)
            k = std::min(k, std::max(a.left, 0));
        int lrc = SIC_OK;
        if (k > 0 && !srv->plan_valid) {
            drop_plans(srv);
            std::vector<sic_sim *> grp[2];
            for (const Active &a : srv->active)
                grp[a.sim->per_q ? 1 : 0].push_back(a.sim);
            for (int g = 0; g < 2 && lrc == SIC_OK; ++g)
                if (!grp[g].empty() &&
                    sic_host::build_plan(srv->plan[g], grp[g].data(), (int)grp[g].size(), srv->stream) != cudaSuccess)
                    lrc = SIC_ECUDA;
            srv->plan_valid = (lrc == SIC_OK);
        }
        if (k > 0 && lrc != SIC_OK) {
            srv->inflight = true;  // nothing launched: the next tick retires them with the error
            srv->launch_rc = lrc;
            cudaEventRecord(srv->ev[0], srv->stream);
            cudaEventRecord(srv->ev[1], srv->stream);
        } else if (k > 0) {
            cudaEventRecord(srv->ev[0], srv->stream);
            for (int32_t st = 0; st < k && lrc == SIC_OK; ++st)
                for (int g = 0; g < 2 && lrc == SIC_OK; ++g)
                    if (srv->plan[g].mem &&
                        sic_host::launch(srv->plan[g], sic::MODE_STEP, 1.0f, 1, 1, srv->stream) != cudaSuccess)
                        lrc = SIC_ECUDA;
            cudaEventRecord(srv->ev[1], srv->stream);
            srv->inflight = true;  // collected by the next tick
            srv->launch_rc = lrc;
        }
    }
    // while it runs: refine the held simulations on the side stream (they are
    // not in the chunk; they join again from the next tick), retire the
    // finished ones there too (their steps are done), then admit
    for (Active &a : to_refine) {
        a.sim->stream = srv->side;
        srv->refinements += 1;
        const size_t before = a.sim->dbytes;
        const int st = sic_host::refine_held(a.sim, nullptr);
        srv->used += a.sim->dbytes - before;
        srv->peak = std::max(srv->peak, srv->used);
        if (st == SIC_OK) {
            srv->fresh.push_back(std::move(a));
        } else {
            retired.push_back(std::move(a));
            rstatus.push_back(st);
        }
    }
    const double t = srv->now();
    for (size_t i = 0; i < retired.size(); ++i) {
        if (retired[i].sim)
            retired[i].sim->stream = srv->side;
        finish(srv, retired[i], rstatus[i], t);
    }
    admit(srv, srv->side, srv->fresh);
    return SIC_OK;
}

int queue_request(sic_server *srv, Request &&r, int64_t *id)
{
    r.id = srv->next_id++;
    r.t_submit = srv->now();
    if (id)
        *id = r.id;
    srv->queue.push_back(std::move(r));
    return SIC_OK;
}

}  // namespace

extern "C" {

int sic_server_create(const sic_server_config *cfg, sic_server **out)
{
    if (!cfg || !out || cfg->hbm_budget <= 0 || cfg->max_active < 1 || cfg->chunk_steps < 1)
        return SIC_EINVAL;
    sic_server *s = new (std::nothrow) sic_server;
    if (!s)
        return SIC_ENOMEM;
    s->cfg = *cfg;
    if (s->cfg.plain)
        s->cfg.max_active = 1;
    if (cfg->stream) {
        s->stream = (cudaStream_t)cfg->stream;
    } else if (cudaStreamCreateWithFlags(&s->stream, cudaStreamNonBlocking) != cudaSuccess) {
        delete s;
        return SIC_ECUDA;
    } else {
        s->own_stream = true;
    }
    if (cudaEventCreate(&s->ev[0]) != cudaSuccess || cudaEventCreate(&s->ev[1]) != cudaSuccess ||
        cudaStreamCreateWithFlags(&s->side, cudaStreamNonBlocking) != cudaSuccess) {
        for (cudaEvent_t e : s->ev)
            if (e)
                cudaEventDestroy(e);
        if (s->own_stream)
            cudaStreamDestroy(s->stream);
        delete s;
        return SIC_ECUDA;
    }
    s->t0 = Clock::now();
    *out = s;
    return SIC_OK;
}

int sic_server_submit(sic_server *srv, const sic_config *cfg, const double *x_host, const double *v_host,
                      const double *w_host, int32_t n_steps, int32_t keep, int64_t *id)
{
    if (!srv || !cfg || !x_host || !v_host || !w_host || n_steps < 0 || !cfg->tracers_per_sheet ||
        !cfg->sheet_closed || cfg->n_sheets < 1)
        return SIC_EINVAL;
    Request r;
    r.horizontal = false;
    r.n_steps = n_steps;
    r.keep = keep;
    r.cfg = *cfg;
    const int M = cfg->n_sheets;
    r.counts.assign(cfg->tracers_per_sheet, cfg->tracers_per_sheet + M);
    r.closed.assign(cfg->sheet_closed, cfg->sheet_closed + M);
    r.winding.assign(M, 0);
    if (cfg->sheet_winding)
        r.winding.assign(cfg->sheet_winding, cfg->sheet_winding + M);
    int64_t n = 0, segs = 0;
    for (int k = 0; k < M; ++k) {
        if (r.counts[k] < 2)
            return SIC_EINVAL;
        n += r.counts[k];
        segs += r.counts[k] - (r.closed[k] ? 0 : 1);
    }
    r.a.assign(x_host, x_host + n);
    r.b.assign(v_host, v_host + n);
    r.c.assign(w_host, w_host + n);
    bool per_q = false;
    {
        int64_t base = 0;
        for (int k = 0; k < M && !per_q; ++k) {
            for (int i = 1; i < r.counts[k]; ++i)
                if (w_host[base + i] != w_host[base]) {
                    per_q = true;
                    break;
                }
            base += r.counts[k];
        }
    }
    r.segments = segs;
    r.bytes = request_bytes(*cfg, r.counts.data(), M, per_q);
    return queue_request(srv, std::move(r), id);
}

int sic_server_submit_horizontal(sic_server *srv, const sic_config *cfg, int32_t n_template,
                                 const double *x_template_host, const double *v_sheet_host,
                                 const double *w_sheet_host, int32_t n_steps, int32_t keep, int64_t *id)
{
    if (!srv || !cfg || n_template < 2 || !x_template_host || !v_sheet_host || !w_sheet_host || n_steps < 0 ||
        cfg->n_sheets < 1)
        return SIC_EINVAL;
    Request r;
    r.horizontal = true;
    r.n_steps = n_steps;
    r.keep = keep;
    r.cfg = *cfg;
    const int M = cfg->n_sheets;
    r.n_template = n_template;
    r.a.assign(x_template_host, x_template_host + n_template);
    r.b.assign(v_sheet_host, v_sheet_host + M);
    r.c.assign(w_sheet_host, w_sheet_host + M);
    r.counts.assign(M, n_template);
    r.segments = (int64_t)n_template * M;
    r.bytes = request_bytes(*cfg, r.counts.data(), M, false);
    return queue_request(srv, std::move(r), id);
}

int sic_server_tick(sic_server *srv, int32_t *pending)
{
    if (!srv)
        return SIC_EINVAL;
    srv->ticks += 1;
    if (!srv->cfg.plain) {
        tick_batched(srv);
        if (pending)
            *pending = (int32_t)(srv->queue.size() + srv->active.size() + srv->fresh.size());
        return SIC_OK;
    }
    // plain: one request at a time, to completion, refining whenever it holds
    // for that (Sec. 2.6)
    admit(srv, srv->stream, srv->active);
    if (!srv->active.empty()) {
        int rc = SIC_OK;
        const bool timed = cudaEventRecord(srv->ev[0], srv->stream) == cudaSuccess;
        Active &a = srv->active.front();
        while (rc == SIC_OK && a.left > 0) {
            rc = sic_step(a.sim, std::min(a.left, srv->cfg.chunk_steps));
            if (rc == SIC_OK)
                rc = read_all(srv);
            if (rc == SIC_OK)
                rc = look(srv, a, srv->scal[0]);
        }
        const bool timed2 = timed && cudaEventRecord(srv->ev[1], srv->stream) == cudaSuccess;
        if (cudaStreamSynchronize(srv->stream) != cudaSuccess && rc == SIC_OK)
            rc = SIC_ECUDA;
        float ms = 0.f;
        if (timed2 && cudaEventElapsedTime(&ms, srv->ev[0], srv->ev[1]) == cudaSuccess)
            srv->busy_s += 1e-3 * ms;
        finish(srv, a, rc, srv->now());
        srv->active.clear();
    }
    if (pending)
        *pending = (int32_t)(srv->queue.size() + srv->active.size());
    return SIC_OK;
}

int sic_server_results(sic_server *srv, sic_result *out, int32_t max, int32_t *n)
{
    if (!srv || !n || max < 0 || (max > 0 && !out))
        return SIC_EINVAL;
    const int32_t k = std::min<int32_t>(max, (int32_t)srv->done.size());
    for (int32_t i = 0; i < k; ++i)
        out[i] = srv->done[i];
    srv->done.erase(srv->done.begin(), srv->done.begin() + k);
    *n = k;
    return SIC_OK;
}

double sic_server_clock(sic_server *srv) { return srv ? srv->now() : 0.0; }

int sic_server_stats(sic_server *srv, sic_server_info *out)
{
    if (!srv || !out)
        return SIC_EINVAL;
    out->bytes_in_use = (int64_t)srv->used;
    out->bytes_peak = (int64_t)srv->peak;
    out->hbm_budget = srv->cfg.hbm_budget;
    out->active = (int32_t)(srv->active.size() + srv->fresh.size());
    out->queued = (int32_t)srv->queue.size();
    out->completed = srv->completed;
    out->segment_updates = srv->segment_updates;
    out->ticks = srv->ticks;
    out->busy_s = srv->busy_s;
    out->waits_slots = srv->waits_slots;
    out->waits_memory = srv->waits_memory;
    out->refinements = srv->refinements;
    return SIC_OK;
}

void sic_server_destroy(sic_server *srv)
{
    if (!srv)
        return;
    cudaStreamSynchronize(srv->stream);
    cudaStreamSynchronize(srv->side);
    drop_plans(srv);
    for (Active &a : srv->active)
        if (a.sim)
            sic_destroy(a.sim);
    for (Active &a : srv->fresh)
        if (a.sim)
            sic_destroy(a.sim);
    for (sic_result &r : srv->done)
        if (r.sim)
            sic_destroy(r.sim);
    cudaStreamSynchronize(srv->stream);
    for (cudaEvent_t e : srv->ev)
        if (e)
            cudaEventDestroy(e);
    if (srv->scal)
        cudaFreeHost(srv->scal);
    cudaStreamSynchronize(srv->side);
    cudaStreamDestroy(srv->side);
    if (srv->own_stream)
        cudaStreamDestroy(srv->stream);
    delete srv;
}

}  // extern "C"
