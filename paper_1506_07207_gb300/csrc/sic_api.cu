// sic_api.cu -- host runtime behind the C ABI of include/sic.h.
//
// Owns each simulation's device memory (one stream-ordered allocation), its
// work items (up to 32 R consecutive tracers of one sheet, one warp's task at
// a time), the launch plans (the simulations of a launch, their claim cursors
// and tickets, a persistent grid of SMs x resident blocks), CUDA-graph
// capture of the step kernel, and batching of several simulations into
// shared launches.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstdlib>
#include <cstring>
#include <new>
#include <vector>

#include "sic.h"
#include "sic_host.h"
#include "sic_internal.h"

using namespace sic;
using namespace sic_host;

namespace {

constexpr int kGraphSteps = 8;  // steps captured in one graph
constexpr double kTwo32 = 4294967296.0;

struct Layout {
    size_t off = 0;
    size_t take(size_t bytes)
    {
        const size_t at = off;
        off = (off + bytes + 255) / 256 * 256;
        return at;
    }
};

int num_sms()
{
    int dev = 0, n = 0;
    if (cudaGetDevice(&dev) != cudaSuccess)
        return 1;
    if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n <= 0)
        return 1;
    return n;
}

constexpr double kPosUnits = 1073741824.0;  // 2^SIC_POS_FRAC_BITS position units per box length

// A position x as P = x / L 2^30 modulo 2^32 (the box length L): the box
// fraction t = x / L is folded into [0, 4) first, so P keeps full precision.
uint32_t to_pos(double x, double L)
{
    double t = x / L;
    t -= 4.0 * std::floor(t * 0.25);
    return (uint32_t)((uint64_t)std::llround(t * kPosUnits) & 0xffffffffull);
}

// Largest |x| / L accepted at creation (the fold into [0, 4) box lengths keeps
// the position to well within a unit below this).
constexpr double kMaxBoxes = 1048576.0;

bool is_finite(double x) { return std::isfinite(x); }

// Test knob: SIC_GRID overrides the block count of the step kernel.  It does
// not change any result: the mesh is an integer sum and every reduction runs
// in a fixed order independent of the blocks.
int env_int(const char *name, int dflt)
{
    const char *v = std::getenv(name);
    if (!v || !*v)
        return dflt;
    const int x = std::atoi(v);
    return x > 0 ? x : dflt;
}

}  // namespace

namespace {

int fail_cuda(sic_sim *s, cudaError_t e)
{
    if (s)
        s->last = e;
    return e == cudaErrorMemoryAllocation ? SIC_ENOMEM : SIC_ECUDA;
}

#define CK(call)                                  \
    do {                                          \
        cudaError_t e_ = (call);                  \
        if (e_ != cudaSuccess)                    \
            return fail_cuda(sim, e_);            \
    } while (0)

int validate(const sic_config *c, bool need_sheets)
{
    if (!c)
        return SIC_EINVAL;
    if (c->nx < 2 || c->nx > SIC_NX_MAX)
        return SIC_EINVAL;
    if (!is_finite(c->box_length) || c->box_length <= 0)
        return SIC_EINVAL;
    if (!is_finite(c->dt) || c->dt <= 0)
        return SIC_EINVAL;
    if (c->n_sheets < 1)
        return SIC_EINVAL;
    if (!is_finite(c->charge_to_mass) || c->charge_to_mass == 0)
        return SIC_EINVAL;
    if (c->history_len < 1)
        return SIC_EINVAL;
    if (c->deposit < SIC_DEPOSIT_BOX || c->deposit > SIC_DEPOSIT_FIRST)
        return SIC_EINVAL;
    // the refinement length: off, or at least 2^-10 of a cell (the hold test
    // measures particles in 2^-16 cells) with a deposit that has particles
    if (!is_finite(c->refine_length) || c->refine_length < 0)
        return SIC_EINVAL;
    if (c->refine_length > 0 && (c->refine_length < c->box_length / c->nx / 1024.0 ||
                                 c->deposit == SIC_DEPOSIT_PIC_NGP || c->deposit == SIC_DEPOSIT_PIC_CIC))
        return SIC_EINVAL;
    if (!is_finite(c->refine_split) || c->refine_split < 0 || c->refine_split > c->refine_length)
        return SIC_EINVAL;
    if (c->max_tracers < 0 || c->max_tracers > SIC_TRACERS_MAX)
        return SIC_EINVAL;
    if (!is_finite(c->charge_unit) || c->charge_unit < 0)
        return SIC_EINVAL;
    if (c->mode_k < 0 || c->mode_k > c->nx / 2)
        return SIC_EINVAL;
    if (need_sheets) {
        if (!c->tracers_per_sheet || !c->sheet_closed)
            return SIC_EINVAL;
        int64_t total = 0;
        for (int s = 0; s < c->n_sheets; ++s) {
            if (c->tracers_per_sheet[s] < 2)
                return SIC_EINVAL;
            total += c->tracers_per_sheet[s];
        }
        if (total > SIC_TRACERS_MAX)
            return SIC_EINVAL;
    }
    return SIC_OK;
}

// Split every sheet into items of at most 32 R tracers (one warp's task);
// each item knows the tracer after its last one (its halo).
void plan_items(sic_sim *sim)
{
    const int item = SIC_K1_WARP_TRACERS;
    sim->items.clear();
    sim->pl_items.clear();
    for (int s = 0; s < sim->M; ++s) {
        const int n = sim->counts[s];
        for (int k = 0; k * item < n; ++k) {
            WorkItem w{};
            w.t0 = sim->sheet_off[s] + (int64_t)k * item;
            w.count = std::min(item, n - k * item);
            w.qh = sim->per_q ? 0 : sim->sheet_qh[s];
            const float qq = sim->per_q ? 1.0f : (float)w.qh;  // rounded as the kernel did
            w.ke_mult = std::ldexp(qq, sim->h.ke_u);
            w.p_mult = std::ldexp(qq, sim->h.p_u);
            const bool last = (k + 1) * item >= n;
            if (!last) {
                w.halo = w.t0 + w.count;
                w.halo_shift = 0u;
            } else if (sim->closed[s]) {
                w.halo = sim->sheet_off[s];
                w.halo_shift = (uint32_t)sim->winding[s] << SIC_POS_FRAC_BITS;
            } else {
                w.halo = -1;
                w.halo_shift = 0u;
            }
            sim->items.push_back(w);
            if (sim->deposit == SIC_DEPOSIT_LINEAR) {
                // the tracer before the first one and the one after the halo;
                // on a closed sheet the other end is one winding away (the
                // kernel subtracts prev_shift and adds next2_shift)
                const uint32_t wind = (uint32_t)sim->winding[s] << SIC_POS_FRAC_BITS;
                const int64_t off = sim->sheet_off[s];
                WorkItemPL p{-1, -1, 0u, 0u};
                if (k > 0)
                    p.prev = w.t0 - 1;
                else if (sim->closed[s]) {
                    p.prev = off + n - 1;
                    p.prev_shift = wind;
                }
                const int64_t after = (int64_t)k * item + w.count + 1;  // sheet index after the halo
                if (!last) {
                    if (after < n)
                        p.next2 = off + after;
                    else if (sim->closed[s]) {
                        p.next2 = off;
                        p.next2_shift = wind;
                    }
                } else if (sim->closed[s]) {
                    p.next2 = off + 1;
                    p.next2_shift = wind;
                }
                sim->pl_items.push_back(p);
            }
        }
    }
}

}  // namespace
namespace sic_host {
int scalars_status(const SimScalars &sc);
}
namespace {

int check_device_errors(sic_sim *sim, SimScalars *out = nullptr)
{
    SimScalars sc;
    CK(cudaMemcpyAsync(&sc, sim->h.sc, sizeof(sc), cudaMemcpyDeviceToHost, sim->stream));
    CK(cudaStreamSynchronize(sim->stream));
    if (out)
        *out = sc;
    return sic_host::scalars_status(sc);
}

// Clear the refinement hold of a synchronised simulation (the epilogue sets it
// again at the next step that leaves a particle longer than the length).
int clear_refine_hold(sic_sim *sim)
{
    SimScalars sc;
    CK(cudaMemcpyAsync(&sc, sim->h.sc, sizeof(sc), cudaMemcpyDeviceToHost, sim->stream));
    CK(cudaStreamSynchronize(sim->stream));
    if (sc.hold & SIC_HOLD_REFINE) {
        const uint32_t hold = sc.hold & ~SIC_HOLD_REFINE;
        CK(cudaMemcpyAsync(&sim->h.sc->hold, &hold, sizeof(hold), cudaMemcpyHostToDevice, sim->stream));
        CK(cudaStreamSynchronize(sim->stream));
    }
    return SIC_OK;
}

// Fixed-point charge scale: every segment charge at most 2^28 units (so the
// sum of a lane's 8 segments fits 32 bits), a power of two.
double choose_sigma(double max_w)
{
    double sigma = std::ldexp(1.0, (int)std::floor(std::log2(std::ldexp(1.0, 28) / max_w)));
    while (std::llround(max_w * sigma * 0.5) * 2 > (1LL << 28))
        sigma *= 0.5;
    return sigma;
}

// Point the descriptor at a device allocation laid out by L and upload the
// work items (and piecewise-linear neighbours) into it.
cudaError_t bind_layout(sic_sim *sim, char *b, const SimLayout &L)
{
    SimDev &h = sim->h;
    const int n_items = (int)sim->items.size();
    h.U[0] = (uint32_t *)(b + L.oU0);
    h.U[1] = (uint32_t *)(b + L.oU1);
    h.V[0] = (float *)(b + L.oV0);
    h.V[1] = (float *)(b + L.oV1);
    h.Qh = sim->per_q ? (const int32_t *)(b + L.oQ) : nullptr;
    h.mesh = (unsigned long long *)(b + L.oMesh);
    h.mesh_last = (long long *)(b + L.oLast);
    h.Ek = (float2 *)(b + L.oEk);
    h.E64 = (double *)(b + L.oE64);
    h.rho64 = (double *)(b + L.oRho);
    h.acc = (SimAccum *)(b + L.oAcc);
    h.items = (const WorkItem *)(b + L.oItems);
    cudaError_t e = cudaMemcpyAsync((void *)h.items, sim->items.data(), sizeof(WorkItem) * (size_t)n_items,
                                    cudaMemcpyHostToDevice, sim->stream);
    h.pl = nullptr;
    h.deposit = sim->deposit;
    h.seg_q = sim->seg_q ? 1 : 0;
    if (e == cudaSuccess && sim->deposit == SIC_DEPOSIT_LINEAR) {
        h.pl = (const WorkItemPL *)(b + L.oPL);
        e = cudaMemcpyAsync((void *)h.pl, sim->pl_items.data(), sizeof(WorkItemPL) * (size_t)n_items,
                            cudaMemcpyHostToDevice, sim->stream);
    }
    h.hist = (double *)(b + L.oHist);
    h.mhist = sim->mode_k > 0 ? (double *)(b + L.oMHist) : nullptr;
    h.spec = (double *)(b + L.oSpec);
    h.mode_k = sim->mode_k;
    h.sc = (SimScalars *)(b + L.oSc);
    h.n_items = n_items;
    return e;
}

// Common part of both constructors: sizes, device layout, descriptor, plan.
// Expects counts, closed, winding, per_q, sigma and sheet_qh to be set.
int setup(sic_sim *sim, const sic_config *cfg)
{
    sim->nx = cfg->nx;
    sim->L = cfg->box_length;
    sim->dt = cfg->dt;
    sim->dx = cfg->box_length / cfg->nx;
    sim->qm = cfg->charge_to_mass;
    sim->strict = cfg->strict_segments ? 1 : 0;
    sim->hist_len = cfg->history_len;
    sim->mode_k = cfg->mode_k;
    sim->half_step_init = cfg->half_step_init ? 1 : 0;
    sim->deposit = cfg->deposit;
    sim->refine_length = cfg->refine_length;
    sim->refine_split = cfg->refine_split > 0 ? cfg->refine_split : cfg->refine_length;
    sim->max_tracers = cfg->max_tracers > 0 ? cfg->max_tracers : SIC_TRACERS_MAX;
    sim->sheet_off.assign(sim->M, 0);
    int64_t off = 0;
    for (int s = 0; s < sim->M; ++s) {
        sim->sheet_off[s] = off;
        off += (sim->counts[s] + SIC_ALIGN_TRACERS - 1) / SIC_ALIGN_TRACERS * SIC_ALIGN_TRACERS;
    }
    sim->n_alloc = std::max<int64_t>(off, SIC_ALIGN_TRACERS);

    if (cfg->stream) {
        sim->stream = (cudaStream_t)cfg->stream;
    } else {
        CK(cudaStreamCreateWithFlags(&sim->stream, cudaStreamNonBlocking));
        sim->own_stream = true;
    }
    // fixed-point units of the lanes' KE and P sums: an item's term (R tracers,
    // old and new velocity, at most the largest half charge, velocities up to
    // 4 times the largest at creation) comes to about 2^44 units, so a lane's
    // 64-bit sum has room for 2^19 items before it spills into the block's
    // 128-bit sum; the unit is never finer than 2^-32
    {
        SimDev &h = sim->h;
        const double qh_max = std::max(1.0, sim->w_max * sim->sigma * 0.5);
        const double vb = 4.0 * sim->v_max;
        auto unit_exp = [](double bound) {
            if (!(bound > 0.0))
                return 32;
            return std::max(-100, std::min(32, (int)std::floor(44.0 - std::log2(bound))));
        };
        h.ke_u = unit_exp(qh_max * 2.0 * SIC_K1_R * vb * vb);
        h.p_u = unit_exp(qh_max * 2.0 * SIC_K1_R * vb);
    }
    plan_items(sim);
    const int n_items = (int)sim->items.size();

    const int nx = sim->nx;
    const SimLayout L = sim_layout(nx, sim->n_alloc, n_items, sim->per_q, sim->hist_len, sim->deposit, sim->mode_k);
    sim->dbytes = L.total;
    CK(cudaMallocAsync(&sim->dmem, L.total, sim->stream));
    char *b = (char *)sim->dmem;
    CK(cudaMemsetAsync(b, 0, L.total, sim->stream));

    SimDev &h = sim->h;
    CK(bind_layout(sim, b, L));
    h.hist_len = sim->hist_len;
    h.nx = nx;
    const double nx2 = (double)nx * (double)nx;
    h.E_scale = 1.0 / (nx2 * sim->sigma);
    // the kick per step in position units: qm E dt^2 / L 2^30
    h.e_scale = sim->qm * sim->dt * sim->dt / sim->L * kPosUnits * h.E_scale;
    h.rho_scale = 1.0 / ((double)nx * sim->sigma * sim->dx);
    // W_E = dx/2 sum E_j^2 = dx/2 E_scale^2 2^120 sum (K_j 2^-60)^2
    h.we_scale = 0.5 * sim->dx * h.E_scale * h.E_scale * std::ldexp(1.0, 120);
    {
        int ex = 0;
        const double mant = std::frexp(h.e_scale, &ex);  // e_scale = mant 2^ex, mant in [0.5, 1)
        h.ek_mant = (float)(mant * 2.0);
        h.ek_exp = ex - 1;
    }
    const double vu = sim->L / (sim->dt * kPosUnits);  // physical velocity of one position unit per step
    h.ke_scale = vu * vu / (2.0 * sim->sigma * sim->qm);
    h.p_scale = vu / (sim->sigma * sim->qm);
    h.strict = sim->strict;
    // hold for refinement once the longest cell-crossing particle (2^-16 cells)
    // exceeds the refinement length
    h.refine_seg = sim->refine_length > 0 ? (long long)std::floor(sim->refine_length / sim->dx * 65536.0) : 0;
    sic_sim *one[1] = {sim};
    CK(build_plan(sim->plan, one, 1, sim->stream));
    return SIC_OK;
}

// Initial deposit + field, then the optional half kick back.
int initialise(sic_sim *sim)
{
    CK(launch(sim->plan, MODE_DEPOSIT, 0.0f, 0, 0, sim->stream));
    if (sim->half_step_init)
        CK(launch(sim->plan, MODE_PUSH, -0.5f, 0, 0, sim->stream));
    return check_device_errors(sim);
}

}  // namespace

namespace sic_host {

int read_scalars(sic_sim *sim, SimScalars *out) { return check_device_errors(sim, out); }

int scalars_status(const SimScalars &sc)
{
    if (sc.err & SIC_ERR_RANGE)
        return SIC_ERANGE;
    if (sc.err & SIC_ERR_SEGLONG)
        return SIC_ESEGMENT_LONG;
    if (sc.err & SIC_ERR_TIMEOUT)
        return SIC_ETIMEOUT;
    return SIC_OK;
}

int64_t segments(const sic_sim *sim)
{
    int64_t n = 0;
    for (int s = 0; s < sim->M; ++s)
        n += sim->counts[s] - (sim->closed[s] ? 0 : 1);
    return n;
}

int refine_held(sic_sim *sim, int64_t *added)
{
    int64_t total = 0;
    int rc = SIC_OK;
    // one pass splits every particle longer than the length once; a particle
    // more than twice as long needs another (a bounded number: each pass
    // halves the longest)
    for (int pass = 0; pass < 64; ++pass) {
        int64_t a = 0;
        rc = sic_refine(sim, sim->refine_split, &a);
        total += a;
        if (rc != SIC_OK || a == 0)
            break;
    }
    if (added)
        *added = total;
    return rc;
}

void free_plan(Plan &p, cudaStream_t s)
{
    if (p.mem)
        cudaFreeAsync(p.mem, s);
    p.mem = nullptr;
}

// Build the device plan of one launch over several simulations (slot order):
// the table of their descriptors, where each one's items start in the
// launch's list, and the zeroed claim cursors, item tickets and block count.
// Every member must share the charge mode.
//
// Scheduling: block b starts on the simulation that holds its proportional
// share of the items; its warps claim runs of consecutive items of that
// simulation from the simulation's cursor (guided self-scheduling: each claim
// a fraction of what is left, at least one item), so no warp waits for
// another while the simulation has items; when none are left unclaimed, the
// block folds its mesh into the simulation's and moves to the simulation with
// the most unclaimed items.
cudaError_t build_plan(Plan &p, sic_sim *const *sims, int n, cudaStream_t s)
{
    std::vector<SimDev> table(n);
    std::vector<int32_t> slot_begin(n + 1, 0);
    int nx_max = 2;
    int64_t n_items = 0;
    for (int slot = 0; slot < n; ++slot) {
        sic_sim *m = sims[slot];
        table[slot] = m->h;
        nx_max = std::max(nx_max, m->nx);
        slot_begin[slot] = (int32_t)n_items;
        n_items += (int64_t)m->items.size();
    }
    slot_begin[n] = (int32_t)n_items;
    const bool per_q = sims[0]->per_q;
    int per_sm = step_blocks_per_sm(nx_max, MODE_STEP, per_q);
    if (per_sm < 1)
        per_sm = 1;
    const int by_items = (int)((n_items + SIC_K1_WARPS - 1) / SIC_K1_WARPS);
    const int grid = std::max(1, std::min(by_items, env_int("SIC_GRID", num_sms() * per_sm)));
    // a claim takes 1 / (D warps) of what is left: a warp's first claim on a
    // simulation that all of them share is 1/D of its fair share, and a small
    // simulation is spread over many warps (D = SIC_CLAIM_DIV, default 4)
    const float claim_q = (float)(1.0 / ((double)env_int("SIC_CLAIM_DIV", 4) * grid * SIC_K1_WARPS));
    Layout lay;
    const size_t oT = lay.take(sizeof(SimDev) * table.size());
    const size_t oS = lay.take(4 * slot_begin.size());
    const size_t oK = lay.take(4 * (size_t)(2 * n + 1));  // cursor[n], tickets[n], done
    cudaError_t e = cudaMallocAsync(&p.mem, lay.off, s);
    if (e != cudaSuccess)
        return e;
    char *b = (char *)p.mem;
    e = cudaMemcpyAsync(b + oT, table.data(), sizeof(SimDev) * table.size(), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(b + oS, slot_begin.data(), 4 * slot_begin.size(), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess)
        e = cudaMemsetAsync(b + oK, 0, 4 * (size_t)(2 * n + 1), s);
    if (e == cudaSuccess)
        e = cudaStreamSynchronize(s);  // host staging vectors go out of scope
    if (e != cudaSuccess)
        return e;
    p.args.sims = (const SimDev *)(b + oT);
    p.args.slot_begin = (const int32_t *)(b + oS);
    p.args.cursor = (unsigned *)(b + oK);
    p.args.tickets = (unsigned *)(b + oK) + n;
    p.args.done = (unsigned *)(b + oK) + 2 * n;
    p.args.n_items = (int32_t)n_items;
    p.args.claim_q = claim_q;
    p.args.claim_min = 1;
    p.args.n_slots = n;
    p.args.nx_max = nx_max;
    p.args.gen = 0;
    for (int slot = 0; slot < n; ++slot)
        p.args.gen |= sims[slot]->deposit != SIC_DEPOSIT_BOX ? 1 : 0;
    p.grid = grid;
    p.per_q = per_q;
    return cudaSuccess;
}

void set_schedule(Plan &p, int claim_div, int staging, int claim_min)
{
    p.args.claim_q = (float)(1.0 / ((double)std::max(1, claim_div) * p.grid * SIC_K1_WARPS));
    p.args.staging = staging;
    p.args.claim_min = std::max(1, claim_min);
}

cudaError_t launch(const Plan &p, Mode mode, float kick_scale, int drift, int record, cudaStream_t s)
{
    LaunchArgs a = p.args;
    a.kick_scale = kick_scale;
    a.drift = drift;
    a.record = record;
    return launch_step_kernel(a, p.grid, mode, p.per_q, s);
}


SimLayout sim_layout(int nx, int64_t n_alloc, int64_t n_items, bool per_q, int hist_len, int deposit, int mode_k)
{
    Layout lay;
    SimLayout L;
    L.oU0 = lay.take(4 * (size_t)n_alloc);
    L.oU1 = lay.take(4 * (size_t)n_alloc);
    L.oV0 = lay.take(4 * (size_t)n_alloc);
    L.oV1 = lay.take(4 * (size_t)n_alloc);
    L.oQ = per_q ? lay.take(4 * (size_t)n_alloc) : 0;
    L.oMesh = lay.take(8 * (size_t)nx);
    L.oLast = lay.take(8 * (size_t)nx);
    L.oEk = lay.take(8 * (size_t)nx);
    L.oE64 = lay.take(8 * (size_t)nx);
    L.oRho = lay.take(8 * (size_t)nx);
    L.oAcc = lay.take(sizeof(SimAccum));
    L.oItems = lay.take(sizeof(WorkItem) * (size_t)n_items);
    L.oPL = deposit == SIC_DEPOSIT_LINEAR ? lay.take(sizeof(WorkItemPL) * (size_t)n_items) : 0;
    L.oHist = lay.take(32 * (size_t)hist_len);
    L.oMHist = mode_k > 0 ? lay.take(8 * (size_t)hist_len) : 0;
    L.oSpec = lay.take(8 * (size_t)(nx / 2 + 1));
    L.oSc = lay.take(sizeof(SimScalars));
    L.total = lay.off;
    return L;
}

int64_t padded_tracers(const int32_t *counts, int M)
{
    int64_t off = 0;
    for (int s = 0; s < M; ++s)
        off += (counts[s] + SIC_ALIGN_TRACERS - 1) / SIC_ALIGN_TRACERS * SIC_ALIGN_TRACERS;
    return std::max<int64_t>(off, SIC_ALIGN_TRACERS);
}

int64_t work_items(const int32_t *counts, int M)
{
    int64_t n = 0;
    for (int s = 0; s < M; ++s)
        n += (counts[s] + SIC_K1_WARP_TRACERS - 1) / SIC_K1_WARP_TRACERS;
    return n;
}

}  // namespace sic_host

extern "C" {

int sic_create(const sic_config *cfg, const double *x_host, const double *v_host, const double *w_host,
               sic_sim **out)
{
    if (!out)
        return SIC_EINVAL;
    *out = nullptr;
    int rc = validate(cfg, true);
    if (rc)
        return rc;
    if (!x_host || !v_host || !w_host)
        return SIC_EINVAL;
    const double L = cfg->box_length;
    int64_t n = 0;
    for (int s = 0; s < cfg->n_sheets; ++s)
        n += cfg->tracers_per_sheet[s];
    double max_w = 0, max_v = 0;
    for (int64_t i = 0; i < n; ++i) {
        if (!is_finite(x_host[i]) || !is_finite(v_host[i]) || !is_finite(w_host[i]) || w_host[i] <= 0)
            return SIC_EINVAL;
        if (std::fabs(x_host[i] / L) >= kMaxBoxes)
            return SIC_ERANGE;
        // a tracer may move less than half a box per step
        if (std::fabs(v_host[i] * cfg->dt / L) >= 0.5)
            return SIC_ERANGE;
        max_w = std::max(max_w, w_host[i]);
        max_v = std::max(max_v, std::fabs(v_host[i] * cfg->dt / L * kPosUnits));
    }
    // every segment shorter than 1.5 box lengths (the position format holds
    // segments up to 2; the step kernels stop a run at 1.5)
    {
        int64_t base = 0;
        for (int s = 0; s < cfg->n_sheets; ++s) {
            const int c = cfg->tracers_per_sheet[s];
            for (int i = 0; i + 1 < c; ++i)
                if (!(std::fabs(x_host[base + i + 1] - x_host[base + i]) < 1.5 * L))
                    return SIC_ERANGE;
            if (cfg->sheet_closed[s]) {
                const double wd = cfg->sheet_winding ? (double)cfg->sheet_winding[s] : 0.0;
                if (!(std::fabs(x_host[base] + wd * L - x_host[base + c - 1]) < 1.5 * L))
                    return SIC_ERANGE;
            }
            base += c;
        }
    }
    sic_sim *sim = new (std::nothrow) sic_sim;
    if (!sim)
        return SIC_ENOMEM;
    sim->v_max = max_v;
    sim->w_max = max_w;
    sim->M = cfg->n_sheets;
    sim->counts.assign(cfg->tracers_per_sheet, cfg->tracers_per_sheet + sim->M);
    sim->closed.assign(cfg->sheet_closed, cfg->sheet_closed + sim->M);
    sim->winding.assign(sim->M, 0);
    for (int s = 0; s < sim->M; ++s) {
        sim->closed[s] = sim->closed[s] ? 1 : 0;
        if (cfg->sheet_winding && sim->closed[s])
            sim->winding[s] = cfg->sheet_winding[s];
    }
    sim->n_tracers = n;
    // weights: one value per sheet when every tracer of every sheet agrees
    sim->per_q = false;
    {
        int64_t base = 0;
        for (int s = 0; s < sim->M && !sim->per_q; ++s) {
            for (int i = 1; i < sim->counts[s]; ++i)
                if (w_host[base + i] != w_host[base]) {
                    sim->per_q = true;
                    break;
                }
            base += sim->counts[s];
        }
    }
    sim->sigma = cfg->charge_unit > 0 ? 1.0 / cfg->charge_unit : choose_sigma(max_w);
    if (std::llround(max_w * sim->sigma * 0.5) * 2 > (1LL << 28)) {
        delete sim;
        return SIC_ERANGE;  // a particle's charge would not fit 2^28 units
    }
    sim->sheet_qh.assign(sim->M, 0);
    {
        int64_t base = 0;
        for (int s = 0; s < sim->M; ++s) {
            sim->sheet_qh[s] = (int32_t)std::llround(w_host[base] * sim->sigma * 0.5);
            base += sim->counts[s];
        }
    }
    rc = setup(sim, cfg);
    if (rc) {
        sic_destroy(sim);
        return rc;
    }
    {
        std::vector<uint32_t> U(sim->n_alloc, 0u);
        std::vector<float> V(sim->n_alloc, 0.f);
        std::vector<int32_t> Q(sim->per_q ? sim->n_alloc : 0, 0);
        const double vscale = cfg->dt / L * kPosUnits;
        int64_t base = 0;
        for (int s = 0; s < sim->M; ++s) {
            const int64_t o = sim->sheet_off[s];
            for (int i = 0; i < sim->counts[s]; ++i) {
                U[o + i] = to_pos(x_host[base + i], L);
                V[o + i] = (float)(v_host[base + i] * vscale);
                if (sim->per_q)
                    Q[o + i] = (int32_t)std::llround(w_host[base + i] * sim->sigma * 0.5);
            }
            base += sim->counts[s];
        }
        cudaError_t e = cudaMemcpyAsync(sim->h.U[0], U.data(), 4 * U.size(), cudaMemcpyHostToDevice, sim->stream);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(sim->h.V[0], V.data(), 4 * V.size(), cudaMemcpyHostToDevice, sim->stream);
        if (e == cudaSuccess && sim->per_q)
            e = cudaMemcpyAsync((void *)sim->h.Qh, Q.data(), 4 * Q.size(), cudaMemcpyHostToDevice, sim->stream);
        if (e == cudaSuccess)
            e = cudaStreamSynchronize(sim->stream);
        if (e != cudaSuccess) {
            sic_destroy(sim);
            return e == cudaErrorMemoryAllocation ? SIC_ENOMEM : SIC_ECUDA;
        }
    }
    rc = initialise(sim);
    if (rc) {
        sic_destroy(sim);
        return rc;
    }
    *out = sim;
    return SIC_OK;
}

int sic_create_horizontal(const sic_config *cfg, int32_t n_template, const double *x_template_host,
                          const double *v_sheet_host, const double *w_sheet_host, sic_sim **out)
{
    if (!out)
        return SIC_EINVAL;
    *out = nullptr;
    int rc = validate(cfg, false);
    if (rc)
        return rc;
    if (n_template < 2 || !x_template_host || !v_sheet_host || !w_sheet_host)
        return SIC_EINVAL;
    if ((int64_t)n_template * cfg->n_sheets > SIC_TRACERS_MAX)
        return SIC_EINVAL;
    const double L = cfg->box_length;
    for (int i = 0; i < n_template; ++i) {
        if (!is_finite(x_template_host[i]))
            return SIC_EINVAL;
        if (std::fabs(x_template_host[i] / L) >= kMaxBoxes)
            return SIC_ERANGE;
        const double next = i + 1 < n_template ? x_template_host[i + 1] : x_template_host[0] + L;
        if (!(std::fabs(next - x_template_host[i]) < 1.5 * L))   // segments below 1.5 box lengths
            return SIC_ERANGE;
    }
    double max_w = 0, max_v = 0;
    for (int s = 0; s < cfg->n_sheets; ++s) {
        if (!is_finite(v_sheet_host[s]) || !is_finite(w_sheet_host[s]) || w_sheet_host[s] <= 0)
            return SIC_EINVAL;
        if (std::fabs(v_sheet_host[s] * cfg->dt / L) >= 0.5)
            return SIC_ERANGE;
        max_w = std::max(max_w, w_sheet_host[s]);
        max_v = std::max(max_v, std::fabs(v_sheet_host[s] * cfg->dt / L * kPosUnits));
    }
    sic_sim *sim = new (std::nothrow) sic_sim;
    if (!sim)
        return SIC_ENOMEM;
    sim->v_max = max_v;
    sim->w_max = max_w;
    sim->M = cfg->n_sheets;
    sim->counts.assign(sim->M, n_template);
    sim->closed.assign(sim->M, 1);
    sim->winding.assign(sim->M, 1);
    sim->n_tracers = (int64_t)n_template * sim->M;
    sim->per_q = false;
    sim->sigma = cfg->charge_unit > 0 ? 1.0 / cfg->charge_unit : choose_sigma(max_w);
    if (std::llround(max_w * sim->sigma * 0.5) * 2 > (1LL << 28)) {
        delete sim;
        return SIC_ERANGE;  // a particle's charge would not fit 2^28 units
    }
    sim->sheet_qh.assign(sim->M, 0);
    for (int s = 0; s < sim->M; ++s)
        sim->sheet_qh[s] = (int32_t)std::llround(w_sheet_host[s] * sim->sigma * 0.5);
    rc = setup(sim, cfg);
    if (rc) {
        sic_destroy(sim);
        return rc;
    }
    std::vector<uint32_t> ut(n_template);
    for (int i = 0; i < n_template; ++i)
        ut[i] = to_pos(x_template_host[i], L);
    std::vector<float> vs(sim->M);
    for (int s = 0; s < sim->M; ++s)
        vs[s] = (float)(v_sheet_host[s] * cfg->dt / L * kPosUnits);
    void *tmp = nullptr;
    // sheet offsets (8-byte) first, then the template and the velocities
    const size_t bytes = 8 * (size_t)sim->M + 4 * (size_t)n_template + 4 * (size_t)sim->M + 64;
    cudaError_t e = cudaMallocAsync(&tmp, bytes, sim->stream);
    if (e == cudaSuccess) {
        char *t = (char *)tmp;
        int64_t *d_off = (int64_t *)t;
        uint32_t *d_ut = (uint32_t *)(t + 8 * (size_t)sim->M);
        float *d_vs = (float *)(t + 8 * (size_t)sim->M + 4 * (size_t)n_template);
        e = cudaMemcpyAsync(d_ut, ut.data(), 4 * ut.size(), cudaMemcpyHostToDevice, sim->stream);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(d_off, sim->sheet_off.data(), 8 * sim->sheet_off.size(), cudaMemcpyHostToDevice,
                                sim->stream);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(d_vs, vs.data(), 4 * vs.size(), cudaMemcpyHostToDevice, sim->stream);
        if (e == cudaSuccess)
            e = launch_expand_horizontal(sim->h.U[0], sim->h.V[0], d_ut, n_template, d_vs, d_off, sim->M,
                                         sim->stream);
        cudaError_t e2 = cudaFreeAsync(tmp, sim->stream);
        if (e == cudaSuccess)
            e = e2;
        if (e == cudaSuccess)
            e = cudaStreamSynchronize(sim->stream);
    }
    if (e != cudaSuccess) {
        sic_destroy(sim);
        return e == cudaErrorMemoryAllocation ? SIC_ENOMEM : SIC_ECUDA;
    }
    rc = initialise(sim);
    if (rc) {
        sic_destroy(sim);
        return rc;
    }
    *out = sim;
    return SIC_OK;
}

int sic_deposit(sic_sim *sim, int64_t *mesh_fixed_host, double *rho_host)
{
    if (!sim)
        return SIC_EINVAL;
    CK(launch(sim->plan, MODE_DEPOSIT, 0.0f, 0, 0, sim->stream));
    CK(launch_field_out(sim->h, sim->stream));
    if (mesh_fixed_host)
        CK(cudaMemcpyAsync(mesh_fixed_host, sim->h.mesh_last, 8 * (size_t)sim->nx, cudaMemcpyDeviceToHost,
                           sim->stream));
    if (rho_host)
        CK(cudaMemcpyAsync(rho_host, sim->h.rho64, 8 * (size_t)sim->nx, cudaMemcpyDeviceToHost, sim->stream));
    return check_device_errors(sim);
}

int sic_moments(sic_sim *sim, int32_t weighting, double *n_host, double *j_host)
{
    if (!sim || (weighting != 0 && weighting != 1))
        return SIC_EINVAL;
    // E64 and rho64 serve as the device buffers: sic_field and sic_deposit
    // rewrite them before reading them
    CK(launch_moments(sim->h, weighting, sim->L, 1.0 / sim->sigma, sim->L / (sim->dt * kPosUnits), sim->h.rho64,
                      sim->h.E64, sim->stream));
    if (n_host)
        CK(cudaMemcpyAsync(n_host, sim->h.rho64, 8 * (size_t)sim->nx, cudaMemcpyDeviceToHost, sim->stream));
    if (j_host)
        CK(cudaMemcpyAsync(j_host, sim->h.E64, 8 * (size_t)sim->nx, cudaMemcpyDeviceToHost, sim->stream));
    return check_device_errors(sim);
}

int sic_refine(sic_sim *sim, double l_ref, int64_t *n_added)
{
    if (!sim || !is_finite(l_ref) || l_ref <= 0)
        return SIC_EINVAL;
    if (sim->deposit == SIC_DEPOSIT_PIC_NGP || sim->deposit == SIC_DEPOSIT_PIC_CIC)
        return SIC_EINVAL;
    if (n_added)
        *n_added = 0;
    int rc = check_device_errors(sim);
    if (rc)
        return rc;
    rc = clear_refine_hold(sim);
    if (rc)
        return rc;
    const double lc = l_ref / sim->L * kPosUnits;  // position units
    if (lc >= 2.0 * kPosUnits)
        return SIC_OK;  // no segment is 2 box lengths long
    const long long lfix = (long long)lc;
    const int n_items = (int)sim->items.size();

    // 1. particles to split, per work item
    void *scratch = nullptr;
    CK(cudaMallocAsync(&scratch, 12 * (size_t)n_items, sim->stream));
    int64_t *d_base = (int64_t *)scratch;  // the 8-byte array first: both stay aligned
    int32_t *d_splits = (int32_t *)((char *)scratch + 8 * (size_t)n_items);
    std::vector<int32_t> splits(n_items);
    cudaError_t e = launch_refine_count(sim->h, lfix, d_splits, sim->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(splits.data(), d_splits, 4 * (size_t)n_items, cudaMemcpyDeviceToHost, sim->stream);
    if (e == cudaSuccess)
        e = cudaStreamSynchronize(sim->stream);
    if (e != cudaSuccess) {
        cudaFreeAsync(scratch, sim->stream);
        return fail_cuda(sim, e);
    }

    // 2. the new layout: sheet sizes, offsets, where each item's tracers go
    std::vector<int32_t> counts = sim->counts;
    int64_t added = 0;
    {
        int k = 0;
        for (int s = 0; s < sim->M; ++s) {
            const int items_s = (sim->counts[s] + SIC_K1_WARP_TRACERS - 1) / SIC_K1_WARP_TRACERS;
            for (int i = 0; i < items_s; ++i, ++k)
                counts[s] += splits[k];
            added += counts[s] - sim->counts[s];
        }
    }
    if (added == 0 || sim->n_tracers + added > sim->max_tracers) {
        cudaFreeAsync(scratch, sim->stream);
        cudaStreamSynchronize(sim->stream);
        return added == 0 ? SIC_OK : SIC_ELIMIT;
    }
    std::vector<int64_t> off(sim->M);
    int64_t n_alloc = 0;
    for (int s = 0; s < sim->M; ++s) {
        off[s] = n_alloc;
        n_alloc += (counts[s] + SIC_ALIGN_TRACERS - 1) / SIC_ALIGN_TRACERS * SIC_ALIGN_TRACERS;
    }
    n_alloc = std::max<int64_t>(n_alloc, SIC_ALIGN_TRACERS);
    std::vector<int64_t> base(n_items);
    {
        int k = 0;
        for (int s = 0; s < sim->M; ++s) {
            const int items_s = (sim->counts[s] + SIC_K1_WARP_TRACERS - 1) / SIC_K1_WARP_TRACERS;
            int64_t at = off[s];
            for (int i = 0; i < items_s; ++i, ++k) {
                base[k] = at;
                at += sim->items[k].count + splits[k];
            }
        }
    }
    const int64_t new_items = work_items(counts.data(), sim->M);
    const SimLayout L = sim_layout(sim->nx, n_alloc, new_items, true, sim->hist_len, sim->deposit, sim->mode_k);
    void *mem = nullptr;
    e = cudaMemcpyAsync(d_base, base.data(), 8 * (size_t)n_items, cudaMemcpyHostToDevice, sim->stream);
    if (e == cudaSuccess)
        e = cudaMallocAsync(&mem, L.total, sim->stream);
    if (e == cudaSuccess)
        e = cudaMemsetAsync(mem, 0, L.total, sim->stream);
    if (e != cudaSuccess) {
        cudaFreeAsync(scratch, sim->stream);
        if (mem)
            cudaFreeAsync(mem, sim->stream);
        return fail_cuda(sim, e);
    }

    // 3. the tracers, with the new ones, and per-particle charges; the mesh,
    //    field, sums, history and scalars carry over unchanged (a box
    //    particle split at its centre into halves deposits the same charge)
    char *b = (char *)mem;
    SimScalars sc;
    CK(cudaMemcpyAsync(&sc, sim->h.sc, sizeof(sc), cudaMemcpyDeviceToHost, sim->stream));
    CK(cudaStreamSynchronize(sim->stream));
    const int cur = (int)(sc.buf & 1);
    const size_t oU = cur ? L.oU1 : L.oU0, oV = cur ? L.oV1 : L.oV0;
    e = launch_refine_scatter(sim->h, lfix, d_base, (uint32_t *)(b + oU), (float *)(b + oV), (int32_t *)(b + L.oQ),
                              sim->stream);
    const size_t nx8 = 8 * (size_t)sim->nx;
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(b + L.oMesh, sim->h.mesh, nx8, cudaMemcpyDeviceToDevice, sim->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(b + L.oLast, sim->h.mesh_last, nx8, cudaMemcpyDeviceToDevice, sim->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(b + L.oEk, sim->h.Ek, nx8, cudaMemcpyDeviceToDevice, sim->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(b + L.oE64, sim->h.E64, nx8, cudaMemcpyDeviceToDevice, sim->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(b + L.oRho, sim->h.rho64, nx8, cudaMemcpyDeviceToDevice, sim->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(b + L.oAcc, sim->h.acc, sizeof(SimAccum), cudaMemcpyDeviceToDevice, sim->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(b + L.oHist, sim->h.hist, 32 * (size_t)sim->hist_len, cudaMemcpyDeviceToDevice,
                            sim->stream);
    if (e == cudaSuccess && sim->mode_k > 0)
        e = cudaMemcpyAsync(b + L.oMHist, sim->h.mhist, 8 * (size_t)sim->hist_len, cudaMemcpyDeviceToDevice,
                            sim->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(b + L.oSc, sim->h.sc, sizeof(SimScalars), cudaMemcpyDeviceToDevice, sim->stream);
    if (e == cudaSuccess)
        e = cudaStreamSynchronize(sim->stream);
    cudaFreeAsync(scratch, sim->stream);
    if (e != cudaSuccess) {
        cudaFreeAsync(mem, sim->stream);
        return fail_cuda(sim, e);
    }

    // 4. switch the simulation over: sheets, items, descriptor, plan
    cudaFreeAsync(sim->dmem, sim->stream);
    if (sim->gexec) {
        cudaGraphExecDestroy(sim->gexec);
        sim->gexec = nullptr;
    }
    free_plan(sim->plan, sim->stream);
    const bool was_seg = sim->seg_q;
    sim->counts = counts;
    sim->sheet_off = off;
    sim->n_tracers += added;
    sim->n_alloc = n_alloc;
    sim->per_q = true;
    sim->seg_q = true;
    sim->dmem = mem;
    sim->dbytes = L.total;
    plan_items(sim);
    CK(bind_layout(sim, b, L));
    if (!was_seg) {  // a tracer's mass is now its particle's charge, Q_s, not 2 Qh
        sim->h.ke_scale *= 0.5;
        sim->h.p_scale *= 0.5;
    }
    sic_sim *one[1] = {sim};
    CK(build_plan(sim->plan, one, 1, sim->stream));
    if (n_added)
        *n_added = added;
    return check_device_errors(sim);
}

int sic_sheet_counts(sic_sim *sim, int32_t *counts_host)
{
    if (!sim || !counts_host)
        return SIC_EINVAL;
    std::copy(sim->counts.begin(), sim->counts.end(), counts_host);
    return SIC_OK;
}

int sic_field(sic_sim *sim, double *E_host)
{
    if (!sim || !E_host)
        return SIC_EINVAL;
    CK(launch_field_out(sim->h, sim->stream));
    CK(cudaMemcpyAsync(E_host, sim->h.E64, 8 * (size_t)sim->nx, cudaMemcpyDeviceToHost, sim->stream));
    return check_device_errors(sim);
}

int sic_push(sic_sim *sim)
{
    if (!sim)
        return SIC_EINVAL;
    CK(launch(sim->plan, MODE_PUSH, 1.0f, 1, 0, sim->stream));
    return SIC_OK;
}

int sic_step(sic_sim *sim, int32_t n_steps)
{
    if (!sim || n_steps < 0)
        return SIC_EINVAL;
    if (n_steps >= kGraphSteps && !sim->gexec) {
        cudaGraph_t g = nullptr;
        CK(cudaStreamBeginCapture(sim->stream, cudaStreamCaptureModeThreadLocal));
        cudaError_t e = cudaSuccess;
        for (int i = 0; i < kGraphSteps && e == cudaSuccess; ++i)
            e = launch(sim->plan, MODE_STEP, 1.0f, 1, 1, sim->stream);
        cudaError_t e2 = cudaStreamEndCapture(sim->stream, &g);
        if (e != cudaSuccess)
            return fail_cuda(sim, e);
        CK(e2);
        e = cudaGraphInstantiate(&sim->gexec, g, 0);
        cudaGraphDestroy(g);
        CK(e);
        count_launches(-kGraphSteps);  // captured, not run
    }
    int32_t left = n_steps;
    while (left >= kGraphSteps && sim->gexec) {
        CK(cudaGraphLaunch(sim->gexec, sim->stream));
        count_launches(kGraphSteps);
        left -= kGraphSteps;
    }
    for (; left > 0; --left)
        CK(launch(sim->plan, MODE_STEP, 1.0f, 1, 1, sim->stream));
    return SIC_OK;
}

int sic_run(sic_sim *sim, int32_t n_steps, int64_t *n_added)
{
    if (!sim || n_steps < 0)
        return SIC_EINVAL;
    if (n_added)
        *n_added = 0;
    SimScalars sc;
    int rc = check_device_errors(sim, &sc);
    if (rc)
        return rc;
    const int64_t target = sc.step + n_steps;
    constexpr int64_t kChunk = 32;  // steps between two looks at the hold flag
    while (true) {
        // refine only before a step that follows: a run that ends holding is
        // refined by the call that continues it
        if (sc.step >= target)
            return SIC_OK;
        if (sc.hold & SIC_HOLD_REFINE) {
            int64_t a = 0;
            rc = refine_held(sim, &a);
            if (n_added)
                *n_added += a;
            if (rc)
                return rc;
        }
        rc = sic_step(sim, (int32_t)std::min<int64_t>(kChunk, target - sc.step));
        if (rc)
            return rc;
        rc = check_device_errors(sim, &sc);
        if (rc)
            return rc;
    }
}

int sic_step_batch(sic_sim *const *sims, int32_t n_sims, const int32_t *n_steps)
{
    if (!sims || n_sims < 1 || !n_steps)
        return SIC_EINVAL;
    for (int i = 0; i < n_sims; ++i) {
        if (!sims[i] || n_steps[i] < 0)
            return SIC_EINVAL;
        for (int k = 0; k < i; ++k)
            if (sims[k] == sims[i])
                return SIC_EINVAL;
    }
    sic_sim *sim = sims[0];
    cudaStream_t bs = sim->stream;
    // order the batch stream after every member's stream
    std::vector<cudaEvent_t> ev;
    for (int i = 1; i < n_sims; ++i) {
        cudaEvent_t e;
        CK(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
        ev.push_back(e);
        CK(cudaEventRecord(e, sims[i]->stream));
        CK(cudaStreamWaitEvent(bs, e, 0));
    }
    std::vector<int32_t> left(n_steps, n_steps + n_sims);
    while (true) {
        // members with steps left, per charge mode (the two modes take
        // different kernel variants)
        int32_t k = INT32_MAX;
        std::vector<sic_sim *> grp[2];
        for (int i = 0; i < n_sims; ++i)
            if (left[i] > 0) {
                k = std::min(k, left[i]);
                grp[sims[i]->per_q ? 1 : 0].push_back(sims[i]);
            }
        if (grp[0].empty() && grp[1].empty())
            break;
        Plan plans[2];
        for (int g = 0; g < 2; ++g)
            if (!grp[g].empty())
                CK(build_plan(plans[g], grp[g].data(), (int)grp[g].size(), bs));
        for (int32_t st = 0; st < k; ++st)
            for (int g = 0; g < 2; ++g)
                if (plans[g].mem)
                    CK(launch(plans[g], MODE_STEP, 1.0f, 1, 1, bs));
        for (int g = 0; g < 2; ++g)
            free_plan(plans[g], bs);
        for (int i = 0; i < n_sims; ++i)
            if (left[i] > 0)
                left[i] -= k;
    }
    cudaEvent_t done;
    CK(cudaEventCreateWithFlags(&done, cudaEventDisableTiming));
    CK(cudaEventRecord(done, bs));
    for (int i = 1; i < n_sims; ++i)
        CK(cudaStreamWaitEvent(sims[i]->stream, done, 0));
    cudaEventDestroy(done);
    for (cudaEvent_t e : ev)
        cudaEventDestroy(e);
    return SIC_OK;
}

}  // extern "C"

struct sic_batch {
    std::vector<sic_sim *> sims;
    cudaStream_t stream = nullptr;
    sic_host::Plan plan[2];
    cudaGraphExec_t gexec = nullptr;
    int64_t segments = 0;
};

namespace {

cudaError_t batch_launch(sic_batch *b)
{
    for (int g = 0; g < 2; ++g)
        if (b->plan[g].mem) {
            const cudaError_t e = sic_host::launch(b->plan[g], MODE_STEP, 1.0f, 1, 1, b->stream);
            if (e != cudaSuccess)
                return e;
        }
    return cudaSuccess;
}

}  // namespace

extern "C" {

int sic_batch_create(sic_sim *const *sims, int32_t n_sims, sic_batch **out)
{
    if (!sims || n_sims < 1 || !out)
        return SIC_EINVAL;
    *out = nullptr;
    for (int i = 0; i < n_sims; ++i) {
        if (!sims[i])
            return SIC_EINVAL;
        for (int k = 0; k < i; ++k)
            if (sims[k] == sims[i])
                return SIC_EINVAL;
    }
    sic_batch *b = new (std::nothrow) sic_batch;
    if (!b)
        return SIC_ENOMEM;
    b->sims.assign(sims, sims + n_sims);
    b->stream = sims[0]->stream;
    sic_sim *sim = sims[0];
    for (int i = 1; i < n_sims; ++i) {
        cudaEvent_t e;
        CK(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
        cudaEventRecord(e, sims[i]->stream);
        cudaStreamWaitEvent(b->stream, e, 0);
        cudaEventDestroy(e);
    }
    std::vector<sic_sim *> grp[2];
    for (sic_sim *m : b->sims) {
        grp[m->per_q ? 1 : 0].push_back(m);
        int64_t segs = 0;
        for (int s = 0; s < m->M; ++s)
            segs += m->counts[s] - (m->closed[s] ? 0 : 1);
        b->segments += segs;
    }
    for (int g = 0; g < 2; ++g)
        if (!grp[g].empty()) {
            const cudaError_t e = sic_host::build_plan(b->plan[g], grp[g].data(), (int)grp[g].size(), b->stream);
            if (e != cudaSuccess) {
                sic_batch_destroy(b);
                return e == cudaErrorMemoryAllocation ? SIC_ENOMEM : SIC_ECUDA;
            }
        }
    *out = b;
    return SIC_OK;
}

int sic_batch_step(sic_batch *b, int32_t n_steps)
{
    if (!b || n_steps < 0)
        return SIC_EINVAL;
    sic_sim *sim = b->sims[0];
    const int launches_per_step = (b->plan[0].mem ? 1 : 0) + (b->plan[1].mem ? 1 : 0);
    if (n_steps >= kGraphSteps && !b->gexec) {
        cudaGraph_t g = nullptr;
        CK(cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal));
        cudaError_t e = cudaSuccess;
        for (int i = 0; i < kGraphSteps && e == cudaSuccess; ++i)
            e = batch_launch(b);
        cudaError_t e2 = cudaStreamEndCapture(b->stream, &g);
        if (e != cudaSuccess)
            return fail_cuda(sim, e);
        CK(e2);
        e = cudaGraphInstantiate(&b->gexec, g, 0);
        cudaGraphDestroy(g);
        CK(e);
        count_launches(-(int64_t)kGraphSteps * launches_per_step);
    }
    int32_t left = n_steps;
    while (left >= kGraphSteps && b->gexec) {
        CK(cudaGraphLaunch(b->gexec, b->stream));
        count_launches((int64_t)kGraphSteps * launches_per_step);
        left -= kGraphSteps;
    }
    for (; left > 0; --left)
        CK(batch_launch(b));
    return SIC_OK;
}

int sic_batch_autotune(sic_batch *b, int32_t steps_each, int32_t *claim_div, int32_t *staging,
                       int32_t *claim_min)
{
    if (!b || steps_each < 1)
        return SIC_EINVAL;
    sic_sim *sim = b->sims[0];
    // (claim divisor, staging, smallest claim): the default first
    const int cand[SIC_AUTOTUNE_CANDIDATES][3] = {{4, 0, 1}, {2, 0, 1}, {8, 0, 1}, {4, 1, 1}, {4, 2, 1},
                                                  {2, 0, 2}, {4, 0, 2}, {2, 0, 4}, {1, 0, 4}, {1, 0, 2}};
    const int n_cand = (int)(sizeof(cand) / sizeof(cand[0]));
    if (b->gexec) {  // captured with the old arguments
        cudaGraphExecDestroy(b->gexec);
        b->gexec = nullptr;
    }
    cudaEvent_t ev[2];
    CK(cudaEventCreate(&ev[0]));
    if (cudaEventCreate(&ev[1]) != cudaSuccess) {
        cudaEventDestroy(ev[0]);
        return SIC_ECUDA;
    }
    int best = 0;
    float best_ms = 0.f;
    cudaError_t e = cudaSuccess;
    for (int c = 0; c < n_cand && e == cudaSuccess; ++c) {
        for (auto &p : b->plan)
            if (p.mem)
                set_schedule(p, cand[c][0], cand[c][1], cand[c][2]);
        e = batch_launch(b);  // settles caches and the function attributes
        if (e == cudaSuccess)
            e = cudaEventRecord(ev[0], b->stream);
        for (int i = 0; i < steps_each && e == cudaSuccess; ++i)
            e = batch_launch(b);
        if (e == cudaSuccess)
            e = cudaEventRecord(ev[1], b->stream);
        if (e == cudaSuccess)
            e = cudaEventSynchronize(ev[1]);
        float ms = 0.f;
        if (e == cudaSuccess)
            e = cudaEventElapsedTime(&ms, ev[0], ev[1]);
        if (e == cudaSuccess && (c == 0 || ms < best_ms)) {
            best = c;
            best_ms = ms;
        }
    }
    cudaEventDestroy(ev[0]);
    cudaEventDestroy(ev[1]);
    if (e != cudaSuccess)
        return fail_cuda(sim, e);
    for (auto &p : b->plan)
        if (p.mem)
            set_schedule(p, cand[best][0], cand[best][1], cand[best][2]);
    if (claim_div)
        *claim_div = cand[best][0];
    if (staging)
        *staging = cand[best][1];
    if (claim_min)
        *claim_min = cand[best][2];
    return SIC_OK;
}

int64_t sic_batch_segments(const sic_batch *b) { return b ? b->segments : 0; }

void sic_batch_destroy(sic_batch *b)
{
    if (!b)
        return;
    if (b->gexec)
        cudaGraphExecDestroy(b->gexec);
    for (auto &p : b->plan)
        sic_host::free_plan(p, b->stream);
    cudaEvent_t done;
    if (cudaEventCreateWithFlags(&done, cudaEventDisableTiming) == cudaSuccess) {
        cudaEventRecord(done, b->stream);
        for (sic_sim *m : b->sims)
            if (m->stream != b->stream)
                cudaStreamWaitEvent(m->stream, done, 0);
        cudaEventDestroy(done);
    }
    delete b;
}

int sic_diagnostics(sic_sim *sim, sic_diag *out)
{
    if (!sim || !out)
        return SIC_EINVAL;
    SimScalars sc;
    int rc = check_device_errors(sim, &sc);
    if (rc)
        return rc;
    out->step = sc.step;
    out->t = (double)sc.step * sim->dt;
    out->field_energy = sc.we;
    out->kinetic_energy = NAN;
    out->momentum = NAN;
    if (sc.step > 0) {
        double row[4];
        const int64_t r = (sc.step - 1) % sim->hist_len;
        CK(cudaMemcpy(row, sim->h.hist + 4 * r, sizeof(row), cudaMemcpyDeviceToHost));
        out->kinetic_energy = row[1];
        out->momentum = row[2];
    }
    out->charge_fixed = sc.q_total;
    out->charge_unit = 1.0 / sim->sigma;
    out->max_segment = (double)sc.maxseg / 65536.0 / (double)sim->nx;
    return SIC_OK;
}

int sic_history(sic_sim *sim, double *hist_host, int32_t max_rows, int32_t *rows)
{
    if (!sim || !hist_host || !rows || max_rows < 1)
        return SIC_EINVAL;
    SimScalars sc;
    int rc = check_device_errors(sim, &sc);
    if (rc)
        return rc;
    const int64_t n = std::min<int64_t>(std::min<int64_t>(sc.step, sim->hist_len), max_rows);
    std::vector<double> ring(4 * (size_t)sim->hist_len);
    CK(cudaMemcpy(ring.data(), sim->h.hist, 8 * ring.size(), cudaMemcpyDeviceToHost));
    for (int64_t i = 0; i < n; ++i) {
        const int64_t step = sc.step - n + i;
        std::memcpy(hist_host + 4 * i, ring.data() + 4 * (step % sim->hist_len), 32);
    }
    *rows = (int32_t)n;
    return SIC_OK;
}

int sic_mode_history(sic_sim *sim, double *out_host, int32_t max_rows, int32_t *rows)
{
    if (!sim || !out_host || !rows || max_rows < 1 || sim->mode_k <= 0)
        return SIC_EINVAL;
    SimScalars sc;
    int rc = check_device_errors(sim, &sc);
    if (rc)
        return rc;
    const int64_t n = std::min<int64_t>(std::min<int64_t>(sc.step, sim->hist_len), max_rows);
    std::vector<double> ring((size_t)sim->hist_len);
    CK(cudaMemcpy(ring.data(), sim->h.mhist, 8 * ring.size(), cudaMemcpyDeviceToHost));
    for (int64_t i = 0; i < n; ++i)
        out_host[i] = ring[(size_t)((sc.step - n + i) % sim->hist_len)];
    *rows = (int32_t)n;
    return SIC_OK;
}

int sic_spectrum(sic_sim *sim, int32_t field, double *out_host)
{
    if (!sim || !out_host || (field != 0 && field != 1))
        return SIC_EINVAL;
    CK(launch_field_out(sim->h, sim->stream));
    CK(launch_spectrum(sim->h, field, sim->stream));
    CK(cudaMemcpyAsync(out_host, sim->h.spec, 8 * (size_t)(sim->nx / 2 + 1), cudaMemcpyDeviceToHost, sim->stream));
    return check_device_errors(sim);
}

int sic_get_state(sic_sim *sim, double *x_host, double *v_host)
{
    if (!sim)
        return SIC_EINVAL;
    SimScalars sc;
    int rc = check_device_errors(sim, &sc);
    if (rc)
        return rc;
    const int b = sc.buf & 1;
    std::vector<uint32_t> U(sim->n_alloc);
    std::vector<float> V(sim->n_alloc);
    CK(cudaMemcpy(U.data(), sim->h.U[b], 4 * U.size(), cudaMemcpyDeviceToHost));
    CK(cudaMemcpy(V.data(), sim->h.V[b], 4 * V.size(), cudaMemcpyDeviceToHost));
    // each sheet unwrapped along its tracers: the first one inside the box,
    // every next one a segment (the 32-bit position difference) further
    const double unit = sim->L / kPosUnits, vs = sim->L / (sim->dt * kPosUnits);
    int64_t base = 0;
    for (int s = 0; s < sim->M; ++s) {
        const int64_t o = sim->sheet_off[s];
        double x = (double)(uint32_t)(U[o] << SIC_POS_WIND_BITS) * (sim->L / kTwo32);
        for (int i = 0; i < sim->counts[s]; ++i) {
            if (i > 0)
                x += (double)(int32_t)(U[o + i] - U[o + i - 1]) * unit;
            if (x_host)
                x_host[base + i] = x;
            if (v_host)
                v_host[base + i] = (double)V[o + i] * vs;
        }
        base += sim->counts[s];
    }
    return SIC_OK;
}

int sic_device_state(sic_sim *sim, uint32_t **pos_dev, float **vel_dev, const int64_t **sheet_offset_host)
{
    if (!sim)
        return SIC_EINVAL;
    SimScalars sc;
    int rc = check_device_errors(sim, &sc);
    if (rc)
        return rc;
    const int b = sc.buf & 1;
    if (pos_dev)
        *pos_dev = sim->h.U[b];
    if (vel_dev)
        *vel_dev = sim->h.V[b];
    if (sheet_offset_host)
        *sheet_offset_host = sim->sheet_off.data();
    return SIC_OK;
}

int sic_sync(sic_sim *sim)
{
    if (!sim)
        return SIC_EINVAL;
    return check_device_errors(sim);
}

void sic_destroy(sic_sim *sim)
{
    if (!sim)
        return;
    if (sim->stream)
        cudaStreamSynchronize(sim->stream);
    if (sim->gexec)
        cudaGraphExecDestroy(sim->gexec);
    if (sim->stream) {
        free_plan(sim->plan, sim->stream);
        if (sim->dmem)
            cudaFreeAsync(sim->dmem, sim->stream);
        cudaStreamSynchronize(sim->stream);
    }
    if (sim->own_stream && sim->stream)
        cudaStreamDestroy(sim->stream);
    delete sim;
}

const char *sic_strerror(int code)
{
    switch (code) {
    case SIC_OK:
        return "ok";
    case SIC_EINVAL:
        return "invalid argument";
    case SIC_ENOMEM:
        return "out of memory";
    case SIC_ECUDA:
        return "CUDA error";
    case SIC_ERANGE:
        return "outside the fixed-point position range (a segment of 1.5 box lengths or a step of half a box)";
    case SIC_ESEGMENT_LONG:
        return "segment longer than the box";
    case SIC_ETIMEOUT:
        return "device wait timed out";
    case SIC_EBUSY:
        return "no capacity";
    case SIC_ELIMIT:
        return "refinement would pass the simulation's tracer limit";
    default:
        return "unknown error";
    }
}

int64_t sic_launch_count(void) { return sic::launches(); }

}  // extern "C"

// ---------------------------------------------------------------------------
// sic_step_batch_static: sic_step_batch with its launch plan in a fixed,
// file-scope device array instead of a per-call allocation.  The paper has no
// counterpart; this serves callers that must not allocate device memory while
// stepping.

#include <mutex>

namespace {

constexpr size_t kStaticScratchBytes = 64 * 1024;
constexpr int kStaticMaxDevices = 64;

// per charge-mode group: descriptor table, item offsets, claim cursors, item
// tickets, finished-block count
constexpr size_t round256(size_t n) { return (n + 255) / 256 * 256; }
constexpr size_t kStaticTable = round256(sizeof(SimDev) * SIC_STATIC_MAX_SIMS);
constexpr size_t kStaticSlots = round256(4 * (SIC_STATIC_MAX_SIMS + 1));
constexpr size_t kStaticCounters = round256(4 * (2 * SIC_STATIC_MAX_SIMS + 1));
constexpr size_t kStaticGroup = kStaticTable + kStaticSlots + kStaticCounters;
static_assert(2 * kStaticGroup <= kStaticScratchBytes, "static plan scratch too small");

static __device__ __align__(256) unsigned char g_step_scratch[kStaticScratchBytes];

std::mutex g_static_mu;
void *g_static_addr[kStaticMaxDevices] = {};

// The scratch's address on device dev, looked up once per device with dev
// current (the caller made it current).
cudaError_t static_scratch(int dev, unsigned char **out)
{
    std::lock_guard<std::mutex> lock(g_static_mu);
    if (dev < 0 || dev >= kStaticMaxDevices)
        return cudaErrorInvalidDevice;
    if (!g_static_addr[dev]) {
        void *p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_step_scratch);
        if (e != cudaSuccess)
            return e;
        g_static_addr[dev] = p;
    }
    *out = static_cast<unsigned char *>(g_static_addr[dev]);
    return cudaSuccess;
}

// Write the plan of one group into its part of the scratch (stream-ordered
// after the previous launches), clear its counters, and return its arguments.
cudaError_t static_plan(unsigned char *region, sic_sim *const *grp, int n, cudaStream_t s, LaunchArgs &a, int &grid)
{
    SimDev table[SIC_STATIC_MAX_SIMS];
    int32_t slot_begin[SIC_STATIC_MAX_SIMS + 1];
    int nx_max = 2;
    int64_t n_items = 0;
    for (int i = 0; i < n; ++i) {
        table[i] = grp[i]->h;
        nx_max = std::max(nx_max, grp[i]->nx);
        slot_begin[i] = (int32_t)n_items;
        n_items += (int64_t)grp[i]->items.size();
    }
    slot_begin[n] = (int32_t)n_items;
    const bool per_q = grp[0]->per_q;
    int per_sm = step_blocks_per_sm(nx_max, MODE_STEP, per_q);
    if (per_sm < 1)
        per_sm = 1;
    const int by_items = (int)((n_items + SIC_K1_WARPS - 1) / SIC_K1_WARPS);
    grid = std::max(1, std::min(by_items, env_int("SIC_GRID", num_sms() * per_sm)));
    unsigned char *t = region, *sb = region + kStaticTable, *ctr = sb + kStaticSlots;
    cudaError_t e = cudaMemcpyAsync(t, table, sizeof(SimDev) * n, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(sb, slot_begin, 4 * (size_t)(n + 1), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess)
        e = cudaMemsetAsync(ctr, 0, 4 * (size_t)(2 * n + 1), s);  // cursors, tickets, done start at zero
    if (e == cudaSuccess)
        e = cudaStreamSynchronize(s);  // the host tables are on this stack frame
    if (e != cudaSuccess)
        return e;
    a = LaunchArgs{};
    a.sims = reinterpret_cast<const SimDev *>(t);
    a.slot_begin = reinterpret_cast<const int32_t *>(sb);
    a.cursor = reinterpret_cast<unsigned *>(ctr);
    a.tickets = reinterpret_cast<unsigned *>(ctr) + n;
    a.done = reinterpret_cast<unsigned *>(ctr) + 2 * n;
    a.n_items = (int32_t)n_items;
    a.claim_q = (float)(1.0 / ((double)env_int("SIC_CLAIM_DIV", 4) * grid * SIC_K1_WARPS));
    a.claim_min = 1;
    a.n_slots = n;
    a.nx_max = nx_max;
    a.drift = 1;
    a.record = 1;
    a.kick_scale = 1.0f;
    a.gen = 0;
    for (int i = 0; i < n; ++i)
        a.gen |= grp[i]->deposit != SIC_DEPOSIT_BOX ? 1 : 0;
    return cudaSuccess;
}

int static_batch(sic_sim *const *sims, int32_t n_sims, const int32_t *n_steps)
{
    cudaStream_t bs = sims[0]->stream;
    // the first member's stream runs the launches: wait for the others' work
    for (int i = 1; i < n_sims; ++i)
        if (cudaStreamSynchronize(sims[i]->stream) != cudaSuccess)
            return SIC_ECUDA;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess)
        return SIC_ECUDA;
    unsigned char *scratch = nullptr;
    if (static_scratch(dev, &scratch) != cudaSuccess)
        return SIC_ECUDA;
    int32_t left[SIC_STATIC_MAX_SIMS];
    for (int i = 0; i < n_sims; ++i)
        left[i] = n_steps[i];
    while (true) {
        int32_t k = INT32_MAX;
        sic_sim *grp[2][SIC_STATIC_MAX_SIMS];
        int ng[2] = {0, 0};
        for (int i = 0; i < n_sims; ++i)
            if (left[i] > 0) {
                k = std::min(k, left[i]);
                const int g = sims[i]->per_q ? 1 : 0;
                grp[g][ng[g]++] = sims[i];
            }
        if (ng[0] == 0 && ng[1] == 0)
            break;
        LaunchArgs a[2];
        int grid[2] = {0, 0};
        for (int g = 0; g < 2; ++g)
            if (ng[g] && static_plan(scratch + g * kStaticGroup, grp[g], ng[g], bs, a[g], grid[g]) != cudaSuccess)
                return SIC_ECUDA;
        for (int32_t st = 0; st < k; ++st)
            for (int g = 0; g < 2; ++g)
                if (ng[g] && launch_step_kernel(a[g], grid[g], MODE_STEP, g == 1, bs) != cudaSuccess)
                    return SIC_ECUDA;
        for (int i = 0; i < n_sims; ++i)
            if (left[i] > 0)
                left[i] -= k;
    }
    // later work on any member's stream comes after these steps
    return cudaStreamSynchronize(bs) == cudaSuccess ? SIC_OK : SIC_ECUDA;
}

}  // namespace

extern "C" int sic_step_batch_static(sic_sim *const *sims, int32_t n_sims, const int32_t *n_steps)
{
    if (!sims || n_sims < 1 || !n_steps)
        return SIC_EINVAL;
    if (n_sims > SIC_STATIC_MAX_SIMS)
        return SIC_EINVAL;  // more simulations than the fixed scratch holds
    int dev = -1;
    for (int i = 0; i < n_sims; ++i) {
        if (!sims[i] || n_steps[i] < 0)
            return SIC_EINVAL;
        for (int k = 0; k < i; ++k)
            if (sims[k] == sims[i])
                return SIC_EINVAL;
        cudaPointerAttributes at{};
        if (cudaPointerGetAttributes(&at, sims[i]->dmem) != cudaSuccess)
            return SIC_ECUDA;
        if (dev < 0)
            dev = at.device;
        else if (at.device != dev)
            return SIC_EINVAL;  // all members on one device
    }
    // run with the members' device current; put the caller's back after
    int prev = 0;
    if (cudaGetDevice(&prev) != cudaSuccess)
        return SIC_ECUDA;
    if (prev != dev && cudaSetDevice(dev) != cudaSuccess)
        return SIC_ECUDA;
    const int rc = static_batch(sims, n_sims, n_steps);
    if (prev != dev)
        cudaSetDevice(prev);
    return rc;
}
