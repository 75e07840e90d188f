// sic_host.h -- host-side structures shared by the C ABI (sic_api.cu) and the
// request server (sic_server.cu).
#pragma once
#include <cuda_runtime.h>

#include <cstddef>
#include <cstdint>
#include <vector>

#include "sic.h"
#include "sic_internal.h"

namespace sic_host {

// Device-side launch plan: table of simulations, items, block ranges, tickets.
struct Plan {
    void *mem = nullptr;
    LaunchArgs args{};
    int grid = 0;
    bool per_q = false;
};

// Device bytes of one simulation's allocation (state, meshes, items, ...).
struct SimLayout {
    size_t oU0, oU1, oV0, oV1, oQ, oMesh, oLast, oEk, oE64, oRho, oAcc, oItems, oPL, oHist, oMHist, oSpec, oSc, total;
};
SimLayout sim_layout(int nx, int64_t n_alloc, int64_t n_items, bool per_q, int hist_len, int deposit, int mode_k);

// Tracer slots (sheets padded to SIC_ALIGN_TRACERS) and work items of M
// sheets of n tracers each.
int64_t padded_tracers(const int32_t *counts, int M);
int64_t work_items(const int32_t *counts, int M);

}  // namespace sic_host

struct sic_sim {
    double refine_length = 0.0;       // Sec. 2.6 refinement length, 0 = never
    double refine_split = 0.0;        // length particles are split to at a hold
    int64_t max_tracers = 0;          // refinement limit (SIC_TRACERS_MAX when not given)
    int nx = 0;
    double L = 0, dt = 0, dx = 0, qm = 1;
    int strict = 0, hist_len = 1, half_step_init = 0;
    int mode_k = 0;                   // Fourier mode of the per-step mode-energy history, 0 = none
    bool per_q = false;
    int M = 0;
    std::vector<int32_t> counts;
    std::vector<uint8_t> closed;
    std::vector<int32_t> winding;
    std::vector<int64_t> sheet_off;
    std::vector<int32_t> sheet_qh;
    int64_t n_tracers = 0, n_alloc = 0;
    double sigma = 1.0;
    double v_max = 0.0;               // largest |v| at creation, position units per step
    double w_max = 0.0;               // largest weight at creation
    std::vector<WorkItem> items;
    int deposit = SIC_DEPOSIT_BOX;    // SIC_DEPOSIT_*
    bool seg_q = false;               // refined: Qh holds per-particle charges
    std::vector<WorkItemPL> pl_items;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    void *dmem = nullptr;
    size_t dbytes = 0;
    SimDev h{};
    sic_host::Plan plan;
    cudaGraphExec_t gexec = nullptr;
    cudaError_t last = cudaSuccess;
};


namespace sic_host {
// The simulation's device scalars (after synchronising its stream) and the
// SIC_E* code of any device error they hold.
int read_scalars(sic_sim *sim, SimScalars *out);
// The SIC_E* code of the device error bits in a simulation's scalars.
int scalars_status(const SimScalars &sc);
// Refine until no particle is longer than the simulation's refinement length
// (sic_refine passes) and clear its refinement hold; *added gets the tracers
// added.
int refine_held(sic_sim *sim, int64_t *added);
// Particles (segments) of the simulation now.
int64_t segments(const sic_sim *sim);
cudaError_t build_plan(Plan &p, sic_sim *const *sims, int n, cudaStream_t s);
// Scheduling knobs of a built plan (results do not depend on them): the claim
// divisor D (a claim takes 1 / (D warps) of what is left) and the staging
// choice (LaunchArgs::staging).
void set_schedule(Plan &p, int claim_div, int staging, int claim_min);
void free_plan(Plan &p, cudaStream_t s);
cudaError_t launch(const Plan &p, sic::Mode mode, float kick_scale, int drift, int record, cudaStream_t s);
}  // namespace sic_host
