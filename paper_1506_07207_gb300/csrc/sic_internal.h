// sic_internal.h -- device-side layout shared by the kernels and the host runtime.
//
// State of one simulation in HBM (all arrays device-resident for its lifetime):
//   U[n_alloc]   int64  tracer position, unwrapped, 32.32 fixed point in cell
//                       units (x / dx * 2^32); sheets start on 32-tracer
//                       boundaries so every thread's tracers are 16-byte aligned.
//   V[n_alloc]   float  velocity in cells per step (v dt / dx).
//   Qh[n_alloc]  int32  half charge of each tracer in fixed-point units (only
//                       when weights differ inside a sheet; otherwise every
//                       work item carries its sheet's value).
//   mesh[nx]     u64    int64 charge accumulator the deposit adds into.
//   mesh_last    int64  charge of the latest completed deposit.
//   Ek[nx]       float2 (Ek_j, Ek_{j+1} - Ek_j): the kick per step
//                       qm E_j dt^2 / dx at node j, paired for one load.
//   E64[nx]      double the node field E_j in physical units.
//   rho64[nx]    double the neutralised density of the latest deposit.
// Charge unit: a segment between tracers of weights w_i, w_{i+1} carries
// Q_s = Qh_i + Qh_{i+1} = round(w_i sigma / 2) + round(w_{i+1} sigma / 2)
// units, sigma chosen so that every Q_s < 2^29.
#pragma once
#include <stdint.h>

#include "sic.h"

#define SIC_ALIGN_TRACERS 32
#define SIC_K1_BLOCK 256
#define SIC_K1_R 8
#define SIC_K1_TILE (SIC_K1_BLOCK * SIC_K1_R)
#define SIC_K2_BLOCK 1024
#define SIC_FIX_ONE 4294967296.0  // 2^32

// error bits raised on the device
#define SIC_ERR_RANGE 1u
#define SIC_ERR_SEGLONG 2u

// periodic cell reduction by a precomputed multiplier (unsigned division by
// an invariant integer: q = (t + ((n - t) >> 1)) >> (l - 1), t = umulhi(m, n))
struct NxDiv {
    int32_t nx;
    uint32_t magic;
    int32_t shift;     // l - 1
    int32_t offset;    // multiple of nx >= 2^30, added before the division
};

// One work item: consecutive tracers of one sheet.
struct WorkItem {
    int32_t sim;        // slot in the launch's simulation table
    int32_t local;      // index of the item inside its simulation
    int64_t t0;         // first tracer (aligned to SIC_ALIGN_TRACERS)
    int32_t count;      // tracers, 1..SIC_K1_TILE * k
    int32_t qh;         // sheet half charge when the simulation has no Qh array
    int32_t seam_next;  // local item whose first tracer ends this item's last
                        // segment, -1 for the open end of a chain
    int32_t pad;
    int64_t seam_shift; // added to that first tracer (winding * nx * 2^32)
};

// Per-step diagnostics that K1 leaves per item, reduced by K2 in fixed order.
struct ItemDiag {
    double ke;          // sum Qh (v_old^2 + v_new^2)   (cells/step)^2 units
    double p;           // sum Qh (v_old + v_new)
    int64_t maxseg;     // longest segment deposited, 2^-32 cells
    int64_t pad;
};

struct SimScalars {
    int64_t step;
    int64_t q_total;    // total charge of the mesh E was solved from
    double we;          // W_E of the current field
    int64_t maxseg;     // longest segment of the latest deposit
    uint32_t err;       // SIC_ERR_* bits
    uint32_t pad;
};

struct SimDev {
    int64_t *U;
    float *V;
    const int32_t *Qh;          // may be null
    unsigned long long *mesh;
    long long *mesh_last;
    float2 *Ek;
    double *E64;
    double *rho64;              // neutralised density n_j - mean(n) of the latest deposit
    const WorkItem *items;      // this simulation's own items
    int64_t *edge_first;        // [n_items]
    int64_t *edge_last;         // [n_items]
    ItemDiag *item_diag;        // [n_items]
    double *hist;               // [hist_len][4]
    SimScalars *sc;
    int32_t n_items;
    int32_t hist_len;
    NxDiv div;
    double e_scale;             // Ek_j = K_j * e_scale
    double E_scale;             // E_j  = K_j * E_scale
    double rho_scale;           // rho_j = (nx mesh_j - Q) * rho_scale
    double half_dx;             // dx / 2 (field energy)
    double ke_scale;            // KE = ke_scale * sum ke
    double p_scale;             // P  = p_scale * sum p
    int32_t strict;
    int32_t pad;
};

// One simulation of a field launch (K2): table slot.
struct FieldJob {
    int32_t slot;
    int32_t pad;
};

// Host-side launch helpers implemented in sic_kernels.cu.
#include <cuda_runtime.h>
namespace sic {
cudaError_t launch_push_deposit(const SimDev *sims, const WorkItem *items, const int32_t *cta_begin,
                                int grid, int nx_max, bool push, bool deposit, bool per_q,
                                float kick_scale, int drift, cudaStream_t s);
cudaError_t launch_field(const SimDev *sims, const FieldJob *jobs, int n_jobs, int nx_max,
                         int record, cudaStream_t s);
cudaError_t launch_expand_horizontal(int64_t *U, float *V, const int64_t *u_template,
                                     int32_t n_template, const float *v_sheet,
                                     const int64_t *sheet_offset, int32_t n_sheets,
                                     cudaStream_t s);
int k1_blocks_per_sm(int nx_max, bool push, bool deposit, bool per_q);
size_t k1_smem_bytes(int nx_max);
void count_launches(int64_t n);
int64_t launches();
}  // namespace sic
