// sic_internal.h -- device-side layout shared by the kernels and the host runtime.
//
// State of one simulation in HBM (all arrays device-resident for its lifetime):
//   U[2][n_alloc] uint32 tracer position P = x / L * 2^30 modulo 2^32: a 30-bit
//                        fraction of the box and 2 bits of winding, so positions
//                        are kept modulo 4 box lengths and the segment between
//                        two tracers is the 32-bit difference of their P
//                        (exact while it is shorter than 2 box lengths).  Two
//                        buffers: a step reads one and writes the other
//                        (sc->buf names the current one).  Sheets start on
//                        32-tracer boundaries so every thread's tracers are
//                        16-byte aligned.
//   V[2][n_alloc] float  velocity in position units per step (v dt / L * 2^30).
//   Qh[n_alloc]   int32  half charge of each tracer in fixed-point units (only
//                        when weights differ inside a sheet; otherwise every
//                        work item carries its sheet's value); after a
//                        refinement (seg_q) the charge of the particle that
//                        starts at the tracer instead.
//   mesh[nx]      u64    int64 charge accumulator the deposit adds into.
//   mesh_last     int64  charge of the latest completed deposit.
//   Ek[nx]        float2 (Ek_j, Ek_{j+1} - Ek_j): the kick per step
//                        qm E_j dt^2 / L 2^30 at node j and its difference to the
//                        next node (the step kernel copies the pairs into
//                        shared memory).
//   E64[nx]       double the node field E_j in physical units.
//   rho64[nx]     double the neutralised density of the latest deposit.
// Charge unit: a segment between tracers of weights w_i, w_{i+1} carries
// Q_s = Qh_i + Qh_{i+1} = round(w_i sigma / 2) + round(w_{i+1} sigma / 2)
// units, sigma a power of two chosen so that every Q_s <= 2^28.
#pragma once
#include <stdint.h>

#include "sic.h"

// Position format: P = x / L * 2^SIC_POS_FRAC_BITS modulo 2^32.
#define SIC_POS_FRAC_BITS 30
#define SIC_POS_WIND_BITS 2      // 32 - SIC_POS_FRAC_BITS

#define SIC_ALIGN_TRACERS 32
#define SIC_K1_BLOCK 256
#ifndef SIC_K1_R
#define SIC_K1_R 8           // tracers per lane: a work item is 32 R tracers
#endif
#ifndef SIC_K1_MIN_BLOCKS
#define SIC_K1_MIN_BLOCKS 2  // resident blocks per SM the registers allow
#endif
#define SIC_K1_WARPS (SIC_K1_BLOCK / 32)
#define SIC_K1_WARP_TRACERS (32 * SIC_K1_R)

// error bits raised on the device
#define SIC_ERR_RANGE 1u
#define SIC_ERR_SEGLONG 2u
#define SIC_ERR_TIMEOUT 4u

// hold bits (SimScalars::hold): set by a step's field epilogue, they stop the
// simulation's later steps until the host clears them
#define SIC_HOLD_ERROR 1u    // an error bit is set: the run ends here
#define SIC_HOLD_REFINE 2u   // a particle is longer than the refinement length

// Per-warp double-buffered staging of the next work item in shared memory
// (filled by bulk copies): positions, velocities and, per-tracer charge mode,
// half charges, each with room for the item's 32 R tracers, its halo and (for
// the published positions of piecewise-linear particles) one more.
#define SIC_STAGE_U_BYTES (((SIC_K1_WARP_TRACERS + 2) * 4 + 15) / 16 * 16)
#define SIC_STAGE_V_BYTES SIC_STAGE_U_BYTES
#define SIC_STAGE_Q_BYTES SIC_STAGE_U_BYTES

// One work item, the task of one warp: up to 32 R consecutive tracers of one sheet.
struct WorkItem {
    float ke_mult;      // the item's KE and P terms are multiplied by these:
    float p_mult;       // the sheet half charge (1 with a Qh array) x 2^ke_u, 2^p_u
    int64_t t0;         // first tracer (aligned to SIC_ALIGN_TRACERS)
    int32_t count;      // tracers, 1..SIC_K1_WARP_TRACERS
    int32_t qh;         // sheet half charge when the simulation has no Qh array
    int64_t halo;       // tracer after the item's last one: the next item's
                        // first, or the sheet's first for a closed sheet; -1
                        // at the open end of a chain
    uint32_t halo_shift; // added to the halo position (winding * 2^30, modulo 2^32)
    uint32_t pad;
};

// The two more tracers a piecewise-linear particle's gradient needs (Sec. 2.5):
// the one before the item's first and the one after its halo; -1 when the
// sheet has none there (open ends).  The shifts move a closed sheet's other
// end by one winding (in position units, modulo 2^32).
struct WorkItemPL {
    int64_t prev;
    int64_t next2;
    uint32_t prev_shift;   // winding * 2^30 modulo 2^32, subtracted or added
    uint32_t next2_shift;
};

// Per-step sums every block adds into and the epilogue reads: the kinetic
// energy and momentum terms as 128-bit fixed-point integers (units of
// 2^-ke_u and 2^-p_u set per simulation, each item's FP32 partial truncated
// to them), so the totals do not depend on the order of the additions; the
// longest segment by atomicMax.  A block adds each 32-bit limb of its
// 128-bit (two's complement) sum into its own 64-bit word, with atomics that
// return nothing; the sum modulo 2^128 is sum_i limb_i 2^(32 i).  The words
// cannot overflow: fewer than 2^32 blocks add to them between epilogues.
struct SimAccum {
    unsigned long long ke[4];   // sum Qh (v_old^2 + v_new^2)  ((cells/step)^2 2^-ke_u), limbs
    unsigned long long p[4];    // sum Qh (v_old + v_new)  (cells/step 2^-p_u), limbs
    unsigned long long maxseg;  // longest segment crossing a cell edge, 2^-16 cells
    unsigned long long pad[3];
};

struct SimScalars {
    int64_t step;
    int64_t q_total;    // total charge of the mesh E was solved from
    double we;          // W_E of the current field
    int64_t maxseg;     // longest segment of the latest deposit crossing a cell edge, 2^-16 cells
    uint32_t err;       // SIC_ERR_* bits
    uint32_t buf;       // which state buffer is current
    uint32_t hold;      // SIC_HOLD_* bits: while nonzero, steps leave the simulation as it is
    uint32_t pad;
    double wk;          // field energy of Fourier mode mode_k of the current field (when recorded)
};

struct SimDev {
    uint32_t *U[2];
    float *V[2];
    const int32_t *Qh;          // may be null
    unsigned long long *mesh;
    long long *mesh_last;
    float2 *Ek;
    double *E64;
    double *rho64;
    SimAccum *acc;
    double *hist;               // [hist_len][4]
    SimScalars *sc;
    const WorkItem *items;      // [n_items] this simulation's work items
    const WorkItemPL *pl;       // [n_items] for piecewise-linear particles, else null
    int32_t deposit;            // SIC_DEPOSIT_*
    int32_t seg_q;              // Qh holds each particle's own charge (refined
                                // sheets: the particle starting at the tracer)
    int32_t n_items;
    int32_t hist_len;
    int32_t nx;
    int32_t pad0;
    double e_scale;             // Ek_j = K_j * e_scale
    double E_scale;             // E_j  = K_j * E_scale
    double rho_scale;           // rho_j = (nx mesh_j - Q) * rho_scale
    double we_scale;            // W_E = we_scale * sum (K_j 2^-60)^2
    float ek_mant;              // e_scale = ek_mant * 2^ek_exp
    int32_t ek_exp;
    double ke_scale;            // KE = ke_scale * sum ke 2^-ke_u
    double p_scale;             // P  = p_scale * sum p 2^-p_u
    int32_t ke_u, p_u;          // the sums count units of 2^-ke_u and 2^-p_u
    int32_t strict;
    int32_t pad1;
    long long refine_seg;       // hold for refinement once the longest segment crossing a
                                // cell edge exceeds this (2^-16 cells); 0: never
    double *mhist;              // [hist_len] field energy of Fourier mode mode_k per step, or null
    double *spec;               // [nx / 2 + 1] Fourier amplitudes (sic_spectrum)
    int32_t mode_k;             // 0: no mode history
    int32_t pad2;
};

// Everything one launch of the step kernel needs.
struct LaunchArgs {
    const SimDev *sims;          // table, one entry per slot
    const int32_t *slot_begin;   // [slots + 1] first item of each slot in the
                                 // launch's list (the slots' items back to back)
    unsigned *cursor;            // [slots] items claimed; zero between launches
    unsigned *tickets;           // [slots] items finished; zero between launches
    unsigned *done;              // blocks finished; zero between launches
    int32_t n_items;             // slot_begin[slots]
    float claim_q;               // a claim takes this fraction of the items a
                                 // simulation has left (guided scheduling)
    int32_t claim_min;           // and at least this many (>= 1)
    int32_t n_slots;
    int32_t nx_max;
    int32_t drift;
    int32_t record;
    float kick_scale;
    int32_t gen;                 // some simulation deposits other than box particles
    int32_t staging;             // 0: staged when it costs no resident block;
                                 // 1: never; 2: whenever it fits (autotuning)
};

#include <cuda_runtime.h>
namespace sic {
enum Mode { MODE_STEP = 0, MODE_DEPOSIT = 1, MODE_PUSH = 2 };
cudaError_t launch_step_kernel(const LaunchArgs &a, int grid, Mode mode, bool per_q, cudaStream_t s);
cudaError_t launch_field_out(const SimDev &sim, cudaStream_t s);
cudaError_t launch_spectrum(const SimDev &sim, int field, cudaStream_t s);
cudaError_t launch_refine_count(const SimDev &sim, long long lfix, int32_t *splits, cudaStream_t s);
cudaError_t launch_refine_scatter(const SimDev &sim, long long lfix, const int64_t *out_base, uint32_t *U2, float *V2,
                                  int32_t *Q2, cudaStream_t s);
cudaError_t launch_moments(const SimDev &sim, int weighting, double box_length, double unit_q, double unit_v,
                           double *n, double *j, cudaStream_t s);
cudaError_t launch_expand_horizontal(uint32_t *U, float *V, const uint32_t *u_template, int32_t n_template,
                                     const float *v_sheet, const int64_t *sheet_offset, int32_t n_sheets,
                                     cudaStream_t s);
int step_blocks_per_sm(int nx_max, Mode mode, bool per_q);
size_t step_smem_bytes(int nx_max, bool staged, bool per_q);
bool step_staged(int nx_max, bool per_q);
void count_launches(int64_t n);
int64_t launches();
}  // namespace sic
