/*
 * sic.h -- C ABI of the GB300-native simplex-in-cell (SIC) library.
 *
 * The library advances the 1D periodic Vlasov-Poisson system with the method
 * of Kates-Harbeck, Totorica, Zrake & Abel (arXiv:1506.07207): phase space is
 * carried by sheets of ordered tracers (Sec. 2.2); each pair of adjacent
 * tracers is a particle whose charge is spread uniformly between them (the box
 * function of Sec. 2.3) and deposited on the charge mesh by exact overlap
 * integration (Eq. overlap, Eq. rho_sum); the field solve, linear gather and
 * push are those of a PIC code (Sec. 2.3, last paragraphs).
 *
 * Conventions (the paper leaves these open):
 *   - Normalised units, C = 1 in the Poisson equation of Sec. 2.1: with
 *     E = -dPhi/dx, dE/dx = n - mean(n) and a tracer accelerates by
 *     charge_to_mass * E.  The neutralising background is the computed mean
 *     density.
 *   - Cells j = 0..nx-1 cover [j dx, (j+1) dx), dx = box_length / nx, left
 *     closed.  rho is the cell average; E lives on the nodes x_j = j dx.
 *   - Segment charge q_s = (w_i + w_{i+1}) / 2.  A zero-length segment puts
 *     its whole charge in the cell holding its point.
 *   - A closed sheet is closed by the segment (x_N, x_1 + winding * L).
 *   - Leapfrog: v^{n+1/2} = v^{n-1/2} + dt qm E^n(x^n), x^{n+1} = x^n + dt v^{n+1/2}.
 *
 * Precision: positions are 32-bit fixed point (SIC position format below),
 * velocities and push arithmetic FP32, charge int64 fixed point (total charge
 * is conserved bit-exactly and the deposit is independent of the order of
 * the atomic adds); the field solve is exact integer arithmetic with one final
 * rounding.  Results are bit-identical however the work is split across
 * thread blocks or batched with other simulations.
 *
 * SIC position format.  A tracer at x is stored as P = x / L 2^30 modulo 2^32
 * (L the box length): 30 bits of box fraction (a resolution of L 2^-30) and
 * 2 bits of winding, so positions are known modulo 4 box lengths and the
 * segment between two tracers is the 32-bit difference of their P, exact
 * while it is shorter than 2 box lengths.  A drift adds the step v dt rounded
 * to whole units of L 2^-30.  Limits, checked: a segment stays shorter than
 * 1.5 box lengths (at creation: SIC_ERANGE; while stepping: the run stops
 * with SIC_ERANGE at the next synchronising call; Sec. 3.2 notes that a run
 * cannot go on once a segment outgrows the box anyway), and a tracer moves
 * less than half a box per step.  Since each end of a segment moves less
 * than half a box per step, no segment can pass from below 1.5 to 2.5 box
 * lengths, where its difference would alias, in one step.  Positions read
 * back (sic_get_state) are unwrapped along each sheet: its first tracer
 * inside [0, L), each next one a segment further.
 *
 * Memory: every pointer argument named *_host is caller-owned host memory that
 * the call only reads or writes during the call.  All device state is owned by
 * the library and freed by sic_destroy.  Calls on one simulation must not run
 * concurrently; distinct simulations are independent.  Every function returns
 * SIC_OK (0) or a negative SIC_E* code; sic_strerror names it.  After a
 * SIC_ECUDA the simulation must be destroyed.
 */
#ifndef SIC_H
#define SIC_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define SIC_OK 0
#define SIC_EINVAL (-1)        /* bad size, NaN/Inf input, nx out of range, ... */
#define SIC_ENOMEM (-2)        /* device or host allocation failed */
#define SIC_ECUDA (-3)         /* a CUDA call failed */
#define SIC_ERANGE (-4)        /* outside the position format: a segment of 1.5 box
                                  lengths or more, a step of half a box or more, |x| of
                                  2^20 box lengths or more at creation */
#define SIC_ESEGMENT_LONG (-5) /* strict mode: a segment is longer than the box */
#define SIC_ETIMEOUT (-6)      /* a bounded device wait gave up */
#define SIC_EBUSY (-7)         /* server: budget or slots exhausted */
#define SIC_ELIMIT (-8)        /* a refinement would take the simulation past its tracer limit */

/* Largest mesh the deposit kernels stage in shared memory. */
#define SIC_NX_MAX 8192
/* Largest tracer count of one simulation (positions are indexed by int64,
 * the cap keeps per-simulation fixed-point sums far from overflow). */
#define SIC_TRACERS_MAX (1LL << 28)

typedef struct sic_sim sic_sim;

/* Charge deposits (sic_config.deposit). */
#define SIC_DEPOSIT_BOX 0     /* box particles: uniform density between two adjacent
                                 tracers (Sec. 2.3, Eq. overlap, Eq. rho_sum) */
#define SIC_DEPOSIT_LINEAR 1  /* piecewise-linear particles: density linear about the
                                 centroid with the central-difference gradient of
                                 Sec. 2.5 (Eq. gradient_rho_estimate), none at a fold
                                 corner, at an open end or for a particle a box
                                 length or longer */
#define SIC_DEPOSIT_PIC_NGP 2 /* PIC comparison: every tracer a point charge w_i in
                                 its cell (nearest grid point, Sec. 2.4) */
#define SIC_DEPOSIT_PIC_CIC 3 /* PIC comparison: every tracer a point charge shared
                                 between the two cells whose centres bracket it
                                 (cloud in cell, Sec. 2.4) */
#define SIC_DEPOSIT_FIRST 4   /* box particles with first-order weighting (Sec. 2.4): each
                                 slice of a particle shared between the two nodes around
                                 it by the hat of half-width dx, so the mesh holds charge
                                 per node x_j = j dx; the field integrates between nodes
                                 by the trapezoid rule, E_{j+1} = E_j + dx (rho_j +
                                 rho_{j+1}) / 2, zero mean */

/*
 * Problem statement (Sec. 2.2-2.3): M sheets of ordered tracers on a periodic
 * box [0, box_length) split into nx cells, stepped with time step dt.
 * tracers_per_sheet[s] >= 2 consecutive tracers form sheet s; sheet_closed[s]
 * != 0 adds the closing segment (last, first + sheet_winding[s] * L)
 * (periodic identification of Sec. 2.3).  sheet_winding may be NULL for all
 * zero windings; it is ignored for open sheets.
 */
typedef struct {
    int32_t nx;                        /* cells, 2..SIC_NX_MAX */
    double box_length;                 /* L > 0 */
    double dt;                         /* > 0 */
    int32_t n_sheets;                  /* M >= 1 */
    const int32_t *tracers_per_sheet;  /* [M], each >= 2 */
    const uint8_t *sheet_closed;       /* [M] */
    const int32_t *sheet_winding;      /* [M] or NULL */
    double charge_to_mass;             /* qm, finite and != 0; the paper's sign is +1 */
    int32_t half_step_init;            /* 1: v^{-1/2} = v^0 - dt/2 qm E^0(x^0) at create */
    int32_t strict_segments;           /* 1: sic_step fails with SIC_ESEGMENT_LONG when a
                                          segment exceeds the box (Sec. 3.2 notes the run
                                          cannot continue then); 0: deposit it anyway,
                                          every periodic image counting */
    int32_t history_len;               /* rows of the per-step diagnostic ring, >= 1 */
    void *stream;                      /* cudaStream_t the simulation runs on, NULL = its own */
    int32_t deposit;                   /* SIC_DEPOSIT_*: what carries the charge onto the mesh;
                                          other values SIC_EINVAL */
    double refine_length;              /* refinement length of Sec. 2.6 (same unit as box_length):
                                          0 = never refine; else >= box_length / nx / 1024, box
                                          and piecewise-linear deposits only.  After a step whose
                                          longest particle exceeds it the simulation holds: later
                                          steps leave it as it is until it is refined (sic_run
                                          and the server do this themselves; sic_refine clears
                                          the hold).  It holds at the same step alone or in any
                                          batch. */
    double refine_split;               /* when a hold for refinement is resolved, every particle
                                          longer than this is split (passes until none is): 0 =
                                          refine_length, else 0 < refine_split <= refine_length.
                                          A shorter one splits ahead, so holds come less often */
    int64_t max_tracers;               /* refinement may grow the simulation to this many tracers:
                                          0 = SIC_TRACERS_MAX.  A refinement that would pass it
                                          is not done and the call returns SIC_ELIMIT (Sec. 2.6:
                                          the tracer count grows about exponentially once the
                                          sheets fold, so a run's length is bounded by memory) */
    double charge_unit;                /* charge of one fixed-point unit: 0 = chosen from the
                                          largest weight; else > 0, and every particle's charge
                                          must fit 2^28 units (SIC_ERANGE otherwise).  Simulations
                                          that hold parts of one set of sheets (split over GPUs)
                                          give the same unit so that their integer meshes add up
                                          to the whole one's bit for bit */
    int32_t mode_k;                    /* Fourier mode whose field energy every step records
                                          (Sec. 3.2: the energy in the excited mode), read with
                                          sic_mode_history: 0 = none, else 1 <= mode_k <= nx/2 */
} sic_config;

/* Diagnostics of the latest completed step (Sec. 3.1: energies and momentum
 * are monitored; W_E is the potential energy E_pot of the paper's figures). */
typedef struct {
    int64_t step;          /* steps taken since create */
    double t;              /* step * dt */
    double field_energy;   /* W_E = 1/2 sum_j E_j^2 dx of the current field */
    double kinetic_energy; /* KE of the last kick, time-centred: 1/2 sum m (v-^2 + v+^2)/2 */
    double momentum;       /* sum m (v- + v+)/2 of the last kick; m = w / qm */
    int64_t charge_fixed;  /* total mesh charge in fixed-point units (constant) */
    double charge_unit;    /* charge of one fixed-point unit */
    double max_segment;    /* longest segment of the last deposit that crosses a cell
                              edge, in box lengths (0 when none does) */
} sic_diag;

/*
 * Create a simulation from host arrays of length sum(tracers_per_sheet):
 * positions x (unwrapped, |x| < 2^20 L), velocities v (|v dt| < L / 2) and
 * charge weights w > 0, all finite; every segment, the closing one included,
 * shorter than 1.5 L (SIC_ERANGE otherwise).  The inputs are copied; the
 * initial charge is deposited and the field solved (and the half step applied
 * if asked).
 */
int sic_create(const sic_config *cfg, const double *x_host, const double *v_host,
               const double *w_host, sic_sim **out);

/*
 * Create M closed horizontal sheets of winding 1 (the "horizontal" set-up of
 * Sec. 3.3) that all share one position template: sheet s has tracers at
 * x_template[0..n-1] with velocity v_sheet[s] and weight w_sheet[s] each.
 * cfg->tracers_per_sheet, sheet_closed and sheet_winding are ignored.  Only
 * the template and the per-sheet values cross the bus.
 */
int sic_create_horizontal(const sic_config *cfg, int32_t n_template,
                          const double *x_template_host, const double *v_sheet_host,
                          const double *w_sheet_host, sic_sim **out);

/*
 * Deposit the current tracer positions (Eq. overlap, Eq. rho_sum) and solve
 * the field.  Outputs, each nullable, host, nx entries: the fixed-point charge
 * per cell (units of sic_diag.charge_unit) and the neutralised density
 * rho_j = n_j - mean(n).
 */
int sic_deposit(sic_sim *sim, int64_t *mesh_fixed_host, double *rho_host);

/*
 * The node field E_j (host, nx entries) solved from the latest deposit: the
 * Poisson equation of Sec. 2.1 with C = 1 against the neutralising
 * background (the mean density), "solve" of the PIC cycle in Sec. 2.3.  E is
 * the exact integral of rho from node to node, shifted to zero mean (periodic
 * potential): E_0' = 0, E_{j+1}' = E_j' + dx rho_j, E_j = E_j' - mean(E').
 * E_host is caller-owned; SIC_EINVAL for a null pointer.
 */
int sic_field(sic_sim *sim, double *E_host);

/*
 * Moments of the current state: number density n (charge per length) and
 * current density j = n v of the box particles, into host arrays of nx
 * doubles (either may be NULL).
 *   weighting 0: zero order onto the cells [j dx, (j+1) dx) (Sec. 2.3,
 *     Eq. rho_sum and Eq. j_sum); a particle moves with the mass-weighted
 *     mean velocity of its two tracers;
 *   weighting 1: first order onto the nodes x_j = j dx (Sec. 2.4): each slice
 *     of a particle weighted by the hat of half-width dx about the node, its
 *     velocity interpolated linearly between the tracers' velocities.
 * The velocities are the stored ones (v^{n-1/2} after a step), the charges
 * the fixed-point ones of the deposit.  Diagnostic only: FP64 with atomics,
 * equal to the FP64 definition within rounding but not bit-reproducible; a
 * particle longer than 64 box lengths is left out (the paper stops a run at
 * one box length, Sec. 3.2).  Other weightings: SIC_EINVAL.
 */
int sic_moments(sic_sim *sim, int32_t weighting, double *n_host, double *j_host);

/*
 * Refinement (Sec. 2.6): every particle of the current state longer than
 * l_ref (same length unit as box_length) gets a new tracer at its centre,
 * with the mean velocity of its two tracers; each half carries half the
 * particle's charge (the first floor(Q/2) fixed-point units, the second the
 * rest), so the total charge stays exact and the deposit does not change.
 * One pass: a particle longer than 2 l_ref needs another call.  From the
 * first refinement on, the simulation carries its charge per particle and a
 * tracer's mass is the charge of the particle it starts (the last tracer of
 * an open sheet has none).  The state is moved to a new, larger device
 * allocation; batches and servers holding the simulation must be rebuilt.
 * Box and piecewise-linear deposits only (SIC_EINVAL for the PIC ones);
 * l_ref must be finite and > 0.  *n_added (nullable) gets the number of new
 * tracers; sic_sheet_counts gives the new tracers per sheet.
 */
int sic_refine(sic_sim *sim, double l_ref, int64_t *n_added);

/* Tracers per sheet now (they grow with sic_refine), into counts_host[M]. */
int sic_sheet_counts(sic_sim *sim, int32_t *counts_host);

/*
 * n_steps full steps, synchronously, refining as Sec. 2.6 describes: whenever
 * a step leaves a particle longer than cfg->refine_length the run holds, the
 * particles longer than cfg->refine_split are split (sic_refine passes until
 * none is), and the run goes on, until n_steps steps are done (a hold after
 * the last of them is resolved by the next call).  Without a refinement length
 * it is sic_step followed by sic_sync.  *n_added (nullable) gets the tracers
 * added.  Errors as for sic_sync (the run stops at the step that raised one).
 */
int sic_run(sic_sim *sim, int32_t n_steps, int64_t *n_added);

/*
 * Gather, kick and drift every tracer with the current field, no deposit:
 * the "gather" and "move" of the PIC cycle, which Sec. 2.3 keeps unchanged
 * for SIC (forces gathered at the tracers by linear weighting between the
 * two nodes around each).  The integrator is the leapfrog kick-drift the
 * paper leaves open: v += dt qm E(x), then x += dt v.  The field is not
 * re-solved, so a second sic_push kicks with the same field; sic_deposit
 * re-solves it.  Asynchronous on the simulation's stream; device-side
 * errors show at the next synchronising call.
 */
int sic_push(sic_sim *sim);

/*
 * n_steps full SIC steps (Sec. 2.3: the PIC cycle with the scatter replaced
 * by the sheet deposit of Eq. overlap and Eq. rho_sum): gather and push with
 * the current field, deposit every particle of the new positions, solve the
 * field (Sec. 2.1).  Each step is one kernel launch, the field solved by the
 * block that finishes last; runs of 8 steps replay a captured CUDA graph.
 * n_steps >= 0.  Asynchronous on the simulation's stream: errors found on
 * the device are returned by the next synchronising call (sic_sync,
 * sic_diagnostics, ...).  A held simulation (an error, or a particle past
 * the refinement length) is left as it is by the remaining steps: check
 * sic_diagnostics' step count, or use sic_run.
 */
int sic_step(sic_sim *sim, int32_t n_steps);

/* Advance several simulations together, n_steps[i] steps each; the work of
 * all of them shares each kernel launch.  Results equal separate sic_step
 * calls bit for bit. */
int sic_step_batch(sic_sim *const *sims, int32_t n_sims, const int32_t *n_steps);

/* A persistent batch: its launch plan is built once, so stepping it costs
 * one kernel launch per step for all members (CUDA graphs of 8 steps when
 * n_steps >= 8).  While the batch exists its members must be advanced only
 * through it; it runs on the first member's stream, ordered after all
 * members' streams at create and before them at destroy.  Every member
 * advances by the same number of steps; results equal sic_step bit for bit. */
typedef struct sic_batch sic_batch;
int sic_batch_create(sic_sim *const *sims, int32_t n_sims, sic_batch **out);
int sic_batch_step(sic_batch *batch, int32_t n_steps);
/*
 * Autotuning of the batch's launch schedule: each of SIC_AUTOTUNE_CANDIDATES
 * candidates (claim divisor D = 1, 2, 4 or 8 for the guided claims of work
 * items, a warp claiming about 1 / (D x warps) of what is left; the smallest
 * claim, 1, 2 or 4 items; staging of the items through shared memory
 * automatic, off, or on whenever it fits) is timed with CUDA events on
 * steps_each real steps (after one untimed step), and the fastest is kept
 * for the batch's later steps.  The schedule never changes results (they
 * are bit-identical under every choice), so the timed steps are ordinary
 * steps: the call advances every member by SIC_AUTOTUNE_CANDIDATES
 * (steps_each + 1) steps.  *claim_div, *staging and *claim_min (nullable)
 * get the choice (staging: 0 automatic, 1 off, 2 on).  steps_each >= 1.
 */
#define SIC_AUTOTUNE_CANDIDATES 10
int sic_batch_autotune(sic_batch *batch, int32_t steps_each, int32_t *claim_div, int32_t *staging,
                       int32_t *claim_min);

/* Segments the batch advances per step (sum over its members). */
int64_t sic_batch_segments(const sic_batch *batch);
void sic_batch_destroy(sic_batch *batch);

int sic_diagnostics(sic_sim *sim, sic_diag *out);

/* Per-step history [rows][4] = {W_E, KE, P, charge_fixed} of the last
 * min(max_rows, history_len, steps taken) steps, oldest first, into hist_host
 * (room for max_rows rows, max_rows >= 1); the row count goes to *rows. */
int sic_history(sic_sim *sim, double *hist_host, int32_t max_rows, int32_t *rows);

/*
 * Field energy in the Fourier mode pair +-k, k = cfg->mode_k (Sec. 3.2: the
 * energy in the excited mode of the two-stream instability), of the last
 * min(max_rows, history_len, steps taken) steps, oldest first, one double per
 * step into out_host (room for max_rows >= 1); the count goes to *rows.  With
 * E^_k = sum_j E_j exp(-2 pi i j k / nx) of the node field, the value is
 * W_k = dx / nx |E^_k|^2 (half that for k = nx/2), so that the W_k of
 * k = 1 .. nx/2 add up to W_E (Parseval).  Row i belongs to the same step as
 * row i of sic_history.  Computed on the device by the field solve, in FP32
 * per thread and FP64 across; SIC_EINVAL when mode_k is 0.
 */
int sic_mode_history(sic_sim *sim, double *out_host, int32_t max_rows, int32_t *rows);

/*
 * Fourier amplitudes |X^_k|, k = 0 .. nx/2 (nx/2 + 1 doubles into out_host),
 * X^_k = sum_j X_j exp(-2 pi i j k / nx), of the latest deposit's neutralised
 * density (field = 0, the rho_j of sic_deposit; Sec. 3.2 shows this transform
 * during the linear growth of the two-stream instability) or of its node
 * field (field = 1, the E_j of sic_field).  FP64 on the device from the exact
 * charge mesh.  SIC_EINVAL for another field or a null pointer.
 */
int sic_spectrum(sic_sim *sim, int32_t field, double *out_host);

/*
 * Copy the tracers back (the sheets of ordered tracers of Sec. 2.2, in the
 * order they were given): positions and current velocities (v^{n-1/2} after
 * n steps), into caller-owned host arrays of sum(tracers_per_sheet) entries
 * each (either may be NULL).  Positions are unwrapped along each sheet (see
 * SIC position format above).
 */
int sic_get_state(sic_sim *sim, double *x_host, double *v_host);

/* Device addresses of the state for zero-copy consumers: positions uint32 in
 * the SIC position format (x / L 2^30 modulo 2^32), velocities float (position
 * units per step, v dt / L 2^30), tracer i of sheet s at sheet_offset[s] + i.
 * Valid until the next sic_step, sic_push or sic_refine (the state is double
 * buffered) or sic_destroy. */
int sic_device_state(sic_sim *sim, uint32_t **pos_dev, float **vel_dev,
                     const int64_t **sheet_offset_host);

/* Synchronise the simulation's stream. */
int sic_sync(sic_sim *sim);

void sic_destroy(sic_sim *sim);

const char *sic_strerror(int code);

/* Kernel launches issued by this process since load (for launch accounting). */
int64_t sic_launch_count(void);

/* ------------------------------------------------------------------------
 * Request server: continuous batching of many simulations on one GPU.
 *
 * A request is a simulation (the arguments of sic_create or
 * sic_create_horizontal) and a step count.  Requests wait in arrival order;
 * the server admits waiting requests while an active slot is free and their
 * device memory fits the budget, advances all active simulations together by
 * up to chunk_steps steps (each step is one kernel launch over all of them,
 * a second one for simulations that carry per-particle charges), and retires
 * the finished ones.  A request that holds for refinement (Sec. 2.6) is
 * refined and goes on.  The batched mode overlaps its host work with the
 * GPU: a tick waits for the chunk launched by the tick before, launches the
 * next one, and then retires, refines and creates beside it on a second
 * stream; admitted and refined requests step again from the next tick on.
 * Results are bit-identical to
 * running each request alone with sic_step.  In plain mode the server runs
 * one request at a time to completion with sic_step, first come first served
 * (the one-simulation-per-launch baseline).  Not thread-safe: one caller
 * drives a server.
 * ---------------------------------------------------------------------- */
typedef struct sic_server sic_server;

typedef struct {
    int64_t hbm_budget;  /* bytes of device memory admitted simulations may hold, > 0 */
    int32_t max_active;  /* simulations advanced together, >= 1 (forced to 1 in plain mode) */
    int32_t chunk_steps; /* steps between two admission points, >= 1 */
    int32_t plain;       /* 1: one request at a time, each run to completion */
    void *stream;        /* cudaStream_t for all server work, NULL = its own */
} sic_server_config;

typedef struct {
    int64_t id;              /* from submit */
    int32_t status;          /* SIC_OK, SIC_EBUSY (larger than the budget) or the error that ended it */
    int32_t pad;
    int64_t steps;           /* steps taken */
    int64_t segment_updates; /* segments x steps */
    double field_energy;     /* final diagnostics, as in sic_diag */
    double kinetic_energy;
    double momentum;
    int64_t charge_fixed;
    double t_submit;         /* server clock (sic_server_clock), seconds */
    double t_admit;
    double t_done;
    sic_sim *sim;            /* the simulation if submitted with keep != 0 (the caller
                                owns it and destroys it), else NULL */
} sic_result;

typedef struct {
    int64_t bytes_in_use;    /* device bytes held by admitted simulations */
    int64_t bytes_peak;
    int64_t hbm_budget;
    int32_t active;
    int32_t queued;
    int64_t completed;
    int64_t segment_updates; /* of completed requests */
    int64_t ticks;
    double busy_s;           /* device time of the steps the ticks launched (CUDA events) */
    int64_t waits_slots;     /* ticks whose admission stopped at the max_active limit */
    int64_t waits_memory;    /* ticks whose admission stopped at the device-memory budget */
    int64_t refinements;     /* refinement holds the server resolved (Sec. 2.6) */
} sic_server_info;

int sic_server_create(const sic_server_config *cfg, sic_server **out);

/* Queue a request; the inputs are copied (host arrays as for sic_create /
 * sic_create_horizontal).  cfg->stream is ignored; cfg->history_len rows of
 * per-step diagnostics (at least 1) are kept, for a caller that keeps the
 * simulation (keep != 0) and reads them with sic_history. */
int sic_server_submit(sic_server *srv, const sic_config *cfg, const double *x_host, const double *v_host,
                      const double *w_host, int32_t n_steps, int32_t keep, int64_t *id);
int sic_server_submit_horizontal(sic_server *srv, const sic_config *cfg, int32_t n_template,
                                 const double *x_template_host, const double *v_sheet_host,
                                 const double *w_sheet_host, int32_t n_steps, int32_t keep, int64_t *id);

/* One scheduling round.  Batched: collect the chunk launched by the previous
 * tick (blocking until it has run), launch the next chunk, then retire, refine
 * and admit while it runs.  Plain: admit one request and run it to completion.
 * *pending (nullable) gets the queued plus admitted, unfinished requests; the
 * caller ticks until it is 0. */
int sic_server_tick(sic_server *srv, int32_t *pending);

/* Move up to max finished requests into out[]; *n gets how many. */
int sic_server_results(sic_server *srv, sic_result *out, int32_t max, int32_t *n);

/* Seconds since sic_server_create on the server's steady clock. */
double sic_server_clock(sic_server *srv);

int sic_server_stats(sic_server *srv, sic_server_info *out);

/* Destroys the server, its queued and active simulations, and kept
 * simulations of results not yet taken. */
void sic_server_destroy(sic_server *srv);

/* ---- stepping without allocation (no counterpart in the paper) ------------
 *
 * sic_step_batch_static: the same steps, and bit-identical results, as
 * sic_step_batch, for callers that may not allocate device memory while they
 * step.  One example is a serving loop whose whole device-memory budget is
 * already promised to resident simulations, so a plan allocation could fail or
 * push it over budget mid-run.  Another is a loop that cannot afford the
 * device-wide synchronisation of cudaFree.  The launch plan is written into
 * one fixed scratch array in device memory per device (64 KiB); the call
 * makes no allocation (no cudaMalloc, cudaMallocAsync or cudaFree, no host
 * heap).
 *
 *   sims     n_sims distinct handles, all on one device (SIC_EINVAL if not);
 *            at most SIC_STATIC_MAX_SIMS, else SIC_EINVAL and nothing is done.
 *   n_steps  per simulation, >= 0; every member with steps left advances in
 *            the same launches, and each stops at its own count.
 *
 * The launches run on sims[0]'s stream, after the other members' streams have
 * been synchronised, and the call returns once they are done.  The plan's
 * counters (claim cursors, item tickets, finished blocks) are cleared before
 * every use.  The first call on a device looks up the scratch address there
 * (one runtime query with that device current); make that first call before
 * any stream capture.  The scratch is shared: calls on the same device that
 * overlap in time (two host threads) race on it, and the caller must
 * serialise them.  Errors as for sic_step_batch; device-side errors of the
 * steps show at the next sic_sync or sic_diagnostics of a member. */
#define SIC_STATIC_MAX_SIMS 64
int sic_step_batch_static(sic_sim *const *sims, int32_t n_sims, const int32_t *n_steps);

#ifdef __cplusplus
}
#endif

#endif /* SIC_H */
