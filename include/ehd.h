/*
 * ehd.h -- C ABI of the GB300 library for the coupled phase-field lattice Boltzmann
 * time step for two-phase electrohydrodynamics (Xiong, Wang, Huang & Luo,
 * arXiv 2407.01654).
 *
 * One simulation is one rectangular D2Q9 lattice (Sec. 3, Eq. weq37) in lattice units
 * (dx = dt = 1), periodic in x, with walls or periodicity in y.  A time step is
 * Algorithm 1 (Sec. 5): the Cahn-Hilliard LBE (Eqs. weq45-weq49), the potential LBE with
 * its large-permittivity-ratio forcing sub-iterated to the relative-change tolerance
 * (Eqs. weq52-weq55, eqA.16), the Nernst-Planck LBE (Eqs. weq56-weq62) and the
 * hydrodynamic LBE (Eqs. weq38-weq43), with the isotropic stencils of Sec. 3.2 and the
 * wetting / electrowetting wall rule (Eqs. weq68, weq69).
 *
 * Conventions for every call:
 *   - Fields are row-major [ny][nx] arrays, x fastest.
 *   - `mem` selects where an array lives: EHD_HOST arrays are double, EHD_DEVICE arrays
 *     are float32 device pointers (e.g. from a torch tensor).  The caller owns every
 *     array it passes; the library keeps no pointer to it after the call returns.
 *   - Work is queued on the CUDA stream given to ehd_create.  Calls that return data to
 *     the host (ehd_step's statistics, ehd_solve_potential, ehd_read_fields to host,
 *     ehd_save_state) synchronise that stream before returning.
 *   - Every call returns an ehd_status; the library never aborts the process and never
 *     traps the GPU.  ehd_error_string names a code.
 */
#ifndef EHD_H
#define EHD_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum ehd_status {
  EHD_OK = 0,
  EHD_ERR_INVALID_ARG = 1,     /* null pointer, bad size, unknown enum value            */
  EHD_ERR_UNSTABLE_PARAMS = 2, /* a relaxation time <= 0.5 + 1e-3, or sigma/eps > 0.5   */
  EHD_ERR_NOMEM = 3,           /* workspace too small or device allocation failed       */
  EHD_ERR_NOT_CONVERGED = 4,   /* a potential loop hit poisson_max_iter (state advanced)*/
  EHD_ERR_NONFINITE = 5,       /* NaN or Inf in phi or q (state advanced)               */
  EHD_ERR_BUSY = 6,            /* batch: no free slot or memory for a request           */
  EHD_ERR_CUDA = 7,            /* a CUDA runtime call failed                            */
  EHD_ERR_TOO_LARGE = 8,       /* lattice exceeds the fixed scratch of the no-allocation
                                  potential solve                                         */
  EHD_ERR_TIMEOUT = 9          /* a bounded device-side wait ran out (the grid barrier of
                                  the on-chip potential loop, 2 s): the kernel returned
                                  early, the results of the call are invalid, the CUDA
                                  context stays usable; destroy the simulation            */
} ehd_status;

enum { EHD_HOST = 0, EHD_DEVICE = 1 };
enum { EHD_FP32 = 0, EHD_FP16DEV = 1 };
/* Implementation of the potential sub-iteration loop (same arithmetic, same results):
 * STREAM runs one kernel per sub-iteration over populations in device memory; RESIDENT
 * runs the whole loop in one cooperative kernel with the populations held on chip (only
 * for lattices that fit, about 600k nodes on a GB300); AUTO picks RESIDENT when it fits. */
enum {
  EHD_LOOP_AUTO = 0,
  EHD_LOOP_STREAM = 1,
  EHD_LOOP_RESIDENT = 2,
  EHD_LOOP_RESIDENT2 = 3,
  EHD_LOOP_RESIDENT3 = 4
};

/* Field selection bits for ehd_read_fields. */
enum {
  EHD_F_PHI = 1u << 0,     /* order parameter phi = sum g (Eq. weq49)                    */
  EHD_F_Q = 1u << 1,       /* charge q = sum l + R/2 (Eq. weq62, lagged R of Alg. 1)     */
  EHD_F_VARPHI = 1u << 2,  /* potential of the last potential solve (Eq. weq55)          */
  EHD_F_EX = 1u << 3,      /* E = -grad(varphi) of the last solve, local (Eq. eqA.16)    */
  EHD_F_EY = 1u << 4,
  EHD_F_UX = 1u << 5,      /* velocity, rho u = sum c f + F/2 (Eq. weq43)                */
  EHD_F_UY = 1u << 6,
  EHD_F_P = 1u << 7,       /* hydrodynamic pressure (Eq. eq32)                            */
  EHD_F_MU = 1u << 8       /* chemical potential hbar (Eq. weq31) of the current phi (its
                              Laplacian with the current wall rule) and the field E that
                              EX / EY return (that of the last potential solve)           */
};
#define EHD_NUM_FIELDS 9

/* Potential LBE schemes (ehd_params.potential_scheme). */
enum { EHD_SCHEME_IMPROVED = 0, EHD_SCHEME_CONVENTIONAL = 1 };

/* Parameters, lattice units.  Phase l is phi = 1, phase v is phi = 0 (Sec. 2.2). */
typedef struct ehd_params {
  int32_t nx, ny;               /* lattice size; x is periodic                           */
  int32_t walls_y;              /* 1: walls half-way below row 0 and above row ny-1;
                                   0: y periodic                                          */
  int32_t precision;            /* EHD_FP32 or EHD_FP16DEV population storage             */
  double rho_l, rho_v;          /* densities (linear in phi, Eq. weq36)                   */
  double mu_l, mu_v;            /* dynamic viscosities (linear); tau_f from
                                   mu = rho c_s^2 (tau_f - 1/2) (Sec. 3.1)                */
  double sigma_l, sigma_v;      /* conductivities (linear)                                */
  double eps_l, eps_v;          /* permittivities (Hermite law, Remark II);
                                   tau_h = 1/2 + eps_v / c_s^2 (Eq. eqA.15)               */
  double alpha;                 /* charge diffusivity; tau_l = 1/2 + alpha / c_s^2       */
  double gamma, width, mobility;/* surface tension, interface width W, mobility M:
                                   beta = 12 gamma/W, kappa = 3 gamma W/2,
                                   tau_g = 1/2 + M / c_s^2 (Secs. 2.2, 3.2)               */
  double theta_bottom_deg;      /* Young contact angles of the walls (Eq. weq68)          */
  double theta_top_deg;
  double ew_bottom;             /* electrowetting number eta/d of the bottom wall         */
  double ew_sign;               /* +1 classical, -1 reversed electrowetting (Sec. 7.2)    */
  double varphi_bottom;         /* Dirichlet wall potentials                              */
  double varphi_top;
  int32_t ramp_steps;           /* wall potentials ramp linearly from 0 over this many
                                   steps (0: applied at once); the electrowetting number
                                   follows the square of the ramp fraction                */
  int32_t neutralize_charge;    /* 1: the potential source is q - mean(q) (for y periodic) */
  double body_gx, body_gy;      /* optional body acceleration, force rho g                */
  double poisson_tol;           /* stopping tolerance of the potential loop (Alg. 1: 1e-5)*/
  int32_t poisson_max_iter;     /* cap on sub-iterations per solve                        */
  int32_t poisson_min_iter;     /* at least this many sub-iterations (>= 1)               */
  int32_t poisson_fixed_iter;   /* > 0: exactly this many sub-iterations, no stopping test*/
  int32_t poisson_loop;         /* EHD_LOOP_AUTO, EHD_LOOP_STREAM, EHD_LOOP_RESIDENT (the
                                   whole loop on chip), EHD_LOOP_RESIDENT2 (on chip, two
                                   sub-iterations per halo exchange; tiles of 24..64 rows,
                                   every tile at least 4 x 4) or EHD_LOOP_RESIDENT3 (three;
                                   48..64 rows, every tile at least 6 x 6).  Every loop
                                   gives the same states, bit for bit                    */
  int64_t start_step;           /* step counter after ehd_set_fields                      */
  int32_t tile_rows;            /* resident potential loop: 0 = tiles chosen from the
                                   lattice size (about 2048 nodes each, at most one per
                                   SM, enough rows of tiles for tiles of at most 64 rows);
                                   8, 16, ..., 64 = tiles of 64 x tile_rows nodes
                                   (as many per SM as fit), e.g. picked by an autotuner;
                                   other values: EHD_ERR_INVALID_ARG.  Results
                                   do not depend on the tiling at a fixed sub-iteration
                                   count.  A batch tiles every slot with its own height
                                   (ehd_batch_set_schedule)                               */
  int32_t potential_scheme;     /* EHD_SCHEME_IMPROVED: the paper's potential LBE with the
                                   large-ratio forcing (Eq. weq53); EHD_SCHEME_CONVENTIONAL:
                                   the conventional scheme of Sec. 3.3 (no forcing,
                                   eps(phi) = chi c_s^2 (tau_varphi - 1/2)), kept as the
                                   paper's comparison baseline; it runs on the streaming
                                   loop and the one- and two-step on-chip loops
                                   (EHD_LOOP_RESIDENT3 with it: EHD_ERR_INVALID_ARG)      */
  double chi;                   /* conventional scheme: the artificial factor chi > 0     */
  int32_t field_mode;           /* E used in hbar, F and R (and returned): 0 the local
                                   first moment of the converged h (Eq. eqA.16); 1 the
                                   isotropic stencil (Sec. 3.2) on varphi (Eq. weq55)
                                   with ghost rows 2 varphi_w - varphi at the electrodes  */
  int32_t lagged_field;         /* 1: hbar of step n uses E of step n-1 (the order in
                                   which Algorithm 1 lists the LBEs); 0: E of step n     */
} ehd_params;

/* Statistics of one ehd_step call. */
typedef struct ehd_stats {
  int64_t step;                 /* step counter after the call                           */
  int32_t steps;                /* time steps made by the call                           */
  int32_t poisson_iters_total;  /* potential sub-iterations over those steps             */
  int32_t poisson_iters_min;
  int32_t poisson_iters_max;
  int32_t not_converged_steps;  /* steps whose potential loop hit poisson_max_iter       */
  int32_t nonfinite;            /* 1 if phi or q held NaN/Inf at some step               */
  double last_rel_change;       /* relative change of the last sub-iteration             */
  double sum_phi;               /* FP64 sum of phi over the lattice, last step's level   */
  double sum_q;                 /* FP64 sum of q, same level                             */
  int64_t kernel_launches;      /* CUDA kernel launches the call queued                  */
} ehd_stats;

/* Device time per kernel kind while profiling is on.  Steps launched as graphs use a
 * profiling form of the step graph with event-record nodes around the moments pass, the
 * potential loop and the coupled pass (one "launch" per part and step, the loop counted
 * whole); steps queued from the host (ehd_use_graphs(0)) record CUDA events around every
 * launch on the simulation's stream.  Kinds: 0 moments, 1 potential loop, 2 potential
 * launches queued after the loop had finished (they return at once; host-queued streaming
 * loop only), 3 coupled collide-and-push. */
typedef struct ehd_kernel_times {
  double ms[4];
  int64_t launches[4];
} ehd_kernel_times;

typedef struct ehd_sim ehd_sim;

/* Device workspace a simulation with these parameters needs, in bytes.
 * Errors: EHD_ERR_INVALID_ARG (null pointer, nx or ny < 1). */
int ehd_workspace_bytes(const ehd_params* params, size_t* bytes);

/* Validates the parameters and creates a simulation.
 *   params      copied; not referenced afterwards.
 *   workspace   device memory of at least ehd_workspace_bytes() bytes, 256-byte aligned,
 *               owned by the caller and kept alive until ehd_destroy; or NULL, in which
 *               case the library allocates (and frees) its own.
 *   stream      cudaStream_t on which every later call queues its work (NULL: the
 *               default stream).
 * The populations are zero until ehd_set_fields.
 * Errors: EHD_ERR_INVALID_ARG, EHD_ERR_UNSTABLE_PARAMS, EHD_ERR_NOMEM, EHD_ERR_CUDA. */
int ehd_create(const ehd_params* params, void* workspace, size_t workspace_bytes,
               void* stream, ehd_sim** out);

/* Initialisation, Algorithm 1 step 1: populations at equilibrium with the given fields
 * (g = g_eq(phi, hbar(phi, E = 0)), l = l_eq(q, u), f = f_eq(p, u)), potential
 * distribution at equilibrium with the potential interpolated linearly between the walls,
 * lagged quantities zero, then one potential solve with the parameters' rule.
 *   phi, q, ux, uy  required, [ny][nx]; p optional (NULL: 0).
 *   mem             EHD_HOST (double) or EHD_DEVICE (float32).
 * Returns the status of the potential solve (EHD_ERR_NOT_CONVERGED if it hit the cap). */
int ehd_set_fields(ehd_sim* sim, const void* phi, const void* q, const void* ux,
                   const void* uy, const void* p, int mem);

/* Advances nsteps time steps (Algorithm 1 steps 2-6).  With `stats` non-NULL the call
 * clears the statistics, synchronises the stream at the end and fills `stats` for these
 * steps.  With `stats` NULL nothing is synchronised and the statistics keep accumulating
 * until ehd_read_stats.  The state always advances; the return code reports
 * EHD_ERR_NOT_CONVERGED / EHD_ERR_NONFINITE if a step met that condition (known only
 * when the statistics are read). */
int ehd_step(ehd_sim* sim, int nsteps, ehd_stats* stats);

/* Launch mode of later ehd_step calls (no counterpart in the paper): enable != 0 (the
 * default) launches steps as captured CUDA graphs (runs of 8 steps as one graph, the
 * rest one graph per step); enable == 0 queues the step's kernels one by one from the
 * host, with the streaming loop's stopping rule checked on the host between chunks of
 * launches.  Both give the same states, bit for bit.  Errors: EHD_ERR_INVALID_ARG (null
 * handle). */
int ehd_use_graphs(ehd_sim* sim, int enable);


/* Which potential loop this simulation runs: EHD_LOOP_STREAM, EHD_LOOP_RESIDENT,
 * EHD_LOOP_RESIDENT2 or EHD_LOOP_RESIDENT3 (negative: invalid handle). */
int ehd_loop_kind(const ehd_sim* sim);

/* Statistics accumulated since they were last cleared (by ehd_step with stats, or by this
 * call); synchronises the stream and clears them.  Returns the status those steps would
 * have returned. */
int ehd_read_stats(ehd_sim* sim, ehd_stats* stats);

/* Runs the potential loop alone for the phi and q of the current populations (the
 * potential sub-iterations of Algorithm 1 step 3), with tolerance `tol` and cap
 * `max_iter` (tol <= 0 or max_iter <= 0: the parameters' values).  Writes the number of
 * sub-iterations and the last relative change when the pointers are non-NULL.
 * Synchronises the stream. */
int ehd_solve_potential(ehd_sim* sim, double tol, int max_iter, int* iters,
                        double* rel_change);

/* Macroscopic fields of the current state.  For each bit set in `mask`, in bit order,
 * the next pointer of `out` receives a [ny][nx] array.  PHI, Q, UX, UY and P are those of
 * the current populations; VARPHI, EX and EY those of the last potential solve (which,
 * after a step, used that step's phi and q); MU combines the two (current phi, last
 * solve's E).  mem: EHD_HOST (double) or EHD_DEVICE (float32).
 * Errors: EHD_ERR_INVALID_ARG (null pointer, a bit beyond EHD_F_MU, bad mem). */
int ehd_read_fields(ehd_sim* sim, unsigned mask, void* const* out, int mem);

/* The contact line of a drop sitting on the bottom wall, from the current populations
 * (the normalised contact-radius histories of Sec. 7.2, Fig. 11, are radius / its initial
 * value): on each of the first two lattice rows the crossings of phi = level are placed
 * by linear interpolation between the outermost nodes with phi >= level and their outside
 * neighbours, and extrapolated linearly to the wall at y = -1/2.  out[0] = left and
 * out[1] = right (x in lattice units, node i at x = i), out[2] = radius = (right - left)/2,
 * all NaN when a row has no node with phi >= level or the drop crosses the periodic seam
 * (the span reaches x = 0 or x = nx - 1).  Host array of 3 doubles; synchronises the
 * stream.  Errors: EHD_ERR_INVALID_ARG (null pointer, a lattice without walls in y or
 * with fewer than 2 rows, a slab, level outside (0, 1)). */
int ehd_contact_line(ehd_sim* sim, double level, double* out);

/* Debugging (no counterpart in the paper): in the index-checking build
 * (libehd_checked.so, `python -m paper_2407_01654_gb300.build --checked`) the kernels test
 * every index they form from lattice coordinates, for the population, potential,
 * history and phi fields, against the field's size, and count and clamp any out of
 * range; *count receives this simulation's count since it was created.  In the normal
 * build nothing is counted and *count is 0.  Synchronises the stream.
 * Errors: EHD_ERR_INVALID_ARG (null pointer). */
int ehd_diag_index_errors(ehd_sim* sim, unsigned* count);

/* Complete state (populations, potential distribution, lagged quantities, step counter)
 * as an opaque host blob: ehd_state_bytes gives its size; ehd_save_state fills `buf`;
 * ehd_load_state restores it into a simulation with the same parameters, after which the
 * run continues bit for bit as if it had not been interrupted. */
int ehd_state_bytes(const ehd_sim* sim, size_t* bytes);
int ehd_save_state(ehd_sim* sim, void* buf, size_t bytes);
int ehd_load_state(ehd_sim* sim, const void* buf, size_t bytes);

/* Kernel timing (ehd_kernel_times): ehd_profile(sim, 1) clears the totals and starts
 * recording, ehd_profile(sim, 0) stops; ehd_profile_read synchronises the stream and
 * returns the totals since profiling was turned on.  Profiled graph steps synchronise the
 * stream after each step. */
int ehd_profile(ehd_sim* sim, int enable);
int ehd_profile_read(ehd_sim* sim, ehd_kernel_times* out);

/* Potential solve that allocates nothing, for callers that cannot allocate device
 * memory: code held to a device-memory budget by someone else, callers that carve every
 * buffer out of their own pool up front, or plug-ins running in a process whose
 * allocator they do not own.  It needs no ehd_sim; it runs the potential sub-iteration
 * loop (the library's streaming potential kernel's arithmetic, the parameters' stopping
 * rule or fixed count) for the given phi and q and returns the converged populations.
 * The paper has no counterpart: it is a deployment variant of the solve, not a step of
 * the method.
 *   params   lattice, permittivities, walls, wall potentials (ramp fraction at
 *            start_step), neutralize_charge and the potential-loop rule; the paper's
 *            scheme only (potential_scheme other than EHD_SCHEME_IMPROVED:
 *            EHD_ERR_INVALID_ARG);
 *   phi, q   device float32 [ny][nx], read only;
 *   h        device float32 [8][ny][nx]: h_1..h_8 in, the solved populations out;
 *   h_work   device float32 [8][ny][nx], overwritten (the loop alternates between the two);
 *   stream   cudaStream_t (NULL: default stream); the call synchronises it.
 * Its only scratch (per-CTA FP64 partial sums and the loop control) is a fixed device
 * array inside the library: a lattice is accepted when its tiling into 32 x 16 tiles has
 * at most 4096 tiles, ceil(nx / 32) * ceil(ny / 16) <= 4096 (at most 2,097,152 nodes);
 * other lattices return EHD_ERR_TOO_LARGE before any work is queued.  The first call on each device
 * looks the array up (with that device current) and should come before any stream
 * capture.  All calls share the array: calls that overlap on the GPU race and must be
 * serialised by the caller.  No cudaMalloc, cudaFree or other allocating routine is
 * called. */
int ehd_potential_solve_noalloc(const ehd_params* params, const float* phi, const float* q,
                                float* h, float* h_work, void* stream, int* iters,
                                double* rel_change);

/* Diagnostics (no counterpart in the paper): arms the next potential solve of a
 * simulation on the on-chip loop so that its grid barrier never completes.  Every CTA's
 * bounded wait then runs out after 2 s, the kernel returns early and the call reports
 * EHD_ERR_TIMEOUT; nothing faults or hangs.  It exists to exercise that failure path in
 * tests.  The simulation's state is invalid afterwards.  EHD_ERR_INVALID_ARG when the
 * simulation does not use the on-chip loop. */
int ehd_diag_expire_barrier(ehd_sim* sim);

/* Measurement helper (no counterpart in the paper): the shared-memory bandwidth of the
 * current device in bytes per second (loads plus stores, all SMs, 16-byte conflict-free
 * accesses, best of four timed launches after one warm-up), the ceiling of the on-chip
 * potential loop's per-node data movement.  Queues its launches on `stream` (NULL:
 * default stream) and synchronises it.  Allocates no device memory.
 * Errors: EHD_ERR_INVALID_ARG (null pointer), EHD_ERR_CUDA. */
int ehd_diag_smem_bandwidth(void* stream, double* bytes_per_second);

/* Measurement helper (no counterpart in the paper): the synchronisation floor of the
 * two-step on-chip potential loop on an nx x ny lattice, in seconds per cycle (one cycle =
 * two sub-iterations).  One cooperative launch of 64 x 56 tiles, 896 threads each, runs
 * the loop's exchange without its arithmetic: each cycle a tile writes its two-node-wide
 * band (464 nodes x 8 populations, FP32) to global memory, meets every tile at a grid
 * barrier (release add, acquire poll; each wait bounded at 2 s) and reads the two-node-wide
 * ring (496 nodes x 8 populations) from its eight neighbours' bands (periodic in x and y).
 * The figure is the difference of the best times of 1088 and 64 cycles over the extra
 * 1024, so the launch and start-up are left out.  Queues its launches on `stream` (NULL:
 * default stream), synchronises it, and allocates and frees its own device buffer (about
 * 30 KB per tile); not for use during stream capture.
 * Errors: EHD_ERR_INVALID_ARG (null pointer; fewer than 3 tiles in x or y);
 * EHD_ERR_TOO_LARGE (more tiles than the device holds at once); EHD_ERR_TIMEOUT (a
 * barrier wait ran out); EHD_ERR_CUDA. */
int ehd_diag_grid_exchange(void* stream, int nx, int ny, double* seconds_per_cycle);

/* Releases the simulation (and its workspace if the library allocated it). */
void ehd_destroy(ehd_sim* sim);

/* ---------------------------------------------------------------------------------------
 * Serving: many simulations resident on one GPU, advanced together.
 *
 * A batch owns a device-memory arena of hbm_budget bytes (allocated by the library, or
 * given by the caller as `arena`, 256-byte aligned).  Each admitted request is a slot: a
 * simulation whose workspace is carved from the arena.  ehd_batch_run advances every live
 * slot by nsteps coupled steps with one CUDA graph per step in which the potential loops of
 * all slots share ONE cooperative launch (a tile work-list across slots); each slot keeps
 * its own stopping rule and reaches exactly the state it would reach alone.  After the
 * steps, each slot's relative L2 change of phi and of u since the previous run call is
 * measured; a slot is steady when both are below steady_tol, or when phi's is and the
 * flow is at rest (RMS speed below 1e-6 lattice units).  Requests that arrive while
 * others run are admitted between run calls as slots and memory free up (continuous
 * batching); the scheduling policy is the caller's.
 * --------------------------------------------------------------------------------------- */
typedef struct ehd_batch ehd_batch;

typedef struct ehd_slot_status {
  int32_t slot;
  int32_t live;
  int64_t request_id;        /* the caller's id given at admission                     */
  int64_t steps;             /* steps made since admission                             */
  int64_t poisson_iters;     /* potential sub-iterations since admission               */
  int32_t steady;            /* 1: both relative changes below steady_tol              */
  int32_t capped;            /* 1: steps reached the batch's step cap                  */
  int32_t status;            /* status of the last run for this slot                   */
  int32_t pad;
  double rel_change_phi;     /* relative L2 change of phi over the last run call       */
  double rel_change_u;       /* relative L2 change of u over the last run call (a flow
                                slower than 1e-6 lattice units counts as rest)         */
} ehd_slot_status;

typedef struct ehd_batch_info_t {
  int32_t live_slots, max_slots;
  size_t arena_bytes, arena_used;
  int32_t tiles_used, tile_capacity;  /* on-chip tiles of the shared potential launch   */
  int64_t steps_run;
  int64_t kernel_launches;            /* kernels launched by run calls                  */
  int32_t tile_rows;                  /* the schedule: tile height of every slot and    */
  int32_t steps_per_graph;            /* steps per captured graph                       */
} ehd_batch_info_t;

/* Creates a batch.  max_slots >= 1; hbm_budget >= 1 MiB; steady_tol > 0; step_cap >= 1.
 * Errors: EHD_ERR_INVALID_ARG, EHD_ERR_NOMEM, EHD_ERR_CUDA (no cooperative launch). */
int ehd_batch_create(size_t hbm_budget, int max_slots, double steady_tol, int64_t step_cap,
                     void* arena, void* stream, ehd_batch** out);
/* Admits a request (host double fields [ny][nx], as ehd_set_fields).  EHD_ERR_BUSY when no
 * slot, arena space or on-chip tile capacity is free; the batch is then unchanged.
 * EHD_ERR_INVALID_ARG for the conventional potential scheme (batches run the paper's) and
 * for poisson_loop = EHD_LOOP_STREAM.  A batch runs every slot's potential loop on chip
 * with one sub-iteration per exchange, whatever on-chip loop params asks for (every loop
 * gives the same states); params' tile_rows is replaced by the batch's. */
int ehd_batch_admit(ehd_batch* b, const ehd_params* params, const double* phi, const double* q,
                    const double* ux, const double* uy, int64_t request_id, int* slot);
/* The batch's schedule (no counterpart in the paper; a launch choice): every slot's
 * potential loop tiles 64 x tile_rows (16, 32 or 64; default 32) and run calls launch
 * captured graphs of steps_per_graph steps (even, 2..64; default 16).  Changes nothing in
 * the results of a request.  Only while no slot is live (EHD_ERR_BUSY otherwise);
 * EHD_ERR_INVALID_ARG for other values. */
int ehd_batch_set_schedule(ehd_batch* b, int tile_rows, int steps_per_graph);
/* Advances every live slot by nsteps steps, then measures steadiness and statistics
 * (synchronises the stream). */
int ehd_batch_run(ehd_batch* b, int nsteps);
/* Status of the live slots: up to `max` entries into `out`, their number into *n. */
int ehd_batch_poll(ehd_batch* b, ehd_slot_status* out, int max, int* n);
/* Fields of a live slot, as ehd_read_fields. */
int ehd_batch_read_fields(ehd_batch* b, int slot, unsigned mask, void* const* out, int mem);
/* Ends a slot (finished, cancelled or capped) and frees its arena space. */
int ehd_batch_retire(ehd_batch* b, int slot);
int ehd_batch_info(ehd_batch* b, ehd_batch_info_t* info);
void ehd_batch_destroy(ehd_batch* b);

/* ---------------------------------------------------------------------------------------
 * Slab decomposition of one lattice: the coupled step of Algorithm 1 computed by nslabs
 * bands of consecutive rows, each with its own device buffers (one ghost row below and
 * one above), exchanging what crosses each cut -- after the moments pass one row of phi and
 * of the potential coefficients each way, after every potential sub-iteration the 8
 * potential populations of the boundary rows, after the coupled pass the 9 populations
 * (3 directions of g, l and f) pushed across -- and combining the global sums (the
 * stopping rule's, and the FP64 sums of phi and q) in a fixed slab order, so every slab
 * takes the same stopping decision.  It is the layout of a lattice spread over several
 * devices, not a step of the method; here every slab lives on the current device and the
 * exchange is a gather kernel between the slabs' buffers.  With a fixed sub-iteration
 * count the fields equal the single-lattice run's bit for bit (except a neutralised
 * source, whose mean charge is summed in another order); with the stopping rule the
 * combined sums round differently, so a decision within rounding of the tolerance can
 * differ.  FP32 storage only; the streaming potential loop.
 * --------------------------------------------------------------------------------------- */
typedef struct ehd_slabs ehd_slabs;

/* Splits params' lattice into nslabs slabs of ny / nslabs rows (the remainder spread over
 * the slabs), 1 <= nslabs <= 64 and <= ny, on `stream`.  The library allocates every
 * buffer.  Errors: EHD_ERR_INVALID_ARG (also for FP16 storage), EHD_ERR_UNSTABLE_PARAMS,
 * EHD_ERR_NOMEM, EHD_ERR_CUDA. */
int ehd_slabs_create(const ehd_params* params, int nslabs, void* stream, ehd_slabs** out);
/* As ehd_set_fields, host double arrays [ny][nx] of the whole lattice (p nullable). */
int ehd_slabs_set_fields(ehd_slabs* t, const double* phi, const double* q, const double* ux,
                         const double* uy, const double* p);
/* As ehd_step (the statistics are those of the whole lattice); synchronises the stream. */
int ehd_slabs_step(ehd_slabs* t, int nsteps, ehd_stats* stats);
/* As ehd_read_fields to host double arrays [ny][nx] of the whole lattice. */
int ehd_slabs_read_fields(ehd_slabs* t, unsigned mask, double* const* out);
/* Bytes crossing all cuts per potential sub-iteration and per step (the rest of the
 * exchange), as a multi-device run would send them.  Either pointer may be NULL. */
int ehd_slabs_exchange_bytes(const ehd_slabs* t, size_t* per_sub_iteration, size_t* per_step);
void ehd_slabs_destroy(ehd_slabs* t);

/* Static description of a status code. */
const char* ehd_error_string(int code);

/* Library version string. */
const char* ehd_version(void);

/* sizeof(ehd_params) and sizeof(ehd_stats) as compiled into the library, so that a
 * binding can check its own struct layouts.  Either pointer may be NULL. */
int ehd_abi_sizes(size_t* params_bytes, size_t* stats_bytes);

#ifdef __cplusplus
}
#endif
#endif /* EHD_H */
