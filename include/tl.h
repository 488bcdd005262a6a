/*
 * tl.h -- C ABI of the GB300 (sm_103a) library for the fine-level transient
 * heat solve of the spatiotemporal two-level method for laser powder bed
 * fusion (Viguerie, Carraturo, Reali, Auricchio; arXiv:2110.12932).
 *
 * The paper's Algorithm 1 (Section 4) advances a coarse global temperature
 * T+ with macro steps Dt and a fine local temperature T- on a patch that
 * follows the laser with m micro steps dt = Dt/m:
 *
 *   for each macro step n:
 *     tl_coarse_step(p, TL_PREDICT)   predictor T~+ at t_n + Dt
 *     tl_fine_substeps(p, m)          m solves of the time-local problem
 *                                     Eq. (localProblemTime)
 *     tl_restrict(p)                  fine -> coarse injection
 *     tl_coarse_step(p, TL_CORRECT)   corrected T+ at t_n + Dt
 *
 * Every solve is one backward-Euler step of the heat equation Eq.
 * (thermalEqn) (Section 2.1, latent heat optional) on a uniform mesh of
 * trilinear hexahedra, with conductivity and heat capacity evaluated at the
 * element-mean temperature of the step's start (lagged), a powder/solid/
 * melted element state, and a preconditioned conjugate gradient solve
 * (tensor-product mass preconditioner by default, Jacobi on request) run
 * entirely on the GPU.
 *
 * Ownership: the library owns every device buffer of a problem; host
 * buffers passed to getters belong to the caller.  Calls are ordered on the
 * configured CUDA stream; getters and tl_sync synchronise it.  No call
 * aborts or leaves the device waiting: every device-side wait has a time
 * limit and failures are reported through tl_status.  A handle is not
 * thread-safe; distinct handles are independent.
 */
#ifndef TL_H
#define TL_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct tl_problem tl_problem;

typedef enum {
  TL_OK = 0,
  TL_EINVAL = -1,   /* invalid configuration or argument                     */
  TL_ENOMEM = -2,   /* a device allocation failed                            */
  TL_ENOCONV = -3,  /* a CG solve reached max_iter; that step left T unchanged */
  TL_ESTATE = -4,   /* call out of order (see the loop above)                */
  TL_ECUDA = -5,    /* a CUDA runtime call failed                            */
  TL_ETIMEOUT = -6  /* a device-side grid barrier exceeded its time limit    */
} tl_status;

typedef enum { TL_FP64 = 0, TL_FP32_REFINED = 1 } tl_precision;
typedef enum { TL_PREDICT = 0, TL_CORRECT = 1 } tl_phase;
typedef enum { TL_COARSE = 0, TL_FINE = 1 } tl_level;

/* One straight laser track on the top surface z = Lz, traversed from
 * (x0, y0) to (x1, y1) at `speed` m/s.  Tracks run back to back from t = 0;
 * the laser is off after the last one (Section 5.2-5.3 scan paths). */
typedef struct { double x0, y0, x1, y1, speed; } tl_track;

/* Problem description (SI units).  The plate is [0,Lx]x[0,Ly]x[0,Lz], z up,
 * held at T_bottom on z = 0 and adiabatic elsewhere apart from the laser.
 * The coarse mesh has NXc x NYc x NZc hexahedra.  The fine patch covers
 * pNXc x pNYc x pNZc coarse elements at the top surface, each refined r
 * times per direction; its origin sits on a coarse node and follows the
 * laser (Section 5.2).  Material (Section 2.2 with linear laws):
 * rho c(T) = rho (c0 + c1 (T - Tref)), k(T) = k0 + k1 (T - Tref), times
 * powder_factor for POWDER elements.  An element is POWDER initially iff its
 * centroid lies within powder_depth of the top surface; after each solve it
 * becomes MELTED if its mean temperature exceeds T_melt, else stays POWDER
 * if it was, else SOLID. */
typedef struct {
  double Lx, Ly, Lz;
  int NXc, NYc, NZc;
  int pNXc, pNYc, pNZc;   /* 1 <= pN*c <= N*c                                  */
  int r;                  /* space refinement ratio, >= 1                      */
  int m;                  /* time ratio: micro steps per macro step, >= 1      */
  double dt_coarse;       /* macro step Dt [s]                                 */
  double T0, T_bottom;    /* initial temperature, bottom Dirichlet value [K]   */
  double rho, c0, c1, k0, k1, Tref;
  double powder_depth, powder_factor, T_melt;
  double P, eta, radius;  /* laser power [W], absorptivity, radius R [m]       */
  const tl_track* path;   /* ntracks tracks, copied at creation                */
  int ntracks;
  /* coarse-level source: 0 = the surface analogue of the paper's distributed
   * source Q+ (Section 5.2): intensity eta P / (R v Dt) on the R-wide
   * rectangle swept during the macro step (tracks must be axis-aligned);
   * 1 = the fine-level Gaussian at t_n + Dt. */
  int coarse_source;
  /* Dirichlet weight of micro step i on gamma_D: 0 -> w = (i+1)/m (the solve
   * produces time t_n + (i+1) dt); 1 -> the printed w = i/m. */
  int bc_weight_literal;
  int energy;             /* 1: accumulate the energy account of every solve   */
  tl_precision precision; /* TL_FP64, or FP32 inner CG with FP64 defect correction */
  double tol;             /* relative residual of each solve (FP64 measure)    */
  double tol_inner;       /* relative residual of each FP32 inner solve        */
  int max_iter;           /* CG iteration cap per solve (inner cap when refined) */
  /* refined path, tiling of the FP32 inner CG: 0 = chosen per solve from the
   * elements each block of the grid (or batch slice) gets (wide from 1024),
   * 1 = element tiles of up to 16 x 8 x ez with the vector update fused into
   * the apply (one grid barrier per iteration; small meshes), 2 = wide tiles
   * of up to 64 x 4 x ez with a separate streaming update (two barriers per
   * iteration; large meshes).  Ignored by TL_FP64. */
  int inner_tiles;
  /* iterated two-level coupling at the correction step (the local and global
   * problems solved in turn until they agree): after the correction, the last
   * micro step is solved again from its start with the corrected coarse field
   * in place of the predictor in its Dirichlet data, injected, and the
   * correction redone from T+^n, until max|T+ change| <= coupling_tol max|T+|
   * or coupling_sweeps corrections were made.  coupling_sweeps <= 1: the
   * plain one-pass correction.  Not available in batches. */
  int coupling_sweeps;
  double coupling_tol;
  /* preconditioner of the CG solves: 1 = Jacobi; 2 = the Jacobi-scaled
   * tensor product of the 1D approximate inverses I - 0.2 L of the consistent
   * mass (L = neighbour sum per direction): 2.5-2.7 x fewer iterations on
   * these mass-dominated steps for one extra pass per iteration; 0 = the
   * default, the same as 2 */
  int precond;
  /* latent heat (Eq. thermalEqn's chi rho d f_pc / dt term) as an apparent
   * heat capacity: rho c(T) becomes rho (c(T) + latent f_pc'(T)) with the
   * sigmoid f_pc(T) = (1 + tanh(pc_sharpness (T - Tm))) / 2,
   * Tm = (T_solidus + T_liquidus) / 2, so f_pc' = (pc_sharpness / 2)
   * (1 - tanh^2(pc_sharpness (T - Tm))) (Eq. 2dPhaseChange of Section 5.1
   * read as this derivative).  latent = 0 [J/kg]: no latent heat.  Both
   * levels use it.  Requires latent >= 0 and, when latent > 0,
   * pc_sharpness > 0 [1/K] and T_liquidus >= T_solidus [K]. */
  double latent, T_solidus, T_liquidus, pc_sharpness;
  /* Picard iterations per backward-Euler step (the nonlinear step with the
   * coefficients evaluated at the new temperature): 0 or 1 = coefficients
   * lagged at the step's start (one solve); K > 1 = K solves per step, solve
   * k taking its coefficients from the element means of solve k-1's result
   * (states stay those of the step's start; only the last solve updates the
   * states and the energy account).  At most 50; not available in batches
   * nor with coupling_sweeps > 1. */
  int picard_iters;
  /* heat loss through the top surface (Section 3.1): convection
   * h_conv (T - T_amb) [W/(m^2 K)] on the top of both levels, radiation
   * sigma_SB emissivity (T^4 - T_amb^4) on the top of the fine patch (the
   * local domain); h_conv = emissivity = 0: adiabatic top.  Backward Euler
   * with the radiation written as h_rad (T - T_amb),
   * h_rad = sigma_SB emissivity (T*^2 + T_amb^2)(T* + T_amb) per top face at
   * the face mean of the temperature the coefficients are taken at (T^k, or
   * the Picard iterate: exact at the fixed point); the consistent surface
   * mass of the bilinear face hats.  Requires h_conv >= 0,
   * 0 <= emissivity <= 1, T_amb > 0 [K] when either is on, and the tensor
   * preconditioner (precond 0 or 2). */
  double h_conv, emissivity, T_amb;
  /* time limit [s] of every device-side grid barrier wait; 0 = 1 s, at most
   * 60 s.  A wait that runs out ends the launch at that barrier in every
   * block (no block passes a barrier that another left), records
   * TL_ETIMEOUT and leaves the problem's fields and states as the last
   * complete solve left them. */
  double barrier_timeout;
  /* 1: time candidate tilings of each level with at least 65,536 nodes at
   * creation and keep the fastest (cached per mesh shape in the process;
   * results then depend on the pick only through the FP32 summation order);
   * 0: cost models only. */
  int autotune;
  /* how the correction step receives the fine solution: 0 = restriction
   * (the fine values injected at the coarse nodes that coincide with free
   * fine nodes, held as Dirichlet data of the coarse step); 1 = the flux
   * jump of the alternate global problem (Section 3, Eq. globalPbmAlternate):
   * tl_restrict forms G_I = int_gamma (kappa_+ - kappa_-) dT-/dn phi_I dA over
   * the patch faces immersed in the plate from the fine field at the end of
   * the macro step (kappa_- the fine element's conductivity there, kappa_+
   * the coarse element's just outside the patch), and the correction solves
   * the coarse step with only the plate's own boundary conditions and G added
   * to its load.  1 requires coupling_sweeps <= 1 and keeps the problem out
   * of batches. */
  int interface_coupling;
  void* stream;           /* cudaStream_t to run on; NULL = legacy default     */
  /* optional device allocator: both NULL -> cudaMalloc / cudaFree; blocks
   * must be 16-byte aligned (else tl_create_problem returns TL_EINVAL) */
  void* (*alloc)(size_t bytes, void* stream, void* ctx);
  void (*free)(void* ptr, void* stream, void* ctx);
  void* alloc_ctx;
} tl_config;

/* Counters and energy account (J) since creation.  stored = sum_e rho c_e
 * int_e (T^{k+1} - T^k), laser = dt sum_i F_i, flux = dt * (sum of the
 * Dirichlet-row reactions), loss = dt * (heat through the top surface,
 * int_top h (T^{k+1} - T_amb)); per solve stored = laser + flux - loss up to
 * the solver tolerance (discrete energy identity). */
typedef struct {
  int64_t macro_steps, substeps;
  int64_t cg_iters_fine, cg_iters_coarse;    /* all inner CG iterations        */
  int64_t outer_iters_fine, outer_iters_coarse; /* defect-correction sweeps (refined) */
  int64_t solves_fine, solves_coarse;       /* solves run (picard_iters per step) */
  int32_t max_iters_fine, max_iters_coarse;  /* largest per-solve inner count  */
  int32_t origin[3];                         /* patch origin, coarse node index */
  int64_t patch_moves;
  int64_t launches;                          /* kernels launched by this handle */
  double energy_fine_stored, energy_fine_laser, energy_fine_flux;
  double energy_coarse_stored, energy_coarse_laser, energy_coarse_flux;
  double time;                               /* simulated time t_n [s]         */
  int64_t coupling_resolves;                 /* extra corrections of the iterated coupling */
  double energy_fine_loss, energy_coarse_loss;  /* top-surface losses (0 with an adiabatic top) */
} tl_stats;

/* Validate *cfg, allocate and initialise (T = T0 on both levels, states by
 * the powder rule, patch origin for the laser position at Dt/2).  *out is
 * set to NULL on error.  Errors: TL_EINVAL (sizes, ratios, non-positive
 * properties, a non-axis-aligned track with coarse_source 0), TL_ENOMEM,
 * TL_ECUDA. */
tl_status tl_create_problem(const tl_config* cfg, tl_problem** out);

/* TL_PREDICT: move the patch for the laser position at t_n + Dt/2 (overlap
 * nodes keep their values, new nodes take the trilinear interpolant of T+^n;
 * Section 5.2: no projection), then solve the coarse backward-Euler step
 * T+^n -> T~+ (Algorithm 1, predictor).  TL_CORRECT: solve the same step
 * again with the injected nodes as Dirichlet data -> T+^{n+1}, update the
 * coarse states, advance n (Algorithm 1, correction step).
 * Errors: TL_ESTATE out of order, TL_EINVAL bad phase. */
tl_status tl_coarse_step(tl_problem* p, tl_phase phase);

/* Solve the next nsub micro steps of the current macro step, Eq.
 * (localProblemTime): Dirichlet data (1-w) I(T+^n) + w I(T~+) on the patch
 * faces interior to the plate, adiabatic patch faces on the plate's sides,
 * T_bottom on the plate's bottom, surface Gaussian source
 * q = 3 eta P/(pi R^2) exp(-3 rho^2/R^2) at the laser position at the end
 * of the micro step.  Errors: TL_ESTATE (no predictor yet, or more than m
 * micro steps in this macro step), TL_EINVAL (nsub < 0). */
tl_status tl_fine_substeps(tl_problem* p, int nsub);

/* Inject the fine temperature into the coarse nodes that coincide with free
 * fine nodes (Algorithm 1, correction input), or, with interface_coupling 1,
 * form the interface load of the flux-jump coupling.  Errors: TL_ESTATE
 * unless all m micro steps of the macro step are done. */
tl_status tl_restrict(tl_problem* p);

/* Convenience: nmacro full macro steps (predict, m micro steps, restrict,
 * correct), then a stream synchronisation; returns the first error. */
tl_status tl_macro_steps(tl_problem* p, int nmacro);

/* Synchronise the stream and return the first device-side error recorded
 * since creation (TL_ENOCONV, TL_ETIMEOUT) or TL_OK. */
tl_status tl_sync(tl_problem* p);

/* Number of nodes of a level (coarse: (NXc+1)(NYc+1)(NZc+1); fine:
 * (r pNXc+1)(r pNYc+1)(r pNZc+1)), or 0 for a bad argument. */
size_t tl_node_count(const tl_problem* p, tl_level level);

/* Copy a level's nodal temperature (x fastest, then y, then z) into the
 * caller's host buffer of exactly n doubles; origin_out (may be NULL)
 * receives the patch origin in coarse node indices.  Synchronises the
 * stream.  Errors: TL_EINVAL (n mismatch, NULL buffer), TL_ECUDA. */
tl_status tl_get_temperature(const tl_problem* p, tl_level level, double* host_out,
                             size_t n, int origin_out[3]);

/* Copy element states (0 POWDER, 1 SOLID, 2 MELTED): coarse, NXc*NYc*NZc;
 * fine, the patch's r pNXc * r pNYc * r pNZc elements; x fastest.
 * Synchronises.  Errors: TL_EINVAL, TL_ECUDA. */
tl_status tl_get_state(const tl_problem* p, tl_level level, uint8_t* host_out, size_t n);

/* Copy the counters (synchronises). */
tl_status tl_get_stats(const tl_problem* p, tl_stats* out);

/* Tilings a level's solves use: out[0..2] element tiles (ex, ey, ez),
 * out[3..5] wide tiles of the refined inner CG (0 when not used), out[6..8]
 * the preconditioner pass's node tiles (columns x, rows y, layers z),
 * out[9] the cooperative grid, out[10] 1 if the autotuner chose them.
 * Errors: TL_EINVAL. */
tl_status tl_get_tiling(const tl_problem* p, tl_level level, int32_t out[11]);

/* Phase timeline of the most recent solve on a level: *n_out pairs
 * (marker, device time in ns) are recorded, the first min(n, cap) are copied
 * to host_out[2*i], host_out[2*i+1].  Markers: 0 start, 1 coefficients /
 * boundary data / load done, 2 right-hand side applies done, 3 initial
 * residual done, 4 end of a CG pass, 5 refined: inner start, 6 refined: FP64
 * correction apply done, 7 refined: outer sweep done, 8 update start, 9 end,
 * 10 block 0 finished its share of a CG pass's apply (before the reduction);
 * value markers, whose second word holds the IEEE bits of a double instead of
 * a time: 11 <r,r> after a CG pass, 12 the recurrence term that stopped a CG
 * on a non-positive value; 13 the vector-update phase of a CG iteration done
 * (grid barrier passed); 14 / 15 block 0 starts / finished its share of that
 * update phase; 16 the preconditioner phase of a CG iteration done (grid
 * barrier passed); 17 / 18 / 19 block 0 has done its share of the setup's
 * element coefficients / Dirichlet increments / laser-load tables; 20 / 21
 * block 0 has done its share of the states and stored energy / Dirichlet
 * reactions at the end of the solve.
 * Synchronises.  Errors: TL_EINVAL, TL_ECUDA. */
tl_status tl_trace_last_solve(const tl_problem* p, tl_level level, uint64_t* host_out, size_t cap,
                              size_t* n_out);

/* ---- Batched jobs (many independent problems in one persistent kernel) ---
 * A batch advances several problems together.  Each round is one cooperative
 * launch of one persistent kernel in which every active problem performs the
 * next launches_per_round solves of its own Algorithm 1 sequence (predictor
 * with the patch motion fused in, fine micro steps, corrector with the
 * restriction fused into its boundary data) back to back on its own slice of
 * the grid: slices are sized in proportion to the round's element counts,
 * and each problem keeps its own buffers, barrier words and reductions, so
 * problems meet only at the end of a round and results match the problem run
 * alone up to rounding (the slice changes the summation order).  The job
 * table of a round is built on the host and copied from pinned memory.
 * Problems join and leave only between macro steps; while in a batch their
 * work runs on the batch's stream.  The paper has no batching; it remarks that
 * the method is embarrassingly parallel (Section 5.3). */
typedef struct tl_batch tl_batch;

/* max_jobs: at most this many active problems (<= 512, and at most the number
 * of co-resident blocks).  Errors: TL_EINVAL, TL_ENOMEM, TL_ECUDA. */
tl_status tl_batch_create(void* stream, int launches_per_round, int max_jobs, tl_batch** out);

/* Add a problem for macro_steps more macro steps; *id_out gets its job id.
 * Errors: TL_ESTATE (not between macro steps), TL_ENOMEM (batch full),
 * TL_EINVAL (a problem with coupling_sweeps > 1, picard_iters > 1 or
 * interface_coupling 1: batched sequences run one solve per step and the
 * one-pass restriction correction). */
tl_status tl_batch_add(tl_batch* b, tl_problem* p, int macro_steps, int* id_out);

/* Enqueue one round (asynchronous after a synchronisation with the previous
 * round); *active_out (may be NULL) gets the number of jobs in its first
 * launch. */
tl_status tl_batch_round(tl_batch* b, int* active_out);

/* Synchronise and report (and remove from the batch) up to cap jobs that
 * finished their macro steps or whose solve failed in a round (a failed job
 * leaves at once; tl_sync on its problem returns the failure); their problems
 * return to their own streams. */
tl_status tl_batch_poll(tl_batch* b, int* ids, int cap, int* n_out);

/* Active jobs and launches (rounds) so far; either pointer may be NULL. */
tl_status tl_batch_info(const tl_batch* b, int* active, long long* launches);

void tl_batch_destroy(tl_batch* b);

/* ---- Single step without device allocation ------------------------------
 * The paper has no counterpart to this entry point; it serves callers that
 * may not allocate device memory while they run (a host application whose
 * allocator owns the whole GPU, a real-time loop that forbids allocation
 * after set-up, a plugin that is handed only its input and output buffers).
 *
 * tl_box_step_noalloc performs one backward-Euler step of the heat equation
 * (the solve behind every tl_fine_substeps micro step) on the whole plate
 * [0,Lx]x[0,Ly]x[0,Lz] meshed with nx*ny*nz hexahedra: T_bottom on z = 0,
 * adiabatic sides and top, the surface Gaussian centred on (xc, yc) when
 * laser_on, coefficients and powder factor from T_in and *state, states
 * updated in place after the solve.  It allocates nothing: the caller passes
 * device pointers to T_in and T_out ((nx+1)(ny+1)(nz+1) doubles, x fastest;
 * they may be the same buffer) and state (nx*ny*nz bytes, read and written);
 * all scratch comes from one fixed device array inside the library, sized for
 * at most TL_NOALLOC_MAX_NODES nodes (about 19.2 MB, held on every GPU that
 * loads the library until the process exits).
 *
 * The first call on a device looks up that array's device address (once per
 * device, with the device current); make that first call before any stream
 * capture.  Every call shares the one array, so calls that overlap on the GPU
 * (other threads, other streams) race and corrupt each other: serialise them.
 * The call runs on `stream` (a cudaStream_t, NULL = legacy default stream),
 * synchronises it and returns the solve's status: TL_OK, TL_ENOCONV (T_out and
 * state left untouched), TL_ETIMEOUT, TL_ECUDA, or TL_EINVAL for NULL pointers,
 * non-positive sizes or properties, or more than TL_NOALLOC_MAX_NODES nodes.
 */
#define TL_NOALLOC_MAX_NODES 65536

typedef struct {
  double Lx, Ly, Lz;      /* plate [m]                                          */
  int nx, ny, nz;         /* hexahedra per direction                            */
  double dt, T_bottom;    /* step [s], bottom Dirichlet value [K]               */
  double rho, c0, c1, k0, k1, Tref, powder_factor, T_melt;  /* as in tl_config */
  double P, eta, radius;  /* laser power [W], absorptivity, radius R [m]        */
  double xc, yc;          /* laser centre at the end of the step [m]            */
  int laser_on;           /* 0: no source                                       */
  double tol;             /* relative CG residual                               */
  int max_iter;           /* CG iteration cap                                   */
} tl_box_step_desc;

tl_status tl_box_step_noalloc(const tl_box_step_desc* d, const double* T_in, double* T_out,
                              uint8_t* state, void* stream);

/* ---- Checkpoint / resume -------------------------------------------------
 * At a macro-step boundary (before PREDICT) the whole state of a problem is:
 * the coarse field T+^n, the fine patch field and its origin, the coarse
 * element states and the plate-wide fine state map, the macro-step index, and
 * the counters / energy account.  tl_checkpoint_save copies it into a
 * caller-owned host buffer of tl_checkpoint_size bytes (an opaque format tied
 * to this library build); tl_checkpoint_load puts it into a problem created
 * from the same configuration, after which the run continues bit-identically
 * to one that never stopped.  Both synchronise the problem's stream.
 * Errors: TL_EINVAL (NULL, wrong size, a buffer from another configuration or
 * build), TL_ESTATE (not between macro steps, or an earlier device failure),
 * TL_ECUDA. */
tl_status tl_checkpoint_size(const tl_problem* p, size_t* bytes);
tl_status tl_checkpoint_save(const tl_problem* p, void* host_out, size_t bytes);
tl_status tl_checkpoint_load(tl_problem* p, const void* host_in, size_t bytes);

/* Release every device buffer of the problem; NULL is ignored. */
void tl_destroy_problem(tl_problem* p);

/* Static description of a status code. */
const char* tl_status_string(tl_status s);

#ifdef __cplusplus
}
#endif

#endif /* TL_H */
