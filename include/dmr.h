/*
 * dmr.h -- C ABI of the GB300 dynamic-mesh-refinement (DMR) EM-plasma library.
 *
 * The library advances the 2D TE EM-plasma fluid model of Ghosh & Chaudhury
 * (arXiv 2105.13276) on one coarse Yee mesh plus one growing fine rectangle:
 *   - Eqs. 1-3 (Sec. II.A): Yee FDTD E/H update in scattered-field form with the
 *     cold-plasma electron current J = -e n v, first-order Mur outer boundary
 *     (Sec. II.B, Fig. 1 caption);
 *   - Eq. 4 (Sec. II.A): electron continuity with nu_i(E_eff/p), effective
 *     diffusion and recombination, once per EM period (Sec. III.C);
 *   - Sec. III.C: r fine sub-steps per coarse step, coarse->fine transfer by
 *     Eq. 5b (coarse-fine boundary) and Eq. 5a (new fine area), fine->coarse;
 *   - Sec. III.A-III.D: threshold / gradient flags and rectangle growth.
 *
 * Conventions (all entry points):
 *   - Every call returns a dmr_status (0 = success) and never aborts;
 *     dmr_last_error() gives a message.
 *   - The caller owns all device memory.  dmr_create() receives one device
 *     buffer of dmr_workspace_bytes() bytes and carves every array out of it;
 *     the library never calls cudaMalloc.  The fine arrays are sized for
 *     patch_cap_cells fine cells up front; growth beyond that is DMR_ECAPACITY.
 *   - Work is queued on the CUDA stream given to dmr_create().  Calls return
 *     after queuing, except where stated (reads to host memory, dmr_stats, and
 *     the once-per-period rectangle decision inside dmr_advance, which reads
 *     16 bytes of flag bounding box back to the host).
 *   - Units are SI; positions are metres from the lower-left domain corner.
 *   - Arrays read or written through the ABI are dense, row-major with y as
 *     the row index and x contiguous:
 *       Ex, vx       : (ny+1) rows x nx       at ((i+1/2)d, j d)
 *       Ey, vy       : ny rows x (nx+1)       at (i d, (j+1/2)d)
 *       Hz           : ny rows x nx           at ((i+1/2)d, (j+1/2)d)
 *       NE, S2, ERMS : (ny+1) rows x (nx+1)   at nodes (i d, j d)
 *       MASK         : (ny+1) rows x (nx+1)   uint8 flags on the coarse nodes
 *     with (nx, ny) the cell counts of the mesh read (coarse, or the current
 *     fine rectangle).  Elements are double for precision 0 and float for
 *     precision 1, except S2 (always double) and MASK (uint8).
 */
#ifndef DMR_H
#define DMR_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct dmr_ctx dmr_ctx;

typedef enum {
  DMR_OK = 0,
  DMR_EINVAL = -1,     /* bad argument or configuration */
  DMR_ECAPACITY = -2,  /* workspace too small or patch beyond patch_cap_cells */
  DMR_ECUDA = -3,      /* a CUDA call failed (message has the CUDA error) */
  DMR_EUNSTABLE = -4,  /* stability guard: Courant, diffusion number, NaN or w_p dt >= 2 */
  DMR_ETIMEOUT = -5,   /* a bounded device wait gave up */
  DMR_ESTATE = -6      /* call not valid in the current state */
} dmr_status;

/* DMR_FIELD_ERMS is the output E_rms(x, y, t) of Sec. II.B / IV at the nodes
 * (read only): within a period the RMS of the total field over the samples
 * taken since the period began (levels after its first, through the present
 * E level), E_rms^2 = S2 / q for q samples; at a period boundary the E_rms of
 * the period just completed, E_rms^2 = S2 / N over its N samples (the value
 * E_eff was taken from), with area the rectangle gained at that boundary
 * filled from the coarse mesh by Eq. 5a. */
typedef enum {
  DMR_FIELD_EX = 0, DMR_FIELD_EY = 1, DMR_FIELD_HZ = 2, DMR_FIELD_VX = 3,
  DMR_FIELD_VY = 4, DMR_FIELD_NE = 5, DMR_FIELD_S2 = 6, DMR_FIELD_MASK = 7,
  DMR_FIELD_ERMS = 8
} dmr_field;

typedef enum {
  DMR_STAT_T = 0,            /* simulated time (s) */
  DMR_STAT_R = 1,            /* refinement region R(t) = fine cells / (r^2 coarse cells), Sec. III.C */
  DMR_STAT_FINE_CELLS = 2,   /* fine cells of the rectangle */
  DMR_STAT_NE = 3,           /* electrons per metre of depth (FP64 composite trapezoid total) */
  DMR_STAT_PABS = 4,         /* period-mean absorbed power per metre of depth (W/m), FP64 */
  DMR_STAT_WABS = 5,         /* absorbed energy per metre of depth since start (J/m), FP64 */
  DMR_STAT_PERIODS = 6,      /* completed EM periods (continuity steps) */
  DMR_STAT_COARSE_STEPS = 7, /* completed coarse EM steps */
  DMR_STAT_NMAX = 8,         /* largest coarse-node density at the last period end */
  DMR_STAT_FLAGS = 9,        /* flagged coarse nodes at the last period end */
  DMR_NSTATS = 10
} dmr_stat;

/*
 * Run description.  Negative values of De, Da, beta_rec, Te, nu_scale, n_th,
 * g_th and patch_cap_cells select the defaults given in brackets.
 */
typedef struct dmr_config {
  int32_t nx, ny;            /* coarse cells along x and y (>= 4 each) */
  int32_t r;                 /* refinement factor (Sec. III.C); 1 = uniform mesh, no patch.
                                Note: the coarse-fine coupling (Eq. 5b into the fine
                                sides, the fine mean back into the coarse E) has a
                                slowly growing mode (spectral radius 1.0005-1.0045 per
                                coarse step in vacuum, more at r = 4 than r = 2 on some
                                shapes).  Collisional plasma damps it in the benchmark
                                runs; long r = 4 runs can end in DMR_EUNSTABLE.  With
                                coupling = 1 (below) the coupled step has no growing
                                mode. */
  int32_t n_lambda;          /* coarse cells per wavelength: dx_c = lambda / n_lambda */
  int32_t steps_per_period;  /* N_T coarse EM steps per period: dt_c = 1/(f N_T);
                                Courant c dt/dx = n_lambda/N_T must be <= 1/sqrt(2) */
  int32_t precision;         /* 0: FP64 everywhere; 1: FP32 fields, FP64 E^2 sums and totals */
  int32_t buffer_cells;      /* growth buffer in coarse cells [4] */
  int32_t growth;            /* 0: the rectangle stays fixed; 1: it grows to the flags'
                                bounding box widened by buffer_cells; 2: threshold
                                lines (Sec. III.D): a side on which n > n_th at some
                                coarse node moves out by m_ex (left/right) or m_ey
                                (bottom/top) coarse cells */
  int64_t patch_cap_cells;   /* fine-cell capacity [(r nx)(r ny)] */
  double freq;               /* EM frequency f (Hz) */
  double E0;                 /* incident amplitude (V/m), E along y, incident from the left */
  double p_torr;             /* gas pressure (Torr); nu_m = 5.3e9 p (Sec. II.A) */
  double De, Da;             /* free / ambipolar diffusion (m^2/s) [0.1*760/p, De/100] */
  double beta_rec, Te;       /* r_ei = beta 1e-13 sqrt(300/Te) m^3/s (Sec. II.A) [1, 300 K] */
  double nu_scale;           /* scale s_nu of the ionization frequency [1] */
  double nu_a;               /* attachment frequency (1/s) [0] */
  double n_th;               /* threshold density (m^-3) [1e-3 n_crit] (Sec. III.A) */
  double g_th;               /* gradient threshold (m^-4) [n_th/(4 dx_c)] (Sec. III.B) */
  int32_t m_ex, m_ey;        /* growth = 2: jumps along x and y in coarse cells
                                [2 buffer_cells, buffer_cells]; the paper takes
                                m_ex > m_ey (Sec. III.B) */
  int32_t nu_model;          /* ionization frequency (Sec. II.A): 0 the air fit
                                s_nu 5.14e11 p exp(-73 (E_eff/p)^-0.44), E_eff/p in
                                V/(cm Torr); 1 the Townsend form s_nu gamma v_d with
                                gamma = A p exp(-B p/E_eff), v_d = e E_eff/(m_e nu_m) */
  double town_A, town_B;     /* nu_model = 1: A in 1/(m Torr) [1500], B in V/(m Torr)
                                [36500] (values <= 0 select the defaults) */
  int32_t boundary;          /* outer boundary of the coarse mesh: 0 first-order Mur on
                                the scattered tangential E (Fig. 1 caption); 1 CPML of
                                pml_cells cells backed by PEC (kappa = 1, cubic sigma
                                grading, sigma_max = 0.8 * 4 / (eta0 dx_c)).  With CPML
                                the fine rectangle must stay pml_cells + 2 coarse cells
                                inside the domain (set_patch: DMR_EINVAL; growth stops
                                there); adjoint and batched runs need boundary = 0 */
  int32_t pml_cells;         /* CPML thickness in coarse cells [8] (values <= 0) */
  int32_t coupling;          /* what the fine mesh gives back to the coarse mesh
                                (Sec. III.C: "fine mesh updated quantities are
                                transferred back"): 0 the fine E means into the
                                coarse E under the rectangle every coarse step and
                                the fine density into the coarse nodes every period
                                (two-way, the default); 1 the density only (one-way
                                for the fields: the coarse E under the rectangle
                                stays the coarse mesh's own; the vacuum coupled step
                                then has spectral radius 1, see the note on r) */
} dmr_config;

/* Bytes of device workspace a run of this configuration needs; 0 if the
 * configuration is invalid (dmr_last_error(NULL) says why). */
size_t dmr_workspace_bytes(const dmr_config* cfg);

/* Create a run.  dev_workspace: device buffer of at least
 * dmr_workspace_bytes(cfg) bytes, 256-byte aligned, owned by the caller and
 * kept alive until dmr_destroy.  cuda_stream: cudaStream_t (NULL = legacy
 * default stream).  All fields start at zero and the density at zero; no
 * fine rectangle exists until dmr_set_patch.  Errors: DMR_EINVAL (bad
 * config), DMR_EUNSTABLE (stability guard), DMR_ECAPACITY (buffer too small),
 * DMR_ECUDA. */
int dmr_create(const dmr_config* cfg, void* dev_workspace, size_t bytes,
               void* cuda_stream, dmr_ctx** out);

/* Release host-side state (the workspace stays the caller's). NULL is ignored. */
void dmr_destroy(dmr_ctx* ctx);

/* Message of the last failed call on ctx (ctx NULL: of the calling thread's
 * last failed dmr_workspace_bytes / dmr_create). Never NULL. */
const char* dmr_last_error(const dmr_ctx* ctx);

/* Gaussian seed n0 exp(-((x-x0)^2/sx^2 + (y-y0)^2/sy^2)) on the nodes of the
 * coarse mesh and of the fine rectangle (Sec. IV), zero where the exponent is
 * below -60; add != 0 adds it to the present density.  The fine density is
 * then copied into the coinciding coarse nodes (Sec. III.C, direct copy).
 * Queued on the stream.  Errors: DMR_EINVAL (sx or sy not > 0). */
int dmr_seed_gaussian(dmr_ctx* ctx, double n0, double x0, double y0, double sx, double sy,
                      int add);

/* Set the fine rectangle to coarse nodes [rect[0], rect[2]] x [rect[1], rect[3]]
 * (i0, j0, i1, j1; i0 < i1 <= nx, j0 < j1 <= ny).  The first call creates the
 * fine mesh with every field interpolated from the coarse mesh (Eq. 5a,
 * frac = 1); later calls must contain the current rectangle and grow it as a
 * flag-driven growth would (Sec. III.D).  Only at a period boundary.
 * Errors: DMR_EINVAL, DMR_ECAPACITY, DMR_ESTATE (r = 1 or mid-period). */
int dmr_set_patch(dmr_ctx* ctx, const int32_t rect[4]);

/* Current rectangle (all -1 when there is none). */
int dmr_get_patch(const dmr_ctx* ctx, int32_t rect[4]);

/* Advance n_coarse_steps coarse EM steps (Sec. III.C sub-cycling; a
 * continuity step, flags and growth at every period end).  Queued on the
 * stream; each period end reads the flag bounding box back (one sync).
 * Errors: DMR_ECAPACITY (growth beyond the cap; the run stops at that period
 * end with the old rectangle), DMR_EUNSTABLE (NaN or w_p dt >= 2 detected at
 * a period end), DMR_ECUDA. */
int dmr_advance(dmr_ctx* ctx, int64_t n_coarse_steps);

/* Checked mode: from the next period end on, the rectangle after period k is
 * rects[4k .. 4k+3] instead of the growth policy of Sec. III.D (a recorded
 * refinement log is replayed).  rects: host memory, 4 n_periods int32,
 * copied by the call.  n_periods = 0 switches replay off.  Errors: DMR_EINVAL
 * (NULL rects with n_periods > 0); a logged rectangle that does not contain
 * the one before, or leaves the domain, stops dmr_advance at that period end
 * with DMR_EINVAL, one beyond patch_cap_cells with DMR_ECAPACITY. */
int dmr_replay_log(dmr_ctx* ctx, const int32_t* rects, int64_t n_periods);

/* Shape (rows, cols) and element size of a field at level 0 (coarse) or 1
 * (fine rectangle), written to shape[2] and *elem_bytes (host memory;
 * elem_bytes may be NULL).  Errors: DMR_EINVAL (unknown field, NULL shape),
 * DMR_ESTATE (a level other than 0 and 1, level 1 without a rectangle, MASK
 * at level 1 or of a uniform run, r = 1). */
int dmr_field_shape(const dmr_ctx* ctx, int field, int level, int32_t shape[2],
                    int32_t* elem_bytes);

/* Copy a field into dst (dense layout above).  dst_is_device != 0: dst is
 * device memory and the copy is queued on the stream; otherwise dst is host
 * memory and the call returns when the copy is done.  bytes must be at least
 * rows*cols*elem_bytes (DMR_ECAPACITY otherwise).  Errors also: DMR_EINVAL
 * (NULL dst, unknown field), DMR_ESTATE (level as in dmr_field_shape),
 * DMR_ECUDA. */
int dmr_read(const dmr_ctx* ctx, int field, int level, void* dst, size_t bytes,
             int dst_is_device);

/* Overwrite a field (EX..NE, S2) from src (same layout).  Used to start from
 * a given state or seed map.  src_is_device as in dmr_read (a host src is
 * copied before the call returns).  Errors: DMR_EINVAL (NULL src, unknown
 * field, MASK or ERMS: derived quantities), DMR_ESTATE (level as in
 * dmr_field_shape), DMR_ECAPACITY (bytes below rows*cols*elem_bytes),
 * DMR_ECUDA. */
int dmr_write(dmr_ctx* ctx, int field, int level, const void* src, size_t bytes,
              int src_is_device);

/* Statistics (dmr_stat indices) into out[DMR_NSTATS] (host memory), after
 * waiting for the stream.  Errors: DMR_ECUDA. */
int dmr_stats(const dmr_ctx* ctx, double out[DMR_NSTATS]);

/* Capture each full period (N_T coarse steps and the period-end kernels) in a
 * CUDA graph and replay it while the rectangle is unchanged (enable = 1);
 * 0 drops the graph and launches directly.  Results are the same either way.
 * Never fails on a valid ctx. */
int dmr_set_graphs(dmr_ctx* ctx, int enable);

/* Per-kernel timing with CUDA events recorded on the run's stream around each
 * launch.  enable is a bit mask of the kernel classes to time (bit k for
 * class k; -1 for all; 0 switches timing off); each call resets the sums.
 * Classes: 0 EM step (the coarse step together with the first fine
 * sub-step), 1 later fine sub-steps (the last also writes the fine->coarse E
 * transfer into the coarse arrays), 2 kept for compatibility (no launches),
 * 3 period-end kernels, 4 growth, 5 persistent period (all EM steps of a
 * period in one launch, dmr_set_persistent).  While timing is on, EM
 * launches do not overlap (no programmatic dependent launch).
 * dmr_kernel_time returns, for a class, the summed device time in ms, the
 * number of timed launches and the algorithmic bytes those launches had to
 * move (each array element read and written once; 0 for classes 3 and 4);
 * dmr_kernel_class_name names a class (NULL past the last one).  Times are
 * collected at period ends. */
int dmr_set_timing(dmr_ctx* ctx, int enable);
int dmr_kernel_time(const dmr_ctx* ctx, int kclass, double* ms, int64_t* launches,
                    double* algorithmic_bytes);
const char* dmr_kernel_class_name(int kclass);

/* Number of kernels the library has launched (graph replays count their
 * kernel nodes), into *launches (host memory). */
int dmr_launch_count(const dmr_ctx* ctx, int64_t* launches);

/* Wait for all work queued on the run's stream.  Errors: DMR_ECUDA (a
 * failure of the queued work). */
int dmr_sync(const dmr_ctx* ctx);

/* Autotuner (at a period boundary): times the run's first EM launch of the
 * present step in its steady form (the coarse step reading the fine E under
 * the rectangle, as every step but the first after a start or growth does)
 * for five strip heights (warps-per-SM targets 8, 16, 32, 48, 96) without
 * changing the run -- 20 back-to-back copies of the launch are captured in a
 * CUDA graph and replayed, as the periods are; they write only next-level
 * buffers that the next step rewrites in full -- keeps the fastest; returns
 * the choice and the per-candidate mean launch times (ms).  With a fine
 * rectangle the choice is then made on the launches of a coarse step as
 * they run: ten coarse steps of the merged launch and fine sub-steps 2..r
 * (each reading the present fine state and writing next-level buffers; their
 * E^2 samples are kept aside and put back) per CUDA graph, programmatic
 * dependent launches in FP32, for the 16 combinations of targets {16, 32, 48,
 * 96} for the merged launch and for the fine sub-steps with launches of
 * their own; times within 1 % of the fastest count as ties, which go to the
 * higher targets (shorter strips).  In FP32 runs without CPML each
 * combination is also timed with two node columns per lane in sub-steps
 * 2..r (dmr_set_strip_columns); two must be more than 1 % faster to be
 * chosen.  *warps_per_sm returns the merged launch's choice
 * (dmr_get_launch_shape gives the whole shape). */
int dmr_autotune(dmr_ctx* ctx, int32_t* warps_per_sm, double trial_ms[5]);

/* Duration of one EM launch form of the present step (at a period boundary;
 * the run is left unchanged): reps back-to-back copies of the launch are
 * captured in a CUDA graph and replayed on the run's stream (best of three
 * timed replays), *ms_per_launch their mean.  form 0: the first launch of a
 * coarse step at a period boundary (coarse step with the first fine
 * sub-step, no E^2 sample); 1: the same launch as the other steps of a
 * period run it, with the E^2 samples of both meshes (the sums are kept
 * aside and put back); 2: the last fine sub-step alone (E^2 sample and the
 * fine->coarse transfer into the coarse arrays).  *algorithmic_bytes: the
 * bytes that launch must move (each element read and written once: 11 words
 * per node, + 16 B per node with an E^2 sample, + the coarse means).
 * Errors: DMR_ESTATE (mid-period, or form 2 without a rectangle), DMR_EINVAL. */
int dmr_time_launch(dmr_ctx* ctx, int form, int reps, double* ms_per_launch, double* algorithmic_bytes);

/* Set the strip height of all EM launches directly, as a warps-per-SM target
 * in [1, 1024] (e.g. the choice dmr_autotune made on an earlier run of the
 * same size).  Results do not depend on it.  DMR_EINVAL otherwise. */
int dmr_set_launch_shape(dmr_ctx* ctx, int32_t warps_per_sm);

/* Node columns each lane of the EM strip kernel advances in the fine
 * sub-steps 2..r of a coarse step (the ones with launches of their own): 1
 * (default) or 2.  With 2, a warp covers 60 columns and each row's loads and
 * stores are 8-byte vector accesses (16-byte for the FP64 E^2 sums).  It
 * applies to FP32 runs without CPML, not in a persistent period; the last
 * sub-step (which writes the fine->coarse means) takes it at r = 2 or 4
 * only.  Results do not depend on it, bit for bit.  dmr_autotune may change
 * it.  Errors: DMR_EINVAL (not 1 or 2), DMR_ESTATE (a run of a batch). */
int dmr_set_strip_columns(dmr_ctx* ctx, int32_t columns_per_lane);

/* The present launch shape: shape[0] the warps-per-SM target of the coarse
 * step's launch, shape[1] that of the fine sub-steps with launches of their
 * own, shape[2] the node columns per lane. */
int dmr_get_launch_shape(const dmr_ctx* ctx, int32_t shape[3]);

/* Persistent period (enable = 1; default 0): every full period that starts
 * at a period boundary runs its N_T coarse steps with their r fine sub-steps
 * (Sec. III.C sub-cycling; r <= 8) as one cooperative launch instead of two
 * launches per coarse step.  Each block of the per-step launches becomes a
 * unit of work that waits only for the units whose output it reads (its
 * neighbouring strips of the previous step; near the fine rectangle, the
 * fine sub-steps and the coarse step it is coupled with through Eq. 5b and
 * the fine->coarse transfer), so the results are the same bit for bit.
 * rows_coarse / rows_fine: node rows per warp of its coarse / fine units in
 * [1, 64], 0 to let the library choose (one unit of a step per resident
 * block where that fits).  Graph capture of a period (dmr_set_graphs)
 * captures the persistent launch.  Every wait inside the launch is bounded;
 * if one gives up, the period end returns DMR_ETIMEOUT and the run refuses
 * to advance (DMR_ESTATE) until dmr_load_state.  Errors: DMR_EINVAL (rows
 * outside [0, 64]), DMR_ESTATE (a run of a batch). */
int dmr_set_persistent(dmr_ctx* ctx, int enable, int32_t rows_coarse, int32_t rows_fine);

/* Test of those bounded waits: with stall = 1, in every later persistent
 * period one unit (the first coarse unit, at the period's second step)
 * waits for a count that nothing reaches; polls (>= 1) bounds every wait of
 * the launch.  The wait gives up after `polls` polls, the launch returns,
 * and the period end reports DMR_ETIMEOUT.  stall = 0 with polls = 4194304
 * restores the default.  Errors: DMR_EINVAL (polls < 1). */
int dmr_test_stall(dmr_ctx* ctx, int stall, int64_t polls);

/* ---- Checkpoint / resume of a run ----
 * The state of a run is everything its later steps depend on: the whole
 * workspace (fields, densities, E^2 sums, E_rms, CPML memory, totals and
 * control block) and the host-side step counter, buffer parities and fine
 * rectangle (the rectangle-growth policy of Sec. III.D and the stepping of
 * Sec. III.C continue from it exactly).  dmr_state_bytes gives the size of a
 * saved state: a 512-byte header followed by an image of the workspace.
 * dmr_save_state copies the present state (after the work already queued on
 * the stream) into dev_dst, a caller-owned device buffer (256-byte aligned),
 * and returns when the copy is done.  dmr_load_state makes the run continue
 * from a state saved by a run of the same configuration (the same context,
 * or another one created with an equal dmr_config); a saved state can be
 * loaded any number of times.  Loading keeps the run's own replay log,
 * resumes it where it stood at the save, drops captured graphs and any
 * adjoint recording.  Neither call is valid for a run of a batch
 * (DMR_ESTATE).  Errors: DMR_EINVAL (null or misaligned buffer, not a saved
 * state, other configuration), DMR_ECAPACITY (buffer too small), DMR_ECUDA. */
size_t dmr_state_bytes(const dmr_ctx* ctx);
int dmr_save_state(dmr_ctx* ctx, void* dev_dst, size_t bytes);
int dmr_load_state(dmr_ctx* ctx, const void* dev_src, size_t bytes);

/* ---- Adjoint (reverse mode) with the refinement schedule held fixed ----
 * Gradients of a loss L(n_coarse(t_end)) with respect to the incident
 * amplitude E0, the ionization scale s_nu and the initial density map of the
 * fine rectangle (the seed map; of the coarse mesh when r = 1).
 *  1. dmr_adjoint_record advances n_steps (a multiple of steps_per_period,
 *     from a period boundary) and keeps a copy of the whole workspace every K
 *     steps (K a multiple of steps_per_period) in ckpt
 *     (dmr_adjoint_checkpoint_bytes), and the rectangle after every period.
 *  2. dmr_adjoint_backward takes dL/dn at t_end (device, dense (ny+1) x
 *     (nx+1) coarse node map in the run's precision) and a device workspace
 *     of dmr_adjoint_workspace_bytes (valid after step 1).  For each segment,
 *     last first, it restores the checkpoint, recomputes the segment with the
 *     recorded rectangles while writing every step's E and v to a tape, and
 *     sweeps the tape backwards with the adjoint kernels; the recompute of
 *     the next segment (on a stream the call creates and destroys) runs
 *     while the sweep of the present one reads the other of two tapes.  The
 *     call returns after all its work is done.  It writes dL/dE0,
 *     dL/ds_nu (host doubles) and dL/d(seed map) (device, dense rows x cols of
 *     the initial fine rectangle's nodes, the run's precision).  Afterwards
 *     the run holds the state at the end of its first recorded segment.
 * The forward loss, the refinement schedule and the gradients are those of
 * the discrete scheme: flags and growth are not differentiated. */
size_t dmr_adjoint_checkpoint_bytes(const dmr_ctx* ctx, int64_t n_steps, int64_t K);
int dmr_adjoint_record(dmr_ctx* ctx, int64_t n_steps, int64_t K, void* ckpt, size_t bytes);
size_t dmr_adjoint_workspace_bytes(const dmr_ctx* ctx);
int dmr_adjoint_backward(dmr_ctx* ctx, const void* dL_dn, void* dev_workspace, size_t bytes,
                         void* ckpt, size_t ckpt_bytes, double* dL_dE0, double* dL_dnu_scale,
                         void* dL_dseed);

/* ---- Batched runs (many independent breakdown runs advanced together) ----
 * A batch holds n runs whose configurations may differ in size, E0, pressure
 * and seeds but share precision, r (1 or even) and an even steps_per_period.
 * Per coarse step one launch advances every run's coarse mesh and first fine
 * sub-step, one launch each later fine sub-step; with graphs on (default)
 * each period (EM steps of all runs, every run's continuity step, flags and
 * totals) is one CUDA graph launch, and all control blocks come back in one
 * read.  Set each run up through its borrowed context (dmr_batch_run:
 * dmr_set_patch, dmr_seed_gaussian, dmr_write, dmr_read, dmr_stats) and
 * advance only through dmr_batch_advance (DMR_ESTATE otherwise). */
typedef struct dmr_batch dmr_batch;

/* Workspace of a batch of n runs; 0 if invalid (dmr_batch_last_error(NULL)). */
size_t dmr_batch_workspace_bytes(const dmr_config* cfgs, int32_t n);

/* Create a batch in one caller-owned device buffer (256-byte aligned) on a
 * non-default stream. */
int dmr_batch_create(const dmr_config* cfgs, int32_t n, void* dev_workspace, size_t bytes,
                     void* cuda_stream, dmr_batch** out);
void dmr_batch_destroy(dmr_batch* b);

/* Context of run k (owned by the batch: dmr_destroy ignores it); NULL if k is
 * out of range. */
dmr_ctx* dmr_batch_run(dmr_batch* b, int32_t k);

/* Advance every run by n coarse steps (growth decided per run each period). */
int dmr_batch_advance(dmr_batch* b, int64_t n_coarse_steps);
int dmr_batch_set_graphs(dmr_batch* b, int enable);

/* Autotuner (at a period boundary): times the batched EM launch for five
 * strip heights (warps-per-SM targets 1, 2, 4, 8, 16) on the present
 * state without changing it (5 copies per CUDA graph replay), keeps the
 * fastest; returns the choice and the per-candidate mean launch times (ms). */
int dmr_batch_autotune(dmr_batch* b, int32_t* warps_per_sm, double trial_ms[5]);
int dmr_batch_launch_count(const dmr_batch* b, int64_t* launches);
const char* dmr_batch_last_error(const dmr_batch* b);

/* Electron total (per metre of depth) of one density map, without any
 * allocation.  The paper has no counterpart to this call: it exists for
 * callers that cannot allocate device memory at all -- a host application
 * that gives all GPU memory to its own pool and lets no plug-in call
 * cudaMalloc, code where an allocation (which synchronises the device) is not
 * allowed, or a caller with no workspace to hand over.  It computes the same
 * composite trapezoid sum as the run totals of a uniform mesh,
 *   total = dx^2 * sum_{i,j} w_i w_j n[j][i],  w = 1/2 on the first and last
 * node of each axis, 1 elsewhere,
 * for a dense (ny+1) x (nx+1) node map n_dev (double for precision 0, float
 * for precision 1) in device memory, and writes one double to total_dev
 * (device memory).  Work is queued on cuda_stream (NULL = legacy default).
 * Its scratch is a fixed array inside the library (16384 doubles, 128 KiB,
 * held on every GPU that loads the library until the process exits), so maps
 * above 67108864 nodes are rejected with DMR_ECAPACITY.  The first call in
 * each CUDA context (per device, and again after a device reset, which makes
 * a new context) looks the array's device address up with that device
 * current (cudaGetSymbolAddress); make that first call before any stream
 * capture.  Every call shares the array:
 * calls that overlap on the GPU (other streams, other threads) race; calls
 * on one stream are ordered and each rewrites the scratch it reads.  Errors:
 * DMR_EINVAL, DMR_ECAPACITY, DMR_ECUDA; dmr_noalloc_last_error() explains. */
int dmr_electron_total_noalloc(const void* n_dev, int32_t nx, int32_t ny, int32_t precision,
                               double dx, void* cuda_stream, double* total_dev);
const char* dmr_noalloc_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* DMR_H */
