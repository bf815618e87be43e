/*
 * lc.h - C ABI of the GB300 lid-driven-cavity library.
 *
 * The library advances the two-dimensional incompressible Navier-Stokes
 * equations in vorticity / stream-function form on the unit square with a
 * moving lid, by the method of N. Cardoso and P. Bicudo, "Time dependent
 * simulation of the Driven Lid Cavity at High Reynolds Number"
 * (arXiv:0809.3098):
 *   - vorticity transport, Sec. 2, Eq. (4); stream-function Poisson
 *     equation, Eq. (3), discretised by the compact fourth-order scheme of
 *     Eq. (14) (default) or the plain 5-point Laplacian;
 *   - spatial operator L(omega), Sec. 3, Eq. (8), velocities from Eq. (22);
 *   - SSPRK(5,4) time step, Sec. 3, Eqs. (9)-(13);
 *   - psi = 0 on the walls, lid speed U, Thom's wall vorticity, Sec. 3.1,
 *     Eq. (25);
 *   - the Poisson equation is solved in every Runge-Kutta stage, warm-started
 *     from the previous solve, by multigrid V-cycles whose smoother is the SOR
 *     update of Eq. (15) in colour order (red-black for the 5-point operator,
 *     four colours (i mod 2, j mod 2) for the compact one), until
 *     ||f - L_h psi||_2 <= tol * ||f||_2 over interior nodes (checked after
 *     every cycle, at least one cycle per solve); the V-cycle ends at the
 *     first level below the fine one with at most 16 intervals, whose
 *     equation is solved exactly (option "coarse_direct");
 *   - steady-state monitors RES_psi, RES_omega, Sec. 3.2, Eqs. (26)-(27).
 *
 * Grid and layout.  N is the number of intervals per side (h = 1/N); fields
 * have (N+1) x (N+1) nodes.  Every host array exchanged through this ABI is
 * FP64, row-major, index j*(N+1) + i, with i the x index (0 = left wall,
 * N = right wall) and j the y index (0 = bottom wall, N = lid).  N must be
 * 2^k, 3*2^k, 5*2^k or 7*2^k with 8 <= N <= 8192 (multigrid halves N down
 * to 2, 3, 5 or 7 intervals).
 *
 * Time step.  One step is one SSPRK(5,4) step: five Runge-Kutta stages and
 * five Poisson solves (psi is re-solved at the end of the step so that the
 * (psi, omega) pair returned by the getters is consistent).  Wall vorticity
 * is recomputed by Thom's formula after every solve and held fixed while L is
 * evaluated; the compact right-hand side at wall-adjacent nodes uses the wall
 * vorticity of the previous solve.
 *
 * Errors.  Functions returning int return LC_OK (0) or a negative LC_ERR_*
 * code and never throw; lc_last_error() gives a message for the calling
 * thread.  A NULL, destroyed or foreign context gives LC_ERR_ARG.
 *
 * Concurrency and ownership.  A context belongs to one host thread at a time.
 * lc_step only enqueues work on the context's CUDA stream and returns; errors
 * raised on the device by that work (LC_ERR_NOCONV, LC_ERR_NONFINITE) are
 * reported by the next call that synchronises the stream (the getters,
 * lc_residual, lc_monitor, lc_synchronize, lc_save).  Host buffers are owned
 * by the caller and only read or written during the call.  Device memory is
 * owned by the library unless the caller binds its own with
 * lc_bind_workspace.
 */
#ifndef LC_H
#define LC_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

#define LC_OK 0
#define LC_ERR_ARG (-1)       /* invalid argument, NULL or destroyed context        */
#define LC_ERR_CUDA (-2)      /* a CUDA runtime call failed                          */
#define LC_ERR_NOCONV (-3)    /* a Poisson solve hit max_cycles above its tolerance  */
#define LC_ERR_NONFINITE (-4) /* NaN or Inf appeared in a residual or the state      */
#define LC_ERR_TIMEOUT (-5)   /* a bounded device-side wait (grid barrier) gave up   */
#define LC_ERR_SIZE (-6)      /* buffer too small or size out of range               */
#define LC_ERR_IO (-7)        /* checkpoint file could not be read or written        */

#define LC_OP_5PT 0     /* (delta_xx + delta_yy) psi = -omega                          */
#define LC_OP_COMPACT 1 /* Eq. (14): compact fourth-order operator (default)           */

#define LC_PREC_FP64 0  /* every kernel computes in FP64 (default)                     */
#define LC_PREC_MIXED 1 /* FP32 smoothing and stencils inside FP64 residual/refinement */

typedef struct lc_ctx lc_ctx;

/* Creates a cavity at rest: omega = 0 in the interior, psi = 0, and the lid's
 * Thom vorticity -2U/h on the top wall (U = 1).  Re > 0 is U L / nu with
 * L = 1, so nu = 1/Re (Sec. 3.2).  dt > 0 is used as given; dt <= 0 selects
 * dt = 0.25 min(h, Re h^2 / 4).  tol > 0 is the relative residual at which
 * each Poisson solve stops.  Device memory is allocated (or taken from
 * lc_bind_workspace) at the first call that needs it, on the device that is
 * current at that time.  Returns NULL on error (see lc_last_error). */
lc_ctx *lc_create(int N, double Re, double dt, double tol);

/* Releases the context, its CUDA graph, stream and any memory it allocated
 * (bound memory is left to the caller).  NULL is ignored. */
void lc_destroy(lc_ctx *ctx);

/* Enqueues nsteps >= 0 SSPRK(5,4) steps on the context's stream (one CUDA
 * graph launch per step) and returns without waiting.  If the "monitor"
 * option is 1 the monitors of lc_monitor are taken over the last of these
 * steps. */
int lc_step(lc_ctx *ctx, int nsteps);

/* Copies psi / omega, (N+1)^2 FP64 values in the layout above, into a host
 * buffer of n_elems >= (N+1)^2 elements (LC_ERR_SIZE otherwise).  Waits for
 * the stream; returns the first pending device error. */
int lc_get_psi(lc_ctx *ctx, double *host_out, size_t n_elems);
int lc_get_omega(lc_ctx *ctx, double *host_out, size_t n_elems);

/* Relative residual ||f - L_h psi|| / ||f|| at the end of the most recent
 * Poisson solve (waits for the stream).  NaN for an invalid context. */
double lc_residual(lc_ctx *ctx);

/* Message describing the last error on the calling thread ("" if none). */
const char *lc_last_error(void);

/* Sets an option; value is converted to the option's type.  Keys:
 *   "op"          LC_OP_5PT or LC_OP_COMPACT (default)       [before first use]
 *   "precision"   LC_PREC_FP64 (default) or LC_PREC_MIXED   [before first use]
 *   "nu1","nu2"   pre/post smoothing sweeps per level (2, 1), 1..16
 *   "coarse_direct" 1 (default): the V-cycle ends at the first level below
 *                 the fine one with at most 16 intervals and solves that
 *                 level's equation exactly (2-D sine transform); 0: it goes
 *                 down to the coarsest level (2, 3, 5 or 7 intervals) and
 *                 smooths it nuc times
 *   "nuc"         sweeps on the coarsest grid with coarse_direct = 0 (16), 1..256
 *   "beta"        relaxation of the SOR update, Eq. (15), in the smoother (or
 *                 the SOR solver), 0 < beta < 2; default 1.1, the value that
 *                 minimised the FP64 and mixed step times at 1024^2 (1.0:
 *                 7.44 ms, 1.05: 6.79, 1.1: 6.73 per FP64 step; 4.75 instead
 *                 of 5.64 V-cycles per solve)
 *   "max_cycles"  cycle cap per solve (100); hitting it raises LC_ERR_NOCONV
 *   "solver"      0 (default) multigrid V-cycles; 1 the paper's SOR iteration
 *                 alone: Eq. (15) swept lexicographically in the order its
 *                 n / n+1 superscripts fix (i outer, j inner), a "cycle" being
 *                 sor_sweeps sweeps followed by the stopping test.  FP64 only.
 *   "sor_sweeps"  sweeps per SOR cycle (16), 1..4096
 *   "fused"       bit mask, 0 (default): one launch per FP64 colour phase;
 *                 bit 0 (1): the fine level's colour phases of one smoothing
 *                 pass run as one cooperative launch with a bounded grid
 *                 barrier between phases; bit 1 (2): the same on the coarser
 *                 phase levels, with as few blocks as their rows need (same
 *                 values; LC_ERR_TIMEOUT if a barrier wait gave up).  On GB300
 *                 a grid barrier costs more than a launch in the step graph
 *                 (1024^2: 8.3 ms per step with 0, 9.5 with 2), so the
 *                 default is 0.
 *   "barrier_extra" test hook (0 default): 1 makes the fused smoother's grid
 *                 barrier wait for one block more than the launch has, so
 *                 every wait runs out (about 0.2 s each) and the next
 *                 synchronising call reports LC_ERR_TIMEOUT
 *   "rhs64"       mixed precision only: 1 (default) evaluates L(omega)
 *                 (Eq. (8)) in FP64 from the FP64 psi and omega; 0 evaluates it
 *                 in FP32 from their FP32 shadows (fewer bytes, but its
 *                 rounding, ~6e-8 of omega / h^2 in the viscous term, grows
 *                 past 1e-6 relative over long unsteady runs at Re >= 2e4 and
 *                 puts a floor under the steady-state monitors).  The
 *                 multigrid corrections stay FP32 either way.
 *   "U"           lid speed (1.0); re-applies Thom to the current state
 *   "profile"     0 uniform lid (default), 1 regularised lid 16x^2(1-x)^2 U
 *   "advect"      1 (default), 0 drops the transport terms of Eq. (8)
 *   "monitor"     1 computes lc_monitor's values over the last step of each
 *                 lc_step call (default 0)
 *   "blocked"     1 (default): levels above the coarse ones run as shared-
 *                 memory tile kernels (all colour phases of a level's smoothing
 *                 in one launch, halos recomputed); 0: one launch per colour
 *                 phase on every level.  FP64 only; results are identical.
 *   "fine_phases" FP64 with "blocked": the number of finest levels that run
 *                 as one launch per colour phase (no recomputed halo); the
 *                 levels between them and the coarse V-cycle run as tile
 *                 kernels.  Default 16: every level above the coarse one (on
 *                 GB300 the tiles' recomputed FP64 halo costs more than the
 *                 extra launches), 0..16.
 *   "coarse_max"  levels with at most this many intervals run as one V-cycle
 *                 in a single thread block (default -1: 32 for FP64, 64 for
 *                 mixed precision), 2..256; used where the cluster form below
 *                 is off or does not apply.
 *   "coarse_cluster" the coarse V-cycle on a thread-block cluster of this
 *                 many blocks, one per SM (-1 default: in FP64 16, else 8,
 *                 whichever the device schedules, in mixed precision off;
 *                 0 off; 2..16): its levels of more than
 *                 cluster_split intervals are split by rows over the blocks
 *                 (barrier between colour phases), the rest run in the first
 *                 block.  Same values as the one-block form.
 *   "cluster_max" the cluster form takes over from the first level below the
 *                 fine one with at most this many intervals (default -1: 128),
 *                 8..512, if its arrays fit shared memory
 *   "cluster_split" levels of at most this many intervals run in the
 *                 cluster's first block alone (16), 4..256
 *   "tile_shape"  -1 (default) picks each level's tile shape; 0..3 forces
 *                 the shared-memory tiles of 110x54, 110x22, 46x22 or 16x16
 *                 owned nodes, 4 the 44x20 register tiles held by one warp
 *                 each (mixed precision, nu1, nu2 <= 2 with the compact
 *                 operator; elsewhere a forced 4 falls back to the default).
 *   "pdl"         1 (default): the step's kernels are launched with
 *                 programmatic dependent launch (each waits for its
 *                 predecessor on entry; the launch overlaps the predecessor's
 *                 drain; 1-2% per step); 0: plain stream order.  Same values.
 *   "graph"       1 (default) replays each step as one CUDA graph whose
 *                 V-cycle loops are device-side while-nodes; 0 launches the
 *                 same kernels one by one and drives the V-cycle loop from the
 *                 host (one stream sync per cycle; for per-kernel profiling,
 *                 since kernels in graphs with conditional nodes cannot be
 *                 profiled)
 * Returns LC_ERR_ARG for an unknown key or a value out of range. */
int lc_set_option(lc_ctx *ctx, const char *key, double value);

/* Makes the context enqueue all later work on cuda_stream (a cudaStream_t,
 * e.g. torch.cuda.current_stream().cuda_stream); NULL is the legacy default
 * stream.  Until this is called the context uses a non-blocking stream of
 * its own.  Work already enqueued is ordered before work on the new stream.
 * The caller keeps the stream alive while the context uses it. */
int lc_set_stream(lc_ctx *ctx, void *cuda_stream);

/* Bytes of device memory a context of size N and precision needs (0 if the
 * arguments are invalid). */
size_t lc_workspace_bytes(int N, int precision);

/* Gives the context caller-owned device memory (256-byte aligned, at least
 * lc_workspace_bytes(N, precision) bytes) instead of allocating its own.
 * Must come before the first use of the context; the caller keeps the memory
 * alive until lc_destroy.  LC_ERR_SIZE if too small or misaligned. */
int lc_bind_workspace(lc_ctx *ctx, void *dev_ptr, size_t bytes);

/* out[0] = max |omega^{n+1} - omega^n| / dt, out[1] = RES_psi,
 * out[2] = RES_omega (Eqs. (26)-(27), with 1/N read as 1/(N+1), the points
 * per side), out[3] = V-cycles of the last Poisson solve; taken over the
 * last step of the most recent lc_step call with the "monitor" option on
 * (zeros otherwise).  Waits for the stream. */
int lc_monitor(lc_ctx *ctx, double out[4]);

/* Installs a state from host arrays ((N+1)^2 FP64 each).  psi is taken as
 * given (its walls are forced to zero); omega's interior is taken and its
 * walls are recomputed from psi by Thom's formula, Eq. (25).  The next step
 * uses psi as the solution for omega (no solve at the first stage). */
int lc_set_state(lc_ctx *ctx, const double *psi, const double *omega);

/* Checkpoint: writes / reads a binary file holding a header (magic "LCCK",
 * version, N, Re, dt, tol, U, steps taken, precision, operator) and the FP64
 * psi and omega in the host layout.  lc_load requires the same N and sets the
 * state as lc_set_state does.  LC_ERR_IO on file errors. */
int lc_save(lc_ctx *ctx, const char *path);
int lc_load(lc_ctx *ctx, const char *path);

/* Copies the V-cycle count of each Poisson solve enqueued so far (oldest
 * first, at most the last 65536) into out[0..max); *n_out receives the
 * number copied.  Waits for the stream. */
int lc_cycle_log(lc_ctx *ctx, int *out, size_t max, size_t *n_out);

/* Waits for the context's stream; returns the first pending device error. */
int lc_synchronize(lc_ctx *ctx);

/* Reads back the resolved parameters: out[0] = N, out[1] = Re, out[2] = dt,
 * out[3] = tol, out[4] = h, out[5] = levels the V-cycle visits, out[6] =
 * steps taken. */
int lc_get_params(lc_ctx *ctx, double out[7]);

/* Kernel launches the context enqueues: out[0] per step outside the Poisson
 * loops, out[1] per V-cycle of a Poisson loop (its residual norm and finisher
 * included).  A step therefore launches out[0] + out[1] * (V-cycles of its
 * five solves); lc_cycle_log gives the cycles. */
int lc_launch_stats(lc_ctx *ctx, double out[2]);

/* Roofline diagnostics: times `reps` >= 1 back-to-back launches of one kernel
 * of the step, with the arguments it has inside the step, between CUDA events
 * on the context stream.  FP64 precision: kernel 0 = fine-level smoother
 * colour phase (the colours taken in turn), 1 = fused L(omega) + stage
 * combination (stage 2), 2 = fine-level residual + full-weighting
 * restriction, 3 = one lexicographic SOR pass of sor_sweeps sweeps, 4 = the
 * fine-level pre-smoothing pass (nu1 colour sweeps in one cooperative
 * launch, LC_ERR_ARG where the device cannot launch it).  Mixed precision: 0 = fine-level FP32 tile kernel (pre-smoothing,
 * residual, restriction), 1 = L(omega) + FP64 stage combination (stage 2;
 * FP64 L with rhs64 = 1, else FP32), 2 = FP64 residual rounded to FP32,
 * 3 = fine-level FP32 tile kernel
 * (prolongation, post-smoothing, FP64 psi += e).  out[0] = mean ms per
 * launch, out[1] = algorithmic bytes per launch (each array element the
 * kernel must read or write, counted once), out[2] = FP64 and out[3] = FP32
 * floating-point operations per launch (an FMA counts two).  The launches
 * change the state: use only on a context whose state no longer matters. */
int lc_bench_kernel(lc_ctx *ctx, int kernel, int reps, double out[4]);

/* Self-test of the library's FP64 -> FP32 (round to nearest even) and
 * FP32 -> FP64 conversions done with integer instructions (the step's
 * mixed-precision kernels use them instead of the hardware conversions, which
 * on GB300 run on the FP64 unit): on the current device, n >= 0 generated
 * values (fixed edge cases, then seeded patterns: raw words, the FP32
 * exponent range, rounding ties, subnormal results) are converted both ways
 * and compared bit for bit with the hardware conversions (two NaNs compare
 * equal).  mismatches[0] / [1]: FP64 -> FP32 / FP32 -> FP64 mismatches.
 * Allocates 16 bytes of device memory for the duration of the call. */
int lc_selftest_conversions(long long n, unsigned long long seed, long long mismatches[2]);

/* ---- Batched engine ------------------------------------------------------
 * Many cavities of different sizes and Reynolds numbers advanced together:
 * each step is one CUDA graph launch whose kernels cover every cavity (a
 * table of per-cavity block ranges maps each thread block to its cavity and
 * tile).  Every cavity runs the mixed-precision step of the single-cavity
 * functions (LC_PREC_MIXED) with its own Poisson stopping rule: a cavity that
 * has converged stops iterating while the others go on, so each cavity makes
 * exactly the V-cycles it would make alone and its result is bit-identical to
 * a single-cavity context with the same options. */
typedef struct lc_batch lc_batch;

/* count (1..256) cavities; N[c] must be 2^k, 3*2^k, 5*2^k or 7*2^k in 128..8192;
 * Re[c] > 0;
 * dt may be NULL or hold dt[c] <= 0 to apply dt = 0.25 min(h, Re h^2 / 4);
 * tol as lc_create; precision must be LC_PREC_MIXED.  All cavities start at
 * rest (as lc_create).  NULL on error (lc_last_error). */
lc_batch *lc_batch_create(int count, const int *N, const double *Re, const double *dt, double tol, int precision);
void lc_batch_destroy(lc_batch *b);

/* Options as lc_set_option: "op", "coarse_max" (8..64), "coarse_direct" [before first use],
 * "nu1", "nu2" (1..4), "nuc", "beta", "max_cycles", "U", "advect", "rhs64",
 * "pdl", "graph". */
int lc_batch_set_option(lc_batch *b, const char *key, double value);
int lc_batch_set_stream(lc_batch *b, void *cuda_stream);
size_t lc_batch_workspace_bytes(int count, const int *N, int precision);
int lc_batch_bind_workspace(lc_batch *b, void *dev_ptr, size_t bytes);

/* Enqueues nsteps steps of every cavity (one graph launch per step). */
int lc_batch_step(lc_batch *b, int nsteps);

/* Copies cavity c's psi (field 0) or omega (field 1), (N[c]+1)^2 FP64 values
 * in the host layout of this header.  Waits for the stream and reports the
 * first pending device error of any cavity. */
int lc_batch_get(lc_batch *b, int cavity, int field, double *host_out, size_t n_elems);

/* Installs cavity c's state as lc_set_state does. */
int lc_batch_set_state(lc_batch *b, int cavity, const double *psi, const double *omega);

/* V-cycle counts of cavity c's solves, as lc_cycle_log. */
int lc_batch_cycle_log(lc_batch *b, int cavity, int *out, size_t max, size_t *n_out);
int lc_batch_synchronize(lc_batch *b);

/* out[0] = N, out[1] = Re, out[2] = dt, out[3] = levels the V-cycle visits, out[4] =
 * first level of the one-block coarse cycle, out[5] = steps taken, out[6] =
 * tile shape of level 0, out[7] = workspace bytes. */
int lc_batch_info(lc_batch *b, int cavity, double out[8]);

/* Autotuner: for every tile level, times `reps` launches of the batch's
 * pre- and post-smoothing tile kernels in each tile shape (0..3: shared-
 * memory tiles of 110x54, 110x22, 46x22, 16x16 owned nodes, those that fit;
 * 4: 44x20 register tiles, one per warp, where the halo fits) on the current
 * state, keeps the fastest, and writes the chosen shape per level to
 * shapes_out[0..max_levels) (-1 past the last tile level).  The tile shape
 * does not change any result (bit-identical); the state is restored. */
int lc_batch_autotune(lc_batch *b, int reps, int *shapes_out, int max_levels);

/* Smoothing-schedule autotuner: for each schedule (nu1, nu2) in (1,1), (2,1),
 * (1,2), (2,2), (3,1), (3,2) it runs one untimed and then `steps` >= 1 timed
 * steps of the whole batch from the current state (tile shapes chosen by the
 * cost model), restores the state (the workspace is snapshotted into a
 * temporary device buffer of lc_batch_workspace_bytes), and keeps the
 * schedule with the least time per step among those whose solves all
 * converged.  Every schedule solves to the same tolerance, so results change
 * only within it; the cycle counts change with the schedule.  Writes the
 * chosen (nu1, nu2) to nu_out[0..1] and sets them as options; tile shapes
 * are reset to the cost model's (call lc_batch_autotune afterwards to tune
 * them for the chosen schedule).  LC_ERR_NOCONV if no schedule converged. */
int lc_batch_autotune_schedule(lc_batch *b, int steps, int nu_out[2]);

/* Largest N accepted by lc_monitor_noalloc: the size of its fixed scratch. */
#define LC_NOALLOC_MAX_N 8192

/* Steady-state monitors of two caller-owned device states, without allocating.
 * The paper has no counterpart: this entry point exists for callers that
 * cannot call cudaMalloc (a host framework that owns all device memory
 * through its own pool, work enqueued while a CUDA graph is being captured,
 * a process with a fixed memory budget).  It computes what lc_monitor's
 * out[0..2] report: out[0] = max |omega1 - omega0| / dt, and out[1], out[2]
 * the RES_psi and RES_omega values that lc_monitor reports, over all
 * (N+1) x (N+1) nodes.
 *   psi0, psi1, omega0, omega1: device FP64 arrays of N+1 rows, element (i, j)
 *     at j*pitch + i (pitch >= N+1; pitch = N+1 is the host layout above);
 *     read only.  out: device pointer to 3 doubles, written.
 *   cuda_stream: the work is enqueued there (NULL = legacy default stream)
 *     and the call returns without waiting.
 * Its scratch (one partial per row and a block counter) is a file-scope
 * device array of about 192 KiB, sized for N <= LC_NOALLOC_MAX_N, that every
 * GPU loading the library holds until the process exits.  The first call on
 * a device looks up the array's device address (cudaGetSymbolAddress) with
 * that device current, so make the first call on each device before any
 * stream capture.  The address found is kept for the life of the device's
 * context: after cudaDeviceReset the library must be reloaded before this
 * entry point is used again on that device.  No call allocates or frees
 * memory.  All calls share the array: calls that overlap on the GPU (two
 * streams, two threads) race; calls in order on one stream are safe.  Returns LC_ERR_SIZE for
 * N > LC_NOALLOC_MAX_N, LC_ERR_ARG for NULL arrays, pitch < N+1, N < 1 or
 * dt <= 0, LC_ERR_CUDA if the set-up or the launch fails. */
int lc_monitor_noalloc(int N, const double *psi0, const double *psi1, const double *omega0,
                       const double *omega1, size_t pitch, double dt, double *out, void *cuda_stream);

#ifdef __cplusplus
}
#endif

#endif /* LC_H */
