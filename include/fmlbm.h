/*
 * fmlbm.h -- C ABI of the GB300 (sm_103a) fugacity-based multicomponent lattice
 * Boltzmann library (libfmlbm.so).
 *
 * The library advances N-component D2Q9 lattices with the fugacity-based
 * free-energy method of Soomro, Ayala, Peng & Ayala (arXiv:2212.10680):
 * per node, the component densities give ln f_i from a cubic EOS with van der
 * Waals mixing rules (Appendix C; density-explicit forms of Section IV,
 * Eqs. eqfugupdatePR / eqfugupdateSRK / eqfugupdateVDW), finite-difference
 * gradients of ln f_i and of sum_j kappa_ij lap(rho~_j) give the component
 * forces (Eqs. eqforcefinal, eqChemPotI2, eqkappa, eq1stder, eq2ndder), and
 * the forces drive the well-balanced multicomponent BGK update (Eqs. eqLBEMCa,
 * eqLBEMCb with rho_0 = 0, eqLBEMCfinal3) in the order of the implementation
 * procedure of Section III.B.
 *
 * Conventions used by every entry point
 * -------------------------------------
 * - Every function returns fmlbm_status; FMLBM_OK == 0.  No C++ exception ever
 *   crosses this interface.  fmlbm_status_str() names a status;
 *   fmlbm_last_error() returns a handle-owned message for the last failure on
 *   that handle (valid until the next call on it).
 * - Host arrays are owned by the caller and only read/written during the call.
 *   Field arrays are float64, C order, component-major: a field f_i(x, y) of an
 *   nx-by-ny lattice is stored at [i][y][x], i.e. index (i*ny + y)*nx + x.
 *   Vector fields (velocity, force) are [2][ny][nx] with x-components first.
 * - Distributions are exchanged as [i][a][y][x] with the D2Q9 direction order
 *   a = 0:(0,0) 1:(1,0) 2:(0,1) 3:(-1,0) 4:(0,-1) 5:(1,1) 6:(-1,1) 7:(-1,-1)
 *   8:(1,-1) (a convention of this library; the paper fixes only the lattice).
 * - The lattice is periodic in x and y.
 * - Device memory of a handle is owned by the library and released by
 *   fmlbm_destroy, except the distribution and force buffers a caller passes to
 *   fmlbm_create_with_buffers, which stay the caller's.  Work is enqueued on the CUDA stream given at creation (NULL:
 *   the legacy default stream); calls that return host data synchronise that
 *   stream.  A handle is not thread-safe: one thread at a time.
 * - Errors raised inside kernels (a node leaving the EOS domain: rho_i <= 0,
 *   rho~ b_m >= 1, or a non-finite value) are latched on the device and
 *   reported as FMLBM_E_NONPHYSICAL by the next synchronising call.
 */
#ifndef FMLBM_H
#define FMLBM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define FMLBM_MAX_COMPONENTS 4

typedef enum fmlbm_status {
    FMLBM_OK = 0,
    FMLBM_E_INVALID_ARG = 1,    /* a NULL pointer, a size out of range, an unknown enum value   */
    FMLBM_E_OOM = 2,            /* device or pinned host allocation failed                      */
    FMLBM_E_CUDA = 3,           /* a CUDA runtime call failed (message in fmlbm_last_error)     */
    FMLBM_E_NONPHYSICAL = 4,    /* a node left the EOS domain; see fmlbm_error_node             */
    FMLBM_E_TIMEOUT = 5,        /* a bounded device-side wait ran out                           */
    FMLBM_E_BUSY = 6,           /* no free slot / budget (never blocks)                         */
    FMLBM_E_NOT_CONVERGED = 7,  /* a solve reached its step limit above its tolerance           */
    FMLBM_E_UNSUPPORTED = 8     /* a valid option this build does not provide                   */
} fmlbm_status;

typedef enum fmlbm_eos { FMLBM_EOS_PR = 0, FMLBM_EOS_SRK = 1, FMLBM_EOS_VDW = 2 } fmlbm_eos;

/* Finite differences for grad and lap.  CENTRAL: the 1-D second-order central
 * differences along each axis of Eqs. eq1stder / eq2ndder.  ISOTROPIC: the D2Q9
 * weighted stencils grad h = 3 sum_a w_a e_a h(r+e_a), lap h = 6 sum_a w_a
 * (h(r+e_a) - h(r)); both coincide on fields uniform along y. */
typedef enum fmlbm_stencil { FMLBM_STENCIL_ISOTROPIC = 0, FMLBM_STENCIL_CENTRAL = 1 } fmlbm_stencil;

/* Storage and arithmetic.  FP64: distributions and all arithmetic in double.
 * FP32: float storage and arithmetic.  FP16DEV / BF16DEV: g_0 stored as float,
 * g_a (a != 0) stored as 16-bit deviations from the rest value w_a rho_0 (= 0),
 * all arithmetic in float (ln f included).  FP16DEV_LNF64 / BF16DEV_LNF64: the same
 * storage and float collide/stream arithmetic, with ln f (the mixing sums, the repulsion
 * and attraction terms of the fugacity coefficient and their logarithms; Eq.
 * eqfugupdatePR/SRK/VDW) evaluated in double from the float densities and rounded to float
 * once.  GB300 executes FP64 at about 1/64 of its FP32 rate, so the _LNF64 forms are several
 * times slower per step; they run the plain step only (no TMA or paired form) and are not
 * accepted by batches or servers (FMLBM_E_UNSUPPORTED).  Every form accumulates the
 * diagnostics sums (masses, residual) in double from 32 x 8 strips up, and exactly to about
 * 44 bits within a strip. */
typedef enum fmlbm_precision {
    FMLBM_FP64 = 0, FMLBM_FP32 = 1, FMLBM_FP16DEV = 2, FMLBM_BF16DEV = 3,
    FMLBM_FP16DEV_LNF64 = 4, FMLBM_BF16DEV_LNF64 = 5
} fmlbm_precision;

/* Which body force enters the velocity of step 1 of Section III.B.  LAGGED
 * (default): the total force sum_i F_i of the previous step, as the procedure
 * states ("body forces ... from the previous time step"); zero before the first
 * step.  CURRENT: the force of the current densities.  The forcing term of step 8
 * always uses the current force. */
typedef enum fmlbm_velocity_force { FMLBM_FORCE_LAGGED = 0, FMLBM_FORCE_CURRENT = 1 } fmlbm_velocity_force;

/* Which lattice Boltzmann formulation carries the fugacity force.  WELL_BALANCED
 * (default, the method of Section III): equilibrium of Eq. eqLBEMCb with rho_0 = 0,
 * forcing term of Eq. eqLBEMCfinal3, force of Eq. eqforcefinal.  STANDARD (Section VI):
 * the standard equilibrium rho_i w_a [1 + ...] and Guo forcing term of Eq. eqLBE per
 * component, with the force of Eq. eqForceGen (Eq. eqforcefinal + c_s^2 grad rho_i);
 * its equilibria deviate slightly from thermodynamics, more for larger density ratios.
 * STANDARD needs FP64 or FP32 storage (the 16-bit forms store deviations from the
 * well-balanced rest state), runs the plain step with 8-row tiles (no TMA form,
 * fmlbm_set_tile_height does not apply) and is not accepted by batches or servers. */
typedef enum fmlbm_formulation { FMLBM_WELL_BALANCED = 0, FMLBM_STANDARD = 1 } fmlbm_formulation;

/* A mixture at fixed temperature in consistent units (the paper's lattice units:
 * R = 1 and a = 2/49, b = 2/21 for the most volatile component, Section V).
 * a_i, b_i, alpha_i follow from Tc, Pc, omega and T by Appendix C. kij is the
 * binary interaction matrix (delta_ij of Appendix C), row-major with a fixed row
 * stride of FMLBM_MAX_COMPONENTS: kij[i*FMLBM_MAX_COMPONENTS + j]. */
typedef struct fmlbm_mixture {
    int32_t n_components;                 /* 1 .. FMLBM_MAX_COMPONENTS               */
    int32_t eos;                          /* fmlbm_eos                               */
    double R, T;                          /* gas constant, temperature               */
    double Tc[FMLBM_MAX_COMPONENTS];
    double Pc[FMLBM_MAX_COMPONENTS];
    double omega[FMLBM_MAX_COMPONENTS];   /* acentric factors                        */
    double M[FMLBM_MAX_COMPONENTS];       /* molar masses, rho~_i = rho_i / M_i      */
    double kappa[FMLBM_MAX_COMPONENTS];   /* interface strengths, Eq. eqkappa        */
    double kij[FMLBM_MAX_COMPONENTS * FMLBM_MAX_COMPONENTS];
} fmlbm_mixture;

typedef struct fmlbm_lattice {
    int32_t nx, ny;                       /* 1 .. 2^16 each, nx*ny <= 2^30            */
    double tau;                           /* BGK relaxation time, > 0.5              */
    int32_t stencil;                      /* fmlbm_stencil                           */
    int32_t precision;                    /* fmlbm_precision                         */
    int32_t velocity_force;               /* fmlbm_velocity_force                    */
    int32_t formulation;                  /* fmlbm_formulation                       */
} fmlbm_lattice;

/* Convergence criteria of batches and servers (the paper runs fixed step counts, Sections
 * V.A-V.C; a criterion is this library's).  RESIDUAL (default): the residual of
 * fmlbm_diagnostics over a check interval, ||rho(t) - rho(t - D)||_2 / ||rho(t)||_2.
 * PHASE: the change of the phase measure over a check interval,
 * max_i |lambda_i(t) - lambda_i(t - D)| with lambda_i = (1 / (nx ny)) sum_x ln rho_i(x)
 * (fmlbm_phase_measure): the volume-averaged relative change of each component's density.
 * It follows every change of the coexisting phases (their densities, compositions and
 * volumes) but not a rigid motion of the density field.  A flat or curved interface in a
 * periodic box keeps the net momentum the initial transient gave it (the discrete force sums
 * to zero only at equilibrium, and viscosity does not damp a rigid motion), so it drifts or
 * sloshes by a fraction of a node and keeps the RESIDUAL near 1e-3 while the phases no
 * longer change. */
typedef enum fmlbm_criterion { FMLBM_CRITERION_RESIDUAL = 0, FMLBM_CRITERION_PHASE = 1 } fmlbm_criterion;

typedef struct fmlbm_handle fmlbm_handle;

/* Creates a lattice: validates the mixture (Appendix C parameters) and lattice,
 * allocates its device buffers (two distribution buffers, two force buffers,
 * a density snapshot for the residual and reduction scratch) and a second stream for
 * diagnostics on the current device, and leaves it uninitialised.  cuda_stream: a cudaStream_t (may be
 * NULL), owned by the caller, must outlive the handle. */
fmlbm_status fmlbm_create(const fmlbm_mixture* mixture, const fmlbm_lattice* lattice,
                          void* cuda_stream, fmlbm_handle** out);

/* Bytes of each caller-provided buffer of fmlbm_create_with_buffers for this component
 * count and lattice (no GPU needed): g_bytes per distribution buffer (N x 9 x ny x nx
 * values of the storage type for FP64/FP32; N x 8 x ny x nx 16-bit values for the
 * deviation forms), g0_bytes per a = 0 buffer (N x ny x nx floats; 0 unless a deviation
 * form), force_bytes per stored-force buffer (2 x ny x nx doubles for FP64, floats
 * otherwise).  FMLBM_E_INVALID_ARG for an invalid lattice or component count. */
fmlbm_status fmlbm_buffer_sizes(int32_t n_components, const fmlbm_lattice* lattice, size_t* g_bytes,
                                size_t* g0_bytes, size_t* force_bytes);

/* As fmlbm_create, but the two distribution buffers g[0], g[1], the two a = 0 buffers
 * g0[0], g0[1] of the deviation forms (g0 may be NULL otherwise) and the two stored-force
 * buffers force[0], force[1] are device memory the caller owns (for example the storage of
 * framework tensors), at least as large as fmlbm_buffer_sizes gives and 16-byte aligned.
 * The handle uses them in place, in its own layout (the ping-pong buffers of the storage
 * form, not the layout fmlbm_get_distributions returns), and never frees them: they must
 * outlive the handle, and the caller must not write them while the handle's work is in
 * flight.  The six buffers must not overlap (a step reads one of each pair while it writes
 * the other).  Everything else (snapshot, reduction scratch, diagnostics stream) the handle
 * allocates itself, as fmlbm_create does.  FMLBM_E_INVALID_ARG for a NULL, host, unaligned
 * or (for non-deviation forms) superfluous g0 pointer, for memory of another GPU than the
 * current one, for overlapping buffers, and for a buffer that does not fit in the device
 * allocation containing it (a buffer carved out of a larger pool allocation is checked
 * against that allocation only). */
fmlbm_status fmlbm_create_with_buffers(const fmlbm_mixture* mixture, const fmlbm_lattice* lattice,
                                       void* cuda_stream, void* const g[2], float* const g0[2],
                                       void* const force[2], fmlbm_handle** out);

/* Fluid at rest: g_{a,i} = g^eq_{a,i}(rho_i, u = 0) (Eq. eqLBEMCb with rho_0 = 0,
 * i.e. rho_i in a = 0 and 0 elsewhere), stored force 0, step counter 0.
 * rho_host: [N][ny][nx] component MASS densities on the host, copied: free to reuse on return.
 * Page-locked memory mapped in the current context (cudaHostAlloc, cudaHostRegister) is read in
 * place by the initialisation kernel and the call waits for it (it synchronises the handle's
 * stream); other host memory is staged through a temporary device buffer from the stream-ordered
 * pool. */
fmlbm_status fmlbm_init(fmlbm_handle* h, const double* rho_host);

/* As fmlbm_init, with rho_device a device pointer of the same layout (read on
 * the handle's stream before the call's work completes; not retained). */
fmlbm_status fmlbm_init_device(fmlbm_handle* h, const double* rho_device);

/* Enqueues nsteps (>= 0) full time steps (steps 1-9 of Section III.B, one fused
 * kernel launch per step; one launch for all of them with FMLBM_VARIANT_MULTI) on the
 * handle's stream.  Asynchronous: kernel-side errors surface at the next synchronising
 * call. */
fmlbm_status fmlbm_step(fmlbm_handle* h, int64_t nsteps);

/* Macroscopic fields of the current state (steps 1-7 without collision):
 * rho [N][ny][nx] mass densities, u [2][ny][nx] the velocity of step 1 (with half
 * the force chosen by velocity_force), lnf [N][ny][nx].  Any pointer may be NULL.
 * Host outputs; synchronises. */
fmlbm_status fmlbm_moments(fmlbm_handle* h, double* rho, double* u, double* lnf);

/* Post-streaming distributions g_{a,i}(x, y, t) [N][9][ny][nx] and the stored
 * force [2][ny][nx] (either may be NULL).  Host outputs; synchronises. */
fmlbm_status fmlbm_get_distributions(fmlbm_handle* h, double* g, double* force);

/* Replaces the state with the given post-streaming distributions [N][9][ny][nx]
 * and stored force [2][ny][nx] (NULL: zero), converting to the storage precision.
 * Resets the step counter to 0 and clears the residual snapshot. */
fmlbm_status fmlbm_set_distributions(fmlbm_handle* h, const double* g, const double* force);

/* Reductions over the lattice (deterministic, fixed-order; double accumulation from each
 * 32 x 8 strip up, exact to about 44 bits within a strip):
 * mass[N] = sum_x rho_i; residual = ||rho(t) - rho(t_prev)||_2 / ||rho(t)||_2
 * where t_prev is the state of the previous diagnostics request (+inf on the first
 * request after init); step = steps taken since init.  Then snapshots rho(t).
 * Any pointer may be NULL.  Host outputs; waits for the result (equivalent to
 * fmlbm_diagnostics_async followed by fmlbm_diagnostics_wait); reports a latched
 * FMLBM_E_NONPHYSICAL. */
fmlbm_status fmlbm_diagnostics(fmlbm_handle* h, double* mass, double* residual, int64_t* step);

/* Asynchronous diagnostics (the paper has none; a convergence monitor for the time
 * loop).  fmlbm_diagnostics_async asks for the diagnostics above of the current state
 * and returns at once with a ticket (requests repeated before the next step share
 * one).  Nothing is computed yet: the next fmlbm_step computes them inside its first
 * time step, from the distributions that step reads anyway (every step variant), so a
 * loop that steps and asks
 * every step adds no extra pass over the lattice; if no step follows,
 * fmlbm_diagnostics_wait runs the separate reduction.  Results are bit-identical either
 * way.  The final sum and the copies to the host of a request served inside a step run
 * on a second, non-blocking stream of the handle at the highest stream priority, ordered
 * by events, with one set of partial sums per kept result, so the next steps do not wait
 * for them.  While the handle's stream is being captured into a CUDA graph
 * they stay on that stream and are not ordered after diagnostics work still running on
 * the second stream: call fmlbm_synchronize before capturing if requests were made.
 * fmlbm_diagnostics_wait blocks until the ticket's results have reached the host
 * (it does not wait for work enqueued after them) and returns them with the state's
 * step count; it reports a latched FMLBM_E_NONPHYSICAL or FMLBM_E_TIMEOUT as of that
 * point.  Four results are kept: a ticket older than the four most recent requests
 * has expired (FMLBM_E_INVALID_ARG), as has a request whose state fmlbm_init,
 * fmlbm_set_distributions or fmlbm_set_state replaced before it was computed. */
fmlbm_status fmlbm_diagnostics_async(fmlbm_handle* h, int64_t* ticket);
/* nsteps time steps (as fmlbm_step) with the diagnostics of every state a step reads, in one
 * call: the loop fmlbm_diagnostics_async, fmlbm_step(h, 1), and fmlbm_diagnostics_wait three
 * requests behind, run inside the library, so each step's diagnostics are computed inside the
 * step and reach the host without a host round trip per step.  mass: host [nsteps][N], residual:
 * host [nsteps] (caller-owned; row k describes the state step k reads, the values
 * fmlbm_diagnostics_async / _wait give for it).  Returns when every row has arrived; a latched
 * FMLBM_E_NONPHYSICAL or FMLBM_E_TIMEOUT is returned with the rows before it filled. */
fmlbm_status fmlbm_step_diagnostics(fmlbm_handle* h, int64_t nsteps, double* mass, double* residual);
fmlbm_status fmlbm_diagnostics_wait(fmlbm_handle* h, int64_t ticket, double* mass, double* residual,
                                    int64_t* step);

/* The phase measure of the current state: lambda[i] = (1 / (nx ny)) sum_x ln rho_i(x) for each
 * component (natural logarithm of the mass densities; a deterministic, fixed-order reduction,
 * double from each 32 x 8 strip up; float logarithms for the float storage forms).  The change of
 * lambda between two states is the PHASE convergence measure (fmlbm_criterion).  lambda:
 * host [N].  Reads the state only (the residual snapshot of fmlbm_diagnostics is not touched);
 * synchronises the handle's stream and reports a latched error. */
fmlbm_status fmlbm_phase_measure(fmlbm_handle* h, double* lambda);

/* First node that left the EOS domain since the last init (after a call returned
 * FMLBM_E_NONPHYSICAL): component, x, y. */
fmlbm_status fmlbm_error_node(fmlbm_handle* h, int32_t* comp, int32_t* x, int32_t* y);

/* Checkpoint / resume: the raw device state (distributions in storage precision,
 * stored force, step counter, a header with N, nx, ny, precision).  state_size
 * gives the byte count; get_state copies it to host memory; set_state restores a
 * state taken from a handle with the same N, nx, ny and precision.  A restored
 * run continues bit-identically to an uninterrupted one. */
fmlbm_status fmlbm_state_size(fmlbm_handle* h, size_t* bytes);
fmlbm_status fmlbm_get_state(fmlbm_handle* h, void* buf, size_t bytes);
fmlbm_status fmlbm_set_state(fmlbm_handle* h, const void* buf, size_t bytes);

/* Tuning: height (8, 16 or 32 rows) of the 32-column tile each thread block of the
 * plain fused step owns (moments always use 8 or 16).  Results do not depend on it
 * (bit-identical).  Default: 8 (the fastest measured on GB300 for two and three
 * components; taller tiles recompute less halo but keep fewer blocks per SM). */
fmlbm_status fmlbm_set_tile_height(fmlbm_handle* h, int32_t tile_y);

/* Which kernel advances the lattice.  PLAIN: the fused step with per-thread pulls from
 * global memory, one node per thread.  PAIR: the same step with two nodes per thread (32
 * columns apart in a 64-column tile) whose float arithmetic runs as packed two-lane
 * instructions; float and 16-bit storage, well-balanced formulation, 8-row tiles.  TMA: a persistent fused step whose blocks copy each wrap-free tile of
 * 32 x 8 nodes (every plane plus a 3-node halo) into shared memory with one bulk tensor
 * copy, double-buffered so the next tile's copy overlaps the current tile's arithmetic;
 * tiles on the periodic edges take the plain path.  TMA_TILE: the same copies with one
 * tile per block and a single stage, as many blocks per multiprocessor as shared memory
 * admits (the pulled values wait in shared memory).  All give bit-identical results.  The
 * TMA forms are available for FP32 and 16-bit storage with nx a multiple of 4 (FP32) or 8
 * (16-bit) and a lattice of at least 38 x 14.  AUTO (default): PLAIN, which matched or beat
 * the other forms on the workloads measured on GB300; fmlbm_autotune measures the lattice
 * at hand instead.  Every form performs the same operations per node, each rounded once,
 * and gives the same bits.  Asking for a form where it is not available returns
 * FMLBM_E_UNSUPPORTED.
 * MULTI (temporal blocking of the periodic update of Eq. eqLBEMCa, Section III.B steps 1-9):
 * the steps of one fmlbm_step call run in a single cooperative launch whose blocks stay
 * resident; a 32 x 8 tile advances to step s + 1 as soon as its 3 x 3 neighbourhood of tiles
 * has completed step s (bounded waits on per-tile step counters; a wait that runs out latches
 * FMLBM_E_TIMEOUT, reported by the next synchronising call, and the lattice state is then
 * undefined), so consecutive steps overlap and a step reads much of the previous step's
 * output from L2.  Results are bit-identical to single steps.  Available for FP32, FP16DEV
 * and BF16DEV storage with the Peng-Robinson EOS, isotropic stencils, the lagged velocity
 * reading and the well-balanced formulation; a call of one step, and the step that serves
 * a pending fmlbm_diagnostics_async request, run as single launches.  The handle keeps 8 bytes
 * of device memory per tile for the counters (allocated on first use). */
typedef enum fmlbm_step_variant {
    FMLBM_VARIANT_AUTO = 0, FMLBM_VARIANT_PLAIN = 1, FMLBM_VARIANT_TMA = 2,
    FMLBM_VARIANT_TMA_TILE = 3,  /* one tile per block, single stage */
    FMLBM_VARIANT_PAIR = 4,      /* two nodes per thread, packed float arithmetic */
    FMLBM_VARIANT_MULTI = 5      /* several steps per launch (temporal blocking) */
} fmlbm_step_variant;
fmlbm_status fmlbm_set_step_variant(fmlbm_handle* h, int32_t variant);
/* Autotuner: times steps_per_trial steps of every available kernel variant and tile
 * height on the handle's own lattice and keeps the fastest.  The trial steps are real
 * steps of the lattice (all variants give bit-identical results); synchronises.
 * Outputs (may be NULL): chosen variant, tile height, ms per step. */
fmlbm_status fmlbm_autotune(fmlbm_handle* h, int32_t steps_per_trial, int32_t* variant, int32_t* tile_y,
                            double* ms_per_step);
/* The kernel fmlbm_step will use (PLAIN, TMA, TMA_TILE, PAIR or MULTI). */
fmlbm_status fmlbm_get_step_variant(fmlbm_handle* h, int32_t* variant);

/* Bound of the device-side waits of the TMA step forms for a tile's bulk copy, in polls of
 * the copy's mbarrier (default 2^24, far beyond any copy's completion; the paper has no
 * counterpart).  A wait that runs out latches FMLBM_E_TIMEOUT, reported by the next
 * synchronising call; its block then waits, at the default bound, for every copy still in
 * flight into its shared memory and returns, so the context stays usable (the state of
 * that step is not computed: re-initialise the lattice).  0 makes the first wait of every
 * block give up at once (a test of the timeout path).  polls < 0: FMLBM_E_INVALID_ARG. */
fmlbm_status fmlbm_set_wait_limit(fmlbm_handle* h, int64_t polls);

/* Waits for the handle's streams (including its diagnostics stream) and reports latched
 * kernel errors. */
fmlbm_status fmlbm_synchronize(fmlbm_handle* h);

/* Device bytes one lattice of this shape and precision holds (for admission
 * control). */
fmlbm_status fmlbm_lattice_bytes(int32_t n_components, const fmlbm_lattice* lattice, size_t* bytes);

/* Allocation-free variant of the reductions of fmlbm_diagnostics, for callers that
 * cannot allocate device memory (a host callback or real-time loop that must not
 * block on cudaMalloc, a process whose device memory is already reserved by
 * another pool, an embedding that forbids allocation after start-up).  The paper
 * has no counterpart; it is an interface convenience of this library.
 *
 * The caller passes every buffer as a device pointer on the current device:
 *   g_device        the distributions in the library's storage layout (the buffer a
 *                   handle steps: [N][9][ny][nx] post-collision values of the last
 *                   step, so that g_a(r) = g_device[a](r - e_a); FP64 double, FP32
 *                   float; for FP16DEV/BF16DEV the 16-bit planes a = 1..8), read only;
 *   g0_device       FP16DEV/BF16DEV only: the float planes a = 0 ([N][ny][nx]); else NULL;
 *   rho_prev_device [N][ny][nx] values in the arithmetic type of the storage (double for
 *                   FP64, float otherwise): read on every call (the values are ignored
 *                   when have_prev == 0, so it may hold anything then), then
 *                   overwritten with this state's densities;
 *   out_device      N + 2 doubles written: sum rho_i for each i, sum (rho - rho_prev)^2
 *                   (0 when have_prev == 0), sum rho^2; residual = sqrt(out[N] / out[N+1]).
 * Work is enqueued on cuda_stream (NULL: legacy default stream); the call returns
 * without waiting.  It allocates nothing: its per-block partial sums live in one
 * fixed device array of 65536 doubles (512 KiB) that every GPU which loads the
 * library keeps until the process exits, so a lattice may have at most
 * 65536 / (N + 2) tiles of 32 x 8 nodes (about 4.2 million nodes for N = 2);
 * larger lattices are rejected with FMLBM_E_INVALID_ARG, as are out-of-range sizes and
 * buffers that are NULL, not device memory of the current GPU, misaligned for their
 * element type or smaller than the lattice needs.  The first call in each CUDA context
 * (each device, and again after that device's context was reset) looks up that array's
 * device address (cudaGetSymbolAddress) with the device current; make that first call
 * before capturing work into a CUDA graph.  All calls share the one array and each
 * call overwrites every entry it later reads, so nothing needs clearing; calls that
 * overlap on the GPU (on different streams) race on it and must be serialised by
 * the caller. */
fmlbm_status fmlbm_diagnostics_noalloc(int32_t n_components, int32_t nx, int32_t ny, int32_t precision,
                                       const void* g_device, const float* g0_device, void* rho_prev_device,
                                       int32_t have_prev, double* out_device, void* cuda_stream);

/* Releases all device memory of the handle.  NULL-safe. */
void fmlbm_destroy(fmlbm_handle* h);

/* ------------------------------------------------------------------------------------
 * Batches: many independent lattices of one component count and storage precision
 * (any sizes, any mixtures) in slots, advanced together by one persistent kernel per
 * time step.  Each lattice's arithmetic is that of a single-lattice plain step, so its
 * results are bit-identical to fmlbm_step on its own handle, whatever else shares the
 * batch.  fmlbm_batch_run captures chunks of steps as a CUDA graph, checks every
 * lattice's residual after each chunk and retires it once converged.  Batches are not
 * thread-safe.  The paper runs its envelope points as independent simulations
 * (Section V.B); a batch runs such sweeps side by side.
 * ------------------------------------------------------------------------------------ */
typedef struct fmlbm_batch fmlbm_batch;

/* capacity: maximum number of slots (1 .. 2^20).  cuda_stream: caller-owned stream, or
 * NULL for a stream the batch creates (graph capture needs a non-default stream). */
fmlbm_status fmlbm_batch_create(int32_t n_components, int32_t precision, int32_t capacity, void* cuda_stream,
                                fmlbm_batch** out);
/* Adds a lattice in a free slot, initialised at rest from rho_host ([N][ny][nx] mass
 * densities, copied) and active.  Its device buffers come from the stream-ordered pool.
 * FMLBM_E_BUSY when every slot is taken, FMLBM_E_OOM when memory runs out. */
fmlbm_status fmlbm_batch_add(fmlbm_batch* b, const fmlbm_mixture* mixture, const fmlbm_lattice* lattice,
                             const double* rho_host, int32_t* slot);
/* Frees a slot and its device memory (synchronises). */
fmlbm_status fmlbm_batch_remove(fmlbm_batch* b, int32_t slot);
/* Pauses (0) or resumes (1) stepping of a slot. */
fmlbm_status fmlbm_batch_set_active(fmlbm_batch* b, int32_t slot, int32_t active);
/* Enqueues nsteps steps of every active slot (asynchronous). */
fmlbm_status fmlbm_batch_step(fmlbm_batch* b, int64_t nsteps);
/* Residual and error check of every active slot (synchronises); results via
 * fmlbm_batch_slot_info.  The first check after a slot is added sets its snapshot
 * (residual +inf). */
fmlbm_status fmlbm_batch_check(fmlbm_batch* b);
/* Runs every active slot until it retires: the batch's convergence measure (fmlbm_criterion:
 * the residual, or the phase-measure change, over the last check interval) < tol at a check
 * (every check_every steps, one graph launch per chunk), a latched error, or max_steps
 * reached (FMLBM_E_NOT_CONVERGED).  Outputs per slot (arrays of capacity entries, may be
 * NULL): steps taken, last value of the convergence measure, status. */
fmlbm_status fmlbm_batch_run(fmlbm_batch* b, int64_t max_steps, int32_t check_every, double tol,
                             int64_t* steps_out, double* residual_out, int32_t* status_out);
/* The convergence measure fmlbm_batch_run compares with its tol (fmlbm_criterion; default
 * FMLBM_CRITERION_RESIDUAL).  Applies from the next retirement decision on. */
fmlbm_status fmlbm_batch_set_criterion(fmlbm_batch* b, int32_t criterion);
/* Change of the phase measure of a slot over the last check interval (+inf before a second
 * check, NaN after a latched error); every check computes it beside the residual. */
fmlbm_status fmlbm_batch_slot_phase_change(fmlbm_batch* b, int32_t slot, double* change);
/* One graph-launched chunk of steps for every active slot followed by a check (the body
 * of fmlbm_batch_run without the retirement decisions; synchronises). */
fmlbm_status fmlbm_batch_run_chunk(fmlbm_batch* b, int32_t steps);
/* Steps taken, last residual (+inf before a second check), status and activity of a slot. */
fmlbm_status fmlbm_batch_slot_info(fmlbm_batch* b, int32_t slot, int64_t* steps, double* residual, int32_t* status,
                                   int32_t* active);
/* As fmlbm_moments / fmlbm_get_distributions for one slot (host outputs; synchronises). */
fmlbm_status fmlbm_batch_moments(fmlbm_batch* b, int32_t slot, double* rho, double* u, double* lnf);
fmlbm_status fmlbm_batch_get_distributions(fmlbm_batch* b, int32_t slot, double* g, double* force);
/* Autotuner: times steps_per_trial steps of the current active slots for each tile
 * height (8, 16) and grid size (1, 2, 4, 8 blocks per multiprocessor) and keeps the
 * fastest (without it a batch runs 8-row tiles, 4 blocks per multiprocessor).  The trial steps are real steps of the lattices (the tiling does not change
 * results).  Outputs (may be NULL): chosen tile height, blocks, ms per step. */
fmlbm_status fmlbm_batch_autotune(fmlbm_batch* b, int32_t steps_per_trial, int32_t* tile_y, int32_t* blocks,
                                  double* ms_per_step);
/* Device bytes held by the batch's lattices. */
fmlbm_status fmlbm_batch_bytes(fmlbm_batch* b, size_t* bytes);
const char* fmlbm_batch_last_error(const fmlbm_batch* b);
/* Synchronises and frees everything.  NULL-safe. */
void fmlbm_batch_destroy(fmlbm_batch* b);

/* The two phases of a slot's current state, a vapour-liquid solve's answer: the molar
 * densities rho~_i = rho_i / M_i averaged over the 2 x 2 block of nodes (nodes 2bx, 2bx + 1
 * by 2by, 2by + 1, periodic at an odd edge) of largest total molar density (rho_liquid[N]) and
 * over the block of smallest (rho_vapour[N]); ties go to the lowest block index (row-major).
 * Block means, not node values: the force differences every field over two nodes (Eqs.
 * eqforcefinal, eq1stder), so a field alternating from node to node feels no force, and at
 * rest the well-balanced equilibrium (rho_0 = 0) keeps each node's mass in its rest
 * population; a checkerboard that the transient of a sharp interface excites therefore stays
 * in both bulk phases, neither sublattice is in equilibrium on its own, and the block mean
 * is the thermodynamic state.  Either pointer may be NULL.  Host outputs; synchronises the
 * batch's stream. */
fmlbm_status fmlbm_batch_phases(fmlbm_batch* b, int32_t slot, double* rho_liquid, double* rho_vapour);

/* ------------------------------------------------------------------------------------
 * Serving: vapour-liquid solves submitted as requests and run with continuous batching.
 * A worker thread owns a batch; between chunks of chunk_steps steps it admits queued
 * requests in arrival order while a slot is free and their device bytes
 * (fmlbm_lattice_bytes) fit hbm_budget_bytes, and retires each running lattice at its
 * own criterion (the configured convergence measure < tol at a check, a latched error, or
 * max_steps).  A request's
 * result does not depend on what else is running.  All server functions are
 * thread-safe and never block on the GPU.
 * ------------------------------------------------------------------------------------ */
typedef struct fmlbm_server fmlbm_server;

typedef struct fmlbm_server_config {
    int32_t n_components;      /* every request has this many components          */
    int32_t precision;         /* and this storage precision                      */
    int32_t max_slots;         /* lattices running at once                        */
    int32_t chunk_steps;       /* steps between admission / retirement decisions   */
    double tol;                /* convergence measure at which a lattice retires  */
    int64_t max_steps;         /* step limit per request (FMLBM_E_NOT_CONVERGED)  */
    size_t hbm_budget_bytes;   /* device bytes the running lattices may hold      */
    int32_t queue_capacity;    /* queued requests beyond which submit is BUSY     */
    int32_t criterion;         /* fmlbm_criterion of the retirement check          */
} fmlbm_server_config;

typedef struct fmlbm_request {
    fmlbm_mixture mixture;
    fmlbm_lattice lattice;
    const double* rho;         /* [N][ny][nx] initial mass densities, copied by submit      */
    double* rho_out;           /* NULL, or [N][ny][nx] receiving the final densities; the
                                  caller keeps it valid until the result has been polled   */
    uint64_t tag;              /* opaque, returned in the result                          */
} fmlbm_request;

typedef struct fmlbm_result {
    uint64_t id, tag;
    int32_t status;            /* FMLBM_OK (converged), FMLBM_E_NOT_CONVERGED, FMLBM_E_NONPHYSICAL, ... */
    int32_t n_components;
    int64_t steps;
    double residual;           /* last value of the server's convergence measure   */
    double t_submit, t_admit, t_done;   /* seconds on the server's steady clock */
    /* the two phases at retirement (fmlbm_batch_phases; zeros for FMLBM_E_NONPHYSICAL):
     * block-mean molar densities rho~_i at the densest and the least dense 2 x 2 block; the
     * compositions are rho~_i / sum_j rho~_j */
    double rho_liquid[FMLBM_MAX_COMPONENTS];
    double rho_vapour[FMLBM_MAX_COMPONENTS];
} fmlbm_result;

/* Creates the server on the current device (its own stream and worker thread). */
fmlbm_status fmlbm_server_create(const fmlbm_server_config* cfg, fmlbm_server** out);
/* Queues a request (copies rho).  FMLBM_E_BUSY when the queue is full (never blocks);
 * FMLBM_E_INVALID_ARG when it does not match the server or could never fit the budget. */
fmlbm_status fmlbm_server_submit(fmlbm_server* s, const fmlbm_request* req, uint64_t* id);
/* Moves up to capacity finished results into out; *n = how many.  Returns the worker's
 * error status if it stopped on a CUDA failure. */
fmlbm_status fmlbm_server_poll(fmlbm_server* s, fmlbm_result* out, int32_t capacity, int32_t* n);
/* Queue length, running lattices, admitted bytes, seconds spent in GPU chunks, and the
 * server clock now (any pointer may be NULL). */
fmlbm_status fmlbm_server_stats(fmlbm_server* s, int32_t* queued, int32_t* running, size_t* bytes_admitted,
                                double* busy_seconds, double* now_seconds);
/* Stops the worker (unfinished requests are dropped) and frees everything.  NULL-safe. */
void fmlbm_server_destroy(fmlbm_server* s);

/* ------------------------------------------------------------------------------------
 * Domain decomposition of one lattice into y-slabs.  The streaming of Eq. eqLBEMCa
 * (Section III.B, step 9) is periodic; a lattice split into slabs needs, before each step,
 * the rows of its neighbours its update reads.  The fused step reads distributions up to
 * three rows away from a node (the pulls of the 2-node halo of rho~ of steps 6-7), so each
 * slab holds its own ny / nslabs rows plus three ghost rows above and below (a lattice of
 * ny / nslabs + 6 rows stepped by the ordinary fused step), and after every step the ghost
 * rows of every distribution plane are refreshed from the neighbouring slabs' boundary rows
 * by cudaMemcpy2DAsync copies (the halo exchange; between devices these would be peer
 * copies).  The slabs' own rows then evolve bit for bit as the undivided lattice does.  All
 * slabs live on the current device and step on cuda_stream (NULL: legacy default stream).
 * ------------------------------------------------------------------------------------ */
typedef struct fmlbm_decomp fmlbm_decomp;

/* The rows [*y0, *y0 + *rows) of the global lattice that slab `slab` of `nslabs` owns (no GPU
 * needed).  FMLBM_E_INVALID_ARG unless ny is a multiple of nslabs with at least 3 rows per
 * slab. */
fmlbm_status fmlbm_decomp_slab_rows(int32_t ny, int32_t nslabs, int32_t slab, int32_t* y0, int32_t* rows);
/* Creates nslabs slab lattices of the global lattice (its nx, ny, tau, stencil, precision,
 * velocity force, formulation) for the mixture, each with its own device buffers. */
fmlbm_status fmlbm_decomp_create(const fmlbm_mixture* mixture, const fmlbm_lattice* lattice, int32_t nslabs,
                                 void* cuda_stream, fmlbm_decomp** out);
/* Fluid at rest (as fmlbm_init) from the global densities rho_host [N][ny][nx] (host, copied). */
fmlbm_status fmlbm_decomp_init(fmlbm_decomp* d, const double* rho_host);
/* nsteps time steps of every slab, each followed by the halo exchange (asynchronous). */
fmlbm_status fmlbm_decomp_step(fmlbm_decomp* d, int64_t nsteps);
/* The global post-streaming distributions [N][9][ny][nx] and stored force [2][ny][nx],
 * gathered from the slabs' own rows (either pointer may be NULL; host outputs; synchronises). */
fmlbm_status fmlbm_decomp_get_distributions(fmlbm_decomp* d, double* g_host, double* force_host);
const char* fmlbm_decomp_last_error(const fmlbm_decomp* d);
/* Frees the slabs and their buffers (synchronises).  NULL-safe. */
void fmlbm_decomp_destroy(fmlbm_decomp* d);

const char* fmlbm_status_str(fmlbm_status s);
const char* fmlbm_last_error(const fmlbm_handle* h);

/* Library version string, e.g. "fmlbm 0.1 sm_103a". */
const char* fmlbm_version(void);

#ifdef __cplusplus
}
#endif

#endif /* FMLBM_H */
