/*
 * bbx.h - C ABI of the GB300 (sm_103a) monodomain reaction-diffusion step.
 *
 * The library (libbbx.so) advances the monodomain model of arXiv:1605.06015,
 * Eq. (monodomain), on a regular finite-difference grid:
 *
 *   dV/dt = -I_ion(V, g)/Cm + (L V) + I_stim/Cm,     dg/dt = f(g, V)
 *
 * with the anisotropic diffusion operator L of Eq. (Lu) discretised by the
 * weights W = Wbar + Wtilde of the section "Monodomain diffusion and boundary
 * conditions" (19 points in 3D, corner weights 0; 9 points in 2D, 5 when
 * isotropic), no-flux boundaries through the grid indicator psi, the
 * transversely isotropic tensor of Eq. (sigma), and the unsplit scheme of the
 * section "Computation of intermediate expressions": forward Euler, Eq.
 * (Euler), for V and the other non-gate variables, Rush-Larsen, Eq. (RL), for
 * gates.  One call of bbx_step with n_steps = 1 is one turn of the paper's
 * diff + euler/rushlarsen ring.
 *
 * Conventions for every call:
 *   - Return value: BBX_OK (0) or a negative BBX_ERR_* code.  No call throws,
 *     exits the process or traps on the GPU.  bbx_status_string() names codes.
 *   - Host arrays use the dense layout, x fastest: index x + nx*(y + ny*z),
 *     n = nx*ny*nz elements.  The caller owns every host buffer; the library
 *     copies what it needs before returning (except where stated).
 *   - Device memory owned by the library is pitched: each x-row holds
 *     px = round_up(nx, 32) elements (bbx_get_info).
 *   - Work is enqueued on the CUDA stream given at bbx_create_grid.  Calls
 *     that return data to the host synchronise that stream first, and report
 *     sticky device errors (BBX_ERR_NAN, BBX_ERR_TIMEOUT) raised by earlier
 *     asynchronous steps.
 *   - A grid handle is not thread-safe; distinct handles are independent.
 */
#ifndef BBX_H
#define BBX_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ------------------------------------------------------ */
#define BBX_OK 0
#define BBX_ERR_ARG (-1)        /* invalid argument (null pointer, size, range) */
#define BBX_ERR_CUDA (-2)       /* a CUDA runtime or driver call failed */
#define BBX_ERR_FIBRE (-3)      /* zero fibre vector at a tissue node */
#define BBX_ERR_UNSTABLE (-4)   /* dt above the explicit diffusion stability bound */
#define BBX_ERR_NAN (-5)        /* a step produced a non-finite V (sticky) */
#define BBX_ERR_TIMEOUT (-6)    /* a bounded in-kernel wait gave up (sticky) */
#define BBX_ERR_STATE (-7)      /* call out of order (e.g. step before a model) */
#define BBX_ERR_NOMEM (-8)      /* device allocation failed */
#define BBX_ERR_UNSUPPORTED (-9) /* no compiled kernel for this configuration */

/* ---- cell models (section "Cell models") ------------------------------- */
/* Parameters in order; a shorter params array keeps the remaining defaults,
 * entries past the model's list are ignored.  bbx_set_ionic_model returns
 * BBX_ERR_ARG for a non-finite parameter, FHN eps = 0, Barkley a or eps = 0,
 * and BBX_BR_FCA Kc or tau_c not positive or eps negative.
 *  BBX_FHN       2 vars (u, v).  eps=0.3 beta=0.71 gamma=0.5.  Eq. (FHN), read
 *                with the cubic u - u^3/3 (fhncub).  threshold 0.
 *  BBX_BARKLEY   2 vars (u, v).  a=0.75 b=0.02 eps=0.02.  Barkley (1991):
 *                du = u(1-u)(u-(v+b)/a)/eps, dv = u - v.  threshold 0.5.
 *  BBX_BR        8 vars (V, Ca, x1, m, h, j, d, f).  gNa=4 gNaC=0.003 ENa=50
 *                gs=0.09.  Beeler-Reuter (1977) ionic model: V and Ca by
 *                Euler, the 6 gates by Rush-Larsen.  Cm = 1 uF/cm^2, V in mV,
 *                t in ms, Ca in mol/L.  threshold -40 mV.
 *  BBX_ZFK       1 var.  alpha=0.13.  dV = V(V-alpha)(1-V), Eq. (ZFKbidomV).
 *                threshold 0.5.
 *  BBX_DIFFUSION 1 var, no reaction (the diffusion equation alone).
 *                threshold 0.5.
 *  BBX_BR_MRL    11 vars (V, Ca, x1, h, j, d, f, P0, P1, P2, P3).  Parameters
 *                and threshold as BBX_BR.  Beeler-Reuter with the sodium
 *                activation m^3 in its Markov form: Pk = probability that k of
 *                the three activation subunits are open (P3 in place of m^3),
 *                du/dt = A(V) u (Eq. markov-generic) with k -> k+1 at
 *                (3-k) alpha_m, k -> k-1 at k beta_m, advanced by the matrix
 *                Rush-Larsen scheme u_{n+1} = exp(dt A(V_n)) u_n (section
 *                "Exponential solvers"), the matrix tabulated in V from
 *                -120 to +80 mV every 0.025 mV and interpolated linearly
 *                (built on the device whenever dt changes; V outside the
 *                range takes the end entry); x1, h, j, d, f by Rush-Larsen
 *                with coefficients from the same V grid (as
 *                bbx_set_tabulation does for BBX_BR).  Unsplit Euler / Rush-Larsen
 *                only: bbx_set_scheme(BBX_SCHEME_LIE), bbx_set_solver(
 *                BBX_SOLVER_RK4) and the surrogate are refused.
 *  BBX_BR_FCA    11 vars (V, Ca, x1, m, h, j, d, Q0, Q1, Q2, Q3).  gNa=4
 *                gNaC=0.003 ENa=50 gs=0.09 Kc=5e-6 (mol/L) tau_c=2 (ms)
 *                eps=0.05 onfly=0.  threshold -40 mV.  Beeler-Reuter with the slow
 *                inward current's inactivation as a channel of two gates, the
 *                voltage gate f of the 1977 model and a calcium gate c
 *                (closed -> open at c_inf/tau_c, open -> closed at
 *                (1-c_inf)/tau_c, c_inf = 1/(1 + Ca/Kc)); Qq = probability of
 *                state q = f + 2c (gate open = 1); a direct transition
 *                (f open, c closed) -> (f closed, c open) at
 *                eps alpha_f (1 - c_inf); I_s = gs d Q3 (V - E_s).  The
 *                generator A(V, Ca) of Eq. (markov-generic) is multivariate;
 *                it is advanced as section "Exponential solvers" describes:
 *                Lie splitting into the V-univariate f gate (Rush-Larsen
 *                coefficients tabulated in V as for BBX_BR_MRL), the
 *                Ca-univariate c gate (closed form: its rates sum to 1/tau_c)
 *                and the small remainder by forward Euler, V and Ca held at
 *                their values at the start of the step.  onfly=1 instead
 *                applies exp(dt A(V_n, Ca_n)) of the whole generator at run
 *                time (the same section's step for a chain with no such
 *                decomposition: rates at the node, no table, the
 *                exponential's action by its Taylor series to nine terms on
 *                2^s substeps that bring dt/2^s |A| to 1/2, s <= 6).
 *                Unsplit Euler / Rush-Larsen only, as BBX_BR_MRL. */
#define BBX_FHN 1
#define BBX_BARKLEY 2
#define BBX_BR 3
#define BBX_ZFK 4
#define BBX_DIFFUSION 5
#define BBX_BR_MRL 6
#define BBX_BR_FCA 7

#define BBX_ACT_NONE 2147483647 /* activation map value of a node never activated */

/* Time-stepping schemes (bbx_set_scheme). */
#define BBX_SCHEME_UNSPLIT 0 /* diff + euler/rushlarsen: L enters the voltage equation */
#define BBX_SCHEME_LIE 1     /* diffstep, then euler/rushlarsen: Lie operator splitting */

/* Kinetics solvers (bbx_set_solver). */
#define BBX_SOLVER_EULER 0 /* forward Euler; Rush-Larsen for the Beeler-Reuter gates */
#define BBX_SOLVER_RK4 1   /* classical fourth-order Runge-Kutta (models given by a right-hand side) */

typedef struct bbx_grid bbx_grid;

typedef struct {
    int nx, ny, nz;          /* grid dimensions (nz = 1: 2D) */
    int px;                  /* device row pitch in elements */
    int nvars;               /* state variables of the current model (0: none) */
    int model;               /* BBX_* model id (0: none) */
    int masked;              /* 1 if a tissue mask was given */
    int anisotropic;         /* 1 if fibres were given */
    int tile_x, tile_y, tile_z; /* brick shape of the step kernel */
    long long n_bricks;      /* bricks with at least one tissue node */
    long long n_tissue;      /* tissue nodes (active cells per step) */
    long long step;          /* steps taken since the model was set */
    double t;                /* model time */
    int wsum_skipped;        /* 1: the W-tilde sums all vanish and a step does not load them */
} bbx_info;

/* Create a grid of nx*ny*nz nodes with spacing h (the paper's hx).
 * mask_host: NULL (every node is tissue) or n bytes, nonzero = tissue (the
 * .bbg status flag, section "Format of BeatBox geometry files"); nodes outside
 * the array are void.  cuda_stream: a cudaStream_t (NULL = legacy default).
 * Idle bricks (no tissue) are elided (section "Domain partitioning").
 * Allocates device memory for the mask and the brick list; the caller keeps
 * its buffer.  Errors: BBX_ERR_ARG (null out, nonpositive size or h,
 * nx*ny*nz >= 2^31), BBX_ERR_NOMEM, BBX_ERR_CUDA. */
int bbx_create_grid(bbx_grid** out, int nx, int ny, int nz, double h, const uint8_t* mask_host,
                    void* cuda_stream);

/* Fibres and diffusivities, Eq. (sigma): D = D_perp I + (D_par - D_perp) f f^T.
 * f_xyz_host: NULL (isotropic, D = D_par I) or 3*n floats, interleaved
 * (fx, fy, fz) per node as in a .bbg line.  Vectors are normalised; values at
 * void nodes are ignored.  Errors: BBX_ERR_FIBRE (zero vector at a tissue
 * node; the grid keeps its previous fibres), BBX_ERR_ARG (negative D). */
int bbx_set_fibres(bbx_grid* g, const float* f_xyz_host, double D_par, double D_perp);

/* Select the cell model and its parameters (copied).  Allocates the two
 * ping-pong state buffers (unless bound by bbx_bind_state), sets every node to
 * the model's rest state, clears the activation map, and resets t and the
 * step counter to 0.  Errors: BBX_ERR_ARG (unknown model, n_params < 0 or
 * params NULL with n_params > 0), BBX_ERR_NOMEM. */
int bbx_set_ionic_model(bbx_grid* g, int model, const double* params, int n_params);

/* Copy one state variable from the host (n = nx*ny*nz floats) into both
 * ping-pong buffers.  Synchronous.  Errors: BBX_ERR_STATE (no model),
 * BBX_ERR_ARG (var out of range, n wrong, null). */
int bbx_write_state(bbx_grid* g, int var, const float* host, size_t n);

/* All state variables at once, [var][z][y][x] (n = nvars*nx*ny*nz floats),
 * into both ping-pong buffers with one synchronisation (one host copy when
 * the rows are not padded).  Errors as bbx_write_state. */
int bbx_write_all(bbx_grid* g, const float* host, size_t n);

/* Let the caller (e.g. PyTorch) own the state: dev_a and dev_b each hold
 * bytes >= nvars*nz*ny*px*4 bytes laid out [var][z][y][x] with row pitch px,
 * 16-byte aligned.  The library never frees them.  Must follow
 * bbx_set_ionic_model; the rest state is written into both.  Errors:
 * BBX_ERR_STATE, BBX_ERR_ARG (null, misaligned, too small). */
int bbx_bind_state(bbx_grid* g, void* dev_a, void* dev_b, size_t bytes);

/* Stimulus current (section "Explicit solvers", I_eff of Eq. (ODE)): amp is
 * added to dV/dt (divided by Cm) at the nodes where region_host is nonzero,
 * on steps whose start time t_n satisfies t_on <= t_n < t_off.  region_host
 * NULL removes the stimulus.  The region is copied. */
int bbx_set_stimulus(bbx_grid* g, const uint8_t* region_host, double amp, double t_on, double t_off);

/* Activation threshold theta (k_poincare device): a node's activation step is
 * the first n+1 with V^n < theta <= V^{n+1}.  Default: the model's threshold. */
int bbx_set_threshold(bbx_grid* g, double theta);

/* Headless output, 1 byte per value (the ppmout device, section "Input and
 * output"): for every node, in the order z, y, x (x fastest), three bytes
 * (R, G, B), channel c = floor(255 t + 0.5) with t = (V_c - lo[c]) / (hi[c] -
 * lo[c]) clamped to [0, 1], evaluated in float32 with one rounding per
 * operation, V_c the current value of state variable layers[c]; layers[c] =
 * -1 gives a dark channel, void nodes are black.  out_dev: device buffer of
 * 3 nx ny nz bytes, owned by the caller.  The sample script's colour map
 * (red = u, green = v / 0.8) is layers {0, 1, -1}, lo {0, 0, 0}, hi {1, 0.8,
 * 1}.  Asynchronous on the grid's stream.  Errors: BBX_ERR_ARG (null pointers, layer out of range,
 * hi == lo or non-finite bounds), BBX_ERR_STATE (no model). */
int bbx_ppm_frame(bbx_grid* g, const int* layers, const double* lo, const double* hi, uint8_t* out_dev);

/* Phase singularities (the singz device, section "Input and output"): in every
 * z cross-section, the intersections of the isolines var_a = iso_a and var_b =
 * iso_b inside grid cells whose four corners are tissue.  An isoline crosses a
 * cell edge where V - iso is > 0 at one end only, at the linearly
 * interpolated point; a cell with exactly two crossings of each isoline holds
 * one piece of each, and their intersection, when it lies on both pieces, is
 * reported as (x, y, z) in grid units (float32).  Up to max_points points are
 * written to xyz_dev (3 floats each, device memory owned by the caller), in
 * no particular order; *n_found receives the number found (which may exceed
 * max_points).  Synchronises the grid's stream.  Errors: BBX_ERR_ARG,
 * BBX_ERR_STATE, BBX_ERR_NOMEM (its 4-byte counter, allocated on first use). */
int bbx_phase_singularities(bbx_grid* g, int var_a, double iso_a, int var_b, double iso_b, float* xyz_dev,
                            int max_points, int* n_found);

/* Resident multi-step mode for small sheets.  With on = 1, bbx_step calls of
 * two or more steps on this grid run as one launch of a cluster of 16 CTAs
 * (8 where the GPU offers no 16-CTA clusters) that keeps the whole sheet in
 * their shared memory (each CTA a band of
 * rows, the rows next to its band read from the neighbours' shared memory),
 * so a step costs neither a kernel launch nor a trip through DRAM.  Serves
 * unmasked isotropic sheets (nz = 1) of FHN, Barkley, ZFK or pure diffusion
 * with the unsplit scheme and Euler solver, up to about 200 KB of state per
 * CTA (for two variables, nx * ny up to ~260 000 with 16 CTAs).  Results agree with the
 * tiled kernel to rounding, not bitwise.  The fused total, time, step count
 * and activation map are kept as by the tiled kernel.  When the grid stops
 * qualifying (fibres, a mask, another scheme), steps go back to the tiled
 * kernel.  Errors: BBX_ERR_ARG, BBX_ERR_STATE (no model), BBX_ERR_UNSUPPORTED
 * (the grid does not qualify or does not fit), BBX_ERR_CUDA. */
int bbx_set_resident(bbx_grid* g, int on);

/* Beeler-Reuter (BBX_BR) with its Rush-Larsen coefficients tabulated in V:
 * the rushlarsen device's tabulation (section "Exponential solvers": A(V)
 * and B(V) of Eq. (RLcoeff) precomputed on a fine grid of V at start time).
 * on != 0: A and B of the six gates and the V factors of I_x1 and I_K1 come
 * from a table of V from -120 to +80 mV every 0.025 mV (FP64-built, stored
 * as float, interpolated linearly; V outside takes the end entry), rebuilt on
 * the device whenever dt changes, instead of being evaluated per node; gates
 * then advance by y' = A y + B.  on = 0: the per-node evaluation (default).
 * Results differ from the default by the interpolation error (about 1e-6
 * relative on the coefficients).  Not used by the surrogate kernels.
 * Errors: BBX_ERR_ARG, BBX_ERR_STATE (no model), BBX_ERR_UNSUPPORTED (model
 * is not BBX_BR), BBX_ERR_NOMEM, BBX_ERR_CUDA. */
int bbx_set_tabulation(bbx_grid* g, int on);

/* Skip loading W-tilde sums that vanish.  The W-tilde part of the weights
 * (Eq. (W), section "Monodomain diffusion and boundary conditions") differences
 * the diffusion tensor across each node; the library stores those sums once
 * per grid.  Where all of them are exactly 0 (fibres in the x-y plane whose
 * direction depends on z only, the paper's rotational anisotropy; uniform
 * fibres), a step of the grid on its own (not in a batch) does not read them
 * from memory: unmasked grids run a kernel variant without the W-tilde term,
 * the others use zeros in its place.  The result is bitwise the same, with
 * 12 bytes per node less to read.  on != 0: skip them where they all vanish
 * (default); on = 0: always read them.  bbx_get_info's wsum_skipped tells
 * whether the current fibres qualify.  Errors: BBX_ERR_ARG (null grid). */
int bbx_set_wsum_elision(bbx_grid* g, int on);

/* Time-stepping scheme.  BBX_SCHEME_UNSPLIT (default; section "Computation of
 * intermediate expressions"): V^{n+1} = V^n + dt (f(V^n, g^n) + L V^n +
 * I_stim), the other variables from (V^n, g^n).  BBX_SCHEME_LIE (section
 * "Operator splitting"): first V^{n+1/2} = V^n + dt L V^n alone, then the
 * kinetics step (Euler / Rush-Larsen, with the stimulus, without diffusion)
 * from (V^{n+1/2}, g^n).  Applies to the following steps, in solo and batch
 * stepping.  The Lie scheme and the RK4 solver run on 7- and 14-row tiles
 * only: a grid on 28-row tiles moves to 14.  Errors: BBX_ERR_ARG (null grid,
 * unknown scheme). */
int bbx_set_scheme(bbx_grid* g, int scheme);

/* Kinetics solver (section "Explicit solvers").  BBX_SOLVER_EULER (default):
 * forward Euler, Eq. (Euler), with Rush-Larsen gates for Beeler-Reuter.
 * BBX_SOLVER_RK4: one classical fourth-order Runge-Kutta step of the model's
 * ODE per time step, with the diffusion term and the stimulus held fixed over
 * the step (unsplit scheme) or absent (Lie scheme); for FHN, Barkley, ZFK and
 * pure diffusion.  Setting a Beeler-Reuter model resets it to Euler.  Errors:
 * BBX_ERR_ARG (null grid, unknown solver), BBX_ERR_UNSUPPORTED (RK4 for
 * Beeler-Reuter). */
int bbx_set_solver(bbx_grid* g, int solver);

/* Advance n_steps explicit steps of size dt (asynchronous on the grid's
 * stream).  Each step also reduces the new V over tissue nodes into one
 * double-precision partial per piece of its schedule (the total is summed
 * from them, in a fixed order, by bbx_step_total).  Errors: BBX_ERR_STATE (no
 * model), BBX_ERR_ARG (dt <= 0, n_steps < 0), BBX_ERR_CUDA (launch),
 * BBX_ERR_UNSTABLE when dt (4 tr D + 2 |D_par - D_perp|) > 2 h^2, tr D =
 * D_par + 2 D_perp (3 D_par when isotropic): a Gershgorin bound on the
 * spectrum of the discrete diffusion operator, above which forward Euler
 * can amplify round-off. */
int bbx_step(bbx_grid* g, double dt, int n_steps);

/* Copy one state variable to the host (n = nx*ny*nz floats).  Synchronises. */
int bbx_read_state(bbx_grid* g, int var, float* host_out, size_t n);

/* All state variables at once, [var][z][y][x] (n = nvars*nx*ny*nz floats;
 * one device-to-host copy when the rows are not padded).  Synchronises;
 * returns sticky device errors as bbx_read_state. */
int bbx_read_all(bbx_grid* g, float* host_out, size_t n);

/* Exchange the whole state with the host in one call: host_out receives the
 * current state ([var][z][y][x], n = nvars*nx*ny*nz floats) while host_in is
 * copied in as the new one, the two copies running at the same time (a
 * second stream; both host buffers should be pinned for the copies to
 * overlap).  Equal to bbx_read_all(host_out) followed by bbx_write_all(host_in),
 * for a loop that feeds new inputs and takes results every step.
 * Synchronises.  Errors as bbx_read_all / bbx_write_all, BBX_ERR_CUDA. */
int bbx_exchange_state(bbx_grid* g, const float* host_in, float* host_out, size_t n);

/* The same exchange, enqueued without waiting (a pipeline of steps fed from and
 * drained to the host: each step's copies overlap the neighbouring steps).
 * The current state (as the grid's stream will hold it when the call's work
 * runs, i.e. after every step enqueued before) goes to host_out and host_in
 * becomes the new state, through two device stages in each direction and
 * their own host-to-device and device-to-host streams; steps enqueued after
 * the call see the new state.  The host buffers must be pinned, stay valid and
 * unchanged (host_in) and unread (host_out) until bbx_exchange_wait returns;
 * the library keeps 4 x nvars x nx*ny*nz floats of stages per grid from the
 * first call on.  Grids with padded rows (nx not a multiple of 32) or 16-bit
 * gates: BBX_ERR_UNSUPPORTED (use bbx_exchange_state).  BBX_ERR_ARG, BBX_ERR_STATE,
 * BBX_ERR_NOMEM, BBX_ERR_CUDA. */
int bbx_exchange_state_async(bbx_grid* g, const float* host_in, float* host_out, size_t n);

/* Wait until every bbx_exchange_state_async of the grid has finished with its
 * host buffers.  BBX_ERR_ARG, BBX_ERR_CUDA. */
int bbx_exchange_wait(bbx_grid* g);

/* Activation steps (BBX_ACT_NONE where not activated), n int32.  Synchronises. */
int bbx_read_activation(bbx_grid* g, int32_t* host_out, size_t n);

/* Restore an activation map (checkpoint/resume).  Synchronous. */
int bbx_write_activation(bbx_grid* g, const int32_t* host, size_t n);

/* Sum of one state variable over tissue nodes (reduce device), accumulated in
 * double precision.  Synchronises. */
int bbx_total(bbx_grid* g, int var, double* out);

/* The tissue sum of V after the most recent step: the fixed-order sum of the
 * per-piece partials that step computed (a small kernel on the grid's stream
 * adds them up the first time it is asked for; deterministic).  Synchronises.
 * BBX_ERR_STATE if no step was taken; BBX_ERR_NAN if V is not finite. */
int bbx_step_total(bbx_grid* g, double* out);

/* Model time and step counter (checkpoint/resume). */
int bbx_get_time(bbx_grid* g, double* t, long long* step);
int bbx_set_time(bbx_grid* g, double t, long long step);

/* Geometry, model and brick-shape information. */
int bbx_get_info(bbx_grid* g, bbx_info* out);

/* Brick ids (bx + nbx*(by + nby*bz)) of the bricks holding tissue, in
 * increasing order, for the current brick shape.  cap: capacity of out;
 * *count receives the number of bricks.  Synchronises. */
int bbx_read_active_bricks(bbx_grid* g, int32_t* out, size_t cap, long long* count);

/* Choose the brick shape of the step kernel: tile_y in {7, 14, 28} rows of 64
 * nodes, and tile_z >= 1 planes per brick (the z-granularity at which idle
 * bricks of a masked grid are elided).  Rebuilds the brick list. */
int bbx_set_tiling(bbx_grid* g, int tile_y, int tile_z);

/* Time candidate brick shapes with CUDA events on the grid's stream (a few
 * steps each, state restored afterwards) and keep the fastest.  best_ms (may
 * be NULL) receives its time per step. */
int bbx_autotune(bbx_grid* g, double dt, double* best_ms);

/* Set the time step used by bbx_batch_step (bbx_step sets it too).  Errors:
 * BBX_ERR_STATE (no model), BBX_ERR_ARG (dt <= 0), BBX_ERR_UNSTABLE. */
int bbx_set_timestep(bbx_grid* g, double dt);

/* Storage of the Beeler-Reuter gates between steps (bbx_set_gate_storage). */
#define BBX_GATES_FP32 0    /* 32-bit floats (default) */
#define BBX_GATES_FP16 1    /* IEEE binary16, round to nearest */
#define BBX_GATES_UNORM16 2 /* 16-bit unsigned fixed point y = u / 65535, round to nearest */

/* Store the six gates of a Beeler-Reuter grid (x1, m, h, j, d, f; variables
 * 2..7) in 16 bits instead of 32 between steps: the precision path of a
 * state whose gates are fractions in [0, 1].  V and Ca stay 32-bit, every
 * operation of the step stays FP32 (the gates are decoded when the tile is
 * read, and the new values rounded to nearest when stored), so a node-update
 * moves 2 (4 + 4 + 6 x 2) bytes of state instead of 2 (8 x 4).
 * BBX_GATES_FP16 has steps of 2^-11 just below 1: a slow gate (f, j, x1)
 * whose Rush-Larsen increment per step is below half a step there stops
 * moving (at dt = 0.02 ms the cell then never repolarises);
 * BBX_GATES_UNORM16 has uniform steps of 1/65535 over [0, 1] and keeps the
 * step within the parity bars.  The current state is converted (read and
 * written back in the new layout).  Device layout with 16 bits: V and Ca
 * planes of floats, then six planes of uint16, [var][z][y][px]; buffers bound
 * by bbx_bind_state need 5 nz ny px floats.  bbx_read_state / bbx_write_state
 * and the whole-state copies convert to and from float; bbx_state_device_ptr
 * returns a uint16 plane for a gate.  With 16-bit gates the grid is stepped
 * alone (no batch), on 7- or 14-row tiles, without surrogate (the Lie scheme
 * and tabulated coefficients are kept), and bbx_total, bbx_ppm_frame and
 * bbx_phase_singularities refuse gate variables (BBX_ERR_UNSUPPORTED).  Setting a model resets the storage
 * to FP32.  Errors: BBX_ERR_ARG (mode), BBX_ERR_STATE (no model, or bound
 * buffers too small), BBX_ERR_UNSUPPORTED (not BBX_BR, or the settings
 * above), BBX_ERR_NOMEM. */
int bbx_set_gate_storage(bbx_grid* g, int mode);

/* ---- z-slab decomposition (section "Domain partitioning") --------------- */
/* The paper's parallel layer cuts the grid into subdomains that exchange a
 * one-node layer of the diffusing variable with their neighbours before
 * every step (the exchange buffers around each subdomain, figure domdec).
 * Here a grid of nz_global planes is cut along z into slabs; each slab is its
 * own bbx_grid holding its planes plus one halo plane on every side that
 * has a neighbour slab, with the mask and fibres of those planes (from the
 * global grid).  Only V diffuses, so only V's halo plane is refreshed.
 *
 * bbx_set_halo_planes: lo, hi in {0, 1}: the first lo and last hi planes of g
 * are halo planes: the stencil reads them as the neighbours they are, the
 * step never computes them (no update, activation, stimulus or tissue sum
 * there); bbx_total and bbx_get_info's n_tissue count only the slab's own
 * planes.  Default 0, 0.  Errors: BBX_ERR_ARG (values, or nz <= lo + hi).
 *
 * bbx_halo_exchange: refresh the halo planes between two slabs of one
 * device, lower directly below upper (lower has hi = 1, upper lo = 1, same
 * nx and ny): upper's lowest own V plane goes into lower's top halo plane
 * and lower's highest own V plane into upper's bottom halo plane, both in
 * the buffers the next steps read (2 nx ny floats, row-pitched).
 * Asynchronous, on lower's stream (after upper's enqueued work, and
 * upper's later work waits for it when the streams differ).  Call it
 * between the steps of the two slabs, once per step.  Errors: BBX_ERR_ARG,
 * BBX_ERR_STATE (no model, no halo plane on the facing sides), BBX_ERR_CUDA.
 *
 * bbx_halo_plane: for slabs on different GPUs, the device address of one V
 * plane of the buffer the next step reads: side 0 = low z, 1 = high z; halo
 * = 1: the halo plane to receive into, 0: the slab's own boundary plane to
 * send.  *bytes (may be NULL) = the plane's size (ny rows of px floats).
 * The caller moves the planes (NCCL send/recv, peer copies) on the grid's
 * stream before the next step; the address changes with every step.
 * Errors: BBX_ERR_ARG, BBX_ERR_STATE (no model, no halo plane on that
 * side). */
int bbx_set_halo_planes(bbx_grid* g, int lo, int hi);
int bbx_halo_exchange(bbx_grid* lower, bbx_grid* upper);
int bbx_halo_plane(bbx_grid* g, int side, int halo, void** dev_ptr, size_t* bytes);

/* ---- batches of independent grids ------------------------------------- */
/* Many independent grids of uneven sizes and parameters (parameter sweeps)
 * advanced together.  Grids of one kernel type (model, masked, anisotropic)
 * share one persistent launch with a balanced schedule over all their
 * columns; the launches of the different types of a step run side by side,
 * each on a share of the GPU proportional to its work.  Steps are replayed
 * from a CUDA graph captured on first use.  Not part of the paper: its
 * parameter studies ran one job per simulation. */
typedef struct bbx_batch bbx_batch;

/* Borrow n grids (distinct, each with a model and a time step, all created
 * on the same stream and device).  The grids must outlive the batch and must
 * not be stepped on their own while a batch step is in flight.  Changing a
 * member's settings is allowed between batch steps (the batch is rebuilt).
 * Errors: BBX_ERR_ARG, BBX_ERR_STATE (a member without model or time step),
 * BBX_ERR_UNSUPPORTED, BBX_ERR_NOMEM, BBX_ERR_CUDA. */
int bbx_batch_create(bbx_batch** out, bbx_grid* const* grids, int n);

/* Advance every member by n_steps steps of its own time step (asynchronous
 * on the members' stream).  Each member's time, step counter, activation map
 * and tissue total advance exactly as with bbx_step. */
int bbx_batch_step(bbx_batch* b, int n_steps);

/* Synchronise the batch's stream and report sticky device errors of batch
 * steps (BBX_ERR_NAN, BBX_ERR_TIMEOUT). */
int bbx_batch_sync(bbx_batch* b);

/* Time the tile rows {7, 14, 28} of each kernel type on a few steps (member
 * states restored afterwards) and keep the fastest.  best_ms may be NULL. */
int bbx_batch_autotune(bbx_batch* b, double* best_ms);

/* Number of kernel-type groups and their tile rows (up to cap entries). */
int bbx_batch_info(bbx_batch* b, int* n_groups, int* tile_y, int cap);

/* Release the batch (the grids are not touched).  NULL is ignored. */
void bbx_batch_destroy(bbx_batch* b);

/* ---- reaction surrogate ------------------------------------------------- */
/* A small perceptron, 8 -> 64 -> 64 -> 8 with ReLU hidden layers, that learns
 * the Beeler-Reuter reaction increment s' - s of one step from (normalised)
 * states s, trained on samples of the plain method's trajectories, and used
 * in the step kernel in place of the exact update wherever the state lies in
 * the training envelope and V is below the upstroke threshold (elsewhere the
 * exact model runs).  Not part of the paper.
 * Parameters are packed as W1[64][8] b1[64] W2[64][64] b2[64] W3[8][64]
 * b3[8] (5256 floats).  Normalisation (48 floats): mu_in[8] sd_in[8]
 * mu_out[8] sd_out[8] lo[8] hi[8]; the network sees (s - mu_in)/sd_in and
 * predicts ((s' - s) - mu_out)/sd_out; [lo, hi] bounds the raw inputs. */
typedef struct bbx_mlp bbx_mlp;

/* Create a network with seeded uniform(+-1/sqrt(fan_in)) weights on the
 * given stream.  Errors: BBX_ERR_ARG, BBX_ERR_NOMEM, BBX_ERR_CUDA. */
int bbx_mlp_create(bbx_mlp** out, unsigned long long seed, void* cuda_stream);
void bbx_mlp_destroy(bbx_mlp* m);
int bbx_mlp_set_params(bbx_mlp* m, const float* params_host, size_t n);  /* resets Adam */
int bbx_mlp_get_params(bbx_mlp* m, float* params_host, size_t n);
int bbx_mlp_set_normalization(bbx_mlp* m, const float* norm_host, size_t n);
int bbx_mlp_get_normalization(bbx_mlp* m, float* norm_host, size_t n);

/* Fit the normalisation and the envelope to n training pairs (device arrays
 * x[n][8] raw states, t[n][8] raw increments), accumulating in double. */
int bbx_mlp_fit_normalization(bbx_mlp* m, const float* x_dev, const float* t_dev, long long n);

/* Gradient of the mean squared error over the first `batch` pairs (no
 * update): grad_host[5256], loss (may be NULL).  Synchronises. */
int bbx_mlp_gradients(bbx_mlp* m, const float* x_dev, const float* t_dev, int batch, float* grad_host, size_t n,
                      double* loss);

/* `steps` Adam steps (beta 0.9/0.999, eps 1e-8) on minibatches of `batch`
 * pairs drawn with replacement from the n pairs by a counter-based hash of
 * (seed != 0, step, index); loss of the last minibatch into final_loss (may
 * be NULL; synchronises if not). */
int bbx_mlp_train(bbx_mlp* m, const float* x_dev, const float* t_dev, long long n, int batch, int steps, double lr,
                  unsigned long long seed, double* final_loss);

/* Use a trained network for the reaction of a Beeler-Reuter grid: its BF16
 * copy (weights rounded to bfloat16, biases and normalisation in float) is
 * made now, so later changes to m do not affect the grid.  Every step then
 * advances each tissue node whose state lies inside the network's envelope
 * and whose V is below v_upstroke (mV) by the network's increment (plus the
 * exact diffusion and stimulus terms), and every other node by the exact
 * model.  m NULL switches back to the exact model everywhere.  Errors:
 * BBX_ERR_STATE (no model), BBX_ERR_UNSUPPORTED (model is not BBX_BR, or the
 * tile shape with the surrogate's buffers does not fit shared memory). */
int bbx_set_surrogate(bbx_grid* g, const bbx_mlp* m, double v_upstroke);

/* Training pairs from a running Beeler-Reuter grid (asynchronous): n tissue
 * nodes drawn by a counter-based hash of (seed, i); x_dev[i][8] = their
 * current state, t_dev[i][8] = the exact reaction increment of one step of
 * the grid's time step (no diffusion, no stimulus).  Call between steps to
 * sample a trajectory.  Errors: BBX_ERR_UNSUPPORTED (model is not BBX_BR),
 * BBX_ERR_STATE (no model or time step), BBX_ERR_ARG. */
int bbx_sample_reaction_pairs(bbx_grid* g, long long n, unsigned long long seed, float* x_dev, float* t_dev);

/* Device pointer of the current buffer of one state variable (pitched
 * layout), for callers that keep data on the GPU. */
int bbx_state_device_ptr(bbx_grid* g, int var, void** dev_ptr);

/* Fault injection for failure-detection tests: when on, the first plane load
 * of CTA 0 in each step waits for bytes no copy delivers, so that CTA's
 * bounded wait (about 1 ms in this mode) runs out; the step then records
 * BBX_ERR_TIMEOUT, which the next synchronising call returns.  No fault, trap
 * or hang reaches the GPU. */
int bbx_debug_poison_first_load(bbx_grid* g, int on);

/* Clear the sticky device error bits (after a reported BBX_ERR_NAN or
 * BBX_ERR_TIMEOUT).  Synchronous. */
int bbx_clear_device_error(bbx_grid* g);

/* Tissue sum of one field, in double precision, for callers that cannot
 * allocate device memory (a framework that owns all allocations through its
 * own pool, a real-time loop that must never call cudaMalloc, a context with
 * a memory budget fixed up front).  The paper has no counterpart; it is the
 * reduction of bbx_total with its scratch held in a fixed device array that
 * the library keeps on every GPU that loads it until the process exits.
 * field_dev: nx*ny*nz floats on the current device in the pitched layout
 * (rows of `pitch` >= nx elements, planes of pitch*ny); mask_dev: NULL (sum
 * every node) or bytes in the same layout, nonzero = tissue; out_dev: one
 * double on the device, written when the work enqueued on cuda_stream runs.
 * No device memory is allocated or freed.  Limits: nx*ny*nz <= 2^28 nodes,
 * else BBX_ERR_ARG.  The first call on a device looks up the scratch array's
 * device address (make that first call before any stream capture); it is
 * looked up again when the device's context changes (after cudaDeviceReset).
 * All calls share the scratch, so calls that overlap on the GPU (concurrent
 * streams) race; serialise them.  An error already pending from the
 * caller's earlier CUDA work makes the call return BBX_ERR_CUDA and is left
 * in place, not cleared.  Errors: BBX_ERR_ARG (checked before any CUDA
 * call), BBX_ERR_CUDA. */
int bbx_total_noalloc(const float* field_dev, const uint8_t* mask_dev, int nx, int ny, int nz, int pitch,
                      double* out_dev, void* cuda_stream);

/* Release every resource of the grid (NULL is ignored). */
void bbx_destroy_grid(bbx_grid* g);

/* Host-only test hooks (no device work, usable without a GPU).
 * bbx_debug_cover_chunks: the pieces a masked 3D grid is cut into, from the
 *   tissue flags of its 16-wide chunks, flags[bz][by][cx] (ncx x nby x nbz
 *   bytes, nonzero = the 16 x ty x zb chunk holds tissue): *count pieces
 *   (x0, y0, z0, z1) into out (4 ints each, at most cap pieces; BBX_ERR_ARG
 *   with *count set if cap is too small).
 * bbx_debug_plan_first_pieces: the first piece (x0, y0, z0, z1) of each CTA
 *   when the segments segs4 (nsegs x (x0, y0, z0, z1), in order) are shared
 *   among ctas CTAs; *used = CTAs used (at most the total plane count; at
 *   most cap written, else BBX_ERR_ARG). */
int bbx_debug_cover_chunks(const uint8_t* flags, int ncx, int nby, int nbz, int ty, int zb, int nz, int* out,
                           int cap, int* count);
int bbx_debug_plan_first_pieces(const int* segs4, int nsegs, int ctas, int* out, int cap, int* used);

/* GPU test hook: out_dev[i] = the e^x - 1 the Beeler-Reuter kernels use
 * (the Taylor series about 0 for |x| < 0.25, else e^x - 1) and ref_dev[i] =
 * CUDA's expm1f, for n floats x_dev (device memory).  Synchronises the
 * stream.  Errors: BBX_ERR_ARG, BBX_ERR_CUDA. */
int bbx_debug_expm1(const float* x_dev, float* out_dev, float* ref_dev, int n, void* cuda_stream);

/* Static text for a status code. */
const char* bbx_status_string(int status);

#ifdef __cplusplus
}
#endif
#endif /* BBX_H */
