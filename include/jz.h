/*
 * jz.h -- C ABI of the GB300 (sm_103a) implementation of the per-stage
 * residual and explicit 5-stage Runge-Kutta update of the filtered
 * compressible Navier-Stokes (LES) equations on a structured curvilinear
 * grid, after "On the Scalability of CFD Tool for Supersonic Jet Flow
 * Configurations" (arXiv 2003.09926).
 *
 *   Section 3, Eqs. les / vec-les / con-prop   the conservation law dQ/dt = -RHS
 *   Section 3, Eq. 2, Eq. q_mod, Eq. sutherland, Eq. tau_mod
 *                                               gas model and viscous terms
 *   Section 3 (numerical method paragraph)      centred 2nd-order fluxes in general
 *                                               curvilinear coordinates, anisotropic
 *                                               scalar dissipation (Turkel & Vatsa),
 *                                               explicit 5-stage Runge-Kutta
 *   Section 3 (boundary-condition paragraph)    supersonic inflow, Riemann far field,
 *                                               the cylindrical domain's centreline
 *                                               (extrapolation plus azimuthal average)
 *                                               and superposed azimuthal points
 *   Section 4.2, Fig. jazzy                     per stage: boundary update,
 *                                               inviscid flux, dissipation, viscous flux
 *   Section 4.3                                 two-layer ghost fringe, five-point stencil
 *   Section 6                                   time statistics of the jet
 *
 * Conventions shared by every entry point:
 *  - Every function returns an int status: JZ_OK (0) or a negative JZ_E* code.
 *    No C++ exception crosses this boundary.  jz_last_error() returns the
 *    calling thread's message for its last failing call.
 *  - Device memory and the CUDA stream belong to the caller.  The library
 *    carves its arrays out of one caller-provided device buffer of
 *    jz_grid_bytes() bytes and never allocates, frees or resizes device
 *    memory on its own.  Host buffers also belong to the caller.
 *  - Work is enqueued asynchronously on the grid's stream unless a function
 *    says it synchronises.  The time step stays on the device.
 *  - Units are non-dimensional: freestream density, sound speed and
 *    temperature 1, jet diameter 1, freestream pressure 1/gamma, jet
 *    velocity = Mach number, viscosity at freestream temperature = mach / re.
 */
#ifndef JZ_H
#define JZ_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* status codes */
#define JZ_OK 0
#define JZ_EINVAL (-1)     /* bad argument, descriptor or call order      */
#define JZ_ENOMEM (-2)     /* caller buffer too small / over budget        */
#define JZ_ECUDA (-3)      /* a CUDA runtime call failed                   */
#define JZ_ENONFINITE (-4) /* state holds non-finite values                */
#define JZ_ETIMEOUT (-5)   /* a bounded device wait gave up                */

/* boundary kinds per face (faces ordered x-, x+, y-, y+, z-, z+).  A
 * direction is periodic when both of its faces are JZ_BC_PERIODIC. */
#define JZ_BC_PERIODIC 0
#define JZ_BC_INFLOW 1   /* jet exit plane: fixed top-hat profile (Section 3) */
#define JZ_BC_FARFIELD 2 /* Riemann invariants against air at rest (Section 3) */
#define JZ_BC_AXIS 4     /* centreline of a cylindrical grid (y- face only)     */

/* grid geometry */
#define JZ_GEOM_BOX 0      /* Cartesian box, optional tanh clustering and mapping */
#define JZ_GEOM_CYLINDER 1 /* the paper's cylindrical jet grid (Section 3)        */

/* precision modes: state/flux arithmetic, metric storage.  FP32 flux
 * arithmetic uses the hardware approximations of sqrt, reciprocal and
 * powers (a few ulp); so do the boundary formulas of JZ_P32 and JZ_P32_M64,
 * while JZ_P32_S64 evaluates them with IEEE FP32 operations.  JZ_P32 and
 * JZ_P32_M64 give bitwise equal states with the scalar stage kernel. */
#define JZ_P64 0     /* FP64 state and fluxes, FP64 metrics                   */
#define JZ_P32_M64 1 /* FP32 state and fluxes, FP64-stored metrics             */
#define JZ_P32 2     /* FP32 state and fluxes, FP64-generated FP32 metrics     */
#define JZ_P32_S64 3 /* FP32 fluxes and stage states, FP64 state between steps,
                      * FP32 metrics: the update adds the FP32 increment to an
                      * FP64 copy of Q^n at the updated nodes, so the state does
                      * not lose the increments smaller than its FP32 spacing */

/* initial conditions */
#define JZ_IC_JET 0       /* top-hat jet column plus seeded velocity noise     */
#define JZ_IC_QUIESCENT 1 /* air at rest (Section 5.1: the paper's start state) */

/* Subgrid-scale eddy viscosity mu_t (Section 3 names an LES formulation,
 * not a model), Delta = J^(-1/3):
 *   JZ_SGS_SMAGORINSKY: mu_t = rho (C_s Delta)^2 |S|, |S| = sqrt(2 S_ij S_ij);
 *   JZ_SGS_VREMAN:      mu_t = rho c sqrt(B_b / (a_ij a_ij)), c = 2.5 C_s^2,
 *     a_ij = du_j/dx_i, b_ij = Delta^2 a_mi a_mj, B_b = b11 b22 - b12^2
 *     + b11 b33 - b13^2 + b22 b33 - b23^2 (0 where a = 0; Vreman's model,
 *     which vanishes in pure shear). */
#define JZ_SGS_SMAGORINSKY 0
#define JZ_SGS_VREMAN 1

/* Grid descriptor.  Nodes are numbered 0..n-1 per direction (i fastest);
 * non-periodic directions need n >= 3 and their first and last nodes are
 * boundary nodes set by the boundary conditions.  At most 2^24 nodes per
 * direction, and nj * nk * ceil(ni / 32) below 2^31 (the reductions index
 * rows of 32 nodes with 32-bit integers).
 *
 * JZ_GEOM_BOX: x is uniform on [lo[0], hi[0]]; y and z (when not periodic
 * and stretch_c > 0) follow a tanh clustering about |y| = cluster_r; every
 * coordinate then receives a seeded sinusoidal offset of amplitude
 * map_amp x local spacing (0 = none).  Periodic directions use uniform
 * spacing (hi - lo)/n.
 *
 * JZ_GEOM_CYLINDER (Section 3, Tab. mesh): i axial (x uniform on
 * [lo[0], hi[0]]), j radial from the centreline, r in [0, hi[1]] with the
 * same tanh clustering about r = cluster_r (lo[1] must be 0), k azimuthal,
 * theta = 2 pi (k mod P) / P with P = nk - 1: the first and last azimuthal
 * nodes coincide (the paper uses nk = 361).  y = r cos(theta),
 * z = r sin(theta).  Faces: bc[2] = JZ_BC_AXIS, bc[4] = bc[5] =
 * JZ_BC_PERIODIC, bc[0], bc[1], bc[3] inflow or far field; P even (the
 * ghosts behind the centreline are the nodes across it, k + P/2), nk >= 5,
 * nj >= 4, map_amp = 0.  Centreline nodes hold the mean over the P
 * distinct azimuthal nodes of the adjacent radial line (summed in
 * azimuthal order, in FP64); the last azimuthal plane holds a copy of the
 * first; J on the centreline (where the conservative metric form gives zero
 * volume) is that of the adjacent radial node.  Blocks of a cylindrical grid
 * may split direction i only. */
typedef struct jz_grid_desc {
  int ni, nj, nk;
  int bc[6];
  double lo[3], hi[3];
  double cluster_r, stretch_c, stretch_w;
  double map_amp;
  uint64_t map_seed;
  int precision; /* JZ_P64, JZ_P32_M64, JZ_P32 or JZ_P32_S64 */
  int geom;      /* JZ_GEOM_BOX or JZ_GEOM_CYLINDER */
} jz_grid_desc;

/* Flow parameters.  re <= 0 means inviscid (no molecular viscosity);
 * cs = 0 disables the eddy viscosity; k2, k4, sigma are the
 * dissipation constants; s1 is the Sutherland constant over T_inf; r0 and
 * theta shape the jet profile u = (M/2)(1 - tanh((r - r0)/(2 theta))); noise
 * is the velocity-noise amplitude relative to the jet velocity. */
typedef struct jz_flow_params {
  double mach, re, gamma, pr, prt, cs, k2, k4, sigma, s1, r0, theta, noise;
  int ic;  /* JZ_IC_JET or JZ_IC_QUIESCENT */
  int sgs; /* JZ_SGS_SMAGORINSKY or JZ_SGS_VREMAN (cs = 0: no eddy viscosity) */
} jz_flow_params;

/* Diagnostics over all grid nodes (ghosts excluded), reduced in a fixed
 * order (bitwise reproducible run to run).  Per-node values are computed in
 * the state's precision (FP32 for JZ_P32 and JZ_P32_M64 grids); the sums are
 * carried in FP64 (FP32 grids: compensated FP32 per thread, then FP64), so
 * an FP32 grid's sums are exact up to the FP32 rounding of 1/J and of the
 * per-node products Q_v * (1/J): within 2^-23 of sum |Q_v|/J. */
typedef struct jz_diag {
  double time;      /* simulated time                                  */
  int64_t step;     /* completed time steps                            */
  double dt;        /* last time step                                  */
  double sum[5];    /* sum over nodes of Q_v / J (conserved integrals) */
  double rho_min, rho_max, p_min, p_max;
  double mach_max;  /* max |u| / c                                     */
  int64_t nonfinite;/* nodes with a non-finite conserved value         */
} jz_diag;

typedef struct jz_grid jz_grid;
typedef struct jz_batch jz_batch;

/* Copy the calling thread's last error message into buf (always
 * NUL-terminated when len > 0).  Returns the message length. */
int jz_last_error(char* buf, size_t len);

/* Device bytes a grid with this descriptor needs (state x3, metrics,
 * coordinate tables, reduction scratch; the FP64 state copy of a JZ_P32_S64
 * grid; the centreline means of a cylinder).  Pure arithmetic: used for
 * HBM-budget admission.  JZ_EINVAL on a bad descriptor. */
int jz_grid_bytes(const jz_grid_desc* desc, size_t* bytes);

/* Create a grid in a caller-owned device buffer (>= jz_grid_bytes, 256-byte
 * aligned) on the caller's stream (cudaStream_t passed as void*; NULL =
 * legacy default stream) and enqueue the metric generation: analytic
 * coordinates, then the conservative metric terms S^k_m = (d xi_k/d x_m)/J
 * and J at every node, in FP64 (Section 3: generalised curvilinear
 * transformation; Section 4.2: Jacobian and metric terms computed once).
 * The handle is host memory owned by the library until jz_grid_destroy. */
int jz_grid_create(const jz_grid_desc* desc, void* dev_buf, size_t bytes, void* stream, jz_grid** out);

/* Release the handle (and any captured graph).  Does not free dev_buf. */
int jz_grid_destroy(jz_grid* g);

/* Enqueue the grid's later work on `stream` (cudaStream_t as void*; NULL =
 * legacy default stream), ordered after everything enqueued so far on its
 * previous stream (an event recorded there, waited for on the new one).
 * The library has no counterpart in the paper: a serving loop uses it to
 * move a case between streams of different priority.  No host sync.
 * Batches keep the stream they were created with. */
int jz_set_stream(jz_grid* g, void* stream);

/* --- blocks of a grid (the paper's domain decomposition, Section 4.2) -----
 * A block holds the nodes [o0[d], o1[d]] (inclusive, d = i, j, k) of the grid
 * `desc` describes, with its own two ghost layers: every jz_grid entry point
 * accepts it and acts on those nodes (jz_state_init gives them the values of
 * the same nodes of the whole grid: the noise is keyed to global indices;
 * jz_state_download / upload and jz_diagnostics cover the block's nodes).  A
 * face of the block inside the grid is an exchange face: its first / last
 * node is updated like an interior node and its ghosts are copies of the
 * neighbouring block's nodes, filled by the halo exchange of a block set
 * (jz_blocks_create).  Periodic directions cannot be split; a block has at
 * least three nodes along a split direction; coordinates and metrics are
 * those of the whole grid at the same nodes.  JZ_EINVAL for a bad range. */
int jz_block_bytes(const jz_grid_desc* desc, const int o0[3], const int o1[3], size_t* bytes);
int jz_block_create(const jz_grid_desc* desc, const int o0[3], const int o1[3], void* dev_buf, size_t bytes,
                    void* stream, jz_grid** out);

/* --- a block whose neighbours live on other ranks (Section 4.1: the
 * partitioned domain, one partition per process; Section 4.3: the
 * non-blocking exchange of two ghost layers of Q at every Runge-Kutta stage;
 * Section 4.2, Fig. jazzy: where the exchanges sit in the stage sequence).
 * The caller moves the face buffers between ranks (point-to-point sends, no
 * collective) and combines the blocks' rates (a maximum over ranks).  One
 * time step of a block, every call enqueued on the block's stream:
 *   exchange of state copy 0 (pack, send / receive, unpack, per direction
 *   i, j, k, so that edge and corner ghosts take values already exchanged);
 *   jz_block_rate; the maximum of the rates over all blocks written back to
 *   *dev_rate; jz_block_advance;
 *   for stage l = 0..4: jz_block_stage(l), then (l < 4) the exchange of
 *   state copy (1, 2, 1, 2)[l].
 * State copies: 0 = Q0 (Q^n, Q^(5)), 1 = QA, 2 = QB.
 *
 * jz_halo_bytes: bytes of the buffer of one face normal to direction dir
 *   (0 = i, 1 = j, 2 = k): 5 variables x 2 layers x the padded node counts
 *   (n + 4) of the other two directions, in the state's type (FP64 for
 *   JZ_P64, else FP32).
 * jz_halo_pack: the two node layers just inside face (dir, side) (side 0:
 *   nodes 0, 1; side 1: nodes n-2, n-1) of state copy `which`, over the
 *   padded extents of the other directions, into buf (device, >=
 *   jz_halo_bytes; layout [v][layer][b][a], a the first of the other two
 *   directions in i, j, k order, fastest).
 * jz_halo_unpack: buf into the two ghost layers behind the face (side 0:
 *   nodes -2, -1; side 1: n, n+1); the neighbour packed its layers in the
 *   same order, nearest-to-low first.
 * jz_block_rate: enqueue this block's largest stable-step rate (Section 3
 *   time step reading R12) into a device FP64 scalar and return its address
 *   (valid while the block lives).
 * jz_block_advance: enqueue dt = cfl / *rate, time += dt, step += 1.
 * jz_block_stage: enqueue Runge-Kutta stage l (0..4) and the boundary pass
 *   of its output copy (exchange ghosts are left to the caller).
 * JZ_EINVAL for a face that is not an exchange face, a bad direction, side,
 * copy or stage, a null pointer, or cfl <= 0. */
int jz_halo_bytes(jz_grid* g, int dir, size_t* bytes);
int jz_halo_pack(jz_grid* g, int which, int dir, int side, void* buf);
int jz_halo_unpack(jz_grid* g, int which, int dir, int side, const void* buf);
int jz_block_rate(jz_grid* g, double** dev_rate);
int jz_block_advance(jz_grid* g, double cfl);
int jz_block_stage(jz_grid* g, int stage);

/* Set the flow parameters and enqueue the initial state (JZ_IC_JET: top-hat
 * profile plus noise drawn from SplitMix64(seed ^ (3 lin + m)); or air at
 * rest), then the boundary conditions.  Resets time and step to 0. */
int jz_state_init(jz_grid* g, const jz_flow_params* flow, uint64_t seed);

/* Enqueue one time step: the time step from the CFL condition (cfl > 0) or
 * the fixed dt_fixed (> 0; exactly one of the two must be positive), then
 * five Runge-Kutta stages Q^(l) = Q^(0) - alpha_l dt J R(Q^(l-1)) with
 * alpha = 1/4, 1/6, 3/8, 1/2, 1, boundary conditions before every stage
 * (Section 3; Section 4.2, Fig. jazzy).  Asynchronous; no host sync. */
int jz_rk_step(jz_grid* g, double cfl, double dt_fixed);

/* Enqueue n steps as replays of a CUDA graph of one step (captured on first
 * use and re-captured when cfl / dt_fixed change).  Asynchronous. */
int jz_nsteps(jz_grid* g, int n, double cfl, double dt_fixed);

/* Compute diagnostics on the device, copy them to *out.  Synchronises the
 * grid's stream.  Returns JZ_ENONFINITE (with *out filled) when any grid
 * node holds a non-finite value. */
int jz_diagnostics(jz_grid* g, jz_diag* out);

/* The diagnostics of jz_diagnostics, enqueued on the grid's stream with their
 * copy to *out, without synchronising: *out holds them once the stream has
 * passed the copy (after a stream synchronisation or an event recorded after
 * this call).  The copy overlaps later work on the stream only when *out is
 * page-locked host memory (cudaHostAlloc, or a pinned torch tensor); *out
 * must stay valid until the copy has run.  Non-finite values are reported in
 * out->nonfinite only, and a bounded-wait timeout of the stage kernel only
 * by the next jz_diagnostics.  JZ_EINVAL for a null handle or output. */
int jz_diagnostics_async(jz_grid* g, jz_diag* out);

/* Diagnostics formed by the steps themselves.  on = 1: the time-step
 * reduction of every later step with a CFL number (jz_rk_step, jz_nsteps)
 * also forms the diagnostics of the state it reads -- the state the step
 * starts from, the previous step's result -- from the same loaded values, so
 * that no separate pass over the grid is needed; a step with a fixed time
 * step forms them by the pass of jz_diagnostics.  The record of the last
 * step is read with jz_step_diagnostics_async.  Its sums are accumulated in
 * another order than those of jz_diagnostics (equal up to rounding); its
 * extrema and non-finite count are the same.  The stepping itself is
 * unchanged.  Affects single-grid steps only (jz_rk_step, jz_nsteps);
 * batches and the per-block entry points ignore it.  on = 0 (the default)
 * switches it off.  JZ_EINVAL for other values of on. */
int jz_set_step_diagnostics(jz_grid* g, int on);

/* Enqueue on the grid's stream the copy of the grid's latest diagnostics
 * record to *out, without a pass over the grid: after a step with step
 * diagnostics on, the diagnostics of the state that step started from
 * (out->time and out->step name that state, out->dt the step before it).
 * The rules for *out are those of jz_diagnostics_async.  JZ_EINVAL for a
 * null handle or output.  jz_diagnostics and jz_diagnostics_async replace
 * the record with the diagnostics of the current state. */
int jz_step_diagnostics_async(jz_grid* g, jz_diag* out);

/* Copy the state to host memory: n = 5*ni*nj*nk doubles, layout [v][k][j][i]
 * (conserved rho, rho u, rho v, rho w, e), ghosts excluded; FP32 states are
 * widened (JZ_P32_S64: the updated nodes come from the FP64 state, boundary
 * nodes from the FP32 one).  Synchronises the stream. */
int jz_state_download(jz_grid* g, double* host, size_t n);

/* Copy the metric terms the kernels use to host memory (Section 3: the
 * generalised curvilinear transformation): n = 10*ni*nj*nk doubles, layout
 * [f][k][j][i], f = 3k+m for S^k_m = (d xi_k / d x_m)/J and f = 9 for J,
 * ghosts excluded, widened from the grid's metric type (FP32 for JZ_P32 and
 * JZ_P32_S64).  Uses the grid's stage buffer as staging, so call it between
 * steps; synchronises the stream.  JZ_EINVAL for a wrong n or a null
 * pointer. */
int jz_metrics_download(jz_grid* g, double* host, size_t n);

/* Replace the state from host memory (layout as jz_state_download; values
 * at boundary nodes are overwritten by the boundary conditions, which are
 * applied after the upload; a JZ_P32_S64 grid keeps the FP64 values of its
 * updated nodes).  Requires jz_state_init to have set the flow parameters.
 * Synchronises the stream (host buffer may be reused on return). */
int jz_state_upload(jz_grid* g, const double* host, size_t n);

/* Batched execution of many grids: per stage, one persistent launch whose
 * CTAs take (grid, tile, k-chunk) work items from a device queue, largest
 * first, plus one batched boundary fill (preceded by the centreline means
 * when a grid is cylindrical); per step one batched time-step reduction.  The batch borrows the grids (one precision mode, flow
 * parameters set; they must outlive the batch and keep the k-chunk length
 * they had at jz_batch_create) and a caller-owned, 256-byte aligned device
 * buffer of jz_batch_bytes bytes for its tables; work goes to `stream`
 * (the grids' own streams are not used, so order them against it).  Every
 * grid keeps its own CFL time step on the device, and its state is bitwise
 * the one it reaches when stepped alone. */
int jz_batch_bytes(jz_grid* const* grids, int n, size_t* bytes);
int jz_batch_create(jz_grid* const* grids, int n, void* dev_buf, size_t bytes, void* stream, jz_batch** out);
/* Enqueue n steps of every grid in the batch (graph-captured; asynchronous). */
int jz_batch_nsteps(jz_batch* b, int n, double cfl);
int jz_batch_destroy(jz_batch* b);

/* A block set: the blocks of one grid (jz_block_create) stepped together as a
 * batch whose members are coupled as the paper's decomposed domain is
 * (Section 4.2): after every stage the ghosts behind each exchange face take
 * the neighbouring block's nodes (halo exchange on the device, direction by
 * direction), and every step takes the one time step of the whole grid (the
 * largest rate over the blocks).  The blocks must partition the grid's nodes
 * as a tensor product of ranges (every exchange face is shared whole with one
 * neighbour) and share one description and precision; JZ_EINVAL otherwise.
 * Each block's nodes then evolve bitwise as the same nodes of the whole grid
 * stepped alone.  Sized by jz_blocks_bytes; stepped by jz_batch_nsteps (CFL
 * only); released by jz_batch_destroy. */
int jz_blocks_bytes(jz_grid* const* blocks, int n, size_t* bytes);
int jz_blocks_create(jz_grid* const* blocks, int n, void* dev_buf, size_t bytes, void* stream, jz_batch** out);

/* --- time statistics and restart (Section 6) --------------------------------
 * The paper's validation averages the solution in time once the jet is
 * statistically steady: the time-averaged axial velocity <U>, the rms of its
 * fluctuation u_rms, radial profiles of both at fixed distances downstream of
 * the inlet (averaged in the azimuthal direction), and the potential core,
 * where <U> is at least 95% of the jet's inlet velocity.
 *
 * jz_stats_bytes / jz_stats_create: running FP64 sums of u = (rho u)/rho and
 *   u^2 over samples for every node of grid g, in a caller-owned device
 *   buffer (256-byte aligned); created zeroed on the grid's stream.
 * jz_stats_sample: adds the grid's current state (enqueued on its stream; in
 *   sample order, so the sums are those of a sequential loop).
 * jz_stats_read: per node ([k][j][i], the grid's nodes), <U> = sum / N and
 *   u_rms = sqrt(max(sum2 / N - <U>^2, 0)); n must be the node count.
 * jz_stats_radial: the i-plane whose axial coordinate (at the node nearest the
 *   axis) is nearest x; its nodes binned by r = sqrt(y^2 + z^2) into nbins
 *   equal bins of [0, r_max): per bin the mean of <U>, the mean of u_rms and
 *   the node count (empty bins 0; a cylinder's last azimuthal plane, a copy
 *   of the first, is not counted).
 * jz_stats_core_length: <U> on the axis (on a box the mean over the node
 *   lines nearest y = z = 0: the middle line of an odd node count, both
 *   middle lines of an even one; on a cylinder the mean over the centreline's
 *   P distinct azimuths) and the axial distance from the inlet to its first
 *   drop below frac * u_jet, interpolated linearly (the last node's x if it
 *   never drops).
 * The read functions synchronise the grid's stream; JZ_EINVAL without samples
 * or for bad arguments.
 * jz_set_clock sets the grid's simulated time and step count (restarting from
 * a saved state: jz_state_upload, then jz_set_clock). */
typedef struct jz_stats jz_stats;
int jz_stats_bytes(jz_grid* g, size_t* bytes);
int jz_stats_create(jz_grid* g, void* dev_buf, size_t bytes, jz_stats** out);
int jz_stats_sample(jz_stats* s);
int jz_stats_count(jz_stats* s, int64_t* samples);
int jz_stats_read(jz_stats* s, double* mean_u, double* rms_u, size_t n);
int jz_stats_radial(jz_stats* s, double x, int nbins, double r_max, double* mean_u, double* rms_u, double* count);
int jz_stats_core_length(jz_stats* s, double u_jet, double frac, double* length);
int jz_stats_destroy(jz_stats* s);
int jz_set_clock(jz_grid* g, double time, int64_t step);

/* --- measurement helpers -------------------------------------------------- */

/* Number of kernel launches this library has issued in this process
 * (graph replays count every kernel node they run). */
int jz_launch_count(uint64_t* out);

/* Per-kernel timing with CUDA events recorded on the grid's stream around
 * every launch jz_rk_step makes while profiling is on (jz_nsteps graphs are
 * not instrumented).  jz_profile_read synchronises the stream and returns,
 * per kernel class (0 = fused RK stage, 1 = boundary fill, 2 = time step,
 * 3 = other), the total milliseconds and launch count since jz_profile_begin. */
int jz_profile_begin(jz_grid* g);
int jz_profile_read(jz_grid* g, double ms[4], int64_t launches[4]);
int jz_profile_end(jz_grid* g);

/* Measured fused multiply-add throughput of the current device in TFLOP/s
 * (2 flops per FMA; fp64 = 1: FP64, 0: FP32): eight independent FMA chains
 * per thread on 8 x 256 threads per SM, timed with CUDA events on `stream`
 * (cudaStream_t as void*; synchronised), best of three after a warm-up.  The
 * denominator of the FP64 stage kernel's roofline (bound by the FP64 pipe)
 * and of the FP32 kernel's arithmetic rate.  JZ_EINVAL for a null output or
 * another fp64 value, JZ_ECUDA on a CUDA error. */
int jz_fma_peak(int fp64, double* tflops, void* stream);

/* Tile shape of the fused stage kernel for this grid (for tuning and for
 * the batched tile table): ti x tj nodes per CTA, kc planes per CTA chunk.
 * jz_set_tiling may change kc (planes per chunk, >= 1); the (i, j) shape is
 * fixed per precision mode except for the FP32 vector-record kernel, whose
 * shape jz_set_tile_shape selects. */
int jz_get_tiling(jz_grid* g, int* ti, int* tj, int* kc);
int jz_set_tiling(jz_grid* g, int kc);

/* Stage kernel variant of a JZ_P32 grid: 2 (default) keeps node records as
 * float4 + float vectors in shared memory (two block barriers per plane);
 * 0 is the scalar kernel (one shared-memory value per load, four barriers
 * per plane).  Both evaluate the same formulas; results agree to FP32
 * rounding.  Measured on the 256x192x192 mapped jet: 0.41 ms (2) and 0.55 ms
 * (0) per stage.  Grids of the other precision modes (JZ_P64, JZ_P32_M64,
 * JZ_P32_S64) run the scalar kernel only: JZ_EINVAL for variant 2 there, and
 * for other variants.  A batch uses its first grid's variant. */
int jz_set_stage_variant(jz_grid* g, int variant);

/* Test of the bounded waits: failure detection exercised without a GPU
 * fault (the paper has no counterpart).  on = 1: every TMA copy that the
 * grid's stage kernels issue expects 16 bytes more than it delivers, so no
 * staging wait can complete,
 * and the waits give up after 2^16 SM cycles instead of about a second.
 * Each stage kernel then takes its timeout path: it records the failure in
 * the grid's sticky error flag, completes the missing bytes itself, waits
 * for its real copies to land and returns; nothing traps or hangs, and
 * jz_diagnostics reports JZ_ETIMEOUT.  The state is invalid afterwards:
 * set on = 0 and call jz_state_init (or jz_state_upload after it) to clear
 * the flag and continue.  Affects single-grid launches only (jz_rk_step,
 * jz_nsteps); batches ignore it.  JZ_EINVAL for other values of on. */
int jz_set_stall_test(jz_grid* g, int on);

/* Tile shape (ti x tj nodes in i and j) of the FP32 vector-record stage
 * kernel of this grid: 16 x 16 (default), 32 x 16 or 16 x 32, each a build of
 * the same kernel (16 x 16 runs two CTAs per SM, the others one; 16 x 16
 * also wastes least of a tile on small grids, 16 x 32 on grids narrow in
 * i).  The per-node arithmetic does not
 * depend on the shape: results are bitwise the same.  Resets the k-chunk
 * length to its default for the shape.  A batch needs one shape for all its
 * grids.  JZ_EINVAL for another shape or for a grid that does not run the
 * vector-record kernel (JZ_P32 with variant 2). */
int jz_set_tile_shape(jz_grid* g, int ti, int tj);

/* --- diagnostics without device allocation --------------------------------
 * The paper has no counterpart to this entry point: it serves callers that
 * may only use device arrays they were handed -- a plug-in called by a host
 * framework with its input and output buffers, or a serving process that
 * reserved all device memory at start-up and treats later allocations as
 * failures -- and so cannot provide the scratch that jz_diagnostics takes
 * from a grid's buffer.  Its reduction scratch is a fixed static device
 * array (about 352 KB, held by every device that loads the library until the
 * process exits); it allocates no device memory and calls no allocating
 * routine.
 *
 * Q:    device, dense [5][n_nodes] conserved variables (rho, rho u, rho v,
 *       rho w, e), FP64 when fp64 = 1, FP32 when fp64 = 0;
 * vol:  device, n_nodes FP64 node volumes (1/J for a grid);
 * out:  device, 11 doubles: sum Q_v * vol (5, in FP64), rho min, rho max,
 *       p min, p max, max |u|/c (pressure and Mach number computed per node
 *       in the state's precision, as jz_diagnostics does), count of nodes
 *       with a non-finite value (nodes with one are left out of the sums and
 *       extrema);
 * stream: cudaStream_t as void* (NULL = legacy default stream).
 * n_nodes must not exceed 268,435,456 (2^28; JZ_EINVAL beyond).  The work is
 * enqueued asynchronously; results are summed in a fixed order (bitwise
 * reproducible).  Every call looks up the static array's device address for
 * the device current at the call (a lookup, no allocation); the first call on
 * a device also loads the library's device code there, so make it before any
 * stream capture.  Every call shares the one array, which keeps the last
 * call's contents (the call clears the counter it needs zeroed); calls whose
 * kernels may overlap on the GPU (unordered streams) race on it and must not
 * be issued. */
int jz_state_diagnostics_static(long long n_nodes, int fp64, const void* Q, const double* vol, double gamma,
                                double* out, void* stream);

#ifdef __cplusplus
}
#endif
#endif /* JZ_H */
