/*
 * tlb.h -- C ABI of the GB300 ternary lattice Boltzmann + immersed boundary
 * library (libtlb.so).
 *
 * The library advances the method of "Modelling ternary fluids in contact
 * with elastic membranes" (Pepona, Shek, Semprebon, Krueger, Kusumaatmaja):
 * a three-component free-energy lattice Boltzmann fluid (populations f_i for
 * the density rho, g_i for phi = C1 - C2 and h_i for psi = C3; Sec. 2.6 and
 * Sec. 3.1, eqs. VariableTransform, LBE, EDF, MomentsDFs) coupled through the
 * immersed boundary method (Sec. 3.3, eqs. Spreading, DiscreteDirac,
 * Interpolation, UpdatedXl) to closed elastic membranes that enclose
 * component 3 (Sec. 3.2, eqs. DiscreteSE, DiscreteBE, DiscreteCE,
 * DiscreteCF).  Every step of the path runs in the library's own CUDA
 * kernels for sm_103a.
 *
 * Conventions shared by every call:
 *  - Units are lattice units, dx = dt = 1, cs^2 = 1/3 (Sec. 3.1).
 *  - A lattice cell (x, y, z) has linear index (z*ny + y)*nx + x.  A 2D
 *    lattice (dim = 2) is nx by ny with index y*nx + x (nz is ignored).
 *  - Device memory is owned by the caller: one arena of tlb_state_bytes()
 *    bytes, 256-byte aligned, passed to tlb_create() and kept alive until
 *    tlb_destroy().  The library allocates no device memory itself.
 *  - Host pointers are borrowed for the duration of the call only; the
 *    library copies what it needs.
 *  - Calls are ordered on the CUDA stream given to tlb_create().  tlb_step
 *    returns once the work is enqueued; every tlb_read_* and
 *    tlb_diagnostics call synchronises that stream before returning.
 *    Inside a tlb_step call the membrane work of a step runs partly on two
 *    internal streams of the context; all of it is joined back into the
 *    context stream before the call returns, so work the caller enqueues on
 *    that stream afterwards sees the finished steps.
 *  - Every call returns a tlb_status; on failure tlb_last_error() returns a
 *    message (thread-local).  A context is not thread-safe.
 */
#ifndef TLB_H
#define TLB_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  TLB_OK = 0,
  TLB_ERR_ARG = 1,       /* invalid argument, size or state of the call     */
  TLB_ERR_CUDA = 2,      /* a CUDA runtime call failed                       */
  TLB_ERR_ALLOC = 3,     /* the arena is too small for the requested state   */
  TLB_ERR_DIVERGED = 4,  /* NaN/Inf or a marker moved more than one cell     */
  TLB_ERR_TIMEOUT = 5,   /* a bounded device-side wait gave up               */
  TLB_ERR_STATE = 6      /* call out of order (e.g. step before init)        */
} tlb_status;

/* Population storage (Sec. 3.1 populations; compute precision follows):
 * TLB_F64 -- double storage and arithmetic;
 * TLB_F32 -- float storage of f_i - w_i (shifted by the rest-density
 *            equilibrium) and of g_i, h_i; float arithmetic;
 * TLB_F16 / TLB_BF16 -- binary16 / bfloat16 storage of f_i - w_i and of
 *            g_i, h_i for i != 0, float storage of the rest populations
 *            g_0, h_0 (they carry phi and psi themselves); float arithmetic. */
enum { TLB_F64 = 0, TLB_F32 = 1, TLB_F16 = 2, TLB_BF16 = 3 };

/* Membrane kinds: a closed ring of markers in 2D (stretching + bending,
 * eqs. DiscreteSE, DiscreteBE) or a closed triangulated surface in 3D
 * (Skalak shear + Helfrich bending). */
enum { TLB_MEM_RING2D = 0, TLB_MEM_TRI3D = 1 };

/* Fields for tlb_read_field (each ncells doubles, or 3*ncells for vectors
 * laid out [component][cell]). */
enum {
  TLB_FIELD_RHO = 0, TLB_FIELD_PHI = 1, TLB_FIELD_PSI = 2,
  TLB_FIELD_C1 = 3, TLB_FIELD_C2 = 4, TLB_FIELD_C3 = 5,
  TLB_FIELD_U = 6,   /* bare velocity u = sum_i c_i f_i / rho (vector)     */
  TLB_FIELD_I = 7    /* membrane profile I of the last step (eq. Iprofile) */
};

typedef struct {
  int dim;            /* 2 (D2Q9, as printed in Sec. 3.1) or 3 (D3Q19)        */
  int nx, ny, nz;     /* lattice size; nz ignored for dim = 2                 */
  int wall_last;      /* 1: halfway bounce-back walls at both ends of the last
                         axis (natural boundary conditions, eq. NaturalBCs);
                         0: periodic                                         */
  int storage;        /* TLB_F64 | TLB_F32 | TLB_F16 | TLB_BF16               */
  double tau, tau_phi, tau_psi;     /* relaxation times (eq. RelaxationTimes) */
  double gamma_phi, gamma_psi;      /* Gamma_phi, Gamma_psi (eq. EDF)         */
  double alpha;                     /* interface width parameter (eq. CmProfile) */
  double kappa[3];                  /* kappa_1..3 (eq. LandauFE)              */
  double kappa_c;                   /* coupling strength (eq. CouplingE)      */
  double dc;                        /* clamp of the signed distance in I     */
  double u0[3];                     /* initial uniform velocity               */
  double interface_pos;             /* default init: flat C1/C2 interface at
                                       this coordinate of the last axis (C1
                                       above); < 0: no interface (all C2)    */
  int forcing;                      /* force in the f collision:
                                       TLB_FORCE_EDM (exact difference method,
                                       eq. LBE; the paper's) or TLB_FORCE_GUO
                                       (Guo, Zheng and Shi 2002: BGK towards
                                       f^eq(rho, v), v = (j + F/2)/rho, plus
                                       (1 - 1/(2 tau)) w_i [3 (c_i - v) +
                                       9 (c_i.v) c_i] . F)                    */
  int state;                        /* TLB_STATE_POPULATIONS (default) or
                                       TLB_STATE_MOMENTS (see below)         */
  int force_form;                   /* free-energy force: TLB_FE_POTENTIAL
                                       (default: -rho grad mu~rho - phi grad
                                       mu_phi - psi grad mu_psi', eq. ForceFE
                                       through eq. GradPT) or
                                       TLB_FE_PRESSURE_TENSOR (grad(rho cs^2)
                                       - div p - psi grad(kappa_c (psi - I)),
                                       eq. ForceFE with the explicit tensor
                                       of App. A, the bulk pressure of eq.
                                       PressureV2); equal to second order in
                                       the lattice spacing                  */
} tlb_params;
enum { TLB_FE_POTENTIAL = 0, TLB_FE_PRESSURE_TENSOR = 1 };
enum { TLB_FORCE_EDM = 0, TLB_FORCE_GUO = 1 };
/* State kept between steps (tlb_params.state):
 * TLB_STATE_POPULATIONS -- the 3Q post-collision populations (any tau);
 * TLB_STATE_MOMENTS     -- at tau = tau_phi = tau_psi = 1 with TLB_FORCE_EDM
 *   (the paper's setting, Sec. 3.1) every post-collision population is an
 *   equilibrium (eq. EDF) of its cell, so 11 values per cell stand for all
 *   of them: rho - 1, u + du, phi, Gamma_phi mu_phi, psi, Gamma_psi mu_psi'
 *   and v (eq. LBE at tau = 1).  The pull of each step rebuilds every
 *   population from the cell it streams from.  The same method, another
 *   executed scheme: 88 bytes of state traffic per cell update in FP32
 *   against 456.  Only with FP32 storage (FP64 or FP32 in 2D); not in
 *   batches.  Initial states and populations written by the caller are
 *   pulled as populations by the next step; reads of populations or fields
 *   see the populations the moments stand for. */
enum { TLB_STATE_POPULATIONS = 0, TLB_STATE_MOMENTS = 1 };

typedef struct {
  int kind;           /* TLB_MEM_RING2D | TLB_MEM_TRI3D                        */
  int n_nodes;        /* markers                                               */
  int n_elems;        /* triangles (3D); ignored for rings (segments l->l+1)   */
  const double* X0;   /* host, n_nodes*3: initial positions (z ignored in 2D);
                         also the reference (stress-free) shape               */
  const int* elems;   /* host, n_elems*3 node indices, counter-clockwise seen
                         from outside (3D only; NULL for rings)              */
  double ks, kb;      /* 2D: stretching modulus kappa_s and bending modulus
                         kappa_b (eqs. DiscreteSE, DiscreteBE); 3D: kb is the
                         Helfrich bending modulus                            */
  double skalak_G, skalak_C;  /* 3D Skalak shear modulus and area ratio       */
} tlb_membrane_desc;

typedef struct {
  long step;          /* steps taken since init                                 */
  double mass[3];     /* FP64 sums of rho, phi, psi over the lattice            */
  double umax;        /* max |u|                                                */
  int n_caps;         /* number of membranes                                    */
  double area[8];     /* FP64 enclosed area (2D) / surface area (3D) per capsule */
  double volume[8];   /* FP64 enclosed volume per capsule (3D; 0 in 2D)         */
} tlb_diag;

/* Arena size (bytes) for a lattice and its membranes.  params and mems are
 * host pointers; n_mem membranes (at most 8).  Fails with TLB_ERR_ARG for
 * invalid sizes (lattice dims < 4, dim not 2/3, wall not along the last axis,
 * capsule larger than half the domain, ...). */
tlb_status tlb_state_bytes(const tlb_params* params, const tlb_membrane_desc* mems, int n_mem,
                           size_t* bytes);

/* Create a context on the current CUDA device.  arena: device pointer to
 * `bytes` bytes (at least tlb_state_bytes), owned by the caller.
 * cuda_stream: a cudaStream_t (NULL = legacy default stream).  The
 * membranes are uploaded here (their X0 is the reference shape).  The
 * context is not usable for stepping until tlb_init_fields. */
tlb_status tlb_create(const tlb_params* params, const tlb_membrane_desc* mems, int n_mem,
                      void* arena, size_t bytes, void* cuda_stream, void** ctx_out);

/* Initial state (the paper prints none; the reading is rho = 1, u = u0,
 * psi = I(X0), a flat C1/C2 interface of tanh profile (eq. CmProfile) along
 * the last axis, C1 = (1 - psi) s, C2 = (1 - psi)(1 - s), populations at
 * equilibrium (eq. EDF) with the chemical potentials of these fields).
 * C: host, 3*ncells doubles C1, C2, C3 (rho = C1+C2+C3, phi = C1-C2,
 *    psi = C3), or NULL for the default fields above.
 * u: host, 3*ncells doubles [component][cell] (z ignored in 2D), or NULL
 *    for the uniform params->u0. */
tlb_status tlb_init_fields(void* ctx, const double* C, const double* u);

/* Advance n_steps time steps (Sec. 3: membrane forces at X(t), spreading,
 * collision with exact-difference forcing, streaming, interpolation of
 * v(t+dt) and marker advection).  Enqueued on the context stream. */
tlb_status tlb_step(void* ctx, long n_steps);

/* Read a field (see TLB_FIELD_*) into host memory as doubles; n_values is
 * the capacity of dst in doubles (ncells, or 3*ncells for TLB_FIELD_U). */
tlb_status tlb_read_field(void* ctx, int field, double* dst, size_t n_values);

/* Marker positions of membrane `capsule` (n_nodes*3 doubles). */
tlb_status tlb_read_nodes(void* ctx, int capsule, double* dst, size_t n_values);

/* Overwrite the marker positions of membrane `capsule` (reference shape is
 * unchanged). */
tlb_status tlb_write_nodes(void* ctx, int capsule, const double* src, size_t n_values);

/* Populations as doubles, layout [set f,g,h][i][cell] with the velocity
 * ordering of the oracle/paper (D2Q9 as printed in Sec. 3.1; D3Q19: rest,
 * +x,-x,+y,-y,+z,-z, then the edge velocities of the xy, xz, yz planes with
 * sign pairs (+,+),(+,-),(-,+),(-,-)).  n_values = 3*Q*ncells.  Writing
 * rounds to the storage format. */
tlb_status tlb_read_populations(void* ctx, double* dst, size_t n_values);
tlb_status tlb_write_populations(void* ctx, const double* src, size_t n_values);

/* FP64 diagnostics of the current state (synchronises the stream). */
tlb_status tlb_diagnostics(void* ctx, tlb_diag* out);

/* The same diagnostics, computed with no device memory from the caller or
 * the arena: the reduction scratch is a fixed array inside the library
 * (about 26 KB on every GPU that loads it, kept until exit).  For callers
 * that cannot supply device memory at the point of the call, e.g. code in a
 * real-time loop where cudaMalloc (which synchronises the device) is not
 * allowed, or whose device memory belongs to another runtime.  The paper has
 * no counterpart; this is an operational variant of tlb_diagnostics.
 * - The first call on a device looks up the array's device address with
 *   that device current; make that first call before any stream capture.
 * - All calls share the one array: calls that overlap on the GPU (other
 *   streams, other contexts on the same device) race.  Serialise them.
 * - Rejects contexts with more than 8 capsules (TLB_ERR_ARG).
 * - Calls no cudaMalloc/cudaFree or any allocating routine. */
tlb_status tlb_diagnostics_static(void* ctx, tlb_diag* out);

/* Contact angle of every capsule with the C1/C2 interface phi = 0, in FP64
 * (synchronises the stream): the equilibrium measure of a capsule at a
 * fluid-fluid interface (Sec. 4.1; the paper prints no discrete recipe).
 * phi is interpolated to the markers with the kernel of eq. DiscreteDirac;
 * each membrane edge whose ends change sign holds a contact point at the
 * linear zero crossing; there the angle between the interface normal (the
 * interpolated lattice gradient of phi, pointing into C1) and the outward
 * membrane normal (the end markers' normals interpolated along the edge).
 * out: host, n_values >= 4*n_caps doubles; per capsule the mean angle over
 * its contact points (degrees), the smallest, the largest and the number of
 * contact points (mean/min/max NaN when it does not cross the interface).
 * Uses the population buffer the next step overwrites as scratch, so it
 * must not overlap a tlb_step of the same context. */
tlb_status tlb_contact_angle(void* ctx, double* out, size_t n_values);

/* Equilibrium residual in FP64 (synchronises the stream).  out[0] and
 * out[1]: the largest change of phi and of psi at any cell; out[2]: the
 * largest change of any coordinate of any membrane marker; each since the
 * reference state, which is the state at the previous tlb_residual call (or
 * at tlb_init_fields).  out[3] = max(out[0..2]) / (steps since the
 * reference), 0 if no step was taken.  The current state becomes the new
 * reference.  A NaN reads as +inf, so a diverged run never looks converged.
 * The paper says only that runs were continued until equilibrium was
 * reached (Sec. 4) and gives no criterion; this residual, taken every K
 * steps and compared with a tolerance, is the library's reading of it. */
tlb_status tlb_residual(void* ctx, double out[4]);

/* Run to equilibrium: tlb_step in chunks of check_every steps, tlb_residual
 * after each chunk, until the residual (out[3]) is at or below tol or
 * max_steps steps were taken.  *steps_done = the step count t at return,
 * *residual = the last residual (NaN if max_steps is 0); either may be NULL.
 * Synchronises the stream. */
tlb_status tlb_run(void* ctx, long max_steps, long check_every, double tol, long* steps_done, double* residual);

/* Checkpoint of the state of a context into host memory, and its restore.
 * The blob holds what a continued run reads (the current populations, the
 * profile I, the markers, the residual's reference state, the step count),
 * so that a context restored from it continues bit for bit as the saved one
 * would have.  tlb_save with host_blob NULL writes the size needed to *bytes;
 * otherwise *bytes is the blob's capacity on entry and its size on return.
 * tlb_load needs a context created with the same parameters and membranes
 * (TLB_ERR_ARG otherwise, or for a truncated or foreign blob); it need not be
 * initialised.  Both synchronise the stream.  Not in the paper: the
 * checkpoint/resume of a long relaxation run. */
tlb_status tlb_save(void* ctx, void* host_blob, size_t* bytes);
tlb_status tlb_load(void* ctx, const void* host_blob, size_t bytes);

/* Per-phase device time of n_steps steps, measured with CUDA events on the
 * context stream around each phase (synchronises the stream).  Phases:
 * moments (streamed-population moments), ibm (profile I, membrane and
 * coupling forces, spreading), collide (force + collision + streaming),
 * interp (interpolation and advection).  Times are totals in ms. */
typedef struct {
  long steps;
  double ms_moments, ms_ibm, ms_collide, ms_interp;
  long launches_per_step;
} tlb_profile;
tlb_status tlb_profile_steps(void* ctx, long n_steps, tlb_profile* out);

/* Choose the tile shape and z chunk of the collide plane sweep by timing
 * the collide kernel on the current state (CUDA events; the state is not
 * advanced).  Writes the chosen variant v = 3 form + tile (tile 0: 32x4,
 * 1: 32x8, 2: 64x4 in 3D; 0: 32, 1: 64, 2: 128 columns in 2D; form 0:
 * registers for 640 threads per SM, 1: 512 with the next population set
 * prefetched, 2: 768, 3: 1024; v = 12: tile 0 at 896) and planes per chunk
 * when the pointers are non-NULL.  Variants 13..18 (tiles 0..2 at 768,
 * then at 1024 threads per SM) are the collide for tau = tau_phi = tau_psi
 * = 1 with TLB_FORCE_EDM, the paper's setting (Sec. 3.1): there every
 * post-collision population is an equilibrium of the cell's moments (eq.
 * LBE), so that collide pulls no population and only stores; the moment
 * pass then also writes j.  Variants 22..27 are the same collide with two
 * x-adjacent cells per thread (tiles 0..2 at 384, then at 512 threads per
 * SM), every stored value of the pair written by one store; they need an
 * even nx.  Variants 28..31 are the tau = 1 collide on 32x16 tiles (3D):
 * one cell per thread at 768 / 1024, two cells per thread (even nx) at 384
 * / 512 threads per SM.  Variants 19..21 are tiles 0..2 of the general collide with the
 * pressure-tensor force.  They are tried only where they apply, and a new
 * context starts on variant 13 there (19 with the pressure-tensor force,
 * else 0).
 * Synchronises the stream.  Not in the paper: an autotuner for this
 * implementation's launch shape. */
tlb_status tlb_autotune(void* ctx, int* tile_variant, int* z_chunk);

/* Set the collide variant (0..31, as written by tlb_autotune; 13..18 and
 * 22..31 only where tau = tau_phi = tau_psi = 1 with TLB_FORCE_EDM and the
 * potential force, 22..27, 30 and 31 only with an even nx, 19..21 only with the
 * pressure-tensor force, else TLB_ERR_ARG)
 * and the planes per z chunk (1..nz) explicitly.  The results do not depend
 * on the choice beyond rounding. */
tlb_status tlb_set_tile(void* ctx, int tile_variant, int z_chunk);

/* Step graphs on (on != 0) or off (the default).  With graphs on, tlb_step
 * and tlb_run issue runs of 8 steps as one CUDA graph launch, captured once
 * per population buffer and collide variant from the same kernels the
 * direct launches use (the results are identical bit for bit); the first
 * step after markers were set from outside, the first step after
 * populations were written with moment storage, the steps of
 * tlb_profile_steps and a remainder below 8 steps run as direct launches.
 * Turning graphs off releases the captured graphs.  On the 128^3 capsule
 * the replay measured slower than direct launches (the captured side-stream
 * kernels lose their stream priority), hence off by default.  Not in the
 * paper: a launch mechanism of this implementation. */
tlb_status tlb_set_graphs(void* ctx, int on);

/* Number of CUDA kernel launches enqueued by the last tlb_step call (a
 * graph replay counts the kernels it holds). */
long tlb_last_launch_count(void* ctx);

/* Release the context (the arena stays owned by the caller). */
void tlb_destroy(void* ctx);

/* ---------------------------------------------------------------- batches
 * A batch advances many independent lattices together -- a parameter sweep
 * whose instances differ in size, parameters and membranes but share dim
 * and storage.  Each of the six phases of a step is one persistent kernel
 * launch over the work of every active instance, and two steps are
 * captured in one CUDA graph, so the launch count does not grow with the
 * number of instances.  Every instance is an ordinary context living in a
 * sub-arena of the batch arena, advanced by the same kernel bodies as
 * tlb_step: the state is the one tlb_step gives it alone (identical bits in
 * FP64; in FP32 the membrane kernels may round differently in the last
 * place, because the compiler may fuse multiply-adds differently inside the
 * batched kernels).  Not in the paper: it is
 * the sweep over capsule and fluid parameters of its Sec. 4 run as one
 * job. */
typedef struct {
  tlb_params params;
  const tlb_membrane_desc* mems; /* host, borrowed for the call */
  int n_mem;
} tlb_instance_desc;

/* Arena bytes of a batch of n_inst instances (each instance's
 * tlb_state_bytes, 256-byte aligned, plus about 2.1 KB of tables per
 * instance).  TLB_ERR_ARG if n_inst is not in 1..4096, an instance is
 * invalid (message names it) or dim/storage differ between instances. */
tlb_status tlb_batch_state_bytes(const tlb_instance_desc* inst, int n_inst, size_t* bytes);

/* Create the batch in `arena` (device, 256-byte aligned, at least
 * tlb_batch_state_bytes; owned by the caller until tlb_batch_destroy).
 * Every instance is created as by tlb_create on the given stream and is
 * active.  Instances must then be initialised (tlb_init_fields on the
 * handles of tlb_batch_instance).  Allocates no device memory. */
tlb_status tlb_batch_create(const tlb_instance_desc* inst, int n_inst, void* arena, size_t bytes,
                            void* cuda_stream, void** batch_out);

/* Context of instance i (borrowed: valid until tlb_batch_destroy; never
 * pass it to tlb_destroy).  Every single-context call works on it;
 * tlb_step on it advances that instance alone. */
tlb_status tlb_batch_instance(void* batch, int i, void** ctx_out);

/* Select the instances the batch calls advance: flags[i] != 0 (n_inst
 * entries, host).  All instances are active after tlb_batch_create. */
tlb_status tlb_batch_set_active(void* batch, const int* flags);

/* Advance every active instance n_steps steps (enqueued on the stream; the
 * host synchronises only while uploading the argument tables).
 * TLB_ERR_STATE if an active instance is not initialised. */
tlb_status tlb_batch_step(void* batch, long n_steps);

/* Run to equilibrium: advance the active instances in chunks of
 * check_every steps; after each chunk take every active instance's
 * residual (tlb_residual's out[3]) in one launch and deactivate the
 * instances at or below tol.  Returns when no instance is active or after
 * max_steps steps.  steps_done[i] = the step count t of instance i and
 * residual[i] = its last residual (NaN if it was inactive throughout); both
 * n_inst entries on the host, or NULL.  Synchronises the stream. */
tlb_status tlb_batch_run(void* batch, long max_steps, long check_every, double tol, long* steps_done,
                         double* residual);

/* Collide tile shape and z chunk of the batch, chosen by timing the batched
 * collide on the current state (not advanced); as tlb_autotune. */
tlb_status tlb_batch_autotune(void* batch, int* tile_variant, int* z_chunk);

/* Device time of each phase of n_steps batched steps (direct launches,
 * CUDA events around each phase; the state advances as by tlb_batch_step).
 * ms_per_phase[0..5] (host) receives the totals in ms of: moments with the
 * marker geometry and brick counts; elastic forces, distance scatter and
 * brick compaction; profile band and brick lists; spreading and profile
 * fill; collide; interpolation and advection.  Synchronises the stream. */
tlb_status tlb_batch_profile_steps(void* batch, long n_steps, double* ms_per_phase);

/* Kernel launches made by the last tlb_batch_step or tlb_batch_run (each
 * kernel of a graph launch counted). */
long tlb_batch_launch_count(void* batch);

/* Destroy the batch and its instance contexts (the arena stays the
 * caller's). */
void tlb_batch_destroy(void* batch);

/* ------------------------------------------------------- learned warm start
 * A 3D convolutional encoder-decoder guesses the equilibrium of a capsule-
 * on-interface run from its plain initial state (undeformed capsule on the
 * flat interface) and five parameters, so that the relaxation starts closer
 * to it.  Not in the paper; an addition of this library.  The plain start
 * stays the fallback, and the relaxation itself decides the equilibrium.
 *
 * Network on an E^3 lattice, channels c_l = base_channels * 2^l at level l
 * (edge E / 2^l), `levels` levels:
 *   input (16 channels): phi0, psi0 of the plain start, the five features,
 *     nine zeros;
 *   encoder: e_l = relu(conv3(relu(conv3(in_l)))), in_0 = input,
 *     in_l = 2x2x2 average pool of e_{l-1};
 *   decoder: d_l = relu(conv3(relu(conv3([nearest 2x upsample of d_{l+1} |
 *     e_l])))), d_{levels-1} = e_{levels-1};
 *   output y = conv1(d_0), 16 channels: y0 = correction of the phase
 *     indicator s = phi / (1 - psi) of the C1/C2 fluid, y2..y4 = displacement
 *     field, the rest (y1 included) unused by the warm start.
 * conv3 is 3x3x3 with zero padding, conv1 is 1x1x1; every conv has a bias.
 * Parameters, in order, per conv: W[tap][ci][co] (tap = (kz*3 + ky)*3 + kx
 * for the input offset (kz-1, ky-1, kx-1)), then b[co]; FP32 on the host.
 * Activations are stored as bf16, the convolutions run on the tensor cores
 * with FP32 accumulation: the 3x3x3 convolutions of the forward pass and of
 * the input gradient on the fifth-generation tensor cores (tcgen05, the
 * accumulator in tensor memory, the operands loaded by TMA; the default) or
 * on the warp-level mma.sync path, the weight gradients and the 1x1x1
 * convolution on mma.sync.
 * Features (normalised by the caller): kappa_1..3, Skalak G, R / E.
 * Training loss for targets t0, t1 of y0, y1 (FP32 [B][E^3]; for the warm
 * start t0 = s_eq - s0 outside the capsule, 0 inside, and t1 = 0) and marker
 * offsets off_t = X_eq - X0 (FP32 [B][max_nodes][3]):
 *   mean over samples and cells of (y0 - t0)^2 + (y1 - t1)^2
 *   + lambda * mean over samples, markers and axes of
 *     (trilinear(y2..y4)(X0) - off_t)^2.
 * Input tensors x are bf16 [B][E^3][16] (device). */
typedef struct {
  int edge;          /* E: multiple of 2^(levels-1), 2^levels..256 */
  int base_channels; /* c_0: 16, 32, 48 or 64 */
  int levels;        /* 2..4 */
  int max_batch;     /* samples per call, 1..64 */
  int max_nodes;     /* markers per sample in training, 0..2^20 */
} tlb_net_desc;

tlb_status tlb_net_param_count(const tlb_net_desc* desc, size_t* n);
tlb_status tlb_net_state_bytes(const tlb_net_desc* desc, size_t* bytes);
/* arena: device, 256-byte aligned, >= tlb_net_state_bytes, the caller's. */
tlb_status tlb_net_create(const tlb_net_desc* desc, void* arena, size_t bytes, void* cuda_stream, void** net_out);
/* Parameters (host FP32, n = tlb_net_param_count); resets the Adam state. */
tlb_status tlb_net_set_params(void* net, const float* host, size_t n);
tlb_status tlb_net_get_params(void* net, float* host, size_t n);
/* Parameter gradient of the last tlb_net_train_step (host FP32). */
tlb_status tlb_net_get_grads(void* net, float* host, size_t n);
/* Input of one sample (x_dev: bf16 [E^3][16], device) from a context that
 * holds its plain initial state, with features feats[5] (host). */
tlb_status tlb_net_input(void* net, void* ctx, const double* feats, void* x_dev);
/* Output y (FP32 [batch][E^3][16], device, or NULL) of batch inputs. */
tlb_status tlb_net_forward(void* net, const void* x_dev, int batch, float* y_dev);
/* Forward, loss (returned in *loss_out, host), backward; then one Adam step
 * (Kingma and Ba 2015; beta1 0.9, beta2 0.999, eps 1e-8, step size lr) when
 * update != 0.  n_nodes: host [batch] marker counts (NULL: no marker term).
 * Every sum is order-independent (the marker term's gradient is scattered
 * in 64-bit fixed point, each contribution clamped to +-2^8), so the same
 * call from the same state gives the same parameters bit for bit.
 * Synchronises the stream. */
tlb_status tlb_net_train_step(void* net, const void* x_dev, const float* t0_dev, const float* t1_dev,
                              const float* X0_dev, const float* off_dev, const int* n_nodes, int batch,
                              double lambda, double lr, int update, double* loss_out);
/* Warm start of a context that holds its plain initial state (tlb_init_fields
 * with NULL fields, no step taken; 3D, edge^3 cells, FP32 arithmetic, one
 * capsule):
 *  - markers: D = trilinear(y2..y4)(X0); X = X0 + T + ((D - T).n) n with T
 *    the mean of D and n the unit vertex pseudo-normals (no tangential
 *    shear of the reference mesh);
 *  - psi = I(X) + l_psi 4 I(X)(1 - I(X)): the profile of the moved
 *    markers, as the plain start takes psi = I(X0);
 *  - phi = (1 - psi)(s + l_phi (1 - s^2)_+) with s = s0 + y0 and
 *    s0 = phi0 / (1 - psi0);
 *  - rho = 1, u = 0; l_psi and l_phi restore the plain totals of psi and
 *    phi (the method conserves them) by moving the membrane's profile and
 *    the C1/C2 interface, leaving the bulk values where they are;
 * then the equilibrium populations of these fields, as tlb_init_fields.
 * Synchronises. */
tlb_status tlb_net_warm_start(void* net, void* ctx, const double* feats);
/* Choose the tensor-core path of the 3x3x3 convolutions: 2 (the default)
 * tcgen05 in a persistent warp-specialised pipeline whose operands arrive by
 * TMA, 1 tcgen05 with cp.async operand staging, 0 mma.sync.  They agree up
 * to the order of the FP32 accumulation.  TLB_ERR_ARG for other values. */
tlb_status tlb_net_set_tcgen05(void* net, int mode);
/* Synchronise the net's stream and read (then clear) its status word: bit 0
 * set when a tcgen05 kernel gave up waiting for the tensor core (its
 * outputs are then not written); TLB_ERR_CUDA in that case.
 * tlb_net_train_step with loss_out and tlb_net_warm_start check it
 * themselves. */
tlb_status tlb_net_status(void* net, unsigned* status);
/* Kernel launches of the last tlb_net_* call that computes. */
long tlb_net_launch_count(void* net);
void tlb_net_destroy(void* net);

/* Message of the last failed call on this thread ("" if none). */
const char* tlb_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* TLB_H */
