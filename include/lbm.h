/*
 * lbm.h -- C ABI of the GB300 (sm_103a) implementation of one time step of the D2Q9
 * chemical-potential multiphase lattice Boltzmann method with the multiphase curved boundary
 * condition of Yao, Liu, Zhong & Wen, "Multiphase curved boundary condition in lattice
 * Boltzmann method" (arXiv 2203.04508).
 *
 * Conventions shared by every entry point
 *  - Every call returns an lbm_status and never aborts the process.  After a failure,
 *    lbm_last_error(ctx) holds a one-line explanation.  A context whose device work failed
 *    (LBM_ECUDA) stays failed: every later call returns the same status.
 *  - Device memory is never allocated by the library.  The caller allocates one device
 *    workspace of at least lbm_workspace_size() bytes (for instance a PyTorch uint8 tensor),
 *    passes it to lbm_create(), and keeps it alive until lbm_destroy().  The context itself
 *    (a small host structure) is owned by the library.
 *  - All device work is issued asynchronously on the CUDA stream given to lbm_create()
 *    (a cudaStream_t; NULL means the legacy default stream).  Calls that return host data
 *    synchronise that stream.
 *  - Node (x, y) of an nx-by-ny lattice has the dense linear index n = y*nx + x in every
 *    array that crosses this interface; x is periodic.  Arrays of populations hold 9 planes of
 *    nx*ny values, plane i for lattice velocity e_i in the order of the columns of the
 *    transformation matrix M (Eq. 2): e_0 = (0,0); e_1..e_4 = (1,0),(0,1),(-1,0),(0,-1);
 *    e_5..e_8 = (1,1),(-1,1),(-1,-1),(1,-1).
 *  - Calls out of order (a step before lbm_init, for example) return LBM_ESTATE.
 */
#ifndef LBM_GB300_H
#define LBM_GB300_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct lbm_ctx lbm_ctx;

typedef enum {
  LBM_OK = 0,
  LBM_EINVAL = 1,     /* invalid argument or configuration */
  LBM_ENOMEM = 2,     /* workspace too small, or a geometry exceeds its link capacity */
  LBM_ECUDA = 3,      /* a CUDA call failed (message in lbm_last_error) */
  LBM_ESTATE = 4,     /* call out of order */
  LBM_EUNSTABLE = 5,  /* a NaN or Inf appeared in the mass audit */
  LBM_ETIMEOUT = 6,   /* a bounded device-side wait gave up */
  LBM_EINTERNAL = 7,
  LBM_ECORRUPT = 8    /* a checkpoint file is truncated, altered or not a checkpoint */
} lbm_status;

/* Equation of state of the nonideal fluid (Sec. 2.2). */
typedef enum {
  LBM_EOS_NONE = 0,   /* no nonideal force: single-phase fluid, force = rho g only */
  LBM_EOS_CS = 1,     /* Carnahan-Starling: p0 = rho R T (1+eta+eta^2-eta^3)/(1-eta)^3 - a rho^2,
                         eta = b rho / 4 */
  LBM_EOS_PR = 2      /* Peng-Robinson, Eqs. 10-11 */
} lbm_eos_kind;

typedef enum { LBM_COLL_BGK = 0, LBM_COLL_MRT = 1 } lbm_coll;  /* Eq. 4 */

/* Treatment of each cut fluid-solid link. */
typedef enum {
  LBM_BC_PRESENT = 0, /* the paper's scheme: Eqs. 16-17 with the nonideal term, plus Eq. 18 */
  LBM_BC_IBC = 1,     /* linear interpolation without the nonideal term and without Eq. 18 */
  LBM_BC_MIBC = 2,    /* IBC plus the mass compensation of Eq. 18 */
  LBM_BC_HBB = 3      /* halfway bounce-back: f_ibar(x1, t+1) = f~_i(x1, t) */
} lbm_bc;

typedef enum { LBM_FP32 = 0, LBM_FP64 = 1 } lbm_prec;

/* Nonideal force. */
typedef enum {
  LBM_FORCE_CHEMPOT = 0, /* the paper's chemical-potential force, Eqs. 9 and 12 */
  LBM_FORCE_PSEUDO = 1   /* the pseudopotential (Shan-Chen) force with a pseudopotential built
                            from the EOS: F = -G psi(x) sum_i w_i psi(x + e_i) e_i, G = -1,
                            w = 1/3 on the axes, 1/12 on the diagonals,
                            psi = [2 (rho c_s^2 - k^2 p0(rho))]^(1/2) (clamped at zero), so that
                            rho c_s^2 + (G/2) psi^2 = k^2 p0; kappa is not used.  Exact-difference
                            forcing, Eq. 15 and Eqs. 16-18 are unchanged.  Single lattices only:
                            the batch and reverse-mode calls return LBM_EINVAL for it. */
} lbm_force_model;

/* How the populations are held in memory (Eq. 5's streaming).
 *  LBM_LAYOUT_AB: two lattices; the collide of each step reads one and pushes into the other.
 *  LBM_LAYOUT_AA: one lattice, updated in place, half the population memory.  Steps alternate:
 *    the first reads each node's own nine slots and writes its post-collision populations back
 *    into the same node's slots, each into the slot of its opposite direction (the state then
 *    holds f_i(x) in slot ibar of node x - e_i); the next reads the populations from those
 *    slots and writes each f~_i(x) into slot i of node x + e_i (the state is in natural order
 *    again).  Each node reads and writes the same nine locations, so no step races with another
 *    node.  The boundary phase, the density pass and every read-out address the slots of the
 *    state's current order; the pre-collision moments the boundary links need (Eq. 17's F_i
 *    uses u at x1) are saved for the boundary nodes before the collide overwrites them.  The
 *    values equal those of LBM_LAYOUT_AB bit for bit, also in a batch (lbm_batch_*, whose
 *    instances may mix both layouts).  The slab and reverse-mode calls return LBM_EINVAL for it,
 *    as do collide kernel 2 and the fused chemical-potential pass (lbm_set_collide_kernel,
 *    lbm_set_mu_kernel). */
typedef enum { LBM_LAYOUT_AB = 0, LBM_LAYOUT_AA = 1 } lbm_layout;

/*
 * Configuration of one lattice.  Geometry: nodes sit at integer (x, y), 0 <= x < nx,
 * 0 <= y < ny.  A node is solid when it lies inside a cylinder, (x-cx)^2 + (y-cy)^2 <= r^2,
 * or, with walls = 1, when y <= y_bottom or y >= y_top; walls = 0 makes y periodic.  The
 * wall lines must satisfy 1 <= y_bottom < 2 and ny-3 < y_top <= ny-2 (two solid rows each,
 * as the fourth-order stencils need), and each cylinder must keep two nodes from the
 * periodic edges.
 *
 * Wettability (Sec. 2.3): solid nodes carry the chemical potential
 *     mu^_w = k^2 mu_sat + dmu_w,
 * where mu_sat is the bulk chemical potential at coexistence; dmu_w = 0 is a neutral wall
 * (90 degrees), dmu_w < 0 hydrophilic, dmu_w > 0 hydrophobic.  With LBM_FORCE_PSEUDO the same
 * fields hold a wall factor c_w > -1 instead: the solid layers carry psi(rho_s) (1 + c_w), rho_s
 * their Eq. 15 density; c_w > 0 hydrophilic, c_w < 0 hydrophobic, c_w = 0 close to neutral.
 */
typedef struct {
  int32_t nx, ny;
  int32_t walls;
  double y_bottom, y_top;
  int32_t eos;                 /* lbm_eos_kind */
  double a, b, R, T_over_Tc;   /* EOS constants; temperature as a fraction of the critical one */
  double omega;                /* acentric factor (Peng-Robinson alpha(T)) */
  double k, kappa;             /* Eq. 12: mu^ = k^2 psi'(rho) - kappa^ lap(rho) */
  int32_t coll;                /* lbm_coll */
  double tau;                  /* BGK relaxation time */
  double s_e, s_eps, s_q, s_nu;/* MRT rates of Eq. 3 (s_nu = 1/tau gives nu = (tau-1/2)/3) */
  double gx, gy;               /* body-force acceleration (force rho g added to Eq. 9) */
  int32_t bc;                  /* lbm_bc */
  int32_t precision;           /* lbm_prec: storage and arithmetic type of the populations */
  double rho_ref;              /* populations are stored as f_i - w_i rho_ref; a negative value
                                  selects the gas coexistence density in FP32 and 0 in FP64 */
  int32_t n_cyl;
  const double* cx;            /* host arrays of n_cyl values, read during lbm_create only */
  const double* cy;
  const double* r;
  const double* dmu_w;
  double dmu_w_walls;          /* dmu_w of the two flat walls */
  int32_t force_model;         /* lbm_force_model */
  int32_t layout;              /* lbm_layout; 0: two lattices */
} lbm_config;

/* Initial state, Eq. 19: around each droplet a tanh profile of width `width` between the
 * Maxwell coexistence densities; velocity (ux0, uy0) weighted by the local liquid fraction;
 * populations at equilibrium. */
typedef struct {
  int32_t n_drop;
  const double* x0;            /* host arrays of n_drop values */
  const double* y0;
  const double* r0;
  const double* ux0;           /* may be NULL: zero */
  const double* uy0;           /* may be NULL: zero */
  double width;
} lbm_init_spec;

/* Bytes of device workspace one lattice of this configuration needs (populations in two
 * lattices, or in one plus three staging planes with LBM_LAYOUT_AA; density and
 * chemical-potential planes, node flags, boundary-link and solid-layer lists sized for the
 * geometry's upper bound, reduction scratch). */
lbm_status lbm_workspace_size(const lbm_config* cfg, size_t* bytes);

/* Validates cfg, solves the EOS set-up on the host (critical point and Maxwell coexistence
 * densities, Sec. 4), and binds the caller's device workspace (device pointer, 256-byte
 * aligned, `bytes` >= lbm_workspace_size).  No device work is issued yet.
 * stream: cudaStream_t of the caller (may be NULL). */
lbm_status lbm_create(const lbm_config* cfg, void* stream, void* workspace, size_t bytes,
                      lbm_ctx** out);

/* Classifies nodes (fluid, first and second solid layer of Eq. 15, deeper solid), finds every
 * cut link (x1 fluid, x1 + e_i solid) with its fraction q (Sec. 3.1; the smaller root of
 * |x1 + q e_i - c|^2 = r^2 for a cylinder, q = y1 - y_bottom or y_top - y1 for a wall),
 * builds the link list sorted by (x1, i), and writes the constant chemical potential of the
 * solid layers.  q is evaluated in FP64 without contractions, so identical inputs give
 * identical bits on any IEEE host.  Synchronises the stream. */
lbm_status lbm_build_links(lbm_ctx* ctx);

/* Counts from lbm_build_links: cut links, boundary-fluid nodes, fluid nodes, first- and
 * second-layer solid nodes. */
lbm_status lbm_counts(lbm_ctx* ctx, int64_t* n_links, int64_t* n_boundary_nodes,
                      int64_t* n_fluid, int64_t* n_solid1, int64_t* n_solid2);

/* Copies the link list to caller-owned HOST arrays of at least n_links entries: node x1,
 * direction i, q (FP64), x2 = x1 - e_i, and whether x2 is fluid. */
lbm_status lbm_get_links(lbm_ctx* ctx, int64_t capacity, int32_t* x1, int32_t* dir, double* q,
                         int32_t* x2, int32_t* x2_fluid);

/* Node classes to a caller-owned HOST array of nx*ny bytes: 0 fluid, 1 first solid layer,
 * 2 second solid layer, 3 deeper solid. */
lbm_status lbm_get_kind(lbm_ctx* ctx, uint8_t* kind);

/* Eq. 19 initial state on the device, then the audit of its mass M0 (FP64), both queued on the
 * context's stream; the host reads M0 at the first call that needs it (lbm_mass, lbm_save).
 * Does not wait for the device; the init arrays may be reused on return. */
lbm_status lbm_init(lbm_ctx* ctx, const lbm_init_spec* init);

/* Advances n time steps, asynchronously on the context's stream (captured into a CUDA
 * graph on first use).  Each step: density (Sec. 2.1); solid-node densities (Eq. 15);
 * chemical potential (Eq. 12); nonideal force (Eq. 9) with exact-difference forcing
 * (Eqs. 13-14), collision (Eq. 4) and streaming (Eq. 5) fused in one kernel; then every cut
 * link by Eq. 16 (q < 1/2) or Eq. 17 (q >= 1/2) with the per-node compensation of Eq. 18
 * accumulated in FP64.  The density pass of the next state overlaps the links on a second
 * stream the context creates on first use (ordered with the context's stream by events; no
 * device memory is allocated); to the caller the work is on the context's stream. */
lbm_status lbm_step(lbm_ctx* ctx, int64_t n);

/* Captures and instantiates the step graphs that lbm_step(n) will launch from the current state,
 * without running them, so that the first such call spends no host time on capture (n >= 0;
 * nothing to do on the legacy default stream, which lbm_step does not capture).  LBM_ESTATE
 * before lbm_init. */
lbm_status lbm_prepare_steps(lbm_ctx* ctx, int64_t n);

/* Density and velocity v = u + F/(2 rho) of the current state (the macroscopic velocity
 * defined under Eq. 14) into caller-owned arrays of nx*ny values of the context's precision
 * (float or double); zero at solid nodes.  on_device != 0: device pointers, written
 * asynchronously; 0: host pointers, the call synchronises (page-locked host arrays are written
 * by the read-out kernel directly, others through device staging memory and copies). */
lbm_status lbm_fields(lbm_ctx* ctx, void* rho, void* vx, void* vy, int32_t on_device);

/* Checkpoint / resume.  lbm_save writes the state of an initialised context to `path`: a
 * header (magic "LBMGBCK1", format version, a hash of the configuration, lattice size,
 * precision, step count, lattice parity, M0), then the current lattice's populations as stored
 * (offset form, padded rows), the per-boundary-node FP64 carry of Eq. 18, the per-step
 * compensation ring with its counter, and a CRC-32 of everything before it.  lbm_load restores
 * such a state into a context created with the same configuration and past lbm_build_links (in
 * place of lbm_init): stepping on from it gives the bits of the run that was saved.  A file
 * that is truncated, altered or not a checkpoint returns LBM_ECORRUPT; a checkpoint of another
 * configuration LBM_EINVAL; I/O failures LBM_EINVAL with the message in lbm_last_error.  Both
 * synchronise the context's stream.  Files carry host byte order (little-endian on the x86 and
 * Arm hosts this targets). */
lbm_status lbm_save(lbm_ctx* ctx, const char* path);
lbm_status lbm_load(lbm_ctx* ctx, const char* path);

/* Density of the current state along one column: rho = sum_i f_i (Sec. 2.1) of the nodes
 * (x, y0 + j), j = 0 .. n-1, NaN at solid nodes, as n FP64 values into `out` (host memory, or
 * device memory if on_device).  Requires 0 <= x < nx, y0 >= 0, n >= 1, y0 + n <= ny, else
 * LBM_EINVAL.  For diagnostics that follow an interface along a line, such as the film on top
 * of a cylinder (Sec. 4.5), without copying the whole field.  Synchronises when copying to the
 * host. */
lbm_status lbm_column_density(lbm_ctx* ctx, int32_t x, int32_t y0, int32_t n, double* out, int32_t on_device);

/* Largest speed |v| over the fluid nodes of the current state, v = u + F/(2 rho) as lbm_fields
 * returns it (the velocity defined under Eq. 14), formed in FP64 from the lattice's precision;
 * NaN when a fluid node's velocity is not a number.  Synchronous (one small read-back); it forms
 * the density and chemical potential of the current state like lbm_fields and leaves the next
 * step's result unchanged.  Status: LBM_ESTATE before lbm_init, LBM_EINVAL for a null pointer. */
lbm_status lbm_max_speed(lbm_ctx* ctx, double* vmax);

/* Populations f_i (not offset) of the current state, 9 planes of nx*ny values of the
 * context's precision; zero at solid nodes.  on_device as for lbm_fields. */
lbm_status lbm_populations(lbm_ctx* ctx, void* f, int32_t on_device);

/* Total mass M = sum over fluid nodes of sum_i f_i (FP64 on the device), the initial mass,
 * and the domain sum of the Eq. 18 compensation of the last step.  FP32 lattices sum each node's
 * nine populations with compensated FP32 arithmetic (TwoSum; within 2.3e-13 of the node's sum
 * of |f_i|) and the nodes in FP64.  Synchronises.  Returns LBM_EUNSTABLE when the populations
 * hold a NaN or Inf. */
lbm_status lbm_mass(lbm_ctx* ctx, double* M, double* M0, double* dM_last);

/* Per-step compensation sums (Eq. 18) of the last min(n, steps taken, 4096) steps, oldest
 * first, to a caller-owned HOST array; *n_out receives the count.  Synchronises. */
lbm_status lbm_dM_history(lbm_ctx* ctx, double* out, int64_t n, int64_t* n_out);

/* Domain sum of the Eq. 18 compensation of the last step (8 bytes read back; synchronises). */
lbm_status lbm_last_dM(lbm_ctx* ctx, double* dM);

/* The same 8 bytes, written on the context's stream into host memory `dM` without waiting: the
 * value is there once the stream has reached this point (any synchronising call, or the
 * stream's own synchronisation).  Page-locked `dM` is stored into by a one-thread kernel, which
 * costs the following steps less than a copy-engine copy would, so a caller can read every
 * step's result without stalling the GPU; pageable memory is copied, and that copy itself
 * waits for the stream. */
lbm_status lbm_last_dM_async(lbm_ctx* ctx, double* dM);

/* Advances n steps like lbm_step, launching the five phases one by one with CUDA events on
 * the context's stream between them, and adds each phase's device time (ms) to ms5:
 * [0] density, [1] solid layers (Eq. 15), [2] chemical potential, [3] force + collision +
 * streaming, [4] boundary links (Eqs. 16-18).  Synchronises after every step. */
lbm_status lbm_profile_steps(lbm_ctx* ctx, int64_t n, double* ms5);

/* EOS summary (host FP64): Tc, rho_c, T, alpha, rho_g, rho_l, mu_sat, p_sat. */
lbm_status lbm_eos_info(lbm_ctx* ctx, double* out8);

/* Number of kernel launches one lbm_step(ctx, 1) issues. */
lbm_status lbm_launches_per_step(lbm_ctx* ctx, int64_t* n);

/* Force + collision + streaming kernel of an FP32 lattice (Eqs. 4, 5, 9 or the pseudopotential
 * force, 13): kind 0 the plain kernel (one 32 x 8 tile per block, populations loaded by each
 * thread), kind 1 the TMA-pipelined one (a persistent grid; each block's next tiles -- the nine
 * population planes, the density and chemical-potential halo -- stream into shared memory by
 * cp.async.bulk.tensor while it computes the current one), kind 2 the same pipeline walking
 * 32-column strips upwards through bands of tile rows, which also sums the populations streaming
 * into the rows it has finished into the next state's density (Sec. 2.1) and psi'(rho), so that
 * the step's separate density pass shrinks to the strips' edge columns and the bands' edge rows.
 * All give the same values, bit for bit.  Kind 2 needs the chemical-potential force with an
 * equation of state, nx a multiple of 32 and ny of 8, and a whole lattice (not a slab); under the
 * fused chemical-potential pass (lbm_set_mu_kernel 3) the step runs kind 1 instead, and
 * lbm_get_collide_kernel reports the kind that runs.  lbm_build_links picks kind 1 where it could
 * encode the tensor maps (FP32 with a driver that has the encoder) and the lattice gives each
 * persistent block at least 16 tiles, kind 0 otherwise; kind 2 runs only when set (on GB300 its
 * added density work slows a collide kernel that is already bound by instruction issue more
 * than the separate density pass costs).  Setting a kind the lattice cannot run returns
 * LBM_EINVAL.  Call after lbm_build_links; the step graphs are captured again.  A
 * bounded wait of kind 1 or 2 that gives up is reported as LBM_ETIMEOUT by the next lbm_mass. */
lbm_status lbm_set_collide_kernel(lbm_ctx* ctx, int32_t kind);
/* The collide kernel lbm_step runs now (0 plain, 1 TMA-pipelined, 2 column sweeps). */
lbm_status lbm_get_collide_kernel(lbm_ctx* ctx, int32_t* kind);

/* The chemical-potential pass (Eq. 12) of the chemical-potential force model: 0 one node a
 * thread, 1 four (FP64: two) consecutive nodes of a row a thread from 16-byte loads, 2 (FP32
 * only) row sweeps, a thread walking down a column of four-node groups with the stencil's rows
 * in registers.  The default is 2 for FP32 lattices of at least four 512 x 16-node blocks per
 * SM, else 1.  All three give the same bits.  Call
 * after lbm_build_links; the step graphs are captured again.  LBM_EINVAL for another value or
 * for 2 on an FP64 lattice. */
lbm_status lbm_set_mu_kernel(lbm_ctx* ctx, int32_t kind);

/* Polls before the TMA-pipelined kernel's wait for a tile's loads gives up (default 2^22, a
 * second or more); 0 makes every such wait give up at once, to test the timeout path.  A block
 * that gives up still waits, with the default limit, for its own copies in flight, then leaves;
 * the next lbm_mass returns LBM_ETIMEOUT and the context stays in that state (the lattice is not
 * a valid state any more).  Call after lbm_build_links; the step graphs are captured again. */
lbm_status lbm_set_spin_limit(lbm_ctx* ctx, int64_t polls);

/* Sets the state (a new initial state, in place of lbm_init) from 9 arrays of ny x nx
 * absolute populations in the context's precision, population i at offset i*nx*ny (the layout
 * lbm_populations writes); values at non-fluid nodes are ignored.  Clears the step counter,
 * the compensation history and the Eq. 18 carries, and takes the state's mass as the new M0.
 * on_device: 1 if f is a device pointer, 0 for host memory (which may be reused on return; the
 * call does not wait for the device, M0 is read when first needed, as after lbm_init).  With
 * FP32 offset storage the values are stored as f_i - w_i rho_ref, so a state read out by
 * lbm_populations comes back to within an ulp of each offset population. */
lbm_status lbm_set_populations(lbm_ctx* ctx, const void* f, int32_t on_device);

/* ---- Objective and reverse mode (gradients through the time integration) ----------------
 * The step (Eqs. 9, 12, 13, 15-18) is differentiable in the populations and in the parameters
 * of the wall: the wall chemical potential offset dmu_w of every cylinder and of the
 * flat walls, and the centre (cx, cy) of every cylinder, which enters only through the cut
 * fractions q of Eqs. 16-17 (the set of cut links stays fixed under an infinitesimal change).
 * lbm_forward_checkpointed advances the lattice and keeps checkpoints in a caller-owned device
 * workspace; lbm_adjoint then runs the step's transpose backwards through those steps
 * (recomputing each segment of `every` steps from its checkpoint) and returns dJ/d(parameters)
 * for a seed dJ/d(final state).  Every step of both passes runs in CUDA kernels.
 *
 * Parameter-gradient layout (3 n_cyl + 1 doubles): [0, n_cyl) dJ/d dmu_w of each cylinder,
 * [n_cyl] dJ/d dmu_w_walls, then dJ/dcx_k, dJ/dcy_k at [n_cyl + 1 + 2k], [n_cyl + 2 + 2k]. */

/* Bytes of device workspace for a checkpointed forward pass of n_steps steps with a
 * checkpoint every `every` steps (0: ceil(sqrt(n_steps))).  The workspace holds
 * ceil(n_steps/every) + every + 1 population lattices plus 2 every + 34 planes (the density
 * and chemical potential of each step of a segment, and the adjoint state). */
lbm_status lbm_adjoint_workspace_size(lbm_ctx* ctx, int64_t n_steps, int64_t every, size_t* bytes);

/* Advances n_steps like lbm_step, storing a checkpoint (populations and Eq. 18 carries) at
 * the start of every segment in `workspace` (device, 256-byte aligned, caller-owned, at least
 * lbm_adjoint_workspace_size bytes; it must stay untouched until lbm_adjoint).  Asynchronous.
 * Any later lbm_step / lbm_init / lbm_build_links invalidates the checkpoints. */
lbm_status lbm_forward_checkpointed(lbm_ctx* ctx, int64_t n_steps, int64_t every, void* workspace, size_t bytes);

/* Droplet objective of the current state for cylinder `body` (0 <= body < n_cyl):
 *   J = y_cm + L_wet,  y_cm = sum (rho - rho_g) y / sum (rho - rho_g) over fluid nodes,
 *   L_wet = (2 pi r_body / N) sum phi over the N fluid nodes with a cut link into the body,
 *   phi = (rho - rho_g)/(rho_l - rho_g)  (the liquid fraction beside the wall).
 * Writes J (host double); if dJ_drho is not NULL also writes dJ/drho, row-major ny x nx in the
 * context's precision (zero off the fluid), to device (on_device = 1) or host memory.
 * Synchronises the stream. */
lbm_status lbm_objective(lbm_ctx* ctx, int32_t body, double* J, void* dJ_drho, int32_t on_device);

/* Reverse sweep through the steps of the last lbm_forward_checkpointed, which must end at the
 * current state (LBM_ESTATE otherwise).  Seeds: dJ_drho (ny x nx, row-major) and dJ_df (9
 * arrays of ny x nx, population i at offset i*nx*ny), both of the final state, in the context's
 * precision; either may be NULL (zero).  Writes the parameter gradient (host, 3 n_cyl + 1
 * doubles, layout above; FP64 accumulation) if grad is not NULL, and dJ/df of the first state
 * (same layout as dJ_df) if dJ_df0 is not NULL.  on_device applies to the three arrays.  The
 * lattice state, step counter, compensation history and carries are those after the forward
 * pass again when it returns; the call may be repeated.  The recomputation of each segment
 * overlaps the reverse steps of the previous one on a second stream the context creates on
 * first use (the workspace holds two segment buffer sets for that).  Synchronises the stream. */
lbm_status lbm_adjoint(lbm_ctx* ctx, const void* dJ_drho, const void* dJ_df, int32_t on_device, double* grad,
                       void* dJ_df0);

/* ---- Batches: many independent lattices advanced together -------------------------------
 * All instances share one precision and the chemical-potential force; sizes, physics, geometry,
 * initial states and population layouts (lbm_config.layout) may differ.
 * Each instance is an ordinary lbm_ctx inside the batch (lbm_batch_instance), so lbm_fields,
 * lbm_mass, lbm_dM_history ... work on it; lbm_step on a single instance is not allowed while it
 * belongs to a batch (lbm_batch_step then returns LBM_ESTATE). */
typedef struct lbm_batch lbm_batch;

/* Device workspace for n instances: their own workspaces plus the batch's work lists. */
lbm_status lbm_batch_workspace_size(int32_t n, const lbm_config* cfgs, size_t* bytes);

/* Creates the n instances (lbm_create each, on sub-ranges of the one workspace). */
lbm_status lbm_batch_create(int32_t n, const lbm_config* cfgs, void* stream, void* workspace, size_t bytes,
                            lbm_batch** out);

/* lbm_build_links for every instance, then the flat work lists of the persistent kernel: tiles
 * of 256 consecutive nodes and chunks of 256 solid-layer / boundary entries across all
 * instances.  Synchronises. */
lbm_status lbm_batch_build_links(lbm_batch* b);

/* lbm_init for every instance with specs[k] (n specs).  Synchronises. */
lbm_status lbm_batch_init(lbm_batch* b, const lbm_init_spec* specs);

/* Advances every instance n steps in ONE cooperative launch of a persistent kernel (captured
 * into a CUDA graph on first use for this n): each step runs the phases of lbm_step over all
 * instances' work, separated by grid barriers; per-instance compensation sums go to each
 * instance's ring as with lbm_step.  Asynchronous; lbm_batch_check reports a barrier timeout. */
lbm_status lbm_batch_step(lbm_batch* b, int64_t n);

/* Synchronises and returns LBM_ETIMEOUT if a grid-barrier wait of the last launches gave up
 * (the kernel then left without finishing its steps). */
lbm_status lbm_batch_check(lbm_batch* b);

/* Polls before a grid-barrier wait gives up (default 2^22, about a second or more); 0 makes
 * every wait give up at once (used to test the timeout path).  Clears the error flag. */
lbm_status lbm_batch_set_spin_limit(lbm_batch* b, int64_t polls);

/* Shape of the node tiles of the persistent kernel: 2^log2w nodes wide and 256 / 2^log2w
 * rows high, log2w in 4 .. 8 (16x16, 32x8, 64x4, 128x2, 256x1; default 5).  Every shape gives
 * identical results; only the speed differs (how well a warp's row segment and the stencils'
 * nearby rows fit the instances' widths).  LBM_EINVAL outside the range.  Synchronises. */
lbm_status lbm_batch_set_tile(lbm_batch* b, int32_t log2w);

/* Schedule of the persistent kernel.  groups = 1: every instance runs the same phase between
 * two grid barriers (lockstep).  groups = 2: the instances are split into two groups of about
 * equal node counts and the second runs three phases behind the first, so that each barrier
 * interval pairs the memory-bound density pass of one group with the instruction-bound chemical
 * potential of the other (and the collision with a solid layer, the boundary links with the
 * other solid layer).  Each instance still runs its phases in order: both schedules give
 * identical results.  Default 2.  LBM_EINVAL for other values.  Synchronises. */
lbm_status lbm_batch_set_schedule(lbm_batch* b, int32_t groups);

/* Autotuner of tile shape and schedule: times `steps` steps of the batch with each tile shape
 * under the current schedule, then with the fastest shape under both schedules (CUDA events on
 * the batch's stream, each after one untimed launch of the same length), and keeps the fastest
 * combination.  Writes the chosen log2w and groups (either pointer may be NULL) and the seven
 * times in ms (tile log2w = 4 .. 8, then groups 1 and 2) to ms (may be NULL).  The trials are
 * real steps: every instance advances 14 * steps steps, so call it on a representative state
 * and re-initialise afterwards if the state matters. */
lbm_status lbm_batch_autotune(lbm_batch* b, int64_t steps, int32_t* chosen_log2w, int32_t* chosen_groups,
                              double* ms);

/* Instance k of the batch (owned by the batch). */
lbm_status lbm_batch_instance(lbm_batch* b, int32_t k, lbm_ctx** ctx);

/* [0] blocks of the persistent grid, [1] node tiles per phase, [2] 1 if the launch is graph-
 * captured, [3] boundary chunks. */
lbm_status lbm_batch_info(lbm_batch* b, int64_t* out4);

const char* lbm_batch_last_error(const lbm_batch* b);
void lbm_batch_destroy(lbm_batch* b);

/* ---- y-slab decomposition of one lattice over several GPUs (one context per slab) ----------
 * The method is a local stencil: a node's next state depends only on nodes within a few rows
 * (the streaming of Eq. 5, the fourth-order stencils of Eqs. 9 and 12, the two solid layers of
 * Eq. 15, the second fluid node x2 of Eq. 16), at most 7 rows in y.  A lattice split into
 * slabs of whole rows therefore advances exactly as the undivided one if, after every step,
 * each slab's halo of H >= 7 rows on either side is overwritten with its neighbour's own rows.
 *
 * lbm_slab_workspace_size / lbm_create_slab take the GLOBAL configuration (cylinders in global
 * coordinates) and the global rows [y0, y1) the slab owns; the context then holds those rows,
 * an H-row halo on each side that has a neighbour (none where a walled lattice ends: the
 * bottom slab owns global rows 0, 1, the top slab rows ny-2, ny-1), and two solid rows beyond
 * each halo that terminate the local lattice (their values never reach the own rows).  With
 * walls = 0 the slabs wrap around in y.  Then lbm_build_links, lbm_init with the global drop
 * positions, and per step: lbm_step(ctx, 1); for each edge with a neighbour, lbm_slab_pack into
 * a device buffer of lbm_slab_message_bytes bytes; the caller moves the message to the
 * neighbour (NCCL send/recv, a peer copy, or host copies) and the neighbour calls
 * lbm_slab_unpack on its facing edge (the bottom slab's top edge faces the next slab's bottom
 * edge).  All four calls are asynchronous on the context's stream.  The message holds the H
 * own rows next to that edge: nine population planes, the density plane, the per-node EOS plane
 * the next step starts from, and the Eq. 18 FP64 carries of the boundary nodes in those rows.
 * Own rows are then bit-identical to the undivided lattice's.
 *
 * lbm_mass and lbm_dM_history of a slab count its own rows and own boundary nodes only: the
 * global M and Delta M are the sums over slabs (an FP64 all-reduce).  lbm_fields and
 * lbm_populations return the whole local lattice (ny = the local rows).
 *
 * lbm_slab_info fills 10 ints: global row of local row 0 (before the periodic wrap), local ny,
 * first and one-past-last own local row, H, bottom edge has a neighbour, top edge has one, first
 * local row of the bottom halo, first local row of the top halo, global lattice periodic in y.
 * Errors: LBM_EINVAL for H < 7, rows outside [0, ny), a slab with a neighbour owning fewer than
 * H rows, wall rows split from their slab, an edge without a neighbour or a short buffer;
 * LBM_ESTATE for a whole-lattice context or a pack/unpack before the first step. */
lbm_status lbm_slab_workspace_size(const lbm_config* cfg, int32_t y0, int32_t y1, int32_t halo, size_t* bytes);
lbm_status lbm_create_slab(const lbm_config* cfg, int32_t y0, int32_t y1, int32_t halo, void* stream,
                           void* workspace, size_t bytes, lbm_ctx** out);
lbm_status lbm_slab_info(lbm_ctx* ctx, int32_t* info10);
lbm_status lbm_slab_message_bytes(lbm_ctx* ctx, size_t* bytes);
lbm_status lbm_slab_pack(lbm_ctx* ctx, int32_t edge, void* device_buffer, size_t bytes);
lbm_status lbm_slab_unpack(lbm_ctx* ctx, int32_t edge, const void* device_buffer, size_t bytes);

/* Mass audit that allocates no device memory (the paper has no counterpart: this serves
 * callers that may not call cudaMalloc -- a host callback, a monitor, or a process whose device
 * memory budget belongs to another allocator -- but already hold populations on the device).
 *
 * f:       device pointer to 9 planes of n_nodes values each (plane i at f + i*n_nodes), of
 *          type float (precision LBM_FP32) or double (LBM_FP64), e.g. from lbm_populations;
 * kind:    device pointer to n_nodes bytes; nodes with kind 0 (fluid) are summed;
 * n_nodes: 1 .. LBM_NOALLOC_MAX_NODES, otherwise LBM_EINVAL and nothing is launched;
 * stream:  cudaStream_t the work is issued on (may be NULL); a stream that is capturing gives
 *          LBM_ESTATE, with nothing issued (the call ends in a synchronising host copy);
 * out2:    HOST pointer to 2 doubles: sum over fluid nodes of sum_i f_i (FP64, deterministic
 *          order), and the number of non-finite values.  The call synchronises the stream.
 *
 * Scratch: a fixed 16.6 kB array in the library's own device memory (a static __device__
 * variable, present on every GPU the library is loaded on until the process exits), whose
 * device address every call looks up with cudaGetSymbolAddress on the current device, so the
 * call stays valid after the device's context has been reset and created again.  Every call
 * reuses the array; calls whose kernels overlap on the GPU race on it and must be serialised
 * by the caller. */
#define LBM_NOALLOC_MAX_NODES (1LL << 30)
lbm_status lbm_mass_noalloc(const void* f, const uint8_t* kind, int64_t n_nodes, int32_t precision,
                            void* stream, double* out2);

void lbm_destroy(lbm_ctx* ctx);
const char* lbm_status_str(lbm_status s);
const char* lbm_last_error(const lbm_ctx* ctx);

#ifdef __cplusplus
}
#endif
#endif
