/*
 * tlbm.h -- C ABI of a single-GPU (sm_103a) engine for the ternary free-energy
 * lattice Boltzmann method of Semprebon, Krueger and Kusumaatmaja,
 * "Ternary free energy lattice Boltzmann model with tunable surface tensions and
 * contact angles" (arXiv:1511.02155).
 *
 * One time step (tlbm_step) is the LBM section of the paper, in order:
 *   moments rho = sum f, rho v = sum f e, phi = sum g, psi = sum k  (Eq. lbconstraint)
 *   concentrations C1 = (rho+phi-psi)/2, C2 = (rho-phi-psi)/2, C3 = psi
 *                                                  (Sec. Auxiliary variables)
 *   wetting ghost values on solid nodes that impose the wall-normal gradients of
 *   rho, phi, psi set by h_1..3                    (Sec. Auxiliary variables)
 *   isotropic gradients and Laplacians; chemical potentials mu_rho, mu_phi, mu_psi
 *   and bulk pressure p_b                          (Sec. Equations of Motion)
 *   pressure-tensor equilibria f_eq, g_eq, k_eq    (Eq. eqdistfbinary)
 *   BGK collision                                  (Eq. latboltCollision)
 *   streaming with halfway bounce-back at solids   (Eq. latboltPropagation)
 *   FP64 totals of rho, phi, psi over fluid nodes  (mass constraints closing the
 *                                                   LBM section)
 *
 * Conventions
 *   Lattice: D2Q9 (nz must be 1) or D3Q19.  Velocity order
 *     D2Q9 : 0; (1,0) (-1,0) (0,1) (0,-1); (1,1) (-1,-1) (-1,1) (1,-1)
 *     D3Q19: 0; +-x +-y +-z; (1,1,0) (1,-1,0) (-1,1,0) (-1,-1,0);
 *            (0,1,1) (0,1,-1) (0,-1,1) (0,-1,-1); (1,0,1) (1,0,-1) (-1,0,1) (-1,0,-1)
 *     (the D3Q19 order is the one the paper's weight table implies).
 *   Node index: x + nx*(y + ny*z), x fastest.  All directions are periodic;
 *   walls are made of solid nodes.
 *   Populations exchanged with the host (tlbm_get_populations /
 *   tlbm_set_populations) are conventional post-streaming values f_i(r, t) as
 *   doubles, laid out [set f,g,k][i][node].  Solid nodes carry zeros.
 *   Relaxation times: tau_rho = tau_f; tau_phi = 1/2 + M_phi/Gamma_phi and
 *   tau_psi = 1/2 + M_psi/Gamma_psi (Eqs. Mobility1, Mobility2) with
 *   Gamma_phi = Gamma_psi = 1 unless tlbm_set_gamma changes them.
 *
 * Ownership: the engine allocates and owns all device memory (cudaMalloc) of a
 *   handle; every host pointer argument is read or written during the call only
 *   and stays owned by the caller.
 * Streams: all device work of a handle is queued on the CUDA stream given at
 *   creation (NULL = the legacy default stream).  tlbm_step returns without
 *   waiting; calls that return host data synchronise that stream.
 * Errors: every call returns a tlbm_status; tlbm_last_error() gives a message.
 *   Nothing throws across the ABI and no kernel traps.
 * Threads: a handle must not be used from two host threads at once.
 */
#ifndef TLBM_H
#define TLBM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct tlbm tlbm; /* opaque handle */

typedef enum {
    TLBM_OK = 0,
    TLBM_ERR_ARG = 1,         /* NULL handle/pointer, bad size, bad enum */
    TLBM_ERR_PARAM = 2,       /* tau <= 1/2, kappa <= 0, |4 h/(alpha kappa)| >= 1, alpha <= 0 */
    TLBM_ERR_CUDA = 3,        /* a CUDA runtime call failed (message has the CUDA error) */
    TLBM_ERR_OOM = 4,         /* device allocation failed */
    TLBM_ERR_NONFINITE = 5,   /* a mass total became NaN or Inf */
    TLBM_ERR_TIMEOUT = 6,     /* a bounded device wait gave up */
    TLBM_ERR_UNSUPPORTED = 7  /* combination not built (e.g. kernel kind for this lattice) */
} tlbm_status;

typedef enum { TLBM_D2Q9 = 9, TLBM_D3Q19 = 19 } tlbm_lattice;

/* Storage / arithmetic of the populations.
 *   TLBM_FP64        : stored and computed in double.
 *   TLBM_FP32        : stored and computed in float.
 *   TLBM_FP16_OFFSET : stored in IEEE half as offsets from the rest state (f_i - w_i,
 *                      g_i and k_i as is), computed in float.
 *   TLBM_BF16_OFFSET : as above with bfloat16 storage. */
typedef enum { TLBM_FP64 = 0, TLBM_FP32 = 1, TLBM_FP16_OFFSET = 2, TLBM_BF16_OFFSET = 3 } tlbm_precision;

/* Which step implementation runs.
 *   TLBM_KERNEL_FUSED: one kernel per step that marches through the lattice,
 *                      recomputing halo moments on chip (no moment arrays).
 *   TLBM_KERNEL_SPLIT: three kernels per step (moments to a device array,
 *                      wetting ghosts, collide+stream).
 *   TLBM_KERNEL_AUTO : FUSED where built, else SPLIT. */
typedef enum { TLBM_KERNEL_AUTO = 0, TLBM_KERNEL_FUSED = 1, TLBM_KERNEL_SPLIT = 2 } tlbm_kernel;

/*
 * Create an engine for an nx x ny x nz lattice and allocate its device memory.
 *   lattice       TLBM_D2Q9 (nz must be 1) or TLBM_D3Q19.
 *   kappa[3]      kappa_1..3 > 0 of the free energy (Eq. energy_functional_general
 *                 with kappa'_m = alpha^2 kappa_m); surface tensions are
 *                 gamma_mn = alpha (kappa_m + kappa_n)/6 (Eq. SurfTens).
 *   alpha         interface width > 0.
 *   tau_f         relaxation time of f (> 1/2), viscosity (tau_f - 1/2)/3.
 *   M_phi, M_psi  mobilities > 0 of the Cahn-Hilliard equations.
 *   h[3]          wetting parameters h_1..3 (Eq. Cahn); may be NULL for zeros.
 *                 Each must satisfy |4 h_m / (alpha kappa_m)| < 1.
 *   solid_mask    host array of nx*ny*nz bytes, nonzero = solid; copied.  NULL =
 *                 no solid nodes.
 *   precision     see tlbm_precision.
 *   cuda_stream   a cudaStream_t (as void*), or NULL for the default stream.
 * On success *out is a new handle; populations are zero until tlbm_init_fields or
 * tlbm_set_populations.  On failure *out is NULL and the status says why.
 */
tlbm_status tlbm_create(tlbm **out, tlbm_lattice lattice, int nx, int ny, int nz,
                        const double kappa[3], double alpha, double tau_f,
                        double M_phi, double M_psi, const double h[3],
                        const uint8_t *solid_mask, tlbm_precision precision,
                        void *cuda_stream);

/* Free all device memory of the handle (NULL is ignored). */
void tlbm_destroy(tlbm *t);

/* Set Gamma_phi, Gamma_psi (> 0) of the g/k equilibria; tau_phi and tau_psi are
 * recomputed from the mobilities (Eqs. Mobility1, Mobility2). */
tlbm_status tlbm_set_gamma(tlbm *t, double gamma_phi, double gamma_psi);

/* Choose the step implementation (see tlbm_kernel). */
tlbm_status tlbm_set_kernel(tlbm *t, tlbm_kernel kind);

/* Which implementation tlbm_step uses now (resolves AUTO). */
tlbm_kernel tlbm_get_kernel(const tlbm *t);

/* Tile of the fused step.  variant = shape | mode << 4: shape 0 = default
 * (D3Q19 shape 7, D2Q9 shape 5), D3Q19 1 = 32x8, 2 = 64x4, 3 = 32x4 nodes
 * per block, 4..7 = 32x4 with part of each node's pulled populations kept in
 * shared memory from the moment pass to the collision (4: the 19 f values;
 * 5: the lane-shifted values first, 28 for FP32, 19 plus a per-warp L2
 * prefetch for the 16-bit formats; 6: 19 lane-shifted values; 7: as 5, the
 * k values first and then the lane-shifted (f, g) pairs); D2Q9 1 = 128,
 * 2 = 256, 3 = 64 nodes per row, 4 = 128 with the 18 lane-shifted values
 * staged, 5 = 128 with all 27 staged.  mode (shapes 1..3) selects the
 * load order and cache hints inside a plane (0 default for the lattice and
 * storage; 1 interleaved halo loads; 2 collision operands loaded first; 3 both;
 * 4 per-warp L2 prefetch three planes ahead; 5 = 1 + 4; 6 plain order;
 * 8 evict-first stores; 9 also evict-first collision loads; 12, 13 = 8, 9 with
 * the prefetch; a mode not built for a shape falls back to its default; the
 * variant must be below 256, its shape below 8).
 * chunk = planes marched per block (0 = chosen from the lattice size).  Double
 * storage ignores the choice.  Results do not depend on the tile. */
tlbm_status tlbm_set_tile(tlbm *t, int variant, int chunk);

/*
 * Set the populations to the equilibria of the given fields.
 *   rho, phi, psi  host double arrays of N = nx*ny*nz values (values on solid
 *                  nodes are ignored);
 *   ux, uy, uz     host double velocity arrays, or NULL for zero.
 * The equilibria use the same derivative stencils and wetting ghosts as a step.
 * Synchronises the stream.
 */
tlbm_status tlbm_init_fields(tlbm *t, const double *rho, const double *phi, const double *psi,
                             const double *ux, const double *uy, const double *uz);

/* Advance nsteps >= 0 time steps.  Queued on the stream; returns without waiting. */
tlbm_status tlbm_step(tlbm *t, int64_t nsteps);

/* Number of steps taken since the last init/set of the populations. */
int64_t tlbm_steps_done(const tlbm *t);

/* Timing mode (on != 0): every step records CUDA events on the stream around
 * its main kernel(s) (not the final mass reduction) and waits for them, adding
 * their elapsed time to a total.  Turning it on or off resets the total.  The
 * waits make tlbm_step synchronous; the kernels themselves are unchanged. */
tlbm_status tlbm_set_timing(tlbm *t, int on);

/* Total main-kernel milliseconds and number of steps timed since timing was set. */
tlbm_status tlbm_kernel_time(const tlbm *t, double *ms_total, int64_t *steps);

/*
 * Copy out macroscopic fields of the current state (host double arrays of N
 * values; u is [3][N]).  Any pointer may be NULL to skip that field.  Solid
 * nodes read 0.  Synchronises the stream.
 */
tlbm_status tlbm_fields(tlbm *t, double *C1, double *C2, double *C3, double *rho, double *u);

/*
 * FP64 totals (sum rho, sum phi, sum psi) over fluid nodes of the current state,
 * reduced in a fixed order (bitwise repeatable).  Returns TLBM_ERR_NONFINITE (and
 * still writes out) if a total is not finite.  Synchronises the stream.
 */
tlbm_status tlbm_mass(tlbm *t, double out[3]);

/*
 * Totals of the state at the start of the most recent step, as accumulated
 * inside that step (NaN before the first step), and the non-finite flag of all
 * steps since the last init.  Synchronises the stream.
 */
tlbm_status tlbm_step_mass(tlbm *t, double out[3]);

/*
 * Conventional populations f_i(r,t), g_i, k_i of the box [x0,x0+bx) x [y0,y0+by)
 * x [z0,z0+bz) (coordinates wrap periodically) as doubles laid out
 * [set][i][bz][by][bx].  host must hold 3*Q*bx*by*bz doubles.  Synchronises.
 */
tlbm_status tlbm_get_populations_box(tlbm *t, int x0, int y0, int z0, int bx, int by, int bz,
                                     double *host);

/* Whole-lattice form of tlbm_get_populations_box (3*Q*N doubles). */
tlbm_status tlbm_get_populations(tlbm *t, double *host);

/* Replace the state by conventional populations (3*Q*N doubles, values on solid
 * nodes ignored), rounded to the storage precision.  Synchronises. */
tlbm_status tlbm_set_populations(tlbm *t, const double *host);

/* Bytes of the raw device state (checkpoint size). */
size_t tlbm_state_bytes(const tlbm *t);

/* Copy the raw device state to / from host memory of tlbm_state_bytes bytes.
 * A state saved by tlbm_get_state resumes bitwise identically.  The bytes are
 * the device layout of this library build (chunked lane words per storage
 * format and lattice), not an interchange format: use tlbm_get_populations /
 * tlbm_set_populations to move a state between builds.  Synchronises. */
tlbm_status tlbm_get_state(tlbm *t, void *host, size_t bytes);
tlbm_status tlbm_set_state(tlbm *t, const void *host, size_t bytes);

/* Kernel launches per tlbm_step(1) of the current configuration. */
int tlbm_launches_per_step(const tlbm *t);

/*
 * One time step on caller-owned device buffers, allocating nothing.
 * The paper has no counterpart: this is an engineering entry point for callers
 * that may not allocate device memory themselves -- a plug-in inside a host
 * framework that owns every device allocation through its own pool and budget
 * (a cudaMalloc behind its back would break its accounting or fail), and
 * real-time loops that must not pay allocation latency or fragment memory.
 *   lattice, nx, ny, nz, kappa, alpha, tau_f, M_phi, M_psi, h: as tlbm_create
 *                 (Gamma_phi = Gamma_psi = 1).
 *   precision     TLBM_FP32 or TLBM_FP64 only.
 *   solid_dev     device array of nx*ny*nz bytes (nonzero = solid) or NULL.
 *   src_dev       device populations in the engine's raw state layout (the bytes
 *                 tlbm_get_state returns, tlbm_state_bytes long); read only.
 *   dst_dev       device buffer of the same size; receives the state one step
 *                 later.  Must not overlap src_dev.
 *   mass_dev      device array of 3 doubles for the FP64 totals of the input
 *                 state (sum rho, phi, psi over fluid nodes), or NULL.  A state
 *                 that has blown up shows as non-finite totals here (there is no
 *                 other non-finite report).
 *   cuda_stream   stream to run on (NULL = default stream).
 * The step is the engine's split implementation (moments, ghosts, collide +
 * stream), the same kernels and parameters tlbm_step runs under
 * TLBM_KERNEL_SPLIT.
 * Its intermediate arrays live in one fixed 8 MiB __device__ buffer per device,
 * which limits the lattice to 349504 nodes in FP64 and 699008 nodes in FP32;
 * larger lattices return TLBM_ERR_ARG before any device work.  Every GPU that
 * loads the library holds that buffer until the process exits.  All calls share
 * it and it keeps the last call's contents, so calls whose kernels overlap on
 * the GPU (other streams, other host threads) race: serialise them.  The first
 * call on a device looks up the buffer's device address (cudaGetSymbolAddress);
 * make that first call outside any stream capture.  Returns without waiting.
 * Errors: TLBM_ERR_ARG / TLBM_ERR_PARAM / TLBM_ERR_UNSUPPORTED on the host
 * checks, TLBM_ERR_CUDA if a launch fails; tlbm_noalloc_last_error() has the
 * message.
 */
tlbm_status tlbm_step_noalloc(tlbm_lattice lattice, tlbm_precision precision, int nx, int ny, int nz,
                              const double kappa[3], double alpha, double tau_f, double M_phi,
                              double M_psi, const double h[3], const uint8_t *solid_dev,
                              const void *src_dev, void *dst_dev, double *mass_dev, void *cuda_stream);

/* ------------------------------------------------------------------ adjoint
 * Discrete adjoint of the time step (the paper has no counterpart; it serves the
 * inverse calibration of surface tensions and contact angles).  Loss:
 *   L = sum over fluid nodes of (C_3(r, T) - target(r))^2
 * after T = nsteps steps from the equilibrium of the initial fields.  The call
 * runs the forward steps (keeping a checkpoint every checkpoint_every steps),
 * then the hand-written adjoint back to the initial fields, recomputing each
 * segment's states from its checkpoint, and returns the gradient of the
 * discrete loss (exact up to rounding):
 *   *loss; dkappa[3] = dL/dkappa_m; dh[3] = dL/dh_m (zero without solid nodes);
 *   dfields (optional, host [3][N], x fastest) = dL/d(rho, phi, psi) of the
 *   initial fields at fluid nodes (0 on solid nodes).
 * target is a host array of N doubles.  Preconditions: TLBM_FP64 or TLBM_FP32
 * storage (else TLBM_ERR_UNSUPPORTED; the adjoint computes in the storage's
 * precision, the loss and the parameter gradients are summed in FP64); the
 * state is the one set by tlbm_init_fields with
 * no velocity and no step since (else TLBM_ERR_ARG).  Device memory: about
 * (ceil(nsteps / checkpoint_every) + checkpoint_every + 3) states plus 22
 * doubles per node (TLBM_ERR_OOM if it does not fit; nothing is run then).
 * Afterwards the engine holds the state after nsteps steps (tlbm_steps_done
 * advanced by nsteps).  If a CUDA error interrupts the run, the engine's
 * populations are unspecified: set them again (tlbm_init_fields) before use. */
tlbm_status tlbm_adjoint_c3_misfit(tlbm *t, int64_t nsteps, int checkpoint_every, const double *target,
                                   double *loss, double dkappa[3], double dh[3], double *dfields);

/* ------------------------------------------------------------------ wetting theory
 * Host-only functions (no GPU involved) of the model's wetting theory,
 * Sec. Surface Thermodynamics and Sec. Inverting the contact angle relations.
 * Solid-fluid tensions gamma_sm = I_m + sum_{n != m} J_n (Eq. solidST), fluid-fluid
 * tensions gamma_mn = alpha (kappa_m + kappa_n)/6 (Eq. SurfTens), angles from
 * Young's equation (Eq. contact angle): cos theta_mn = (gamma_sn - gamma_sm)/gamma_mn,
 * theta_mn measured through fluid m.  The closed form used,
 *   cos theta_mn = (D_m - D_n) / (2 alpha (kappa_m + kappa_n)),
 *   D_j = [(alpha kappa_j + 4 h_j)^{3/2} - (alpha kappa_j - 4 h_j)^{3/2}] / sqrt(alpha kappa_j),
 * is what I_m, J_n and Young's equation give; the printed Eq. invertCA has the
 * opposite sign and no 1/alpha.
 */

/* theta_deg[0..2] = theta_12, theta_23, theta_31 in degrees for wetting parameters
 * h[0..2].  TLBM_ERR_ARG for NULL pointers or kappa_m, alpha not > 0;
 * TLBM_ERR_PARAM unless |4 h_m| < alpha kappa_m for every m. */
tlbm_status tlbm_contact_angles(const double kappa[3], double alpha, const double h[3], double theta_deg[3]);

/* Wetting parameters h[0..2] that give the contact angles theta_12 and theta_13
 * (both measured through fluid 1, degrees, in (0, 180)), with the gauge
 * sum_m h_m / kappa_m = 0 (Eq. Redundancy: zero wall-normal gradient of rho).
 * theta_23 then follows from the Girifalco-Good relation.  TLBM_ERR_PARAM when no
 * admissible h exists (theta_23 would not exist, or some |4 h_m| would reach
 * alpha kappa_m); h is written only on success. */
tlbm_status tlbm_wetting_from_angles(const double kappa[3], double alpha, double theta12_deg,
                                     double theta13_deg, double h[3]);

/* ------------------------------------------------------------------ batches
 * The paper has no counterpart: this is an execution feature for parameter
 * sweeps such as the contact-angle runs of Sec. Contact Angles.
 * Many independent lattices of one lattice type and storage format (for example
 * a contact-angle or kappa sweep over lattices of uneven size) advanced by ONE
 * kernel launch per step plus one launch for all their FP64 totals.  A batch
 * groups existing engines; each keeps its own state, parameters, solid mask and
 * accessors (tlbm_fields, tlbm_mass, ...), and a batched step gives bit for bit
 * the same populations as stepping each member alone with the same tile.
 */
typedef struct tlbm_batch tlbm_batch;

/* Group count >= 1 engines: same device, stream, lattice and precision, all with
 * or all without solid nodes, each at the same step parity (equal parity of
 * steps taken since initialisation).  The members stay owned by the caller and
 * must outlive the batch.  Returns TLBM_ERR_ARG if they do not match. */
tlbm_status tlbm_batch_create(tlbm_batch **out, tlbm *const *members, int count);

/* Advance every member by nsteps.  Fails with TLBM_ERR_ARG if a member was
 * stepped alone since the last batched step (its parity differs). */
tlbm_status tlbm_batch_step(tlbm_batch *b, int64_t nsteps);

/* Tile for every member (tlbm_set_tile encoding).  On failure the previous tile
 * stays in use. */
tlbm_status tlbm_batch_set_tile(tlbm_batch *b, int variant, int chunk);

/* Time candidate tiles (shape and planes per block) for trial_steps steps each
 * with CUDA events on the members' stream, keep the fastest, and report it.
 * The trial steps are real steps: every member advances by them. */
tlbm_status tlbm_batch_autotune(tlbm_batch *b, int trial_steps, int *variant, int *chunk);

/* on != 0: replay the steps as a CUDA graph of two batched steps (captured on
 * a private stream at the next tlbm_batch_step, launched on the members' stream). */
tlbm_status tlbm_batch_set_graph(tlbm_batch *b, int on);

/* on != 0: record CUDA events around each batched step's main kernel and add
 * its duration up (steps then run one by one, without the graph; the autotuner's
 * trial steps are timed too).  Turning it on or off resets the sums. */
tlbm_status tlbm_batch_set_timing(tlbm_batch *b, int on);

/* Summed main-kernel time (ms) and the number of timed batched steps. */
tlbm_status tlbm_batch_kernel_time(const tlbm_batch *b, double *ms_total, int64_t *steps);

/* Blocks of one batched step launch. */
int64_t tlbm_batch_blocks(const tlbm_batch *b);

/* Message of the last failed batch call ("" if none; NULL b: last create). */
const char *tlbm_batch_last_error(const tlbm_batch *b);

/* Release the batch (not its members). */
void tlbm_batch_destroy(tlbm_batch *b);

/*
 * Bounds-checked step (a debugging aid; the paper has no counterpart).  With
 * on != 0 the fused step of an engine with TLBM_FP32 storage runs checked
 * variants of its default kernels: every population address of a pull, a
 * bounce-back and a store is validated against the population buffer and its
 * 32-node chunk layout, and every index into the on-chip moment ring and the
 * neighbour mask against its extent.  The first violation is recorded in a
 * device word as (code << 56 | offending offset or index), codes 1 pull
 * source, 2 bounce-back source, 3 store target, 4 moment-ring index, 5 mask
 * index; the access is redirected to a valid address and the kernel carries on
 * (no trap, no fault).  The checked kernels use the default tile and compute
 * the same results as the unchecked ones.  The checked kernels are those of
 * the pressure-tensor coupling (an engine under TLBM_COUPLING_FORCING runs its
 * unchecked kernels).  TLBM_ERR_UNSUPPORTED for other storage formats.
 * tlbm_bounds_check_word waits for the engine's stream,
 * returns the word (0: no violation) and clears it.
 */
tlbm_status tlbm_set_bounds_check(tlbm *t, int on);
tlbm_status tlbm_bounds_check_word(tlbm *t, uint64_t *word);

/*
 * How the thermodynamic force enters the momentum equation (Sec. Equations of
 * Motion offers both routes).
 *   TLBM_COUPLING_PRESSURE_TENSOR: the paper's default: the second moment of
 *       f_eq is the full pressure tensor P_ab (every kernel kind).
 *   TLBM_COUPLING_FORCING: Guo forcing: f_eq is the ideal-gas equilibrium and
 *       the body force F_a = -d_b (P_ab - rho c_s^2 delta_ab), the divergence of
 *       the same tensor's non-ideal part by the isotropic gradient stencil,
 *       enters through the source of Guo, Zheng and Shi (2002) at the fluid
 *       velocity u = (j + F/2)/rho.  In the continuum F = -(rho grad mu_rho +
 *       phi grad mu_phi + psi grad mu_psi); on the lattice sum_r F = 0 exactly.
 *       g and k are unchanged.  TLBM_KERNEL_FUSED (the AUTO choice) runs one
 *       marching kernel per step (moments with a two-node halo and a ring of
 *       Pi planes in shared memory); TLBM_KERNEL_SPLIT three kernels
 *       (moments; Pi_ab, mu_phi, mu_psi node arrays; collide+stream).
 */
typedef enum { TLBM_COUPLING_PRESSURE_TENSOR = 0, TLBM_COUPLING_FORCING = 1 } tlbm_coupling;

/*
 * Select the coupling.  TLBM_COUPLING_FORCING needs a lattice without solid
 * nodes (TLBM_ERR_UNSUPPORTED otherwise); it allocates (NPI + 2) node arrays
 * of the compute type for the split kernels, NPI = 3 on D2Q9 and 6 on D3Q19
 * (TLBM_ERR_OOM if that fails), which tlbm_destroy frees.  The populations are left as they are: call
 * tlbm_init_fields afterwards to start from the coupling's own equilibrium
 * (under forcing, the u given there is the stored momentum over rho; the
 * fluid velocity adds F/(2 rho)).  Under forcing, tlbm_fields returns the
 * fluid velocity (j + F/2)/rho, and batches and the adjoint refuse the engine
 * (TLBM_ERR_UNSUPPORTED).  tlbm_step_noalloc always uses the pressure tensor.
 */
tlbm_status tlbm_set_coupling(tlbm *t, tlbm_coupling coupling);
tlbm_coupling tlbm_get_coupling(const tlbm *t);

/* Message of the last failed tlbm_step_noalloc call on this host thread ("" if none). */
const char *tlbm_noalloc_last_error(void);

/* Message of the last failed call on this handle ("" if none; never NULL). */
const char *tlbm_last_error(const tlbm *t);

/* Name of a status code. */
const char *tlbm_status_string(tlbm_status s);

#ifdef __cplusplus
}
#endif

#endif /* TLBM_H */
