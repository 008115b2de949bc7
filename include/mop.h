/*
 * mop.h - C ABI of the B300 engine for the metadynamics-of-paths effective potential.
 *
 * The engine evaluates, for one or more discretised trajectories ("paths") of N beads each,
 * the Onsager-Machlup effective potential of Eq. 3 of the paper (arXiv 2501.11962, Sec. 1.1)
 *
 *     V_eff = U(R^1) + sum_{n=1}^{N-1} K/2 |R^{n+1} - R^n - L^n|^2,
 *     K_i = m_i nu / (2 dt),   L^n_i = (dt / (m_i nu)) F^n_i,   F = -grad U,
 *
 * and its exact gradient dV_eff/dR, which is minus the effective force of Eqs. 5-7.  The
 * Hessian-vector product H(R^n) eta^n that the gradient needs (the finite-difference term of
 * Eq. 5) is computed by an adjoint kernel (MOP_HVP_ADJOINT) or, for comparison, by the paper's
 * central difference F(R + eps eta) - F(R - eps eta) (MOP_HVP_FD).  The physical potential U is
 * Lennard-Jones (Lorentz-Berthelot) + reaction-field Coulomb with a cutoff modifier, plus
 * harmonic bonds and angles.  A metadynamics bias on a centroid-distance CV (Sec. 1.2, Eq. 8)
 * and path dynamics (Eq. 4) are provided as well.
 *
 * Conventions
 *   - Every call returns a mop_status; nothing throws across the ABI.  On failure the handle
 *     keeps a one-line message, read with mop_last_error().
 *   - Units: nm, ps, atomic mass units, elementary charges, kJ/mol.
 *   - Coordinate arrays are [bead][atom][3], atoms in the caller's order, unwrapped; the engine
 *     applies periodic wrapping only for its neighbour search and pair minimum images.  Bead
 *     differences R^{n+1} - R^n are taken on the caller's coordinates as given.
 *   - Pointers are host pointers unless flags contain MOP_DEVPTR, in which case they are device
 *     pointers on the handle's device and the work is only enqueued on `cuda_stream` (a
 *     cudaStream_t; NULL = the legacy default stream).  Host-pointer calls are synchronous.
 *   - The caller owns every buffer it passes; the handle owns all memory it allocates.
 *   - A handle is not thread safe; use one handle per host thread.
 */
#ifndef MOP_H_
#define MOP_H_

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct mop_handle mop_handle; /* opaque; owns all device memory of one system */

typedef enum {
  MOP_OK = 0,
  MOP_ERR_ARG = 1,       /* invalid argument (NULL pointer, size out of range, ...) */
  MOP_ERR_CUDA = 2,      /* a CUDA runtime call failed; see mop_last_error() */
  MOP_ERR_OOM = 3,       /* device allocation failed */
  MOP_ERR_NONFINITE = 4, /* NaN or Inf in the input coordinates, parameters or result */
  MOP_ERR_BOX = 5,       /* cutoff not below half the shortest box edge, or box edge <= 0 */
  MOP_ERR_STATE = 6,     /* call out of order (e.g. evaluating a path that was never set) */
  MOP_ERR_TIMEOUT = 7    /* a bounded device-side wait gave up */
} mop_status;

/* cutoff modifiers of the nonbonded potential phi(r), r < rc */
enum { MOP_SHIFTED_FORCE = 0, /* phi(r) - phi(rc) - (r - rc) phi'(rc) (default) */
       MOP_POT_SHIFT = 1 };   /* phi(r) - phi(rc) */
/* Hessian-vector product of the spring-term gradient */
enum { MOP_HVP_ADJOINT = 0, /* exact, forward-over-reverse pair/bond/angle kernels */
       MOP_HVP_FD = 1 };    /* paper Eq. 5: [F(R + eps eta) - F(R - eps eta)] / (2 eps),
                               eps = fd_h / max_i |eta_i| per bead */
/* arithmetic of the pair kernels */
/* MOP_PREC_MIXED: FP32 pair arithmetic; forces F, eta and the gradient G in double-float (an
 * FP32 hi + lo pair, error-free transformations on the FP32 pipes; G written as FP64); H eta in
 * FP32; energies summed as double-floats and in FP64; the Ewald exclusion and SPME terms add
 * into int64 fixed point.  MOP_PREC_FP64: FP64 everywhere. */
enum { MOP_PREC_MIXED = 0,
       MOP_PREC_FP64 = 1 };

/* call flags */
#define MOP_DEVPTR 1       /* pointer arguments are device pointers; call is asynchronous */
#define MOP_INPUT_F64 2    /* mop_set_path: xyz is double* instead of float* */
#define MOP_E2E 4          /* mop_add_bias: CV = s(R^N) - s(R^1) (Eq. 8) instead of s(R^N) */
#define MOP_COM 8          /* mop_add_bias: mass-weighted group centres (centres of mass) */
#define MOP_ASYNC 16       /* mop_set_path / mop_veff_and_grad with host pointers: enqueue and
                              return (see mop_wait) */

#define MOP_ELEC_RF 0      /* reaction-field electrostatics */
#define MOP_ELEC_PME 1     /* Ewald electrostatics (real space + smooth particle-mesh Ewald) */

/* fields for mop_get_field, each [N][Q][3] FP64 in the caller's atom order */
enum { MOP_FIELD_FORCE = 0, /* F^n = -grad U(R^n) on the beads that need it */
       MOP_FIELD_ETA = 1,   /* eta^n = R^{n+1} - R^n - L^n, n < N */
       MOP_FIELD_HETA = 2 };/* H(R^n) eta^n (adjoint) or its FD estimate, n < N */

/* Host description of a system; every pointer is a host array read during mop_create only. */
typedef struct {
  int32_t n_atoms;           /* Q >= 1 */
  double box[3];             /* rectangular periodic box edges, nm */
  const int32_t* type;       /* [Q] LJ type, 0 <= type < n_types */
  int32_t n_types;           /* 1 <= n_types <= 16 */
  const double* lj_sigma;    /* [n_types] nm; pairs use sigma_ij = (sigma_i + sigma_j) / 2 */
  const double* lj_eps;      /* [n_types] kJ/mol; pairs use eps_ij = sqrt(eps_i eps_j) */
  const double* charge;      /* [Q] e */
  const double* mass;        /* [Q] u, > 0 */
  const int32_t* mol_id;     /* [Q] molecule id */
  const int32_t* mol_local;  /* [Q] index inside the molecule; pairs with equal mol_id and
                                |mol_local_i - mol_local_j| <= 2 have no nonbonded term */
  int32_t n_bonds;
  const int32_t* bond_ij;    /* [n_bonds][2] */
  const double* bond_r0;     /* [n_bonds] nm */
  const double* bond_k;      /* [n_bonds] kJ/mol/nm^2; U = k/2 (d - r0)^2 */
  int32_t n_angles;
  const int32_t* angle_ijk;  /* [n_angles][3], j is the vertex */
  const double* angle_th0;   /* [n_angles] rad */
  const double* angle_k;     /* [n_angles] kJ/mol/rad^2; U = k/2 (theta - theta0)^2 */
  double rc;                 /* cutoff, nm; 0 < rc < min(box) / 2 */
  double eps_rf;             /* reaction-field dielectric (>= 1) */
  int32_t cutoff_mode;       /* MOP_SHIFTED_FORCE | MOP_POT_SHIFT */
  double dt_path;            /* ps, time step of the discretised trajectory (Sec. 1.1) */
  double nu_path;            /* 1/ps, friction coefficient nu of Eq. 1 */
  double temperature;        /* K, used by mop_step's thermostat */
  int32_t hvp_mode;          /* MOP_HVP_ADJOINT | MOP_HVP_FD */
  double fd_h;               /* nm, largest atomic displacement of the FD mode */
  int32_t precision;         /* MOP_PREC_MIXED | MOP_PREC_FP64 */
  /* electrostatics: MOP_ELEC_RF (reaction field, eps_rf) or MOP_ELEC_PME (Ewald: erfc(beta r)/r
   * in real space with the cutoff modifier, the erf correction of excluded pairs and the self
   * term, plus smooth particle-mesh Ewald in reciprocal space on a pme_grid grid with B-splines
   * of pme_order; a grid of 0 x 0 x 0 leaves the reciprocal part out).  MOP_ELEC_PME needs
   * MOP_PREC_MIXED. */
  int32_t elec;
  double ew_beta;            /* 1/nm, Ewald splitting parameter (> 0 with MOP_ELEC_PME) */
  int32_t pme_grid[3];       /* grid points per box edge (each 0, or >= pme_order) */
  int32_t pme_order;         /* 4..8 */
} mop_system_desc;

/* Validates `desc` and uploads it to `device`.  Errors: MOP_ERR_ARG (bad sizes, indices or
 * masses), MOP_ERR_NONFINITE, MOP_ERR_BOX (rc >= min(box)/2), MOP_ERR_CUDA, MOP_ERR_OOM.
 * On success *out owns the device memory until mop_destroy. */
mop_status mop_create(const mop_system_desc* desc, int device, mop_handle** out);

/* Frees everything the handle owns (NULL is allowed). */
mop_status mop_destroy(mop_handle* h);

/* Stores the coordinates of path `path_id` (0 <= path_id < 64): n_beads >= 1 beads of
 * [n_beads][Q][3] float (double with MOP_INPUT_F64), copied into the handle.  Resets the
 * path's velocities to zero.  In mixed precision with float input, the integrator's FP64 copy
 * of the coordinates and the zeroed velocities are formed by the next mop_step or
 * mop_kinetic_energy on the path (the evaluation reads the float coordinates only).  Errors: MOP_ERR_ARG, MOP_ERR_NONFINITE (host input is checked
 * here; device input is checked by mop_veff_and_grad through the result), MOP_ERR_CUDA,
 * MOP_ERR_OOM. */
mop_status mop_set_path(mop_handle* h, int32_t path_id, int32_t n_beads, const void* xyz,
                        int32_t flags, void* cuda_stream);

/* Copies the current coordinates of a path (after mop_step) into xyz [N][Q][3] float. */
mop_status mop_get_path(mop_handle* h, int32_t path_id, float* xyz, int32_t flags, void* cuda_stream);

/* Evaluates V_eff (Eq. 3, plus the bias if one is set) and its gradient for path `path_id`, or
 * for every set path when path_id = -1, in one pass of the kernels.  veff: [1] or [P] doubles
 * (P = number of set paths, in path-id order); grad: [N][Q][3] doubles (concatenated over
 * paths in path-id order when path_id = -1), dV_eff/dR (not the force); grad may be NULL.
 * Host buffers: the call returns when they are filled.  (With MOP_PAIR_KERNELS=half, a pinned
 * host grad of one mixed-precision path without an SPME grid is filled while the kernels run:
 * the HVP pass runs in bead chunks and each chunk's rows are copied on a second stream as soon
 * as they are final; the bead-lane kernels take 64 beads at once, so there the copy follows the
 * kernels.)  The result is bitwise that of a device-pointer call.
 * Errors: MOP_ERR_STATE (path not set), MOP_ERR_NONFINITE (non-finite V_eff, host calls
 * only), MOP_ERR_CUDA, MOP_ERR_OOM. */
mop_status mop_veff_and_grad(mop_handle* h, int32_t path_id, double* veff, double* grad,
                             int32_t flags, void* cuda_stream);

/* Asynchronous host calls.  With MOP_ASYNC, mop_set_path and mop_veff_and_grad take host
 * pointers but only enqueue their work: the coordinates are copied to one of two staging buffers
 * on an upload stream of the handle, the evaluation runs on `cuda_stream`, and V_eff and the
 * gradient are copied back on a download stream, so that the copies of one call overlap the
 * evaluation of the next (page-locked host buffers are needed for that).  The host arrays must
 * stay valid and untouched until mop_wait returns; a later evaluation's gradient kernel waits
 * for the earlier download on the device.  Non-finite input is not reported by these calls: it
 * shows in V_eff.  mop_step and mop_metadynamics wait for pending downloads first.
 * mop_wait returns when every enqueued upload and download has finished.  Errors: MOP_ERR_CUDA. */
mop_status mop_wait(mop_handle* h);

/* Copies one field of the last evaluation of `path_id` into out [N][Q][3] doubles (rows of
 * beads where the field is undefined are zero). */
mop_status mop_get_field(mop_handle* h, int32_t path_id, int32_t field, double* out,
                         int32_t flags, void* cuda_stream);

/* Parts of the last evaluation of `path_id`: out[0] = U(R^1), out[1] = spring energy,
 * out[2] = bias energy, out[3] = CV value (0 without a bias).  Synchronous. */
mop_status mop_get_energies(mop_handle* h, int32_t path_id, double out[4]);

/* Metadynamics bias (Sec. 1.2): defines the CV of path `path_id` as the distance between the
 * centroids of atom groups A and B (minimum image; each centroid taken with its group
 * unwrapped relative to the group's first atom; mass-weighted, i.e. centres of mass as in
 * Sec. 3, with MOP_COM) at the last bead, or, with MOP_E2E, its difference between the last
 * and the first bead (Eq. 8); then appends one Gaussian
 * height * exp(-(S - s_center)^2 / (2 width^2)).  grpA/grpB may be NULL to keep the groups of
 * the previous call.  Groups hold 1..1024 atom indices (host pointers); at most 4096
 * Gaussians per path.  Errors: MOP_ERR_ARG, MOP_ERR_STATE (no groups yet), MOP_ERR_CUDA. */
mop_status mop_add_bias(mop_handle* h, const int32_t* grpA, int32_t nA, const int32_t* grpB,
                        int32_t nB, double s_center, double height, double width,
                        int32_t path_id, int32_t flags);

/* Advances every set path by n_steps of the path dynamics M d2R/dt2 = -dV_eff/dR (Eq. 4),
 * fictitious masses = physical masses: velocity Verlet when gamma = 0, BAOAB Langevin at the
 * system temperature otherwise (noise from Philox-4x32-10 keyed by seed, counter = (atom,
 * bead, step)).  Positions are kept in FP64 and the force is evaluated at their float32
 * rounding (MOP_PREC_MIXED).  Errors: MOP_ERR_STATE, MOP_ERR_ARG, MOP_ERR_CUDA. */
mop_status mop_step(mop_handle* h, int32_t n_steps, double dt_md, double gamma, uint64_t seed,
                    void* cuda_stream);

/* Adds collective variable number *index (0, 1, ...; at most 4 per path) to the bias of path
 * `path_id`: the distance of the centres of groups A and B, with the MOP_E2E and MOP_COM flags of
 * mop_add_bias.  With several CVs the bias is a sum of multivariate Gaussians
 *     h_k exp(-sum_q (S_q - c_kq)^2 / (2 w_kq^2)).
 * deposit_width (nm, >= 0) is the width mop_metadynamics gives its Gaussians along this CV (0:
 * the width passed to mop_metadynamics).  CVs can only be added while the path holds no
 * Gaussians.  Errors: MOP_ERR_ARG, MOP_ERR_STATE (Gaussians present), MOP_ERR_CUDA. */
mop_status mop_add_cv(mop_handle* h, int32_t path_id, const int32_t* grpA, int32_t nA, const int32_t* grpB,
                      int32_t nB, int32_t flags, double deposit_width, int32_t* index);

/* Appends one Gaussian on all CVs of path `path_id`: height and, per CV, centres[n_cv] and
 * widths[n_cv] (host arrays).  Errors: MOP_ERR_ARG (widths <= 0, more than 4096 Gaussians),
 * MOP_ERR_NONFINITE, MOP_ERR_STATE (no CV), MOP_ERR_CUDA. */
mop_status mop_add_gaussian(mop_handle* h, int32_t path_id, double height, const double* centers,
                            const double* widths);

/* Metadynamics of paths (Sec. 1.2, with the deposition rule of Sec. 3: a new Gaussian every
 * `stride` MD steps, 500 in the paper).  Runs n_deposits rounds; each round is mop_step(stride,
 * dt_md, gamma, seed) on V_eff plus the bias deposited so far, then appends to every path with
 * CVs (mop_add_bias, mop_add_cv) one Gaussian of the given height centred at the CVs' values at
 * the current positions (computed on the device), with the width of each CV's deposit_width, or
 * `width` where that is 0 (always for the CV of mop_add_bias).  The gradient is then
 * evaluated again before the next round, so its first half kick sees the new Gaussian.  Works
 * in graph mode (the rounds replay the captured step).  Synchronous.  Errors: MOP_ERR_ARG
 * (n_deposits < 0, stride < 1, non-finite height, width <= 0, more than 4096 Gaussians),
 * MOP_ERR_STATE (no path has a CV), and those of mop_step. */
mop_status mop_metadynamics(mop_handle* h, int32_t n_deposits, int32_t stride, double dt_md, double gamma,
                            uint64_t seed, double height, double width, void* cuda_stream);

/* Copies the Gaussians of path `path_id` (those of mop_add_bias, mop_add_gaussian and
 * mop_metadynamics, in the order they were added): centers and widths as [k][n_cv] and heights
 * as [k] (host arrays with room for `cap` Gaussians; any may be NULL), their number into *n (may
 * exceed cap; then only cap are copied) and the number of CVs into *n_cv (may be NULL).
 * Synchronous.  Errors: MOP_ERR_ARG, MOP_ERR_CUDA. */
mop_status mop_get_gaussians(mop_handle* h, int32_t path_id, double* centers, double* heights, double* widths,
                             int32_t cap, int32_t* n, int32_t* n_cv);

/* Graph mode of mop_step (off by default).  When on, mop_step captures one MD step of all set
 * paths (integrator kernels plus a full V_eff + gradient evaluation, with no host
 * synchronisation inside) into a CUDA graph on a stream of the handle, and replays it n_steps
 * times.  The graph is captured again when the set of paths, dt, gamma or seed changes.  The
 * pair lists keep the capacity sized by the last synchronous evaluation (with 25% headroom).  If a
 * list outgrows it during the replays, mop_step restores the positions, velocities, gradients and
 * noise counter it held before them, grows the capacity to 1.25 times the largest list the replays
 * met and at least to twice the old one, captures the step again and replays the n_steps again
 * (mop_get_list_overflows counts these repeats); after four attempts it returns MOP_ERR_STATE and
 * the steps are invalid. */
mop_status mop_set_graph_mode(mop_handle* h, int32_t on);

/* *overflows = number of graph-mode step batches of path `path_id` that were run again because a
 * pair list outgrew its capacity (mop_set_graph_mode).  No counterpart in the paper.  Errors:
 * MOP_ERR_ARG, MOP_ERR_STATE (path not set). */
mop_status mop_get_list_overflows(const mop_handle* h, int32_t path_id, int64_t* overflows);

/* Geometry of the neighbour search, chosen by the autotuner.  col_factor scales the x-y width of
 * the columns that are cut into 8-atom clusters (1 = near-cubic clusters); bin_factor sets the
 * bin edge of the cluster-pair search in units of rc.  Neither changes any result, only the
 * number of pairs the kernels evaluate and the cost of the list build. */
typedef struct {
  double col_factor;  /* default 1.0 */
  double bin_factor;  /* default 0.5 */
} mop_tuning;

mop_status mop_set_tuning(mop_handle* h, const mop_tuning* t);
mop_status mop_get_tuning(const mop_handle* h, mop_tuning* t);

/* Times full evaluations of path `path_id` for col_factor in {0.85, 1, 1.2} and bin_factor in
 * {0.5, 1} (CUDA events, a warm-up call and two timed calls each), keeps the fastest setting on
 * the handle and returns it with its time per evaluation in ms (either output may be NULL).
 * Synchronous.  Errors: MOP_ERR_STATE (path not set), MOP_ERR_CUDA. */
mop_status mop_autotune(mop_handle* h, int32_t path_id, mop_tuning* best, double* best_ms);

/* Verlet skin of the cluster-pair lists (NEXT row "shared list with a skin across steps").
 * skin_nm > 0: each path's list is built for the cutoff rc + skin_nm (every atom's union sphere
 * over the beads grows by skin_nm / 2) together with a device copy of the coordinates, and later
 * evaluations keep the sort, the clusters and the list as long as no atom of any bead has moved
 * more than skin_nm / 2 from that copy (a device reduction and one 4-byte read per evaluation);
 * only the cluster-local coordinates are then recomputed.  Results differ from a rebuilt list
 * only by rounding (the pair kernels still test r < rc).  0 (default): rebuild at every
 * evaluation.  Applies to mixed-precision evaluations outside CUDA-graph capture (a captured step
 * always rebuilds).  Errors: MOP_ERR_ARG (negative or non-finite skin, or skin >= L/2 - rc). */
mop_status mop_set_list_skin(mop_handle* h, double skin_nm);

/* Lists built and lists reused by the evaluations of `path_id` since it was set (instrumentation
 * of mop_set_list_skin; either output may be NULL). */
mop_status mop_get_list_stats(const mop_handle* h, int32_t path_id, int64_t* builds, int64_t* reuses);

/* Kinetic energy sum_i m_i |v_i|^2 / 2 over all beads of `path_id` (synchronous). */
mop_status mop_kinetic_energy(mop_handle* h, int32_t path_id, double* ke);

/* Number of kernel launches the last mop_veff_and_grad made (instrumentation). */
int32_t mop_last_launch_count(const mop_handle* h);

/* Instrumentation.  With profiling on, mop_veff_and_grad records CUDA events on its stream
 * around each pass; mop_last_pass_ms then returns the device time of the last call's passes in
 * milliseconds: out[0] sort + pair list, [1] pair force, [2] bonded + eta, [3] pair HVP (or
 * FD), [4] bonded HVP + gradient, [5] bias + V_eff reduction (n <= 6 values, synchronous). */
mop_status mop_set_profiling(mop_handle* h, int32_t on);
mop_status mop_last_pass_ms(mop_handle* h, float* out, int32_t n);

/* Counts, for the last evaluation of `path_id`, the nonbonded pairs inside the cutoff (minus
 * exclusions) over all beads that need forces: *unique = number of unordered pairs, *listed =
 * number of atom pairs the cluster-pair list makes the force kernel evaluate (ordered, padding
 * included).  Synchronous. */
mop_status mop_count_pairs(mop_handle* h, int32_t path_id, int64_t* unique, int64_t* listed);

/* Measured FP32 throughput of `device` in TFLOP/s (FFMA = 2 flops): a kernel of independent
 * dependent-FMA chains over a grid of SMs x resident blocks, best of three timed launches after
 * a warm-up.  No counterpart in the paper; the pair kernels' roofline is quoted against it
 * beside the nominal lanes x maximum clock figure.  Synchronous; allocates and frees a small
 * buffer.  Errors: MOP_ERR_ARG (NULL output), MOP_ERR_OOM, MOP_ERR_CUDA. */
mop_status mop_measure_fp32_peak(int32_t device, double* tflops);

/* Spring energy without any device allocation.  No counterpart in the paper: this is a service
 * for callers that cannot allocate device memory, for example code that runs inside a CUDA
 * graph that another framework captures and replays, or a plug-in whose host application owns
 * every allocation.  Returns, in *out (device pointer, one double), the spring energy
 *     sum_{n < n_springs} sum_i K_i/2 |eta^n_i|^2,   K_i = mass_i nu_path / (2 dt_path),
 * of eta [n_springs][n_atoms][3] (device, FP64, as mop_get_field returns it) and mass
 * [n_atoms] (device, FP64).  The reduction is deterministic and fixed-order (FP64 sums over
 * tiles of 256 atoms, then over the tiles); it is not the engine's reduction, so the result
 * agrees with the E_spring of mop_veff_and_grad to rounding (within 1e-6 relative), not bit for
 * bit.  No handle is needed and nothing is allocated: the block partial sums live in a fixed
 * array of 65,536 doubles (512 KiB) that every GPU loading the library keeps until the process
 * exits.  n_springs * ceil(n_atoms / 256) must not exceed 65,536 (MOP_ERR_ARG otherwise; for
 * example up to 65,536 springs of at most 256 atoms).  Errors are taken from this call's own
 * runtime calls: an error the caller left pending is neither cleared nor reported as this
 * call's.  Work is enqueued on cuda_stream on the current device; the first call on a
 * device looks up the array's device address, so make it before any stream capture.  All calls
 * share the array: calls that overlap on the GPU race.  Errors: MOP_ERR_ARG, MOP_ERR_CUDA. */
mop_status mop_spring_energy_noalloc(const double* eta, const double* mass, int32_t n_springs, int32_t n_atoms,
                                     double dt_path, double nu_path, double* out, void* cuda_stream);

/* Text of the last error of the handle ("" if none); valid until the next call. */
const char* mop_last_error(const mop_handle* h);

#ifdef __cplusplus
}
#endif
#endif /* MOP_H_ */
