/*
 * sdpd.h -- C ABI of libsdpd, the GB300 (sm_103a) implementation of the
 * per-timestep SDPD-DEM particle-interaction step of Tsuzuki, "DEMocritus: an
 * open source framework for simulating slurry flows using an SDPD-DEM coupled
 * model" (arXiv 2002.03120).
 *
 * One call of each stage below performs, on the GPU, the routine of the
 * paper's Algorithm 1 (per velocity-Verlet sub-step "velver") or Algorithm 2
 * (inside compute_force) named in its comment.  All stages are asynchronous on
 * the CUDA stream passed as `stream` (a cudaStream_t; NULL = legacy default
 * stream) unless stated otherwise.
 *
 * Conventions
 *  - Every function returns an sdpd_status; no C++ exception crosses the ABI
 *    and no function calls exit, abort or a device trap.  On failure
 *    sdpd_last_error() returns a message (thread-local).
 *  - Errors raised by kernels (capacity overflow, non-finite state) are
 *    recorded in a device word and reported by the next synchronising call
 *    (sdpd_get_*, sdpd_check, sdpd_step) as SDPD_E_CAPACITY / SDPD_E_NONFINITE.
 *  - Arrays are row-major [n][3] doubles (x, y, z) unless stated; pointers may
 *    be host or device memory (unified addressing); the library copies what it
 *    needs and never keeps or frees caller memory.
 *  - A context owns all its device buffers (allocated by sdpd_init, released
 *    by sdpd_destroy).  A context is not thread-safe; distinct contexts are
 *    independent.
 *  - Particle types: 0 fluid, 1 rigid (DEM sphere), 2 inner wall, 3 outer wall
 *    (the frozen dummy particles of Section 2.5).
 *  - Particle index within an instance = global id (gid) of the counter-based
 *    noise (Philox4x32-10 keyed by the seed and the instance, counter
 *    (min gid, max gid, step, block)).
 */
#ifndef SDPD_H
#define SDPD_H

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    SDPD_OK = 0,
    SDPD_E_INVALID = 1,   /* bad argument or parameter set                  */
    SDPD_E_CUDA = 2,      /* a CUDA runtime call failed                      */
    SDPD_E_OOM = 3,       /* device allocation failed                        */
    SDPD_E_CAPACITY = 4,  /* neighbour list / cell / contact table overflow  */
    SDPD_E_NONFINITE = 5, /* NaN or Inf detected in the state                */
    SDPD_E_DOMAIN = 6,    /* particle left the grid on a wall axis           */
    SDPD_E_TIMEOUT = 7,   /* a bounded device wait gave up                   */
    SDPD_E_STATE = 8      /* stage called out of order                       */
} sdpd_status;

/* Pair-force precision of a context. */
enum {
    SDPD_PREC_FP64 = 0,   /* all pair arithmetic in double                     */
    SDPD_PREC_SPLIT = 1   /* pair arithmetic in float; positions, momenta,
                             density/pressure and the integrator in double    */
};

typedef struct sdpd_ctx sdpd_ctx;

/* Parameters of one instance: Table 1 of the paper (Section 3.1) plus the
 * constants of the readings where the paper is silent.  SI or mesoscale units,
 * the caller's choice, as long as they are consistent. */
typedef struct {
    double dx;            /* initial particle spacing (--dx)                        */
    double r_c;           /* kernel radius h: support of the Lucy kernel (--h)       */
    double dt;            /* time step (--dt)                                        */
    double rho0, p0, alpha, beta_p; /* Eq. prtcpres (--dens0 --pres0 --alpha --beta) */
    double eta, xi, kBT;  /* shear and bulk viscosity, energy level (Section 2.1)   */
    double coeff_c, coeff_d, coeff_r, coeff_t; /* --Coeff_fcij .. --Coeff_ftij       */
    double origin[3], box[3]; /* domain (--orgx.. --Lx..); fluid region on wall axes */
    double g[3];          /* uniform acceleration (--gx --gy --gz)                  */
    double body_amp;      /* reverse-Poiseuille forcing (accel.): +amp on the lower,
                             -amp on the upper half of split_axis (--gravity_type)  */
    double artvis_alpha, artvis_e; /* collision-method range (x dx), restitution     */
    double kn, restitution, nu_p, E_p, mu_fric; /* DEM (Section 2.2; --Edem --Pdem --Fdem) */
    double lub_gap_min;   /* lubrication gap floor as a fraction of R_i + R_j       */
    double eps_min;       /* lower clamp of the fluid volume fraction               */
    int periodic[3];      /* per-axis periodic (1) or wall (0) (--periodic_type)    */
    int body_axis, split_axis;
    int pressure_filter, clamp_negative_p, artvis; /* switches (Sections 2.1, 2.5, 4.4) */
    int dem_law;          /* 0: Eqs. deminputA-F as printed; 1: linear kn + restitution */
    int density_reinit;   /* 1: Shepard density reinitialisation at every evaluation (after
                             Colagrossi & Landrini; text under Algorithm 1), 0: off       */
    unsigned long long seed; /* noise seed                                          */
} sdpd_params;

/* Upper bound of max_neighbors: the sphere kernel stages the rigid entries of
 * four lists (4 B each) in the 48 KB of shared memory a launch gets by
 * default; list positions are 16-bit. */
#define SDPD_MAX_NEIGHBORS 3072

/* Create a context for n_instances independent instances (batched viscometer
 * sweep: one launch per stage covers all instances).  params[k] and
 * n_particles[k] describe instance k.  precision: SDPD_PREC_*.  max_neighbors:
 * capacity of each particle's neighbour list (0 = 384, at most
 * SDPD_MAX_NEIGHBORS, else SDPD_E_INVALID).  max_contacts: DEM
 * contact-history slots per rigid particle (0 = 16).  Validates the parameters
 * (gamma^a, gamma^b >= 0 i.e. 40 eta/51 <= xi <= 5 eta/3; periodic axes at
 * least 3 kernel radii wide; positive dx, r_c, dt, rho0).  Allocates the
 * device buffers.  Synchronous. */
sdpd_status sdpd_init(const sdpd_params *params, int n_instances, const long long *n_particles,
                      int precision, int max_neighbors, int max_contacts, sdpd_ctx **out);

/* Release a context and all its device memory (NULL is ignored). */
void sdpd_destroy(sdpd_ctx *ctx);

/* Upload the particles of instance `inst` (n must equal its n_particles).
 * x, v, w: [n][3]; type: [n] int32; radius, mass: [n].  Walls must have zero
 * velocity and spin.  Resets the contact history of the instance.
 * Synchronous. */
sdpd_status sdpd_set_particles(sdpd_ctx *ctx, int inst, long long n, const double *x,
                               const double *v, const double *w, const int *type,
                               const double *radius, const double *mass);

/* Upload positions, velocities and spins of all instances at once ([N][3],
 * N = sum of n_particles; any pointer may be NULL to keep that field).
 * Asynchronous on `stream` (host memory should be pinned).  When the context
 * has current neighbour lists they are kept: the particles move by their
 * displacement and the next step rebuilds only if one moved more than half
 * the Verlet skin since the last build (results do not depend on it). */
sdpd_status sdpd_upload_state(sdpd_ctx *ctx, const double *x, const double *v, const double *w,
                              void *stream);

/* Download positions, velocities, spins, total force and torque of all
 * instances ([N][3]; NULL skips a field).  Asynchronous on `stream`. */
sdpd_status sdpd_download_state(sdpd_ctx *ctx, double *x, double *v, double *w, double *F,
                                double *N, void *stream);

/* Set the time-step counter (keys the random stream).  Synchronous. */
sdpd_status sdpd_set_step(sdpd_ctx *ctx, long long step);
sdpd_status sdpd_get_step(sdpd_ctx *ctx, long long *step);

/* Number of neighbour-list builds the context has run (forced ones and
 * those the Verlet skin triggered inside the steps), a measurement aid.
 * Synchronous.  SDPD_E_INVALID for a NULL argument. */
sdpd_status sdpd_build_count(sdpd_ctx *ctx, long long *builds);

/* compute_neighbor_list (Algorithm 1; Section 3.2): background grid of cells
 * at least max(h, largest sphere diameter) wide, counting sort of the
 * particles into Morton-ranked cells (deterministic order within a cell), the
 * cell-sorted particle mirrors, and each particle's list of neighbours
 * j != i with r_ij < h (plus rigid pairs in contact beyond h).  Neighbour
 * decisions are exact in double precision. */
sdpd_status sdpd_build_cells(sdpd_ctx *ctx, void *stream);

/* compute_particle_dens, compute_particle_pres, smoothe_particle_pres
 * (Algorithm 1; Eqs. compdens, prtcpres; pressure filter): number density
 * d_i = C_n sum_j W_ij (self included), rho_i = rho0 dx^3 d_i, pressure from
 * the equation of state (clamped at 0 if clamp_negative_p), Shepard-filtered if
 * pressure_filter; also the fluid sums each rigid particle needs for the drag.
 * Requires sdpd_build_cells for the current positions. */
sdpd_status sdpd_compute_density(sdpd_ctx *ctx, void *stream);

/* compute_fpi_action (Algorithm 2; Eqs. fvfdef, beta, F_fpi_DG): per rigid
 * particle the fluid volume fraction, the mean fluid velocity around it and
 * the drag force.  Requires sdpd_compute_density. */
sdpd_status sdpd_couple_drag(sdpd_ctx *ctx, void *stream);

/* compute_fluid + compute_fpi_reaction + compute_rigid (Algorithm 2; Eqs.
 * FijC, FijD, FijR, FijT, F_fpi_PG, F_fpi_DG_reac, dem_fnij .. slideref,
 * lubri) and the external force (Eq. govern): total force and torque of every
 * particle for velocity-Verlet sub-step `velver` (1 or 2) at the current step
 * counter.  velver 2 commits the tangential contact history.  Requires
 * sdpd_couple_drag. */
sdpd_status sdpd_compute_forces(sdpd_ctx *ctx, int velver, void *stream);

/* update(velver) (Algorithm 1; Eqs. newton1, newton2): velocity-Verlet half
 * kick of v and w; velver 1 also drifts x and applies the periodic wrap / wall
 * reflection; velver 2 applies the artificial viscosity (collision method) if
 * enabled and advances the step counter. */
sdpd_status sdpd_integrate(sdpd_ctx *ctx, int velver, void *stream);

/* Algorithm 1 for n_steps full steps (both sub-steps, all stages), replayed
 * from a CUDA graph captured on the first call.  Positions unchanged since the
 * last neighbour build (velver 1 after velver 2) reuse that build and its
 * density exactly.  Synchronises at the end and reports kernel errors. */
sdpd_status sdpd_step(sdpd_ctx *ctx, long long n_steps, void *stream);

/* Reverse-Poiseuille viscometer read-out (Section 4.1; Eqs. poiseuanasol,
 * poiseuave) of instance `inst`: mean velocity along body_axis of the fluid
 * particles in n_bins slabs of split_axis (profile_out[n_bins], host), and the
 * apparent viscosity mu = rho0 a D^2 / (12 V) from the mean speed V of the two
 * counter-flowing halves (D = half the box).  Synchronous. */
sdpd_status sdpd_viscosity_probe(sdpd_ctx *ctx, int inst, int n_bins, double *profile_out,
                                 double *mu_app_out);

/* Viscosity from the curvature of the steady profile (Section 4.1: the
 * parabola of Eq. poiseuanasol fitted to the convex and concave halves): for
 * each half of the split axis a least-squares parabola through the slab mean
 * velocities at the slabs' mean particle positions (n_bins slabs as
 * sdpd_viscosity_probe), over the slabs at least h from the ends of the
 * half, mu = -+ rho0 g / v''; the mean of the two halves in
 * *mu_fit_out.  Independent of where a wall's no-slip plane lies.  Needs at
 * least 4 such slabs per half (else SDPD_E_INVALID).  Synchronous. */
sdpd_status sdpd_viscosity_fit(sdpd_ctx *ctx, int inst, int n_bins, double *mu_fit_out);

/* Host copies of one instance's state (NULL skips a field): x, v, w, F, N
 * [n][3]; d (number density), p (pressure) [n].  Synchronous. */
sdpd_status sdpd_get_state(sdpd_ctx *ctx, int inst, double *x, double *v, double *w, double *F,
                           double *N, double *d, double *p);

/* Per rigid particle of instance `inst`, in gid order of the rigid particles:
 * fluid volume fraction eps[nr], drag force F_dg[nr][3].  Synchronous. */
sdpd_status sdpd_get_drag(sdpd_ctx *ctx, int inst, double *eps, double *F_dg);

/* Neighbour pairs (i < j, instance-local gids) with r_ij < h of instance
 * `inst` from the last build: writes min(cap, count) pairs into ij[2*cap] and
 * the count into *n_out.  Synchronous. */
sdpd_status sdpd_get_pairs(sdpd_ctx *ctx, int inst, long long cap, int *ij, long long *n_out);

/* Number of unordered pairs within h that the force pass evaluates (at least
 * one mobile particle), all instances, from the last build.  Synchronous. */
sdpd_status sdpd_count_pairs(sdpd_ctx *ctx, long long *n_pairs);

/* Diagnostics of instance `inst` (Synchronous): out[0..2] total momentum,
 * out[3] kinetic energy, out[4] kinetic temperature m<v^2>/3 of the mobile
 * particles (mean removed), out[5] max |v|, out[6] min d, out[7] max d,
 * out[8] number of non-finite values in x, v, w. */
sdpd_status sdpd_diagnostics(sdpd_ctx *ctx, int inst, double out[16]);

/* Force-pass variant: newton3 = 1 (default) evaluates each unordered pair once
 * (one of the two particles owns it, chosen by a hash of the pair so that
 * each owns about half of its list; its result goes to the partner through a
 * pair buffer; deterministic, no atomics); newton3 = 0 evaluates every pair
 * from both sides, one thread per particle walking its list; newton3 = 2 is
 * the same pass as 0 with the pairs streamed through shared memory: a warp
 * compacts the pairs within h of its 32 particles' lists and evaluates them
 * 32 at a time, each particle summing its own in list order (forces equal to
 * those of 0 bit for bit); newton3 = 3 is that pass with its registers
 * capped for three 256-thread blocks per SM instead of two (a tuning choice;
 * FP32 pairs only, FP64 runs 2); newton3 = 4 is the Newton-3 pass with the
 * owner writing each finished pair result (force, e x o) straight into the
 * partner's column, which the partner then reads coalesced, as the FP64
 * pass always does (for FP32 pairs, 1 keeps {o, ce} in the owner's column
 * and the partner gathers it through the reverse index; 4 and 1 give the
 * same bits); newton3 = 5 is the direct pass with only the list index and
 * the partner's position fetched ahead, which needs fewer registers and runs
 * more warps per SM, its other records coming at the first evaluation through
 * an asynchronous shared-memory ring (FP32 pairs; FP64 runs 0; the same bits
 * as 0).  All give
 * the same forces up to summation order.
 * Invalidates the current neighbour build and graph.  Synchronous. */
sdpd_status sdpd_set_force_mode(sdpd_ctx *ctx, int newton3);

/* Normals cache (default on = 1): the second force evaluation of a step
 * (velver 2) reads the six standard normals of each pair that the first one
 * drew, where the neighbour list was not rebuilt in between, instead of
 * drawing them again.  The draws are keyed by (pair, step) (Section 2.1,
 * Eq. FijT; one dW per pair and step), so both give the same bits; off
 * (0) draws every time.  Invalidates the current graph.  Synchronous. */
sdpd_status sdpd_set_noise_cache(sdpd_ctx *ctx, int on);

/* Threads per block of the pair kernels (density, filter, force passes):
 * 64, 128 (default) or 256.  A tuning knob; results do not change.
 * Synchronous. */
sdpd_status sdpd_set_block_size(sdpd_ctx *ctx, int threads);

/* Lanes per particle of the direct force pass (force mode 0): 1 (default), 2
 * or 4.  With more than one, the lanes of a particle take every tpp-th entry
 * of its list and their sums are added by a fixed butterfly of shuffles, so
 * small workloads fill more of the GPU; the result differs from tpp = 1 only
 * by summation order and is the same on every run.  A tuning knob.
 * Invalidates the current graph.  Synchronous. */
sdpd_status sdpd_set_threads_per_particle(sdpd_ctx *ctx, int tpp);

/* Cells of the neighbour search per minimum cell width (Algorithm 1, Section
 * 3.2, the background grid): 1 (default) or 2.  The minimum width is
 * max(h (1 + skin), largest sphere diameter + skin h); with 2 the cells are
 * half as wide, the stencil reaches 2 cells each way (125 cells, about 0.58
 * of the 27-cell volume) and the lists are built with one lane per candidate
 * instead of one per particle.  The listed pairs are the same (every pass
 * re-decides r_ij < h exactly); particles are ordered by the finer cells,
 * so results differ only by summation order.  A tuning knob.  Invalidates
 * the grid and the graph.  Synchronous.  SDPD_E_INVALID for any other value. */
sdpd_status sdpd_set_cell_factor(sdpd_ctx *ctx, int cells);

/* Verlet skin as a fraction of h (default 0.03): neighbour lists hold the
 * pairs within h (1 + skin) and are reused by later evaluations until some
 * particle has moved skin h / 2 since the build (decided on the device each
 * drift; the rebuild happens inside the step).  Every pass re-decides
 * r_ij < h exactly, so results do not depend on the skin beyond summation
 * order.  Invalidates the grid and the graph.  Synchronous. */
sdpd_status sdpd_set_skin(sdpd_ctx *ctx, double skin);

/* Number of kernel nodes in the captured one-step graph of sdpd_step (0 if
 * sdpd_step has not run yet).  Synchronous. */
sdpd_status sdpd_graph_kernels(sdpd_ctx *ctx, long long *n_kernels);

/* Largest particle and cell counts sdpd_density_noalloc accepts. */
#define SDPD_NOALLOC_MAX_PARTICLES 131072
#define SDPD_NOALLOC_MAX_CELLS 65536

/* Number density d and pressure p ([n] doubles, device memory) of one
 * particle set -- positions x ([n][3] doubles) and types ([n] int32), both in
 * device memory -- under parameters *params, without allocating any device
 * memory.  The paper has no counterpart: this exists for callers that cannot
 * let a library allocate, such as applications whose own allocator owns the
 * whole device and code that cannot afford the device-wide synchronisation
 * cudaMalloc/cudaFree may cause.  The results equal those of
 * sdpd_build_cells + sdpd_compute_density in FP64 with the filter off, up to
 * summation order.
 * Input domain: origin and box finite with box > 0 on every axis, dx > 0,
 * r_c > 0 and r_c / dx <= 32; otherwise SDPD_E_INVALID before any launch.
 * Positions on periodic axes may lie anywhere (they are folded into the
 * box); on wall axes positions outside the box are used as given.  A
 * particle whose position is not finite gets d = p = NaN and is nobody's
 * neighbour; the other particles are unaffected.
 * Scratch: one file-scope __device__ array of about 2 MB (cell keys, slots,
 * counts, starts, permutation) held by every GPU that loads the library until
 * the process exits.  At most SDPD_NOALLOC_MAX_PARTICLES particles and
 * SDPD_NOALLOC_MAX_CELLS cells of width >= r_c (periodic axes: floor(box/r_c)
 * cells, >= 3; wall axes: the box plus 2 r_c on each side); larger inputs are
 * rejected with SDPD_E_INVALID.  The first call on a device resolves the
 * array's device address (with that device current) and should come before
 * any stream capture; the address is kept for the process, so the library
 * must not be used across a device reset.  Every call reuses the same array
 * and leaves its contents behind: calls whose work overlaps on the GPU
 * (different streams, different host threads) race and give wrong results;
 * serialise them.  Asynchronous on `stream`; no cudaMalloc, cudaFree or
 * allocating library call is made. */
sdpd_status sdpd_density_noalloc(const sdpd_params *params, long long n, const double *x,
                                 const int *type, double *d_out, double *p_out, void *stream);

/* The six standard normals z0..z5 of the random term of Eq. FijT for n
 * pairs (gi[k], gj[k]) at `step`, exactly as the pair kernels draw them:
 * Philox4x32-10 (Salmon et al., SC'11) keyed (seed low word, seed high word
 * XOR inst), counter (min gid, max gid, step, block 0/1), uniforms
 * ((u >> 9) + 1/2) 2^-23, Box-Muller in the given precision (SDPD_PREC_FP64
 * or SDPD_PREC_SPLIT, FP32).  gi, gj: host [n]; z_out: host [n][6] doubles.
 * Synchronous; needs no context.  Symmetric in (gi, gj). */
sdpd_status sdpd_noise_normals(int precision, unsigned long long seed, int inst, unsigned step, long long n,
                               const unsigned *gi, const unsigned *gj, double *z_out);

/* The counter-based generator of the random term (Eq. FijT's dW; Philox4x32-10
 * of Salmon, Moraes, Dror and Shaw, SC'11, the stream that replaces the
 * paper's per-pair Mersenne Twister) on the GPU, exactly as the pair kernels
 * run it: for each k < n, the 128-bit block philox(ctr[k][0..3],
 * key[k][0..1]) into out[k][0..3].  ctr [n][4], key [n][2], out [n][4]: host
 * uint32 arrays.  Synchronous; needs no context.  For checking the
 * generator against published known-answer vectors. */
sdpd_status sdpd_philox4x32_10(long long n, const unsigned *ctr, const unsigned *key, unsigned *out);

/* Measured arithmetic throughput of this GPU (a measurement utility; the
 * paper has no counterpart): out[0] FP32 fused multiply-add rate in TFLOP/s
 * (2 flops each), out[1] the FP64 one, out[2] 32-bit integer multiply-adds in
 * tera-operations/s, out[3] the number of SMs.  Register-resident
 * independent chains on every SM, timed with CUDA events at the clock the
 * GPU runs at; these are the denominators of the pair kernels' rooflines.
 * Synchronous, about 0.2 s; allocates a small scratch buffer. */
sdpd_status sdpd_alu_peaks(double *out);

/* Checkpoint and restart (the restart files of Section 3.1): the dynamic
 * state of all instances -- positions, velocities and angular velocities
 * [N][3] FP64 in particle order, the step counter (it keys the random
 * stream) and the tangential contact histories of the rigid particles -- as
 * one byte image in caller (host) memory.  sdpd_checkpoint_size gives its
 * length; sdpd_checkpoint waits for the context and writes it; sdpd_restore
 * reads it into a context of the same shape (same particle count, rigid
 * particles and max_contacts; created from the same sdpd_set_particles data)
 * and fails with SDPD_E_INVALID otherwise.  Both make the next step rebuild
 * the neighbour lists, so a run restored from an image continues bit for bit
 * as the run that wrote it. */
sdpd_status sdpd_checkpoint_size(sdpd_ctx *ctx, long long *bytes);
sdpd_status sdpd_checkpoint(sdpd_ctx *ctx, void *buf, long long bytes);
sdpd_status sdpd_restore(sdpd_ctx *ctx, const void *buf, long long bytes);

/* Wait for all work of the context and report a pending kernel error. */
sdpd_status sdpd_check(sdpd_ctx *ctx);

/* ---------------------------------------------------------------------------
 * Apparent-viscosity surrogate (a build component; the paper has none): a
 * multilayer perceptron 3 -> 128 -> 128 -> 128 -> 128 -> 1 with GELU (erf
 * form), MSE loss and Adam (lr given, beta = (0.9, 0.999), eps = 1e-8).  The
 * three 128 x 128 layers run on the tensor cores (tcgen05, BF16 operands,
 * FP32 accumulation); the input/output layers and element-wise work in FP32.
 * Parameters are one flat FP32 vector of mlp_param_count() values in the
 * order W0 [128][3], b0 [128], W1 [128][128], b1, W2, b2, W3, b3, W4 [128],
 * b4 [1] (W[out][in], row-major).  X is [n][3] FP32 (inputs scaled to about
 * [0, 1] by the caller), targets and outputs [n] FP32, all in device memory.
 * A network object is not thread-safe. */
typedef struct sdpd_mlp sdpd_mlp;

/* Create the network (in = 3, width = 128, depth = 4 are the only shape);
 * He-uniform weights from `seed`, zero biases; training batches up to
 * batch_max rows.  Synchronous. */
sdpd_status mlp_init(int in, int width, int depth, unsigned long long seed, int batch_max, sdpd_mlp **out);
void mlp_destroy(sdpd_mlp *net);
int mlp_param_count(void);
/* Replace the parameters (host or device pointer; resets Adam).  Synchronous. */
sdpd_status mlp_set_params(sdpd_mlp *net, const float *params);
/* Copy parameters and the last gradients out (NULL skips).  Synchronous. */
sdpd_status mlp_get_params(sdpd_mlp *net, float *params, float *grads);
/* Forward + backward of one batch without updating: gradients of the mean
 * squared error; *loss (host, may be NULL) written after a synchronisation. */
sdpd_status mlp_gradients(sdpd_mlp *net, const float *X, const float *T, int batch, float *loss, void *stream);
/* One Adam step on one batch; *loss as for mlp_gradients. */
sdpd_status mlp_train_step(sdpd_mlp *net, const float *X, const float *T, int batch, float lr, float *loss,
                           void *stream);
/* Predictions for n rows (persistent launch over 128-row tiles). */
sdpd_status mlp_infer(sdpd_mlp *net, const float *X, float *Y, long long n, void *stream);
/* Wait and report a pending error (a tensor-core completion wait that timed
 * out is SDPD_E_TIMEOUT). */
sdpd_status mlp_check(sdpd_mlp *net);

/* Last error message of the calling thread (never NULL). */
const char *sdpd_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* SDPD_H */
