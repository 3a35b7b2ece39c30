/*
 * mlswlbm.h -- C ABI of the GB300 (sm_103a) multilayer shallow-water lattice
 * Boltzmann solver for the n-layer thin-film equation (Richter, Malgaretti &
 * Harting, "Modeling of thin liquid films with arbitrary many layers").
 *
 * One time step, for every lattice cell and liquid layer i = 1..n:
 *   - moments h_i = sum_k f_ki, h_i U_i = sum_k c_k f_ki        (section LBM)
 *   - interfaces z_i = sum_{j<=i} h_j, their lattice gradient and Laplacian
 *   - Laplace pressure Lambda_i (Eq. Laplace_pressure) with the wetting
 *     potential phi_k (Eq. wetting_potential) and disjoining pressure Pi_i
 *     (Eq. disjoining_pressure); p_i - p_atm = sum_{j>=i} (Lambda_j + Pi_j)
 *   - friction 2 mu_i h_i a_i from the velocity boundary conditions
 *     (Eqs. u_ansatz, no_slip, flux, viscous_boundary, friction_force)
 *   - force F_i = -h_i grad p_i + 2 mu_i h_i a_i (Eq. force)
 *   - BGK collision with forcing and streaming (Eqs. BGK,
 *     equilibrium_distribution) on a D1Q3 or D2Q9 lattice, periodic.
 *
 * Conventions for every entry point:
 *   - Return value: MLSW_OK (0) or a negative MLSW_ERR_* code; no exception
 *     or signal crosses the ABI. mlswlbm_strerror() names the code.
 *   - Host arrays are owned by the caller and copied; the library never
 *     keeps a caller pointer. Device memory of a handle is owned by the
 *     handle and released by mlswlbm_destroy().
 *   - All device work of a handle runs on the CUDA stream bound at create
 *     (a cudaStream_t passed as void*, NULL = legacy default stream), so a
 *     PyTorch stream's cuda_stream can be used. Entry points that return
 *     host data synchronise that stream; the others are asynchronous.
 *   - A handle is used by one host thread at a time.
 *   - Layouts (row-major, x fastest, all FP32):
 *       heights      h[i][y][x],          i = 0..n-1 (layer i+1)
 *       populations  f[i][k][y][x],       k = lattice direction, paper order:
 *         D1Q3: c = 0, +1, -1;
 *         D2Q9: c = (0,0),(1,0),(1,1),(0,1),(-1,1),(-1,0),(-1,-1),(0,-1),(1,-1).
 *     A state is stored post-streaming: f[i][k] at cell x arrived from x - c_k.
 *   - Inside a handle the rest population of layer i is stored shifted by a
 *     per-layer constant H_i (f_0 - H_i; H_i = median of the layer in
 *     h_init), which keeps the long-wave height differences and the small
 *     fluxes of precursor films representable in FP32. mlswlbm_get_state /
 *     mlswlbm_set_state convert to and from the true populations;
 *     mlswlbm_save_state / mlswlbm_load_state move the
 *     internal representation unchanged (bit-exact checkpoints).
 */
#ifndef MLSWLBM_H
#define MLSWLBM_H

#ifdef __cplusplus
extern "C" {
#endif

#define MLSW_MAX_LAYERS 5
#define MLSW_D1Q3 1
#define MLSW_D2Q9 2

/* flags */
#define MLSW_FLAG_SKIP_STABILITY_CHECK 1
/* D1Q3 lattices that fit one CTA's shared memory normally run all the
 * steps of one mlswlbm_step call in a single persistent launch; this flag
 * keeps them on one launch per step (same results, bit for bit). */
#define MLSW_FLAG_NO_PERSISTENT 2

/* return codes */
#define MLSW_OK 0
#define MLSW_ERR_ARG (-1)         /* invalid argument or parameter             */
#define MLSW_ERR_NOMEM (-2)       /* device or host allocation failed          */
#define MLSW_ERR_CUDA (-3)        /* a CUDA call failed                        */
#define MLSW_ERR_NONFINITE (-4)   /* a kernel saw h <= 0 or a non-finite value */
#define MLSW_ERR_UNSTABLE (-5)    /* explicit friction update not contractive  */
#define MLSW_ERR_TIMEOUT (-6)     /* a bounded device wait ran out             */
#define MLSW_ERR_UNSUPPORTED (-7) /* no kernel for this configuration          */

/*
 * Problem statement (section Model). Index conventions:
 *   gamma[i-1]      gamma_{i,i+1}, tension of the interface above layer i,
 *                   i = 1..n (layer n+1 is the gas).
 *   spread[i][k-1]  spreading coefficient S_{ik} of Eq. (spreading_parameters),
 *                   i = 0..n-1 (0 = substrate), k = 1..n-i; other entries
 *                   are ignored.
 *   mu[i-1]         viscosity mu_i > 0.
 *   beta[i-1]       slip length beta_i >= 0 of Eq. (no_slip): beta_1 at the
 *                   substrate, beta_{i>1} at the interface below layer i.
 *   wet_n, wet_m    exponents of Eq. (wetting_potential), wet_n > wet_m >= 1
 *                   (with wet_kind 0, the power law).
 *   hstar           precursor thickness h* > 0.
 *   tau             BGK relaxation time of Eq. (BGK), tau > 1/2 (paper: 1).
 *   nx, ny          periodic lattice size; D1Q3 needs ny == 1.
 * The arithmetic is FP32 on the device; these doubles are rounded once.
 */
typedef struct mlsw_params {
  int n_layers; /* 1..MLSW_MAX_LAYERS */
  int lattice;  /* MLSW_D1Q3 or MLSW_D2Q9 */
  int nx, ny;
  double tau;
  double gamma[MLSW_MAX_LAYERS];
  double spread[MLSW_MAX_LAYERS][MLSW_MAX_LAYERS];
  double mu[MLSW_MAX_LAYERS];
  double beta[MLSW_MAX_LAYERS];
  int wet_n, wet_m;
  double hstar;
  int flags; /* MLSW_FLAG_* */
  /* substrate height z_0(x, y) = sub_amp cos(2 pi (sub_kx x / nx + sub_ky y / ny))
   * (section Model: z_0 is the possibly corrugated substrate); sub_amp = 0
   * is the flat substrate of the paper's runs. It enters the interface
   * heights z_i = z_0 + sum_{j<=i} h_j, hence every Laplace and slope term,
   * and the factor (1 + |grad z_0|^2 / 2) of the substrate's terms in
   * Eq. (disjoining_pressure). D1Q3 needs sub_ky = 0. */
  double sub_amp;
  int sub_kx, sub_ky;
  /* wetting potential: wet_kind 0 is the power law of Eq. (wetting_potential)
   * with exponents (wet_n, wet_m); 1 is the exponential decay the paper
   * quotes for charged surfaces (the discussion before that ansatz), in the
   * form phi_k(d) = 2 e^{-kappa (d - k h*)} - e^{-2 kappa (d - k h*)} with
   * kappa = wet_kappa > 0. It keeps the power law's limits phi_k(k h*) = 1,
   * phi_k'(k h*) = 0 and phi_k -> 0, and wet_n, wet_m are not used. */
  int wet_kind;
  double wet_kappa;
} mlsw_params;

typedef struct mlsw_handle mlsw_handle;

/*
 * Fills p->spread (Eq. spreading_parameters) and p->gamma from the full
 * tension table gamma_full[a * (n+2) + b] = gamma_{a,b}, a, b = 0..n+1
 * (0 = substrate, n+1 = gas). Host only. Sets p->n_layers = n_layers.
 * Errors: MLSW_ERR_ARG for a NULL pointer or n outside 1..MLSW_MAX_LAYERS.
 */
int mlswlbm_spreading_from_tensions(int n_layers, const double* gamma_full,
                                    mlsw_params* p);

/* Validates p without touching the GPU. MLSW_OK or MLSW_ERR_ARG. */
int mlswlbm_check_params(const mlsw_params* p);

/*
 * Creates a solver: validates p, allocates two population buffers of
 * n*Q*nx*ny floats plus small scratch on the current CUDA device, uploads
 * h_init (host, [n][ny][nx], every value finite and > 0) and sets
 * f = f_eq(h_init, U = 0) (Eq. equilibrium_distribution), i.e. the rest
 * population carries h and the moving ones are zero.
 * Unless p->flags has MLSW_FLAG_SKIP_STABILITY_CHECK, the explicit update of
 * a uniform flux, J <- (1 + K) J with the friction matrix K of
 * Eq. (friction_force), must be contractive at the per-layer minimum, mean
 * and maximum of h_init and with every layer at h*; otherwise
 * MLSW_ERR_UNSTABLE. MLSW_ERR_UNSUPPORTED when one layer's padded planes
 * exceed 2^31 - 1 floats (about 15000 x 15000 cells for D2Q9).
 * stream: cudaStream_t or NULL.
 * On failure *out is set to NULL and nothing is leaked.
 */
int mlswlbm_create(const mlsw_params* p, const float* h_init, void* stream,
                   mlsw_handle** out);

/* Enqueues nsteps >= 0 time steps on the handle's stream; asynchronous.
 * One fused kernel launch per step, except for D1Q3 lattices small enough
 * for one CTA (8 n nx floats of shared memory), which run up to 16384 steps
 * per persistent launch with the lattice held on chip (see
 * MLSW_FLAG_NO_PERSISTENT). MLSW_ERR_ARG for a NULL handle or nsteps < 0;
 * MLSW_ERR_CUDA if a launch fails. */
int mlswlbm_step(mlsw_handle* h, long nsteps);

/* Heights h_i = sum_k f_ki into out (host, n*nx*ny floats). Synchronises.
 * Returns MLSW_ERR_NONFINITE if any step since create or the last status
 * query flagged h <= 0 or a non-finite value (out is still written).
 * Page-locked memory (cudaHostAlloc, cudaHostRegister) is written by the
 * read-out kernel directly; other memory through a device buffer. */
int mlswlbm_get_heights(mlsw_handle* h, float* out);

/* Same into device memory dev_out (n*nx*ny floats, caller-owned, on the
 * handle's device); asynchronous, no status check. */
int mlswlbm_get_heights_device(mlsw_handle* h, float* dev_out);

/* Restarts the state from heights in device memory (n*nx*ny floats,
 * [layer][y][x], on the handle's device): f = f_eq(h, U = 0), as
 * mlswlbm_set_heights does for host heights. Asynchronous; heights <= 0 or
 * non-finite set the handle's status, which the next status query reports. */
int mlswlbm_set_heights_device(mlsw_handle* h, const float* dev_in);

/* Restarts from heights (host, [n][ny][nx]): f = f_eq(h, U = 0). The
 * values are checked on the device: a value <= 0 or non-finite is reported
 * as MLSW_ERR_NONFINITE by the next status query (mlswlbm_status,
 * mlswlbm_get_heights, mlswlbm_get_diagnostics). The shift H_i of create is
 * kept. Asynchronous on the handle's stream; h_in must stay valid until the
 * stream reaches the copy (pageable memory is copied before return).
 * Page-locked memory is read by the initialisation kernel directly, so it
 * must stay unchanged until that kernel has run. */
int mlswlbm_set_heights(mlsw_handle* h, const float* h_in);

/* True population state (host, n*Q*nx*ny floats, layout above): copy out
 * (synchronises) and copy in. The copy out rounds f_0 = H_i + (f_0 - H_i)
 * to FP32, so a get/set round trip is not bit-exact; use save/load for
 * that. */
int mlswlbm_get_state(mlsw_handle* h, float* f_out);
int mlswlbm_set_state(mlsw_handle* h, const float* f_in);

/* Internal representation, unchanged: H_out / H_in = the n shifts H_i,
 * g_out / g_in = n*Q*nx*ny floats laid out like f with the rest planes
 * holding f_0 - H_i. Save then load resumes bit-exactly. Both synchronise.
 * MLSW_ERR_ARG for NULL pointers or a non-finite shift. */
int mlswlbm_save_state(mlsw_handle* h, float* H_out, float* g_out);
int mlswlbm_load_state(mlsw_handle* h, const float* H_in, const float* g_in);

/*
 * Diagnostics of the current state, reduced on the device in double:
 *   mass[i]   = sum_x h_i(x)                                (n doubles)
 *   *kinetic  = sum_{i,x} |J_i(x)|^2 / (2 h_i(x))
 *   *hmin     = min_{i,x} h_i(x)
 * Any output pointer may be NULL. Synchronises. Returns MLSW_ERR_NONFINITE
 * as mlswlbm_get_heights does.
 */
int mlswlbm_get_diagnostics(mlsw_handle* h, double* mass, double* kinetic,
                            double* hmin);

/* Free energy of Eq. (free_energy_n_layer) in its long-wave form,
 *   F = sum_x [ sum_{i=1..n} gamma_{i,i+1} (1 + |grad z_i|^2 / 2)
 *             + sum_{i=0..n-1} sum_{k=1..n-i} S_ik phi_k(z_{i+k} - z_i)
 *               (1 + |grad z_i|^2 / 2) ]     (z_0 = 0, flat substrate),
 * with the lattice gradient of the step, summed on the device in FP64 from
 * the current heights and the parameters of create (in double). A quantity
 * the relaxation lowers (section Model); with the kinetic energy of
 * mlswlbm_get_diagnostics it serves as the stop criterion of equilibrium
 * runs. Synchronises; status as mlswlbm_get_heights. */
int mlswlbm_get_free_energy(mlsw_handle* h, double* F);

/* Radially averaged power spectrum of every layer's heights (the quantity
 * the paper's spinodal-dewetting section follows and sets against its
 * linear stability analysis): out[i * nbins + b] = mean of |H_i(k)|^2 over
 * the integer wavevectors k = (kx, ky), kx in (-nx/2, nx/2] and likewise
 * ky, with round(|k|) = b, for b < nbins; H_i is the unnormalised 2-D DFT of
 * h_i with its mean removed (0 where a bin holds no wavevector). D1Q3
 * lattices (ny = 1) give the 1-D spectrum by |kx|. Computed on the device by
 * FP32 radix-2 FFTs of h_i - H_i (the height minus the layer's
 * rest-population shift) with FP64 bin sums. nx and ny must be powers of two
 * up to 8192 and 1 <= nbins <= 8192 (MLSW_ERR_UNSUPPORTED otherwise);
 * out is host memory of n_layers * nbins doubles. Allocates stream-ordered
 * scratch of 8 n nx ny bytes for the call (MLSW_ERR_NOMEM if that fails).
 * Synchronises; returns the handle's status like mlswlbm_get_heights. */
int mlswlbm_get_spectrum(mlsw_handle* h, int nbins, double* out);

/* Azimuthal averages of the interface heights around (cx, cy), the
 * profiles the paper's droplet-equilibrium section fits circular arcs to:
 * out[m * nbins + b] = mean of z_m over the cells whose periodic
 * (minimum-image) distance r from (cx, cy) has floor(r) = b, for the
 * interfaces m = 0..n (z_0 the substrate, z_m = z_0 + h_1 + ... + h_m) and
 * b < nbins; 0 for an empty ring. counts (optional, nbins values) receives
 * the cells per ring. Per-cell heights are those of mlswlbm_get_heights
 * (FP32); interfaces and ring sums are FP64, summed on the device. D2Q9
 * only (MLSW_ERR_UNSUPPORTED otherwise); MLSW_ERR_ARG for nbins < 1 or a
 * non-finite centre. out is host memory of (n_layers + 1) * nbins doubles.
 * Allocates stream-ordered scratch for the call; synchronises; returns the
 * handle's status like mlswlbm_get_heights. */
int mlswlbm_get_radial_profile(mlsw_handle* h, double cx, double cy, int nbins, double* out,
                               long long* counts);

/* Contact angle of an axisymmetric cap (the paper's droplet-equilibrium
 * fit), host only: the circular arc through the profile's apex prof[0] at
 * r = 0 that meets the level `base` at angle theta; theta minimises the
 * relative volume difference E = sum_b a_b |prof_b - arc(r_b)| /
 * sum_b a_b (prof_b - base), r_b = b + 1/2, a_b = area[b] (the cells per
 * ring). Scan from 0.5 to 60 degrees in 0.05-degree steps, then 40
 * golden-section steps between the neighbours of the best one. Writes theta
 * in degrees and, if err is not NULL, E. MLSW_ERR_ARG for NULL arrays,
 * nbins < 2 or prof[0] <= base. For a lens, pass the upper surface above its
 * far level, or the far level minus the lower surface, with base 0. */
int mlswlbm_fit_cap_angle(const double* prof, const double* area, int nbins, double base,
                          double* theta_deg, double* err);

/* Steps until the kinetic energy sum_{i,x} |J_i|^2 / (2 h_i) (as in
 * mlswlbm_get_diagnostics) is below ke_threshold, checked after every
 * check_every >= 1 steps (a run starting from rest has none, so at least
 * min(check_every, max_steps) steps are taken), or until max_steps >= 0
 * steps are done. *steps_done and *kinetic (either may be NULL) receive the
 * steps taken and the last kinetic energy; the caller compares it with the
 * threshold to see which limit ended the run. Synchronises at every check;
 * errors as mlswlbm_step and mlswlbm_get_diagnostics. */
int mlswlbm_step_until(mlsw_handle* h, long max_steps, long check_every, double ke_threshold,
                       long* steps_done, double* kinetic);

/* Synchronises and returns MLSW_OK or MLSW_ERR_NONFINITE (a kernel saw
 * h <= 0 or a non-finite value since create or the last call); clears it. */
int mlswlbm_status(mlsw_handle* h);

/* Self-test of failure detection, without a GPU fault: one CTA waits on
 * an mbarrier with the bounded wait the step kernels use for their tile
 * copies (limit iterations of try_wait, 1 <= limit <= 2^22). With
 * arrive != 0 the barrier receives its arrival and the call returns
 * MLSW_OK; with arrive == 0 nothing arrives, every wait runs out, the
 * kernel records the timeout in a status word and returns, and the call
 * returns MLSW_ERR_TIMEOUT, the code mlswlbm_status gives when a step's
 * wait runs out. The CUDA context stays usable. Allocates one int of device
 * memory; synchronises the stream (cudaStream_t or NULL). */
int mlswlbm_selftest_bounded_wait(int arrive, unsigned limit, void* stream);

/* Binds another stream to the handle (cudaStream_t or NULL). The caller
 * orders work already queued on the old stream. */
int mlswlbm_set_stream(mlsw_handle* h, void* stream);

/* Number of GPU kernel launches this handle has issued since create. */
long mlswlbm_launch_count(const mlsw_handle* h);

/* Frees the handle and its device memory; NULL is accepted. Synchronises. */
void mlswlbm_destroy(mlsw_handle* h);

/* Static string for a return code; never NULL. */
const char* mlswlbm_strerror(int code);

/*
 * Bounds-checked build. A library compiled with -DMLSW_DEBUG checks every
 * padded-layout index, every shared-memory access and global store of the
 * step kernels and the coordinates of every tile copy; an access out of
 * range is counted and sent to a padding cell instead of faulting, so the
 * results are wrong but the GPU is not. This call synchronises the device,
 * returns in *count the accesses out of range since the previous call and
 * clears the counters. It checks the implementation, not a passage of the
 * paper.
 * Errors: MLSW_ERR_ARG (count NULL), MLSW_ERR_CUDA (the counters could not be
 * read), MLSW_ERR_UNSUPPORTED (a release build: *count = 0).
 */
int mlswlbm_debug_bounds_violations(unsigned long long* count);

/*
 * Per-cell friction 2 mu_i h_i a_i (Eq. friction_force) for ncell
 * independent cells, on the device. h, Jx, Jy, Rx, Ry: device pointers of
 * n*ncell floats, layout [i][cell]; Jy/Ry may be NULL (one component).
 * Only n_layers, mu and beta of p are used. Runs the same device routine
 * the step kernels use; asynchronous on stream. Allocates nothing.
 * Errors: MLSW_ERR_ARG (bad p or pointers), MLSW_ERR_CUDA (launch).
 */
int mlswlbm_friction_eval(const mlsw_params* p, long ncell, const float* h,
                          const float* Jx, const float* Jy, float* Rx,
                          float* Ry, void* stream);

/*
 * Diagnostics without any allocation. The paper has no counterpart; this
 * entry point serves callers that cannot call cudaMalloc: applications
 * whose device memory is already reserved by a pool allocator (a plain
 * cudaMalloc there fails or fragments the pool) and latency-critical loops
 * in which cudaMalloc / cudaFree would synchronise the whole device.
 *
 * Computes what mlswlbm_get_diagnostics computes -- out[i] = mass of layer
 * i (i < n), out[n] = kinetic energy sum |J|^2 / (2h), out[n+1] = min h --
 * for a population array that the caller owns, without a handle.
 *   p       problem statement; n_layers, lattice, nx, ny are used.
 *   f       device, n*Q*nx*ny floats in the population layout above.
 *   H       host, n floats: the rest planes of f hold f_0 - H_i (as written
 *           by mlswlbm_save_state); NULL when f holds the true populations.
 *   out     device, n + 2 doubles, caller-owned; written asynchronously.
 *   stream  cudaStream_t or NULL.
 * Scratch: a static device array of 224 KiB (4096 blocks x 7 doubles) in
 * the library, held by every GPU that loads the library until exit. One
 * block is used per 16384 cells, so lattices above 4096 * 16384 cells
 * (67,108,864) return MLSW_ERR_UNSUPPORTED. The first call on a device looks
 * up the array's device address (with that device current) and should come
 * before any stream capture; only a successful look-up is kept, so after a
 * failed one (MLSW_ERR_CUDA) the next call on that device tries again.
 * Every call shares the array and overwrites the partials it uses; calls
 * that overlap on the GPU race on it. Calls no cudaMalloc, cudaFree or other
 * allocating routine.
 * Errors: MLSW_ERR_ARG (NULL pointer, invalid p, non-finite H),
 * MLSW_ERR_UNSUPPORTED (lattice beyond the scratch, device ordinal >= 64),
 * MLSW_ERR_CUDA (symbol look-up or launch failed).
 */
int mlswlbm_diagnostics_noalloc(const mlsw_params* p, const float* f, const float* H,
                                double* out, void* stream);

/*
 * ------------------------------------------------------------------------
 * Batches: many independent D2Q9 lattices (e.g. the instances of a
 * stability or equilibrium sweep: layer counts, sizes and parameters may all
 * differ) advanced together. One step of a batch is one persistent kernel
 * launch over a table of every instance's tiles, in which the instances
 * sharing the layer count, the kernel mode (tau = 1 or not, exponents
 * (3, 2), spreading only between neighbouring interfaces) and the tile
 * height (a group) form a contiguous range; CTAs draw tiles from one
 * counter and pass from range to range without waiting for each other.
 * The launch is captured once in a CUDA graph per buffer parity and
 * replayed. Each instance is stepped with exactly the arithmetic of
 * mlswlbm_step (section LBM, Eq. BGK).
 * ------------------------------------------------------------------------
 */
typedef struct mlsw_batch mlsw_batch;

/* batch flags */
#define MLSW_BATCH_TILE8 1    /* 8-row tiles for every instance (default: 16 rows for n <= 3) */
#define MLSW_BATCH_AUTOTUNE 2 /* at create, time 8- and 16-row tiles for every class of
                                 instances with the same n, kernel mode and size (n <= 3)
                                 and keep the faster; the states are then reset to h_init */

/* Creates a batch of count >= 1 lattices: params[j] and h_init[j] (host,
 * [n_j][ny_j][nx_j]) as for mlswlbm_create, every lattice D2Q9 (else
 * MLSW_ERR_UNSUPPORTED). Errors of an instance are those of mlswlbm_create.
 * One device allocation holds all population buffers. On failure *out is
 * NULL and nothing is leaked. */
int mlswlbm_batch_create(int count, const mlsw_params* params, const float* const* h_init,
                         int flags, void* stream, mlsw_batch** out);

/* Enqueues nsteps >= 0 steps of every instance; asynchronous. */
int mlswlbm_batch_step(mlsw_batch* b, long nsteps);

/* Heights of instance index (host, [n][ny][nx]); synchronises; status as
 * mlswlbm_get_heights (for the whole batch). MLSW_ERR_ARG for a bad index. */
int mlswlbm_batch_get_heights(mlsw_batch* b, int index, float* out);

/* Device variants for one instance (dev: device, [n][ny][nx] FP32),
 * asynchronous on the batch's stream. get writes the instance's heights;
 * set restarts the instance from the given heights at rest, f = f_eq(h,
 * U = 0) as at create (the rest-population shift of create is kept), and
 * ORs MLSW_ERR_NONFINITE into the batch status where h <= 0 or h is not
 * finite. MLSW_ERR_ARG for a bad index or NULL pointer. */
int mlswlbm_batch_get_heights_device(mlsw_batch* b, int index, float* dev);
int mlswlbm_batch_set_heights_device(mlsw_batch* b, int index, const float* dev);

/* The same for `count` instances in one call (indices: host ints, any order;
 * an instance listed twice is read twice, or set from its later heights):
 * dev is the concatenation, in list order, of the instances' [n][ny][nx]
 * FP32 heights. One kernel launch per instance, no synchronisation.
 * MLSW_ERR_ARG for an index out of range, count < 0 or a NULL pointer with
 * count > 0; nothing is enqueued then. */
int mlswlbm_batch_get_heights_device_many(mlsw_batch* b, int count, const int* indices,
                                          float* dev);
int mlswlbm_batch_set_heights_device_many(mlsw_batch* b, int count, const int* indices,
                                          const float* dev);

/* One Fourier mode of every layer of every instance:
 * out[2 (j MLSW_MAX_LAYERS + i) + 0 / 1] = Re / Im of
 * sum_{x,y} h_i(x, y) exp(-2 pi i (kx[j] x / nx_j + ky[j] y / ny_j)),
 * zero for i >= n_j. kx, ky: count host ints; out: 2 MLSW_MAX_LAYERS count
 * host doubles. Synchronises; status as mlswlbm_get_heights. */
int mlswlbm_batch_modes(mlsw_batch* b, const int* kx, const int* ky, double* out);

/* MLSW_OK, MLSW_ERR_NONFINITE or MLSW_ERR_TIMEOUT for the whole batch since
 * create or the last query (then cleared); synchronises. */
int mlswlbm_batch_status(mlsw_batch* b);

/* Tile rows (8 or 16) that instance index runs with, or MLSW_ERR_ARG. */
int mlswlbm_batch_tile_rows(const mlsw_batch* b, int index);

/* Chooses the instances that mlswlbm_batch_step advances: the nsel distinct
 * indices (host ints, 0 <= index < count; nsel = 0 leaves none, and the
 * step then does nothing). Every instance starts selected. An instance left
 * out keeps its state unchanged through later steps, and its heights can be
 * read and set as before; selected again, it continues from that state.
 * A selected instance steps with exactly the arithmetic it has in the full
 * batch. Synchronises the batch's stream and rebuilds the step's launch
 * plan (milliseconds): meant for occasional changes, such as dropping the
 * instances that a caller finishes another way. MLSW_ERR_ARG for an index
 * out of range, a repeated index, or nsel outside [0, count]. */
int mlswlbm_batch_select(mlsw_batch* b, int nsel, const int* indices);

/* Kernel launches issued since create (graph replays counted by the
 * kernels they contain: one per step), and groups (ranges of the step's
 * tile table). */
long mlswlbm_batch_launch_count(const mlsw_batch* b);
int mlswlbm_batch_groups(const mlsw_batch* b);

void mlswlbm_batch_destroy(mlsw_batch* b);

/* ---------------------------------------------------------------------
 * U-Net surrogate of 64 LBM steps on the 5th-generation tensor cores.
 * Not a part of the paper's method: a learned stand-in for 64 steps of
 * the LBM step above (heights in, heights 64 steps later out),
 * trained on trajectories the solver generates and judged by it.
 *
 * Network: four levels of 32, 64, 128 and 256 channels at full, 1/2, 1/4
 * and 1/8 resolution; two 3 x 3 periodic convolutions with ReLU per level
 * on the way down (2 x 2 average pooling between levels) and on the way up
 * (nearest 2x upsampling, concatenated with the way down's features of the
 * same level), then a 3 x 3 convolution to 16 channels whose first n are
 * the layers' change times out_scale / s. Every sample is normalised by the
 * RMS s of its deviations h_i - mean h_i over all its layers (a flat
 * sample, s = 0, does not change). Input planes (16): (h_i - mean h_i)
 * in_scale / s, then the n_extra problem parameters as constant planes,
 * then zeros. The change is made mean-free per layer, so every prediction
 * keeps each layer's mass, as the LBM does.
 * Arithmetic: BF16 activations and weights, FP32 accumulation in tensor
 * memory (tcgen05.mma, operands staged by TMA), FP32 master weights and
 * Adam moments. Arrays are device memory, [batch][n][ny][nx] FP32 unless
 * stated; work is enqueued on the stream given at create.
 * ------------------------------------------------------------------- */
typedef struct mlswlbm_unet mlswlbm_unet;

/* Number of FP32 parameters: for each of the 15 convolutions in order,
 * its weights [out][tap][in] (tap = 3 (dy + 1) + (dx + 1)), then its bias. */
long mlswlbm_unet_param_count(void);

/* Creates a network for n_layers (1..MLSW_MAX_LAYERS) on nx x ny lattices
 * (powers of two from 128 to 4096) and batches of up to max_batch samples;
 * extra: n_extra values (host; n_layers + n_extra <= 16) for the parameter
 * planes. He-normal weights from a generator seeded with `seed`, zero
 * biases. Errors: MLSW_ERR_ARG, MLSW_ERR_UNSUPPORTED (lattice size),
 * MLSW_ERR_NOMEM, MLSW_ERR_CUDA; *out is NULL on failure. */
int mlswlbm_unet_create(int n_layers, int nx, int ny, int max_batch, int n_extra,
                        const double* extra, unsigned long long seed, double in_scale,
                        double out_scale, void* stream, mlswlbm_unet** out);

/* out = h + the predicted, mass-projected change over 64 steps, for
 * `batch` samples (device arrays; out may not alias h). Asynchronous. */
int mlswlbm_unet_predict(mlswlbm_unet* u, const float* h, float* out, int batch);

/* One Adam step (learning rate lr, betas 0.9 / 0.999, eps 1e-8) on the mean
 * squared error between the first n output channels and
 * (target - h) out_scale / s; *loss (optional, host) receives that error
 * before the step, and the call then synchronises. */
int mlswlbm_unet_train_step(mlswlbm_unet* u, const float* h, const float* target, int batch,
                            double lr, double* loss);

/* MLSW_ERR_TIMEOUT if a bounded wait of a tensor-core kernel ran out since
 * create, else MLSW_OK. Synchronises. */
int mlswlbm_unet_status(mlswlbm_unet* u);

/* Parameters to / from host memory (count = mlswlbm_unet_param_count());
 * setting them resets the Adam moments. Synchronise. */
int mlswlbm_unet_set_params(mlswlbm_unet* u, const float* host, long count);
int mlswlbm_unet_get_params(mlswlbm_unet* u, float* host, long count);

/* Copies an internal array of the last pass to host memory, for tests:
 * kind 0 the activation tensor `id`, kind 1 its gradient (BF16, NHWC with a
 * one-pixel periodic halo, [max_batch][h + 2][w + 2][C]), kind 2 the
 * parameter gradients (FP32), kind 3 the network output (FP32
 * [max_batch][n][ny][nx]), kind 4 the gradient that reaches the way down's
 * features of level `id` (0..2) through the skip connection. Tensor ids:
 * X0 A0 S0 P1 A1 S1 P2 A2 S2 P3 A3 S3 U2 B2 D2 U1 B1 D1 U0 B0 D0 YG = 0..21
 * (YG: the output gradient). Synchronises. */
int mlswlbm_unet_debug(mlswlbm_unet* u, int kind, int id, void* out, long bytes);

void mlswlbm_unet_destroy(mlswlbm_unet* u);

/* The height error by which the LBM judges a surrogate window (the largest
 * height difference between the surrogate's prediction and the LBM's
 * heights after the same 64 steps from the same state): for each of
 * `count` items of `elems` FP32 values each (a and b device arrays, the
 * items contiguous, [count][elems]), out[j] = max_e |a[j][e] - b[j][e]|; a
 * NaN or infinite difference counts as +inf, so a non-finite prediction
 * fails any bound. out: device, count floats, caller-owned. Asynchronous on
 * `stream` (a cudaStream_t, or NULL). Errors: MLSW_ERR_ARG (NULL pointer,
 * count < 1 or elems < 1), MLSW_ERR_CUDA. */
int mlswlbm_max_abs_diff(const float* a, const float* b, int count, long elems, float* out,
                         void* stream);

#ifdef __cplusplus
}
#endif
#endif /* MLSWLBM_H */
