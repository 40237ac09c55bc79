/*
 * okmc.h -- C ABI of the GB300 hot path of object kinetic Monte Carlo with exact
 * FFT elastic interactions (Santos-Gueemes, Ortiz, Segurado, arXiv:2403.09158).
 *
 * One handle (okmc_grid) owns one periodic voxel grid on one GPU: the voxelised
 * eigenstrain of all defects, its stress, the defect table, the per-defect
 * coverage stencils and self-term tables, and the kinetic state.  All device
 * memory is allocated and freed by the library.  No C++ exception crosses this
 * boundary; every call returns an okmc_status and okmc_last_error() gives the
 * message of the last failure on that handle.  A handle is not thread safe: use
 * one handle per host thread (handles on different streams run concurrently).
 *
 * Units: lengths nm, stresses GPa, energies eV, frequencies 1/s, time s.
 * Symmetric tensors are stored as 6 components in the order
 * (xx, yy, zz, yz, xz, xy) -- true tensor components, so a : b counts the three
 * off-diagonal products twice.  Fields are structure-of-arrays,
 * field[c][z][y][x] with x fastest (c = component).
 * Defect positions are integers in units of a0/2 on the bcc lattice (all three
 * coordinates even or all odd), 0 <= pos[a] < 2 n[a]; the lattice parameter a0
 * equals the voxel edge h.  The parity of a position is its rasterisation class.
 */
#ifndef OKMC_H
#define OKMC_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  OKMC_OK = 0,
  OKMC_EINVAL = 1,    /* bad argument (sizes, defect records, null pointers)      */
  OKMC_ENOMEM = 2,    /* device allocation failed or exceeded hbm_budget          */
  OKMC_ECUDA = 3,     /* a CUDA runtime call or kernel launch failed              */
  OKMC_ETIMEOUT = 4,  /* a bounded device-side wait gave up                       */
  OKMC_ESTATE = 5,    /* call out of order (e.g. energies before set_defects)     */
  OKMC_ERANGE = 6     /* a value left the representable range (eigenstrain sum)  */
} okmc_status;

enum { OKMC_LOOP_111 = 0, OKMC_LOOP_100 = 1, OKMC_SIA_CLUSTER = 2 };
enum { OKMC_IMMOBILE = 0, OKMC_ONE_D = 1, OKMC_THREE_D = 2 };
enum { OKMC_MEAN_STRESS_ZERO = 0, OKMC_MEAN_STRAIN_ZERO = 1 };
enum { OKMC_FP32_FIELDS = 0, OKMC_FP64_FIELDS = 1 };
enum { OKMC_RESIDENCE = 0, OKMC_FIXED_DT = 1 };

typedef struct okmc_grid okmc_grid;

/* Grid description.  n[a]: edges; each a multiple of 16 of the form 2^p 3^q 5^r,
 * 16 <= n[a] <= 512.  voxel_nm: voxel edge h (= a0).  C11, C12, C44: cubic
 * stiffness in GPa along the grid axes (an isotropic solid passes
 * C44 = (C11 - C12)/2).  k0_mode: OKMC_MEAN_STRESS_ZERO (the stress has zero
 * mean) or OKMC_MEAN_STRAIN_ZERO (the strain has zero mean, Appendix B).
 * precision: OKMC_FP32_FIELDS (FP32 transforms, FP64 energies) or
 * OKMC_FP64_FIELDS (FP64 everywhere).  nu0: attempt frequency (Eq.
 * unbiased_boltzmann; 0 selects 1e13 1/s).  seed: Philox4x32-10 key.
 * stream: cudaStream_t to run on (NULL = the legacy default stream).
 * hbm_budget: upper bound on the handle's device bytes (0 = no bound). */
typedef struct {
  int32_t n[3];
  int32_t k0_mode;
  int32_t precision;
  int32_t reserved;
  double voxel_nm;
  double C11, C12, C44;
  double nu0;
  uint64_t seed;
  void* stream;
  size_t hbm_budget;
} okmc_grid_desc;

/* One defect (48 bytes).  type: OKMC_LOOP_111 (prismatic interstitial loop with
 * b = (a0/2)<111>, normal n = b/|b|), OKMC_LOOP_100 (b = a0<100>), or
 * OKMC_SIA_CLUSTER (size self-interstitial atoms, relaxation volume 1.5 Omega
 * per atom).  axis: index into {[111],[-111],[1-11],[11-1]} (loops 111 and SIA
 * clusters) or {[100],[010],[001]} (loops 100); a 1D migrant jumps +-(a0/2)*axis.
 * radius_nm: loop radius (ignored for SIA clusters).  Em_eV: migration barrier.
 * mobility: OKMC_IMMOBILE, OKMC_ONE_D (needs a <111> axis) or OKMC_THREE_D (all
 * eight (a0/2)<111> jumps).  reserved must be 0. */
typedef struct {
  int32_t type;
  int32_t pos[3];
  int32_t axis;
  int32_t size;
  int32_t mobility;
  int32_t reserved;
  double radius_nm;
  double Em_eV;
} okmc_defect;

/* Step parameters.  T_K: temperature.  mode: OKMC_RESIDENCE (one event per
 * step on the frequency line of every allowed jump of every defect; clock
 * advance -ln(u)/R_tot) or OKMC_FIXED_DT (Algorithm 1: delta t = 1/nu_max with
 * nominal barriers, Poisson event counts, one jump per defect that fires, all
 * decisions from the start-of-step field).  t_end: if > 0, okmc_step stops
 * early once the clock reaches it. */
typedef struct {
  double T_K;
  int32_t mode;
  int32_t reserved;
  double t_end;
} okmc_step_params;

/* Cumulative kinetic statistics of a handle since okmc_set_defects. */
typedef struct {
  int64_t events;             /* executed jumps                                  */
  int64_t steps;              /* okmc_step iterations                            */
  int64_t solves;             /* stress solves                                   */
  int64_t negative_barriers;  /* jumps whose E_m + dE/2 was < 0 (not clamped)     */
  double clock;               /* simulated time, s                               */
  double dt_last;             /* last time increment, s                          */
} okmc_step_stats;

/* Create a grid handle and allocate its device memory.  Errors: EINVAL (sizes,
 * constants, k0_mode, precision), ENOMEM (allocation or budget), ECUDA. */
int okmc_grid_create(const okmc_grid_desc* d, okmc_grid** out);

/* Free everything the handle owns; NULL is accepted. */
int okmc_grid_destroy(okmc_grid* g);

/* Message of the last failing call on g (static text for g == NULL). */
const char* okmc_last_error(const okmc_grid* g);

/* Change the stream later work runs on (cudaStream_t; NULL = legacy stream). */
int okmc_set_stream(okmc_grid* g, void* stream);

/* Replace the defect set (host array, copied).  Builds the coverage stencils of
 * every defect for both rasterisation classes (Sec. 3.1 eigenstrains on the
 * Sec. 3.4 voxel grid), the self-term tables W (the energy of a defect's own
 * eigenstrain at its current site or after a jump, against its own field), and
 * the voxelised eigenstrain.  Resets the step counter and the statistics.
 * Errors: EINVAL (type, axis, mobility, parity, radius, stencil larger than
 * half the grid), ENOMEM, ECUDA. */
int okmc_set_defects(okmc_grid* g, const okmc_defect* defs, int32_t n);

/* Immobile dislocation lines as eigenstrain, by static field dislocation mechanics
 * (Sec. 2.2: Eqs. curlUe, Nye2, eq_EIG_fourier, plastic_0).  On the device: the Nye
 * tensor alpha_ij = b_i t_j ds / h^3 of every sub-segment (each segment cut into
 * ceil(L / ds_max) equal parts) spread to the 8 voxel centres (i + 1/2) h around the
 * sub-segment's midpoint with trilinear weights; the incompatible plastic distortion
 * U_ij = -i xi_k / |xi|^2 eps_jkl alpha_il at xi != 0; at xi = 0 the compatible part
 * sum over closed lines of (b (x) A + A (x) b) / (2 V), with A = -1/2 sum x_a x x_{a+1}
 * (a closed line runs clockwise seen from the tip of its oriented area); the symmetric
 * part, rounded to the grid's eigenstrain quantum, is kept as a background to which the
 * defects' eigenstrain is added from then on (okmc_set_defects keeps it; the stress,
 * the energies and the kinetics see the lines' field; the lines do not move).  On a
 * Nyquist plane the operator is averaged over the sign of the Nyquist component.
 * points: double[sum counts][3], vertices in nm, the lines one after another (host).
 * counts[n_lines]: vertices per line (>= 2; >= 3 when closed).  closed[n_lines]: 1 for
 * a loop (its last vertex joins its first), 0 for an open line (an open line whose
 * last vertex is a lattice translate of its first is one period of an infinite line;
 * a net Burgers vector drops out with the xi = 0 term).  burgers: double[n_lines][3]
 * in nm.  ds_max_nm: largest sub-segment length (<= 0 selects h/4).  n_lines = 0
 * removes the background.  Temporary device memory: 9 N int64 and a nine-component
 * half spectrum.  Errors: EINVAL (counts, closed flags, non-finite or coincident
 * vertices, too many sub-segments), ENOMEM, ERANGE (the plastic strain leaves the
 * fixed-point range), ECUDA; on error the background is removed. */
int okmc_set_dislocations(okmc_grid* g, const double* points, const int32_t* counts, const int32_t* closed,
                          const double* burgers, int32_t n_lines, double ds_max_nm);

/* Copy the current defect records (positions included) to host memory. */
int okmc_get_defects(okmc_grid* g, okmc_defect* out, int32_t n);

/* Positions as int32[n][3].  set: the field is updated incrementally for the
 * defects whose position changed (parity must be kept consistent per defect).
 * on_device != 0 means the pointer is device memory. */
int okmc_set_positions(okmc_grid* g, const int32_t* pos, int32_t n, int on_device);
int okmc_get_positions(okmc_grid* g, int32_t* pos, int32_t n, int on_device);

/* Periodic elastic solve (Sec. 3.2 Eqs. EIG_elastic_fourier, basicgammacomplete,
 * summaryEL, on the discrete frequencies of Sec. 3.4): forward 3D R2C transform
 * of the six eigenstrain components, Green operator per frequency, inverse C2R.
 * sigma_out (nullable): 6*nx*ny*nz values, float for FP32 fields and double for
 * FP64 fields, layout [c][z][y][x]; out_on_device says where it lives.  The
 * stress stays resident for the energy calls. */
int okmc_solve_stress(okmc_grid* g, void* sigma_out, int out_on_device);

/* The voxelised eigenstrain eps* (6*nx*ny*nz, same type and layout as sigma). */
int okmc_eigenstrain(okmc_grid* g, void* eps_out, int out_on_device);

/* Interaction energy of each defect at its site (Eq. interaction_energy3 in the
 * form E_i = -int eps*_i : (sigma - sigma_i) dV): E[n] in eV (FP64).  Solves
 * first if the stress is stale. */
int okmc_interaction_energies(okmc_grid* g, double* E, int out_on_device);

/* The same energy after each of the eight jumps lambda_j = (a0/2)(sx,sy,sz),
 * j = 4(sx>0) + 2(sy>0) + (sz>0): E[n][8] (FP64).  valid[n][8] (nullable)
 * marks the jumps the defect's mobility allows (Sec. 5). */
int okmc_candidate_energies(okmc_grid* g, double* E, uint8_t* valid, int out_on_device);

/* Dipole approximation of the same energies (Sec. 2.1, Eq. interaction_energy4 with
 * the dipole tensor P = C : int eps* of Eq. dipole_def2): the external field is taken
 * constant over the defect, E_i(Y) = -P_i : eps_ext(Y) = -(int eps*_i) : sigma^(-i)(Y),
 * sigma^(-i) = sigma - sigma_i read at the defect's centre (the base voxel of a class-1
 * site, the mean of the 8 voxels around the corner of a class-0 site).  E[n] at the
 * sites, Ec[n][8] (nullable) after the eight jumps (order as above), eV (FP64).
 * Solves first if the stress is stale.  Same ownership and errors as
 * okmc_interaction_energies. */
int okmc_dipole_energies(okmc_grid* g, double* E, double* Ec, int out_on_device);

/* Point defects of given dipole tensor in the grid's current field (Sec. 2.1, Eq.
 * interaction_energy4; Table 1 gives the <110> dumbbell self-interstitial's):
 * E[k] = -P_k : eps(Y_k), eps = C^-1 : sigma read at the centre of site Y_k (the rule
 * of okmc_dipole_energies).  The probes are not part of the grid: they feel every
 * defect and dislocation line and change nothing.  pos: int32[m][3] bcc sites (units
 * of a0/2, 0 <= pos[a] < 2 n[a], all even or all odd); P: double[m][6] in eV, order
 * (xx, yy, zz, yz, xz, xy); E: double[m] in eV.  on_device != 0: all three pointers are
 * device memory (a bad site then gives NaN in E and OKMC_EINVAL).  Solves first if the
 * stress is stale.  Errors: EINVAL (null pointers, m < 0, sites, non-finite P), ENOMEM,
 * ECUDA. */
int okmc_point_dipole_energies(okmc_grid* g, const int32_t* pos, const double* P, int32_t m, double* E, int on_device);

/* The paper's evaluation at continuous positions (Sec. 3.3, Eq. shift; Eq.
 * interaction_energy3 in its elastic-strain form): the interaction energy of defect i if
 * it sat at X_k instead of its site, E[k] = kappa int sigma^(-i) : eps^e_i(. - X_k) dV.
 * eps^e_i is the elastic strain C^-1 : sigma of defect i alone with its class-0 stencil
 * placed at the origin (centre X0 = 0), moved to X_k by exp(-i xi.X_k) and summed by
 * Parseval over the discrete frequencies; sigma^(-i) is the stress of everything on the
 * grid (defects and dislocation lines) except defect i at its current site.  At a
 * whole-voxel move of a class-0 defect this is its stencil energy there (up to the
 * Nyquist terms of even edges); between lattice sites it is the band-limited reading of
 * an off-lattice defect.  X: double[m][3] in nm (any finite values; periodic);
 * E: double[m] in eV.  on_device != 0: X and E are device memory.  Cost: two forward
 * transforms and one pass over the half spectrum per 8 positions, with temporary
 * device memory for 8 spectrum components and 2 fixed-point fields.  Errors: EINVAL
 * (i out of range, m < 0, null or non-finite X), ENOMEM, ECUDA. */
int okmc_shift_energies(okmc_grid* g, int32_t i, const double* X, int32_t m, double* E, int on_device);

/* Self part of the dipole energies, D[n][2][9] in GPa nm^3 (FP64): D[i][c][k] =
 * (int eps*_i) : sigma_i(Y_k), defect i's own field at the centre of a class-c site
 * (k = 0) or of its jump k - 1; the dipole energy is -kappa ((int eps*_i) : sigma(Y) -
 * D).  Translation invariant, summed in Fourier space with the self-term table. */
int okmc_dipole_self_terms(okmc_grid* g, double* D, int out_on_device);

/* Self-term table W[n][2][9] in eV (FP64): W[i][c][0] is the self energy of
 * defect i's eigenstrain at a class-c site against its own periodic field,
 * W[i][c][1+j] the same after jump j.  Translation invariant. */
int okmc_self_terms(okmc_grid* g, double* W, int out_on_device);

/* Coverage stencil of defect i, class c: k entries of (dx, dy, dz) voxel offsets
 * from the base voxel floor(pos/2) and subsample counts 1..64, sorted by
 * (dz, dy, dx); the voxel weight is count*alpha.  Pass capacity 0 to query k.
 * offs: int32[k][3], counts: int32[k] (host). */
int okmc_get_stencil(okmc_grid* g, int32_t i, int32_t c, int32_t* offs, int32_t* counts,
                     int32_t capacity, int32_t* k, double* alpha);

/* Run n_steps kinetic steps (Sec. 5, Algorithm 1), each: solve if stale,
 * energies at the sites and after every jump, rates (Eqs.
 * biased_forward/backward_boltzmann with prefactor 1/z over the z allowed jumps),
 * selection on the frequency line (Eqs. frequency_line, selection_jump),
 * position update and incremental eigenstrain update.  Uniforms come from
 * Philox4x32-10 with key = seed and counter = (step, defect or 0xFFFFFFFF, mode).
 * out (nullable, host): the cumulative statistics after the last step. */
int okmc_step(okmc_grid* g, const okmc_step_params* p, int64_t n_steps, okmc_step_stats* out);

/* Cumulative statistics (host). */
int okmc_get_stats(okmc_grid* g, okmc_step_stats* out);

/* Restores the kinetic state (clock, step counter, events, negative-barrier count,
 * last time step, solve count) saved by okmc_get_stats, e.g. after re-creating a
 * handle from defects saved with okmc_get_defects: the step counter drives the
 * Philox counters, so the trajectory then continues exactly as it would have.
 * s is read (host); OKMC_EINVAL for negative counts or non-finite times. */
int okmc_set_kinetic_state(okmc_grid* g, const okmc_step_stats* s);

/* okmc_step replays a captured CUDA graph of one step (solve, energies and rates,
 * event, incremental field update), one graph per (mode, T), captured on first use
 * and dropped by okmc_set_defects.  enable = 0 launches kernel by kernel instead
 * (kernel timing, see okmc_set_profiling, always does). */
int okmc_set_graphs(okmc_grid* g, int enable);

/* Batches: many independent replicas (handles of any grid size and defect count on
 * the same GPU) advanced together, one CUDA graph launch per step on the batch stream.
 * Two forms of that graph:
 *   OKMC_BATCH_KERNELS: one persistent kernel per stage of the step (forward plane
 *     pass, pencil pass, inverse plane pass, energies and rates, event, field update),
 *     each walking a device work list of (replica, plane / tile / defect) items of
 *     every replica, whatever its edge; six launches per step for the whole batch.
 *     Needs FP32-field replicas with nx = ny and edges in {64, 96, 128, 160, 192, 256}.
 *   OKMC_BATCH_GRAPHS: every replica's own step as an independent branch of the graph
 *     (fork/join over private streams), so the replicas' kernels overlap.
 * OKMC_BATCH_AUTO (the default) takes the kernels when every replica qualifies, else
 * the branches.  params[n] and stats[n] (nullable) are per replica; t_end must be 0.
 * The graph is rebuilt when a replica's mode or temperature changes, after
 * okmc_set_defects on a replica, or after okmc_batch_set_mode.  The handles stay
 * owned by the caller and must outlive the batch; their own streams are synchronised
 * before the batch runs.  Results are those of okmc_step on each handle alone, bit for
 * bit, in either form. */
typedef struct okmc_batch okmc_batch;
enum { OKMC_BATCH_AUTO = 0, OKMC_BATCH_KERNELS = 1, OKMC_BATCH_GRAPHS = 2 };
int okmc_batch_create(okmc_grid* const* grids, int32_t n, void* stream, okmc_batch** out);
int okmc_batch_step(okmc_batch* b, const okmc_step_params* params, int64_t n_steps, okmc_step_stats* stats);
/* Chooses the form (OKMC_BATCH_*); OKMC_BATCH_KERNELS on a batch with a replica that
 * does not qualify makes the next okmc_batch_step fail with OKMC_EINVAL.
 * okmc_batch_get_mode reports the form the last step used (0 before the first). */
int okmc_batch_set_mode(okmc_batch* b, int32_t mode);
int okmc_batch_get_mode(const okmc_batch* b, int32_t* mode);
int okmc_batch_destroy(okmc_batch* b);
const char* okmc_batch_last_error(const okmc_batch* b);

/* Cubic constants of an isotropic solid, for okmc_grid_desc: C[0] = C11 =
 * lambda + 2 mu, C[1] = C12 = lambda, C[2] = C44 = mu, with the Lame constant
 * lambda = 2 mu nu / (1 - 2 nu) (so C44 = (C11 - C12)/2).  mu_GPa > 0 and
 * -1 < nu < 1/2, else OKMC_EINVAL.  Host only; C (host, 3 doubles) is written. */
int okmc_isotropic_stiffness(double mu_GPa, double nu, double C[3]);

/* Device bytes held by the handle. */
size_t okmc_device_bytes(const okmc_grid* g);

/* Device bytes okmc_grid_create allocates for a description (fields, spectra and
 * tables; defect data come on top with okmc_set_defects); 0 for a bad description. */
size_t okmc_estimate_field_bytes(const okmc_grid_desc* d);

/* Kernel timing: when enabled, every kernel launch of the handle is bracketed
 * with CUDA events on the handle's stream and its time is accumulated per
 * kernel name.  okmc_kernel_times fills up to cap entries (names point to static
 * strings, ms = total milliseconds, count = launches) and returns how many
 * kernels were seen; okmc_reset_kernel_times clears the totals. */
int okmc_set_profiling(okmc_grid* g, int enable);
int okmc_kernel_times(okmc_grid* g, const char** names, double* ms, int64_t* count, int cap);
int okmc_reset_kernel_times(okmc_grid* g);

/* Number of CTAs in each launch of the pass kernels and the cluster size the
 * handle picked for its grid (diagnostics): out[0..2] = cluster size of the
 * forward plane pass, CTAs of the pencil pass, cluster size of the inverse pass.
 * out[0] = out[2] = -1 when the grid runs the register-FFT passes (FP32 fields,
 * nx = ny and nx, nz in {32, 48, 64, 96, 128, 160, 192, 256, 320}). */
int okmc_launch_shape(const okmc_grid* g, int32_t out[3]);

/* Launch variants of the three FFT passes (forward plane pass = 0, pencil pass = 1,
 * inverse plane pass = 2), for diagnostics and tests.  okmc_grid_create times every
 * variant that exists for the grid's shape (three interleaved rounds, best of each)
 * and keeps variant 0 unless another is more than 2% faster.  The picks are kept per
 * grid shape for the life of the process and in a JSON file keyed by device name, SM
 * count, grid shape and variant schema: $OKMC_TUNE_CACHE (set and empty: no file),
 * else $XDG_CACHE_HOME/okmc/tune.json or ~/.cache/okmc/tune.json; a shape found there
 * is not timed again.  OKMC_TUNE=0 keeps variant 0 without timing (e.g. under a
 * profiler) and OKMC_VARIANTS=a,b,c pins variants a, b and c of the three passes, each
 * where it exists.  The variants differ in cluster size, threads per CTA and how data
 * reaches shared memory, not in arithmetic, so results are bitwise the same under
 * every variant.  Pencil variants: 0 swizzled tile by 16-byte asynchronous copies,
 * 1 padded tile by 8-byte copies, 2 swizzled tile by TMA box copies onto an mbarrier
 * (present when the driver encodes the spectra's tensor maps).  Variant 2 waits for its
 * copies for at most 0.5 s: a CTA whose copies have not arrived by then sets the
 * device error word and returns, and the next call that synchronises with the host
 * (okmc_solve_stress with a host output, okmc_get_stats, okmc_step) returns
 * OKMC_ETIMEOUT; the grid then stays failed, the context usable.
 * okmc_get_variants: current[p] = variant in use, available[p] = bit mask of the
 * variants that exist.  okmc_set_variant: OKMC_EINVAL if the variant does not exist
 * for this grid; drops captured step graphs. */
int okmc_get_variants(const okmc_grid* g, int32_t current[3], int32_t available[3]);
int okmc_set_variant(okmc_grid* g, int32_t pass, int32_t variant);

/* ---------------------------------------------------------------- serving
 * Request server over resident replicas (the paper runs one simulation at a time;
 * this is the library's serving loop: continuous batching of solve and step
 * requests for many independent replicas on one GPU).
 *
 * okmc_server_create starts `lanes` worker threads, each with its own non-blocking
 * CUDA stream on the device current at the call; a lane takes the oldest runnable
 * request, runs it on its stream and waits for it, so requests for different
 * replicas overlap on the device.  Replicas are registered with a grid description
 * and defects (both copied; the description's stream and hbm_budget are ignored)
 * and become resident (a live handle) at the first request that needs them.
 * Requests for one replica run in submission order, one at a time.  Admission: a
 * replica becomes resident only while the device bytes of all resident replicas
 * stay within hbm_budget (0 = no limit); idle replicas are evicted least recently
 * used first to make room, their defects and kinetic state kept on the host and
 * restored on re-admission, so every replica's trajectory is the one it would
 * follow alone.  While the oldest request that needs memory waits, no other replica
 * is admitted ahead of it.
 *
 * Requests: OKMC_REQ_SOLVE computes the stress and the site energies (energies:
 * host array of the replica's defect count, required); OKMC_REQ_STEP runs n_events
 * steps with params (positions: nullable host array of 3 x defect count, filled
 * after the steps).  The arrays must stay valid until the request completes.
 * okmc_server_wait returns the result of a ticket once (timeout_ms < 0 waits
 * without limit; OKMC_ETIMEOUT if not done in time); times are seconds since
 * okmc_server_create on the host's steady clock.  okmc_server_destroy stops the
 * lanes after their current request (queued requests are dropped) and frees every
 * replica; no other call on the server may be in progress. */
typedef struct okmc_server okmc_server;

typedef struct {
  size_t hbm_budget;  /* bytes the resident replicas may hold, 0 = no limit */
  int32_t lanes;      /* worker threads and streams, 1..64 */
  int32_t reserved;   /* must be 0 */
} okmc_server_desc;

enum okmc_request_kind { OKMC_REQ_SOLVE = 0, OKMC_REQ_STEP = 1 };

typedef struct {
  int32_t replica;          /* id from okmc_server_add_replica */
  int32_t kind;             /* okmc_request_kind */
  int64_t n_events;         /* STEP: number of steps */
  okmc_step_params params;  /* STEP: temperature, mode, t_end */
  double* energies;         /* SOLVE: host, defect count */
  int32_t* positions;       /* STEP: host, 3 x defect count, nullable */
} okmc_request;

typedef struct {
  int32_t status;           /* OKMC_OK or the error of the failing call */
  int32_t admitted;         /* 1 if this request made its replica resident */
  double t_submit, t_start, t_end;
  okmc_step_stats stats;    /* the replica's statistics after the request */
} okmc_result;

typedef struct {
  int64_t submitted, completed, failed, admissions, evictions, resident, queued;
  size_t device_bytes;      /* bytes held or reserved by resident replicas */
} okmc_server_stats;

int okmc_server_create(const okmc_server_desc* d, okmc_server** out);
int okmc_server_add_replica(okmc_server* s, const okmc_grid_desc* d, const okmc_defect* defs, int32_t nd, int32_t* id);
int okmc_server_submit(okmc_server* s, const okmc_request* r, uint64_t* ticket);
int okmc_server_wait(okmc_server* s, uint64_t ticket, int32_t timeout_ms, okmc_result* out);
int okmc_server_get_stats(okmc_server* s, okmc_server_stats* out);
const char* okmc_server_last_error(const okmc_server* s);
int okmc_server_destroy(okmc_server* s);

/* Allocation-free stress solve (the paper has no counterpart; this is a service for
 * callers that cannot allocate device memory -- code that runs after its process
 * has handed all device memory to a pool it does not own, code inside a region
 * where allocation would synchronise the device or break a caller-owned memory
 * plan, or embedded callers whose allocator forbids cudaMalloc after start-up).
 * It does what okmc_solve_stress does for a grid, from an eigenstrain field the
 * caller provides: eps and sigma are device pointers to 6*nx*ny*nz floats each,
 * layout [c][z][y][x], both owned by the caller and 8-byte aligned (rows are read
 * and written as float pairs; a misaligned pointer returns OKMC_EINVAL before any
 * launch); n = {nx, ny, nz} as for
 * okmc_grid_create; C11, C12, C44 in GPa; k0_mode as in okmc_grid_desc; stream is
 * a cudaStream_t (NULL = legacy stream).  It allocates nothing: the half spectrum
 * and twiddle tables live in one static device array of 6.5 MB (room for
 * 6*(nx/2+1)*ny*nz <= 6*33*64*64 complex values, e.g. 64^3 voxels) that every GPU
 * loading this library keeps until the process exits.  Larger grids return
 * OKMC_EINVAL.  The first call on a device looks up the array's device address
 * (with that device current), so make that first call outside any stream capture;
 * that lookup is done once per device under a lock, so first calls from several
 * host threads at once are safe.
 * All calls share the array and leave their data in it: two calls whose work
 * overlaps on the GPU (different streams, different host threads) race and give
 * wrong results; serialise them.  Returns OKMC_OK, OKMC_EINVAL or OKMC_ECUDA
 * (asynchronous: launch errors only; sync the stream to see execution errors). */
int okmc_solve_stress_static(const float* eps, float* sigma, const int32_t n[3], double C11, double C12, double C44,
                             int32_t k0_mode, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* OKMC_H */
