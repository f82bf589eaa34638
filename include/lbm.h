/*
 * lbm.h -- C ABI of the GB300 D3Q27 MRT pipe-flow lattice Boltzmann library.
 *
 * Method: Magacho, Moriconi and Loureiro, "Persistence of large scale coherent
 * structures in a turbulent pipe flow through an improved lattice Boltzmann
 * approach" (arXiv 2405.12082).  One time step is the collision of Eq. (collision)
 * with the MRT operator of Eqs. (mrt), (lambda), (m*) and the sixth-order Hermite
 * equilibrium of Eq. (BoltzmannEquilibriumDistribution), the Guo forcing moments
 * of Eq. (Rmrti), and the streaming of Eq. (streaming), with bounce-back at the
 * pipe wall (Eqs. (fbc1)-(fbc2)) and periodic streamwise boundaries (Sec. II.B).
 *
 * Conventions used by every call below.
 *   Grid layout.   A field over one pipe is stored [comp][nz][ny][nx] (x fastest);
 *                  a cell (x, y, z) has flat index (z * ny + y) * nx + x.
 *   Populations.   Exchanged unshifted, in the paper's velocity order (Appendix A),
 *                  as double [27][nz][ny][nx].  On the device they are stored
 *                  shifted by the rest weights, f_i - w_i, in the chosen precision.
 *   Acceleration.  The body force F of Eq. (macroscopic_u) is taken as an
 *                  acceleration g: u = sum_i c_i f_i / rho + g / 2.
 *   Pointers.      Caller buffers may be host or device memory; the library asks
 *                  the CUDA runtime which.  A call that writes into host memory
 *                  synchronises the context's stream before returning; a call that
 *                  only touches device memory is asynchronous on that stream.
 *                  The caller keeps ownership of every buffer it passes.
 *   Errors.        Every call except lbm_free returns LBM_OK (0) or a negative
 *                  status below; lbm_last_error gives the reason.  No call aborts,
 *                  traps or waits without bound.
 */
#ifndef LBM_H
#define LBM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ------------------------------------------------------------ */
#define LBM_OK            0
#define LBM_EINVAL       -1   /* an argument is out of range or inconsistent       */
#define LBM_ENOMEM       -2   /* a device or host allocation failed                */
#define LBM_ECUDA        -3   /* a CUDA runtime call or a kernel launch failed     */
#define LBM_EUNSTABLE    -4   /* non-finite populations or mass drift detected     */
#define LBM_ETIMEOUT     -5   /* a bounded device-side wait expired                */
#define LBM_EUNSUPPORTED -6   /* valid request this build or state cannot serve    */

/* ---- storage precision of the populations (collision runs in FP32 for all but F64) */
#define LBM_F64   0   /* double storage, double collision                            */
#define LBM_F32   1   /* float storage of f - w, float collision                     */
#define LBM_F16S  2   /* IEEE half of (f - w) * 2^s, float collision                 */
#define LBM_BF16  3   /* bfloat16 of f - w, float collision                          */

/* ---- geometry ------------------------------------------------------------------- */
#define LBM_PIPE  0   /* circular pipe along z, axis at ((nx-1)/2, (ny-1)/2); a cell is
                         fluid iff its distance to the axis is < R; periodic in z       */
#define LBM_BOX   1   /* fully periodic box, every cell fluid (R unused)              */

/* ---- wall treatment (Sec. II.A) ------------------------------------------------- */
#define LBM_HALFWAY 0 /* half-way bounce-back: Eqs. (fbc1)-(fbc2) at Delta = 1/2      */
#define LBM_FULLWAY 1 /* full-way bounce-back: solid cells reverse their populations  */
#define LBM_BOUZIDI 2 /* Eqs. (fbc1)-(fbc2) with the exact wall distance Delta        */

/* ---- initial velocity profiles ---------------------------------------------------- */
#define LBM_REST    0 /* u = 0                                                         */
#define LBM_LAMINAR 1 /* Hagen-Poiseuille u_z = g_z (R^2 - r^2) / (4 nu)              */
#define LBM_LOGLAW  2 /* Sec. II.B mean profile U+ = delta+ (delta+ <= 10.8), else
                         ln(delta+) / 0.4 + 5, with u* = sqrt(g_z R / 2)               */

/* ---- objectives of the adjoint ---------------------------------------------------- */
#define LBM_J_UBULK 0 /* J = (1/T) sum_t (1/N_fluid) sum_x u_z(x, t)                  */
#define LBM_J_WSS   1 /* J = (1/T) sum_t tau_w(t), axial momentum exchanged with the
                         wall per step divided by the wall area 2 pi R nz              */

#define LBM_MAX_TRIGGER_MODES 8
#define LBM_MAX_MEMBERS       64

typedef struct lbm_ctx lbm_ctx;

/* Grid of one pipe.  nx, ny, nz >= 1 (a pipe also needs nx, ny >= 3).  A pipe must
 * leave at least one solid cell between the fluid and the box edge in x and y.
 * f16_log2_scale: exponent s of the LBM_F16S scale 2^s (0 selects 16; 1..24 valid). */
typedef struct {
    int32_t nx, ny, nz;
    int32_t geometry;       /* LBM_PIPE | LBM_BOX                                   */
    double  R;              /* pipe radius in lattice units (LBM_PIPE)               */
    int32_t precision;      /* LBM_F64 | LBM_F32 | LBM_F16S | LBM_BF16               */
    int32_t wall;           /* LBM_HALFWAY | LBM_FULLWAY | LBM_BOUZIDI               */
    int32_t f16_log2_scale;
} lbm_grid;

/* Relaxation matrix.  rates == NULL: Lambda of Eq. (lambda), diag[1,1,1,1, omega x5,
 * 1 x18] (or omega I under lbm_set_collision's LBM_BGK), with omega = 1/tau =
 * (nu / c_s^2 + 1/2)^{-1}, 0 < omega < 2.  rates != NULL: 27 rates lambda_k in [0, 2], Lambda =
 * diag(rates) in Eq. (m*), in the moment order of Eq. (Mmatrix) (the library copies them;
 * the rates of the conserved moments 0..3 have no effect); omega then only sets the
 * viscosity of the LBM_LAMINAR and LBM_LOGLAW initial profiles.  A context with rates on
 * any member runs the general collision (both transforms of Eq. (m*) per cell, the
 * equilibrium chosen by lbm_set_collision), in F32 or F64 storage only, in the default
 * launch shape, without adjoint. */
typedef struct {
    double omega;
    const double *rates;    /* NULL or 27 relaxation rates, moment order of Eq. (Mmatrix) */
} lbm_relax;

/* Acceleration g(x, t) acting on every fluid cell (Sec. II.B):
 *   g = (g[0], g[1], g[2])                                   constant part (h along z)
 *     + trigger force of Eq. (TurbForce), while trigger != 0 and t < t_end
 *     + (0, 0, gz_field[cell])                               if gz_field != NULL
 * The trigger is a sum over n_modes azimuthal modes; mode q has wavenumber
 * k_theta[q] >= 1, amplitude A0 * weight[q] and enters as cos(k_theta theta +
 * phase[q]) and sin(k_theta theta + phase[q]).  The paper's force is n_modes = 1,
 * k_theta = 2, weight = 1, phase = 0, kz = 3, A0 = 50, kappa = 0.5, l0 = 0.2 R,
 * l = 0.4 R, period = 0.052 T_LET, h = g[2].  theta = atan2(y - y_c, x - x_c), the
 * streamwise coordinate is the cell index z and L = nz.  The force is applied in
 * the band R - l0 - l <= r <= R - l0.
 * gz_field: device pointer, [nz][ny][nx] of double for LBM_F64 and of float for
 * the other precisions; caller-owned, must stay valid while steps run. */
typedef struct {
    double  g[3];
    int32_t trigger;
    int32_t n_modes;
    int32_t k_theta[LBM_MAX_TRIGGER_MODES];
    double  weight[LBM_MAX_TRIGGER_MODES];
    double  phase[LBM_MAX_TRIGGER_MODES];
    double  A0, kappa, l0, l, period, h;
    int32_t kz;
    int64_t t_end;
    const void *gz_field;
} lbm_force;

/* Cross-section ring analysis of Sec. II.C (see lbm_modes). */
typedef struct {
    int32_t n_sections;     /* sections at z_s = floor(s nz / n_sections), >= 1      */
    int32_t n_rings;        /* 1..16 rings                                           */
    double  r_over_R[16];   /* ring radius / R; the paper uses 0.78                  */
    int32_t n_theta;        /* samples per ring, 8..4096                             */
    int32_t n_modes;        /* highest mode M reported, 0 <= M < n_theta             */
} lbm_modes_cfg;

typedef struct {
    int64_t n_cells;        /* nx * ny * nz of the selected member                   */
    int64_t n_fluid;        /* fluid cells of the selected member                    */
    int64_t t;              /* completed time steps                                  */
    int64_t population_bytes; /* device bytes of the population array (all members)*/
    int32_t n_members;
    int32_t precision;
    int64_t launches;       /* kernels this context has launched so far              */
    int32_t variant;        /* launch shape of the step kernel (lbm_set_variant)     */
    int32_t step_threads;   /* threads per block of that shape                       */
    int32_t n_variants;     /* launch shapes available for this precision            */
    int32_t graph_chunk;    /* steps per captured graph, 0 = direct launches         */
    int32_t variant_odd;    /* launch shape of the odd steps (variant: the even ones) */
} lbm_info;

/* ==== life cycle ====================================================================== */

/* Creates a context holding one pipe: allocates its populations on the device
 * (owned by the library, freed by lbm_free) and sets them to rest, f = w, t = 0.
 * stream: a cudaStream_t (NULL = legacy default stream) on which every later call
 * of this context runs.  Errors: LBM_EINVAL (bad grid, omega, force),
 * LBM_EUNSUPPORTED (27 x cells of the context reach 2^32: the kernels index the
 * population array with 32-bit element offsets, about 159 M cells at most),
 * LBM_ENOMEM, LBM_ECUDA.  *out is NULL on error. */
int lbm_create(lbm_ctx **out, const lbm_grid *grid, const lbm_relax *relax,
               const lbm_force *force, void *stream);

/* Device-memory hooks for the contexts created after this call (process-wide; a
 * context keeps the hooks it was created with until lbm_free).  alloc(bytes, stream,
 * user) returns device memory of at least `bytes` bytes, 256-byte aligned, usable on
 * `stream` (the context's stream), or NULL; free(ptr, stream, user) releases it.  The
 * library synchronises the context's stream before it frees anything.  Every device
 * buffer a context owns (populations, tables, statistics, staging, graph tables, the
 * adjoint's and the autotuner's temporaries) comes from the hooks; pinned host memory
 * and events do not.  A NULL result, or one not 256-byte aligned, is reported as
 * LBM_ENOMEM by the call that needed it.  Both NULL: cudaMalloc / cudaFree (the
 * default).  Errors: LBM_EINVAL (one hook NULL, the other not).  This serves callers
 * whose device memory belongs to a pool of their own (a framework's caching allocator). */
typedef void *(*lbm_alloc_fn)(size_t bytes, void *stream, void *user);
typedef void (*lbm_free_fn)(void *ptr, void *stream, void *user);
int lbm_set_allocator(lbm_alloc_fn alloc, lbm_free_fn free_fn, void *user);

/* An ensemble of n independent pipes (1 <= n <= LBM_MAX_MEMBERS) advanced together
 * by one kernel launch per time step.  grids[k], relax[k], force[k] describe member
 * k; all members share precision and wall.  Per-member calls act on the member
 * chosen by lbm_select_member (default 0). */
int lbm_ensemble_create(lbm_ctx **out, int32_t n, const lbm_grid *grids,
                        const lbm_relax *relax, const lbm_force *force, void *stream);

/* Releases everything the context owns.  NULL-safe.  Synchronises its stream. */
void lbm_free(lbm_ctx *ctx);

/* Text of the last error of ctx (or, if ctx is NULL, of the calling thread's last
 * failed call that takes no context: lbm_create, lbm_ensemble_create,
 * lbm_set_allocator, lbm_reduce_static).  Never NULL. */
const char *lbm_last_error(const lbm_ctx *ctx);

int lbm_set_stream(lbm_ctx *ctx, void *stream);
int lbm_select_member(lbm_ctx *ctx, int32_t member);
int lbm_get_info(lbm_ctx *ctx, lbm_info *info);

/* Replace the relaxation or the force of the selected member (Eq. (lambda),
 * Sec. II.B).  Takes effect for the next step. */
int lbm_set_relax(lbm_ctx *ctx, const lbm_relax *relax);
int lbm_set_force(lbm_ctx *ctx, const lbm_force *force);

/* Collision model of every member, for ablations (default LBM_MRT, LBM_EQ_HERMITE6).
 * model LBM_MRT: Lambda of Eq. (lambda) in Eq. (m*); LBM_BGK: Lambda = omega I, the
 * single-relaxation-time operator of Eq. (srt) with the forcing term of Eq. (collision),
 * f* = f - omega (f - f^eq) + (1 - omega/2) F.  equilibrium LBM_EQ_HERMITE6: Eq.
 * (BoltzmannEquilibriumDistribution); LBM_EQ_ORDER2: its second-order truncation (the
 * "LBM-O(2)" of Sec. III.B's comparison), w rho (1 + 3 c.u + 9/2 (c.u)^2 - 3/2 u.u).
 * In every case F_i = g . grad_u f_i^eq (with the second-order equilibrium these are
 * the forcing populations of Guo et al. 2002).  The equilibrium also sets the initial
 * state written by lbm_init and lbm_init_fields.  Takes effect for the next step; drops
 * a captured graph.  Models other than (LBM_MRT, LBM_EQ_HERMITE6) run in the default
 * launch shape only (lbm_set_variant of another shape and lbm_autotune then fail with
 * LBM_EUNSUPPORTED) and have no adjoint.  Errors: LBM_EINVAL (unknown value),
 * LBM_EUNSUPPORTED (an ablation model with LBM_F16S or LBM_BF16 storage). */
#define LBM_MRT 0
#define LBM_BGK 1
#define LBM_EQ_HERMITE6 0
#define LBM_EQ_ORDER2 1
int lbm_set_collision(lbm_ctx *ctx, int32_t model, int32_t equilibrium);

/* ==== initial state ================================================================== */

/* Every member: f = f^eq(rho = 1, u_0) (Eq. (BoltzmannEquilibriumDistribution)) on
 * fluid cells, f = w elsewhere; t = 0; statistics cleared.  u_0 is the profile plus
 * noise_amp times a standard normal per cell and component drawn from SplitMix64
 * (seed + member index) with Box-Muller: normal number (3 c + k) of cell c, component
 * k, uses outputs 2(3c+k) and 2(3c+k)+1.  Errors: LBM_EINVAL. */
int lbm_init(lbm_ctx *ctx, int32_t profile, double noise_amp, uint64_t seed);

/* Selected member: f = f^eq(rho, u) on fluid cells from caller fields
 * rho [nz][ny][nx] and u [3][nz][ny][nx] (double, host or device); t = 0. */
int lbm_init_fields(lbm_ctx *ctx, const double *rho, const double *u);

/* ==== time stepping ================================================================== */

/* Enqueues n >= 0 time steps of every member (Eqs. (collision), (streaming)):
 * collision with the MRT operator, forcing, streaming with the wall rule and
 * periodic z.  Steps whose index t is a multiple of the statistics interval also
 * accumulate the statistics (lbm_stats_enable).  Asynchronous unless a stability
 * check is due (lbm_set_check), which synchronises and may return LBM_EUNSTABLE. */
int lbm_step(lbm_ctx *ctx, int64_t n);

/* Steps in CUDA graphs: from now on lbm_step replays a captured graph of `chunk`
 * steps (even, 2..4096; 0 = direct launches) whenever at least `chunk` steps remain
 * and t is even (and a multiple of the statistics interval when statistics are on);
 * the rest run as direct launches.  The graph is captured once per launch shape and
 * statistics setting; every node reads its step index and trigger phase from a
 * device table that the host refreshes before each replay, so results are
 * bit-identical to direct launches.  Allocates the tables (device + pinned host). */
int lbm_set_graph(lbm_ctx *ctx, int32_t chunk);

/* Launch shape ("variant") of the step kernel: 0 = 256 threads, registers for 4
 * blocks per SM; 1 = 256 x 3; 2 = 128 x 8; 3 = 512 x 2; for LBM_F32 also the
 * software-pipelined persistent kernel, 4 = 256 x 3 and 5 = 128 x 6 (each thread
 * copies its next cell's 27 populations into shared memory with cp.async while it
 * computes the current one); 6 = 128 x 8 with each thread taking 2 consecutive planes
 * of one in-plane position (the default for F32 storage), 7 = the same with 4 planes
 * (the default for the 16-bit formats and for LBM_BOUZIDI walls), 8 = 256 x 4, 9 = 128 x 7 and 10 = 128 x 6 with 2
 * planes; 11 and 12 = the staged persistent kernel (512 threads with 3 tiles in flight,
 * one CTA per SM; 256 threads, 3 tiles, two CTAs per SM): a tile is a group of whole
 * fluid rows of one plane, whose populations the kernel copies into shared memory with
 * bulk copies (cp.async.bulk, completing on an mbarrier) several tiles ahead, so loads
 * are in flight without holding registers; available in every storage for pipes with
 * half-way or Bouzidi walls whose rows fit its shared-memory segments.  LBM_F64 has shape
 * 0 (256 x 2) and the staged shapes.  The direct shapes (0-3, 6-10) and the staged shapes
 * give bit-identical results; the pipelined kernel is compiled separately and agrees
 * with them to rounding (the compiler may contract different multiply-adds).  Errors:
 * LBM_EINVAL (a shape not available for the storage), LBM_EUNSUPPORTED (an ablation
 * collision model is set, or a staged shape the context's walls or rows cannot use). */
int lbm_set_variant(lbm_ctx *ctx, int32_t variant);

/* Launch shapes per parity of the AA pattern: `even` for the steps with even t (own
 * slots), `odd` for the others (neighbour slots); lbm_set_variant sets both.  The defaults
 * are the fastest pair measured on GB300 (F32: 6 even, 9 odd; 16-bit formats: 7 and 9;
 * Bouzidi walls: 7 and 7; F64: 0 and 0).  Same errors as lbm_set_variant. */
int lbm_set_variants(lbm_ctx *ctx, int32_t even, int32_t odd);

/* Failure-detection tests of the staged shapes (11, 12): the next step launched directly
 * leaves the copies of staged tile `tile` (0-based, in launch order) unissued, so the CTA
 * waiting for it gives up after its bounded wait (about 2 s, then about 2 s more for its
 * copies in flight), records the expiry in the context's device status word and returns
 * without faulting; that step's results are then incomplete.  The next lbm_reduce or
 * stability check (lbm_set_check) returns LBM_ETIMEOUT and clears the word; the context
 * stays usable.  A tile beyond the last one has no effect.  Errors: LBM_EINVAL (tile < 0),
 * LBM_EUNSUPPORTED (the current shape is not staged). */
int lbm_test_expire_wait(lbm_ctx *ctx, int32_t tile);

/* Project autotuner for the launch shapes: times `steps` steps (2..10000) of every
 * shape on the context's own problem, the even and the odd steps separately, restores
 * the populations, t and statistics afterwards, selects the fastest shape for each parity
 * (lbm_set_variants) and returns the even one in *variant (lbm_get_info reports both) with
 * the mean time per step of the chosen pair (microseconds).  Synchronises; allocates one
 * temporary copy of the populations. */
int lbm_autotune(lbm_ctx *ctx, int32_t steps, int32_t *variant, double *best_us);

/* Every `every` steps (0 = never), lbm_step reduces mass and checks for
 * non-finite populations; a relative mass drift above max_mass_drift or any
 * non-finite value returns LBM_EUNSTABLE. */
int lbm_set_check(lbm_ctx *ctx, int64_t every, double max_mass_drift);

/* ==== observables ==================================================================== */

/* Eqs. (macroscopic_rho), (macroscopic_u) of the selected member at the current t:
 * rho [nz][ny][nx] and u [3][nz][ny][nx], u = sum c f / rho + g(x, t) / 2.  Element
 * type double for LBM_F64, float otherwise.  Solid cells get rho = 0, u = 0. */
int lbm_moments(lbm_ctx *ctx, void *rho, void *u);

/* Populations of the selected member at the current t, unshifted, double
 * [27][nz][ny][nx].  Solid cells of a half-way or Bouzidi wall read as w. */
int lbm_get_populations(lbm_ctx *ctx, double *f);

/* Overwrite the populations of the selected member (same layout); solid cells
 * of a half-way or Bouzidi wall are ignored. */
int lbm_set_populations(lbm_ctx *ctx, const double *f);

/* The raw device population array of the whole context (population_bytes of
 * lbm_get_info), in storage precision, in the layout of the current t.  Used to
 * save and restore a state bit-exactly. */
int lbm_get_raw(lbm_ctx *ctx, void *buf, size_t bytes);
int lbm_set_raw(lbm_ctx *ctx, const void *buf, size_t bytes);

/* Checkpoint and resume (the paper keeps snapshots, Sec. II.B; the file format is this
 * library's own): lbm_save writes the raw populations, t and the statistics
 * accumulators (if enabled) to `path`; lbm_load restores them into a context created
 * with the same grids, precision and wall (LBM_EINVAL otherwise), so that stepping on
 * gives bit-identical results.  lbm_load checks the whole header against the context
 * (layout, population bytes, statistics bytes 0 or exactly 4 doubles per cell with an
 * interval >= 1 and a count >= 0) and reads the whole file into host memory before it
 * changes anything: a mismatched, corrupt or truncated file returns LBM_EINVAL and
 * leaves the context as it was.  Both synchronise the context's stream. */
int lbm_save(lbm_ctx *ctx, const char *path);
int lbm_load(lbm_ctx *ctx, const char *path);

/* Sum over fluid cells of the selected member, in FP64: out[0] = sum (rho - 1),
 * out[1..3] = sum of momentum sum_i c_i f_i, out[4] = number of cells with a
 * non-finite population.  out is host memory; the call synchronises. */
int lbm_reduce(lbm_ctx *ctx, double *out);

/* Point statistics of Sec. III.B: from now on, every step t with t % every == 0
 * adds u_z^k (k = 1..4) of every fluid cell of every member to FP64 accumulators
 * (u_z before the collision of step t, as lbm_moments reports it).  every >= 1;
 * resets the accumulators. */
int lbm_stats_enable(lbm_ctx *ctx, int32_t every);

/* Accumulators of the selected member: acc [4][nz][ny][nx] double (sum of u_z^k),
 * and the number of samples taken. */
int lbm_stats_get(lbm_ctx *ctx, double *acc, int64_t *count);

/* Profiles of the point statistics of Sec. III.B: for every fluid cell of the selected
 * member the time mean, u_rms = <du^2>^(1/2), S3 = <du^3>/u_rms^3 and S4 = <du^4>/u_rms^4
 * of u_z (du = u_z - <u_z>_t, from the FP64 sums of lbm_stats_enable), averaged over the
 * cells whose distance to the axis falls in [b dr, (b+1) dr).  out: host [nbins][6] =
 * bin centre, cells, mean, u_rms, S3, S4.  1 <= nbins <= 1024.  Synchronises. */
int lbm_stats_profile(lbm_ctx *ctx, int32_t nbins, double dr, double *out);

/* Coherent-structure analysis of Sec. II.C for the selected member at the
 * current t: for every section s and ring j, u_z is sampled bilinearly at
 * theta_n = 2 pi n / n_theta on the circle of radius r_over_R[j] R and
 * E[s][j][m] = |sum_n u_z(theta_n) exp(-i m theta_n)|^2 / n_theta^2, m = 0..n_modes,
 * in double.  For m >= 1 E_m is proportional to the Fourier power of the
 * correlation R_uu of Eq. (newcorrelation) at Delta r = 0 (Wiener-Khinchin); the
 * dominant mode is its argmax over 1 <= m <= 10. */
int lbm_modes(lbm_ctx *ctx, const lbm_modes_cfg *cfg, double *E);

/* ==== analysis of the dominant-mode series (Sec. II.C, Sec. III.C), host functions ==== */

/* Dominant azimuthal mode k* of every section: the m in [m_lo, m_hi] with the largest
 * E[s][ring][m] (the smallest such m on a tie), E as written by lbm_modes (host memory,
 * [n_sections][n_rings][n_modes + 1]).  kstar: [n_sections]. */
int lbm_dominant_modes(const double *E, int32_t n_sections, int32_t n_rings, int32_t n_modes, int32_t ring,
                       int32_t m_lo, int32_t m_hi, int32_t *kstar);

/* Transition matrix of a mode series (Sec. III.C): over all pairs (k*(t), k*(t + lag))
 * with both values in [m_lo, m_hi], T[i][j] = P(k*(t + lag) = m_lo + i | k*(t) = m_lo + j),
 * column-stochastic (a column without visits is zero); lag = d for the series decimated
 * by d (all d phases pooled).  counts (optional): the raw pair counts, same layout. */
int lbm_transition_matrix(const int32_t *series, int64_t n, int32_t m_lo, int32_t m_hi, int32_t lag, double *T,
                          int64_t *counts);

/* Self-mode correlation of Sec. III.C: F[m - m_lo][tau] = <V_m(t) V_m(t + tau)>_t - <V_m>^2,
 * V_m(t) = 1 if k*(t) = m else 0, for tau = 0..max_lag (< n); the product is averaged
 * over the n - tau available pairs and <V_m> over the whole series. */
int lbm_mode_correlation(const int32_t *series, int64_t n, int32_t m_lo, int32_t m_hi, int32_t max_lag, double *F);

/* ==== adjoint ======================================================================== */

/* Runs T >= 1 forward steps of the selected single-pipe context from its current
 * state and returns J (objective LBM_J_UBULK or LBM_J_WSS) together with its
 * gradient with respect to the per-cell axial acceleration, dJ_dgz [nz][ny][nx]
 * (double, host or device), and to the shear rate omega (*dJ_domega).  The
 * reverse sweep recomputes the forward from checkpoints taken every
 * `checkpoint_every` steps (0 = about sqrt(T)); the steps of the last segment store
 * their moments during the forward pass and are not recomputed.  On return the
 * context holds the state after the T steps.  Needs a context with LBM_HALFWAY wall,
 * LBM_F32 or LBM_F64 precision, no trigger and the default collision model
 * (LBM_EUNSUPPORTED otherwise).  Allocates its temporaries (checkpoints, moments of
 * two segments, two adjoint fields, one per-segment gradient buffer) for the duration of
 * the call (LBM_ENOMEM).  The reverse sweep recomputes segment s - 1 on a second stream,
 * created and destroyed by the call and ordered against the context's stream by events,
 * while the backward steps of segment s run on the context's stream; dJ_dgz is summed per
 * segment in the storage's compute type and added to FP64 totals after each segment.  The
 * call synchronises the context's stream before it returns. */
int lbm_adjoint(lbm_ctx *ctx, int64_t T, int32_t objective, int64_t checkpoint_every,
                double *J, double *dJ_dgz, double *dJ_domega);

/* ==== timing =========================================================================== */

/* While enabled, every step-kernel launch is bracketed by CUDA events on the
 * context's stream; lbm_profile_read returns the summed device time (ms) and the
 * number of timed launches, then clears them.  lbm_profile_read synchronises. */
int lbm_profile_enable(lbm_ctx *ctx, int32_t on);
int lbm_profile_read(lbm_ctx *ctx, double *ms, int64_t *launches);

/* Fills the pipe's per-column fluid mask mask[ny][nx] (1 fluid, 0 solid) of the
 * selected member, exactly as the kernels decide it.  Host memory. */
int lbm_fluid_mask(lbm_ctx *ctx, uint8_t *mask);

/* ==== reduction without allocation ====================================================== */

/* The paper has no counterpart to this call; it serves callers that may not allocate
 * device memory at the moment they need the sum -- an application whose device memory
 * belongs wholly to its own pool, or a latency-critical loop that cannot afford the
 * device-wide synchronisation of cudaMalloc/cudaFree.  It computes what lbm_reduce
 * computes, from a population array the caller passes in, and allocates nothing.
 *
 * pops: device array [27][n_cells] in the storage precision `precision`, holding
 *       f_i - w_i (scaled by 2^f16_log2_scale for LBM_F16S; 0 selects 16) in the
 *       natural layout of an even time step, e.g. a copy made by lbm_get_raw at even t.
 * out:  device memory for 5 doubles: sum (f - w), the three momentum sums
 *       sum c_i (f_i - w_i) and the number of cells with a non-finite value.  For a
 *       context with half-way walls at even t, whose solid and padding slots hold
 *       zero, this equals lbm_reduce of that context.
 * The block partials live in a fixed static device array of
 * LBM_STATIC_REDUCE_MAX_BLOCKS x 5 + 8 doubles (48,704 bytes) that every GPU loading
 * the library keeps until the process exits.  The first call on a device looks up
 * the array's device address (cudaGetSymbolAddress) with that device current; make
 * that first call before any stream capture.  All calls on a device share the array
 * and each overwrites what it reads, so nothing needs clearing, but calls whose
 * kernels overlap on the GPU race: order them (one stream).  Asynchronous on
 * `stream` (a cudaStream_t, NULL = default stream).
 * Errors: LBM_EINVAL (NULL pointer, n_cells < 1 or above LBM_STATIC_REDUCE_MAX_CELLS,
 * unknown precision or scale, pops or out neither device nor managed memory),
 * LBM_ECUDA (no current device, symbol lookup or launch failure); the reason is
 * reported by lbm_last_error(NULL) in the calling thread.  Calls no cudaMalloc,
 * cudaFree or other allocating routine. */
#define LBM_STATIC_REDUCE_MAX_BLOCKS 1216
#define LBM_STATIC_REDUCE_MAX_CELLS  159072862   /* floor((2^32 - 1) / 27) */
int lbm_reduce_static(const void *pops, int32_t precision, int32_t f16_log2_scale, int64_t n_cells,
                      double *out, void *stream);

/* Measured FP32 arithmetic rate of the current device: the instruction-issue side of the
 * step's roofline (the DRAM side is the measured copy bandwidth).  Not an operation of the
 * method: a probe, used by bench.py.  Runs kernels of independent fused multiply-adds on
 * every SM (8 blocks of 256 threads per SM, 8 dependency chains per thread), first as
 * scalar FFMA, then as paired FFMA2 (two FMAs per instruction), each the best of three
 * timed launches (CUDA events on `stream`, a cudaStream_t, NULL = default stream) after
 * one untimed launch, about 30-60 ms in all.  The kernels write no memory.
 * out: HOST memory for 4 doubles: [0] scalar FP32 rate in TFLOP/s (2 flops per FMA),
 *      [1] paired rate in TFLOP/s, [2] scalar FFMA warp instructions per second per SM
 *      sub-partition (the issue rate: divide by the SM clock for instructions per
 *      cycle), [3] the scalar launch's milliseconds.
 * Synchronises `stream`; allocates nothing.  Errors: LBM_EINVAL (out NULL), LBM_ECUDA (no
 * device, event or launch failure); the reason is reported by lbm_last_error(NULL). */
int lbm_probe_fp32(double *out, void *stream);

#ifdef __cplusplus
}
#endif
#endif /* LBM_H */
