/* teuk.h -- C ABI of the GB300 Lax-Wendroff Teukolsky stepper.
 *
 * One handle holds one problem: a spin-weight-s, azimuthal-m perturbation of a Kerr black
 * hole (mass M, spin a) on an (r*, theta) grid, evolved by the two-step Lax-Wendroff
 * scheme of Ginjupalli & Khanna, "High-Precision Numerical Simulations of Rotating Black
 * Holes Accelerated by CUDA" (arXiv:1006.0663): the Teukolsky equation (Eq. 1) reduced with
 * Psi = e^{i m phi~} r^3 Phi (Eq. psiphi) to the first-order system u_t + D u_{r*} = S for
 * u = {Phi_R, Phi_I, Pi_R, Pi_I} (Sec. 3.B, Eqs. new_teu2, d_matrix), advanced by Eqs. lw1
 * and lw2, with 10th-order centred theta differences (Sec. 3.D), Phi = Pi = 0 on the r*
 * boundaries and axis parity conditions (Sec. 3.B). Arithmetic is FP64, double-double or
 * quad-double (Sec. 3.D "double, quadruple and octal precision").
 *
 * Conventions
 *  - Every call returns 0 on success or a negative TEUK_ERR_* code; teuk_strerror() gives
 *    a message, teuk_last_error() the detail of the last failure on a handle.
 *  - Host buffers are owned by the caller and are only read or written during the call
 *    (the call synchronises the handle's stream before returning host data).
 *  - Multi-word values are passed as word planes: a real in precision p (words w = p) is the
 *    exact sum of w doubles, stored plane by plane. A field array [C][w][n_r][n_theta] holds
 *    component c, word k, row i, column j at ((c*w + k)*n_r + i)*n_theta + j; the components
 *    of the state are Phi_R, Phi_I, Pi_R, Pi_I.
 *  - All double parameters are taken as exact binary values in every precision.
 *  - A handle is not thread-safe; all its work is queued on its CUDA stream in order.
 *  - No call uses more than the one CUDA device that is current when the handle is created.
 */
#ifndef TEUK_H
#define TEUK_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum { TEUK_FP64 = 1, TEUK_DD = 2, TEUK_QD = 4 } teuk_precision; /* = words per real */

enum {
  TEUK_OK = 0,
  TEUK_ERR_INVALID_ARG = -1,   /* a parameter is out of range (message in teuk_last_error) */
  TEUK_ERR_CUDA = -2,          /* a CUDA runtime call failed */
  TEUK_ERR_OOM = -3,           /* device or host allocation failed */
  TEUK_ERR_NONFINITE = -4,     /* the evolution produced Inf/NaN (instability) */
  TEUK_ERR_STATE_MISMATCH = -5,/* a state or observer request does not fit this handle */
  TEUK_ERR_NO_DEVICE = -6,     /* no CUDA device is available */
  TEUK_ERR_TIMEOUT = -7        /* a bounded wait inside a step kernel reached its limit */
};

/* Grid and time stepping (Sec. 3.B: r* nodes r*_i = rstar_min + i dr*, i = 0..n_r-1,
 * dr* = (rstar_max - rstar_min)/(n_r - 1); cell-centred theta_j = (j + 1/2) pi / n_theta).
 * dt is the outer (sampling) step; each outer step is `substeps` Lax-Wendroff iterations
 * of dt/substeps (the explicit scheme needs several iterations per dt = 0.25 dr* to stay
 * stable with 10th-order theta differences near the poles). */
typedef struct {
  double rstar_min, rstar_max;
  int32_t n_r;          /* >= 3 */
  int32_t n_theta;      /* 6 .. 1024 */
  double dt;            /* outer step; 0 selects 0.25 dr* */
  int32_t substeps;     /* >= 1, chosen by the caller: the smallest stable count comes from an
                           eigenvalue study of the discrete operator (the midpoint-rule growth
                           of the largest theta frequencies, those of the pole cells' (m + s cos
                           th)^2 / sin^2 th potential for s != 0) that is run once per problem on
                           the host; this library has no host arithmetic, so it does not pick k */
  int32_t theta_order;  /* 10 (Sec. 3.D, default if 0) or 2 (Sec. 3.B) */
  int32_t parity;       /* sign of the axis reflection of Phi and Pi: 0 selects (-1)^(m+s)
                           (regularity of the spin-weighted harmonics), 2 the paper's rule
                           (+1 for even |m|, -1 for odd, Sec. 3.B), +1 / -1 explicit */
  int32_t reserved;     /* must be 0 */
  double ko_sigma;      /* r* dissipation (teuk_set_dissipation), not in the paper: 0 = off */
  double ko_theta;      /* theta dissipation (teuk_set_theta_dissipation), not in the paper:
                           0 = off; both are applied at creation with the setters' rules */
  int32_t theta_filter; /* theta filter (teuk_set_theta_filter), not in the paper: 0 = off,
                           else l_cut; applied at creation with the setter's rules */
  int32_t theta_filter_period; /* its period in outer steps (0 = 1) */
} teuk_grid;

typedef struct teuk_s* teuk_t;

/* Creates a problem and evaluates its coefficients on the device (tortoise inversion r(r*)
 * and the system coefficients at every node and half node, in the target precision).
 * M > 0, |a| < M, stream = a cudaStream_t or NULL for a stream owned by the handle.
 * Allocates about (4 + 4 + 4*8) * w * n_r * n_theta doubles of device memory. */
int teuk_create(teuk_t* out, double M, double a, int s, int m, const teuk_grid* grid,
                teuk_precision precision, void* cuda_stream);
int teuk_destroy(teuk_t h);

/* r* slabs: one problem split along r* over several handles (the paper's decomposition of
 * the grid over processing elements, Sec. 4, applied across GPUs or streams). A slab handle
 * advances the global nodes own_lo .. own_hi (0 <= own_lo <= own_hi <= n_r - 1) of the grid
 * `grid` and holds one halo row beyond each end that lies inside the grid: local row 0 is
 * global row row0 = max(own_lo - 1, 0). Its tables are those of the global rows, so one
 * iteration gives bit for bit the values the whole-grid handle gives on the owned rows,
 * provided the halo rows hold the neighbours' rows of the same iteration. Advance with
 * teuk_substep(h, 1) (more than one iteration per call and teuk_step are refused), after
 * copying the neighbours' edge rows in: per iteration, teuk_get_halo_rows on every slab, then
 * teuk_set_halo_rows on every slab, then teuk_substep(h, 1). Array arguments of the slab
 * calls (teuk_set_initial, teuk_get_state, ...) cover its local rows; the observer must be one
 * of its owned nodes; no dissipation, batches or persistent launches. At least three local
 * rows. The caller owns the exchange and its ordering between streams. */
int teuk_create_slab(teuk_t* out, double M, double a, int s, int m, const teuk_grid* grid,
                     teuk_precision precision, void* cuda_stream, int own_lo, int own_hi);
/* The slab's first and last owned rows (global own_lo and own_hi), [4][w][n_theta] doubles
 * each, into lo_out / hi_out (device or page-locked host memory; NULL to skip), queued on the
 * handle's stream: what the neighbours below / above need as their halo rows. */
int teuk_get_halo_rows(teuk_t h, double* lo_out, double* hi_out);
/* Writes the halo rows (global own_lo - 1 from lo_in, own_hi + 1 from hi_in; same layout and
 * memory kinds; NULL to skip), queued on the handle's stream. There is no halo beyond global
 * row 0 or n_r - 1: a non-NULL pointer there is TEUK_ERR_INVALID_ARG. */
int teuk_set_halo_rows(teuk_t h, const double* lo_in, const double* hi_in);
/* Global index of local row 0 and the owned rows (a whole-grid handle: 0, 0, n_r - 1). */
int teuk_slab_rows(teuk_t h, int* row0, int* own_lo, int* own_hi);

/* Initial data from host word planes phi_pi[4][w][n_r][n_theta] (copied to the device).
 * Rows 0 and n_r-1 are set to zero (Sec. 3.B). Resets the step counter. */
int teuk_set_initial(teuk_t h, const double* phi_pi);
/* Gaussian pulse Phi = A exp(-((r* - center)/width)^2) sY_{ell m}(theta) with A = amp_re +
 * i amp_im, zero initial time derivative (Pi = b Phi_{r*}), evaluated on the device in the
 * target precision; sY is the spin-weighted harmonic without its normalisation constant.
 * max(|m|, |s|) <= ell <= 40. */
int teuk_set_initial_pulse(teuk_t h, double center, double width, double amp_re, double amp_im,
                           int ell);

/* Arithmetic engine of a double-double or quad-double handle (the paper's "quadruple" and
 * "octal" precisions, Sec. 3.D): 0 = FP64 error-free transforms (the default), 1 = integer
 * engine: every dot product of the step is formed in fixed-point mantissas (128-bit for dd,
 * 256-bit for qd) on the integer pipe and rounded once (error about 2^-105 / 2^-208 of the
 * result plus N 2^-122 / N 2^-249 of the largest of its N terms; subnormal operands count as
 * zero).
 * GB300 issues far more integer than FP64 operations per cycle. Results of the two engines
 * agree to the precision's rounding, not bit for bit; engine 1 evaluates the theta operator in
 * its factored form A2 D2 + (A1 cot theta) D1 with exact integer stencil sums. Engine 1
 * converts the coefficient tables once (nine planes: about 1.4x (dd) / 1.3x (qd) their size of
 * extra device memory) and runs the rows-per-block kernels (launch-shape variants 0..2).
 * FP64 handles accept 0 only. */
int teuk_set_engine(teuk_t h, int engine);
int teuk_engine(teuk_t h);
/* Test hook of the bounded waits (no counterpart in the paper). Integer engine: from the next
 * launch on, thread block `block` of each engine step kernel arms its copy barrier with the
 * expected byte count but issues no copy, so its wait gives up after 2^wait_log2 tries
 * (10 <= wait_log2 <= 20) with nothing in flight; the kernel then skips that block's rows and
 * teuk_sync reports TEUK_ERR_TIMEOUT. The kernels stage at least their table rows while the
 * hook is set. Persistent launches (teuk_set_persistent): block `block` never publishes its
 * progress counters, so its neighbours' waits give up after 2^wait_log2 polls, every other
 * wait ends on the abort word, and teuk_sync reports TEUK_ERR_TIMEOUT. block = -1 restores
 * normal operation. Handles on the integer engine or on persistent launches only. */
int teuk_test_stall_copies(teuk_t h, int block, int wait_log2);

/* r* dissipation. NOT part of the paper's method (sigma = 0, the default, is the paper's
 * scheme). With several Lax-Wendroff iterations per dt = 0.25 dr*, the scheme's own damping
 * of short r* wavelengths is too weak for long runs: modes of near-zero numerical group
 * velocity grow where the lower-order terms of the system (c Phi_{r*}, V/Sigma^2 Phi) make a
 * frozen wave grow. With sigma > 0, every outer step (whenever the iteration count is a
 * multiple of substeps) begins with
 *   u_i <- u_i - eps (u_{i-2} - 4 u_{i-1} + 6 u_i - 4 u_{i+1} + u_{i+2}),  eps = sigma dt / (16 dr*),
 * for all four components at rows 2 .. n_r - 3 (fourth-order Kreiss-Oliger dissipation over
 * one outer step; an O(dr*^3) change for smooth fields). 0 <= sigma <= 4. Allocates one
 * state-sized device buffer. Handles with sigma > 0 cannot join a batch or use
 * teuk_substep_noalloc. */
int teuk_set_dissipation(teuk_t h, double sigma);
/* theta dissipation. NOT part of the paper's method (sigma = 0, the default, is the paper's
 * scheme). The theta terms sit in the source S, so for them each Lax-Wendroff iteration acts
 * like the explicit midpoint rule, which amplifies every oscillation; the grid-scale theta
 * modes have the largest frequencies and set how many iterations per dt are needed. With
 * sigma > 0 the dissipation step at the start of every outer step (the one of
 * teuk_set_dissipation; both terms read the same input) also subtracts
 *   eps_th(i) (d_th^2)^6 u,   eps_th(i) = sigma c_th(i) dt / (4096 dtheta),
 *   (d_th^2)^6 u_j = sum_{q=-6..6} (-1)^q C(12, 6+q) u_{j+q} (parity ghosts at the poles),
 * c_th(i) = max_j sqrt(Delta/Sigma^2) at node i, from every component at rows 1 .. n_r - 2: the
 * 12th-order Kreiss-Oliger operator integrated over one outer step (an O(dtheta^11) change for
 * smooth fields: the 10th-order theta accuracy is kept; the grid-scale mode is multiplied by
 * 1 - sigma c_th dt / dtheta). 0 <= sigma <= 4 and sigma max_i c_th(i) dt / dtheta <= 2, else
 * TEUK_ERR_INVALID_ARG and the sigma in use is kept. Allocates one state-sized buffer and one row table; handles with it
 * cannot join a batch or use teuk_substep_noalloc. It damps grid-scale theta modes only: the
 * pole-cell modes of the (m + s cos th)^2 / sin^2 th potential and resolved multipoles are
 * left as they are. teuk_theta_dissipation returns the sigma in use. */
int teuk_set_theta_dissipation(teuk_t h, double sigma);
double teuk_theta_dissipation(teuk_t h);
/* theta filter. NOT part of the paper's method (l_cut = 0, the default, is the paper's
 * scheme). A multipole l oscillates near the photon sphere (r ~ 3M) at about
 * (l + 1/2) / (3 sqrt(3) M). Once that frequency exceeds what the central r* differences of
 * the iteration carry (they stop at 1/dr*), the grid traps the multipole there and the
 * first-order term c Phi_{r*} of the r^3-scaled system makes it grow (rates ~0.1/M on
 * r* in [-100, 400] with 1024 points from l = 7 at a = 0.99); neither substeps nor the
 * dissipation terms remove that. With l_cut > 0, every period-th outer step begins (after
 * the dissipation kernel, when there is one) by replacing every interior row of every
 * component with its projection onto the harmonics of the problem's s and m below l_cut:
 *   f_j <- sum_l sY_lm(theta_j) c_l,  c_l = sum_j' 2 pi w_j' sY_lm(theta_j') f_j',
 *   max(|s|, |m|) <= l < l_cut,
 * sY_lm normalised, w_j Fejer's first-rule weights on the cell centres; with
 * 2 (l_cut - 1) < n_theta the harmonics are exactly orthonormal in that sum, so the map is an
 * orthogonal projection. The tables are computed once, in quad-double, and kept in the run's
 * words. Rules: l_cut = 0, or max(|s|, |m|) < l_cut <= 41 and 2 (l_cut - 1) < n_theta, else
 * TEUK_ERR_INVALID_ARG (also on slabs) and the filter in use is kept. Allocates one table of
 * 2 (l_cut - max(|s|, |m|)) n_theta words and a two-word counter; handles with it cannot
 * join a batch or use teuk_substep_noalloc. The projection runs at the outer steps whose
 * index (iterations done / substeps, counted from the iteration count given with the state)
 * is a multiple of period (0 or 1: every outer step; at most 1024; the kernel runs at every
 * outer step and keeps the count on the device): the trapped multipoles grow by at most a factor
 * e^{rate period dt} between projections, so a period of about 1 M keeps them at the level
 * the projection leaves while the projection's cost (multi-word dot products on the FP64 pipe)
 * falls by the period. teuk_theta_filter / teuk_theta_filter_period return the values in use
 * (-1 for a null handle). */
int teuk_set_theta_filter(teuk_t h, int l_cut, int period);
int teuk_theta_filter(teuk_t h);
int teuk_theta_filter_period(teuk_t h);

/* Advances n outer steps (n * substeps Lax-Wendroff iterations), asynchronously on the
 * handle's stream. The observer ring (if any) gets one sample per outer step. */
int teuk_step(teuk_t h, int64_t n_outer_steps);
/* CUDA graphs: teuk_step captures one outer step (its 2 * substeps kernel launches and the
 * observer bookkeeping) as a CUDA graph on first use and replays it, which removes most of
 * the launch overhead of small problems. On by default; not used while per-kernel timing is
 * on or when the handle runs on the legacy default stream. enable = 0 launches kernels one
 * by one. Results are identical either way. */
int teuk_use_graphs(teuk_t h, int enable);
/* Advances n single Lax-Wendroff iterations of dt/substeps (no observer samples). */
int teuk_substep(teuk_t h, int64_t n_iterations);
/* Waits for the handle's stream; returns TEUK_ERR_NONFINITE if any Inf/NaN was produced, and
 * TEUK_ERR_TIMEOUT if a step kernel's wait for its own copies into shared memory reached its
 * iteration limit (the kernel then skipped its rows). Either error stays until the state is
 * replaced (teuk_set_initial, teuk_set_initial_pulse, teuk_set_state clear it). */
int teuk_sync(teuk_t h);

/* Phi at the node nearest rstar_obs (ties toward the lower index): out[2][w][n_theta]. */
int teuk_observe(teuk_t h, double rstar_obs, double* out_phi, double* rstar_used);
/* Records Phi(i_obs, .) after every outer step into a device ring of `capacity` samples. */
int teuk_set_observer(teuk_t h, double rstar_obs, int64_t capacity);
/* Copies the recorded samples, oldest first: out[n][2][w][n_theta], n = min(recorded,
 * capacity) returned in *n_samples. out may be NULL to query n only. */
int teuk_read_waveform(teuk_t h, double* out, int64_t* n_samples);

/* The data flow of the paper's first CUDA design (Sec. 4): the time loop runs on the host and
 * every iteration the state travels from main memory to the GPU and back, which over PCIe
 * gave no overall gain. Here all arithmetic stays on the device: each of the n iterations
 * copies host_planes [4][w][n_r][n_theta] (host memory, page-locked for full link speed) to
 * the device, runs one Lax-Wendroff iteration (Eqs. lw1, lw2), copies the state back and
 * waits for it. Rows 0 and n_r-1 are used as given (keep them zero, Sec. 3.B). The caller
 * owns host_planes; the device state of the handle is overwritten. */
int teuk_substep_host_state(teuk_t h, double* host_planes, int64_t n);

/* Multipoles of the recorded waveform (Sec. 3.C: the late-time decay of each multipole l of the
 * field at the observer, Fig. 1): for every recorded sample t (oldest first) and
 * l = ell_min .. ell_max,
 *   c_l(t) = 2 pi int_0^pi Phi(t, r*_obs, theta) sY_lm(theta) sin(theta) dtheta,
 * sY_lm the normalised spin-weighted spherical harmonic of the handle's s and m (Goldberg et
 * al. 1967 sum with the (-1)^m sign, phi = 0). Quadrature: Fejer's first rule in x = cos(theta)
 * on the cell centres, exact when Phi sY_lm is a polynomial in x of degree < n_theta. Weights,
 * harmonics and sums are in the handle's precision, on the device.
 * Needs max(|m|, |s|) <= ell_min <= ell_max <= min(40, n_theta - 1) and an observer
 * (TEUK_ERR_STATE_MISMATCH otherwise). out: host [n][ell_max - ell_min + 1][2 (re, im)][w]
 * doubles, or NULL to query n only; *n_samples = n = min(recorded, capacity). Synchronises
 * the handle's stream. */
int teuk_read_multipoles(teuk_t h, int ell_min, int ell_max, double* out, int64_t* n_samples);

/* Whole state as host word planes [4][w][n_r][n_theta], and the substep counter. */
int teuk_get_state(teuk_t h, double* planes, int64_t* substeps_done);
int teuk_set_state(teuk_t h, const double* planes, int64_t substeps_done);
/* Same, device to device (a caller-owned device buffer of the same layout). */
int teuk_get_state_device(teuk_t h, double* dev_planes);

/* The raw system coefficients (b, c_R, c_I, Re B/S^2, Im B/S^2, Delta/S^2, Re V/S^2,
 * Im V/S^2) at nodes (which = 0, [8][w][n_r][n_theta]) or half nodes (which = 1,
 * [8][w][n_r-1][n_theta]), and the grid tables x = r - r+ at nodes / half nodes ([w][rows]). */
int teuk_get_coeffs(teuk_t h, int which, double* out);
int teuk_get_tortoise(teuk_t h, int which, double* x_out);

/* Sizes: words per real, rows, columns, substeps, outer dt (rounded to double). */
int teuk_info(teuk_t h, int* words, int* n_r, int* n_theta, int* substeps, double* dt_outer);

/* Number of step kernels launched by this handle so far (two per Lax-Wendroff iteration). */
int64_t teuk_kernel_launches(teuk_t h);

/* Batched execution. Several problems (members) advance together in one cooperative launch
 * per up to 200 outer steps: the paper's data-parallel decomposition of the grid over cores
 * (Sec. 4) applied across independent problems of uneven size. In round q of an outer step
 * every member with more than q Lax-Wendroff iterations per step does one iteration; work
 * items of equal size (rows x theta columns) from all active members share the GPU, with a
 * grid-wide barrier between the half-step and full-step phases. Results are bit-identical to
 * stepping each member alone with teuk_step. Members must use the same precision, arithmetic
 * engine (teuk_set_engine, chosen before the batch is made: a later change makes
 * teuk_batch_step fail with TEUK_ERR_INVALID_ARG) and device, have no r* dissipation, stay
 * alive while the batch exists, and not be stepped by other calls meanwhile; the batch runs on
 * the first member's stream. Observer rings of members receive one sample per outer step, as
 * with teuk_step. */
typedef struct teuk_batch_s* teuk_batch_t;
int teuk_batch_create(teuk_batch_t* out, const teuk_t* members, int n_members);
int teuk_batch_step(teuk_batch_t b, int64_t n_outer_steps);
/* Waits for the batch; returns TEUK_ERR_NONFINITE if any member produced Inf/NaN. */
int teuk_batch_sync(teuk_batch_t b);
/* Grid size of the cooperative launch, largest substep count, grid-point updates per outer
 * step over all members, cooperative launches so far. Any pointer may be NULL. */
int teuk_batch_info(teuk_batch_t b, int* grid_blocks, int* k_max, int64_t* points_per_outer_step,
                    int64_t* launches);
int teuk_batch_destroy(teuk_batch_t b);

/* Autotuner: times a few Lax-Wendroff iterations for each candidate launch shape (threads
 * along theta x rows of theta per thread block, one warp per 32 columns, register budgets)
 * on a copy of the current state; when an outer step is short (under 5 ms) the four fastest
 * are timed again over four outer steps as teuk_step runs them (a replayed CUDA graph), and the
 * persistent launches are tried against them. Grids of up to 2^20 points also try the fused
 * iterations (variant 10), which allocate a second state-sized buffer kept with the handle. It keeps the fastest for this handle, restores
 * the state and
 * returns in *rows_per_block (may be NULL) the rows per block of the chosen shape, 0 when the
 * one-warp-per-32-columns kernels won (teuk_launch_shape reports the whole shape). Allocates
 * and frees one state-sized device buffer; call it before timing-critical work. */
int teuk_tune(teuk_t h, int* rows_per_block);
/* The step kernels' launch shape in use: threads along theta per row, rows per block, and the
 * kernel variant: 0, 1, 2 = whole rows per block with <= 255 and <= 128 registers per thread
 * (blocks of up to 256 threads), or <= 102 registers in blocks of up to 128 threads;
 * 3, 4, 5 = one warp per (row, 32 theta columns) with <= 255, 128, 85 registers;
 * 6, 7, 8 = balanced: as many blocks of threads_theta threads as fit on the GPU at once,
 * each taking the same number of (row, theta) points, budgets as for 0, 1, 2; 9 = persistent
 * (teuk_set_persistent); 10 = fused iterations: one launch per Lax-Wendroff iteration, each block
 * forming the R + 1 half-step rows its R full-step rows need (rows_per_block = R) in shared
 * memory, so one half row per block is formed twice, and writing a second state buffer (the
 * iterations alternate between the two; a sequence that ends in the second one is copied back,
 * so the state is in place between calls): the bits of the two-kernel form with half the
 * launches, for grids whose iterations are shorter than a launch. */
int teuk_launch_shape(teuk_t h, int* threads_theta, int* rows_per_block, int* variant);
/* Sets the launch shape explicitly (same meaning as above; threads_theta a multiple of 32,
 * threads_theta * rows_per_block <= 256; both ignored for variants 3..5, rows_per_block
 * ignored for 6..8; with variants 2 and 8 the block is cut to 128 threads; on the integer
 * engine only variants 0..2, and rows_per_block rows must fit one block's shared memory,
 * else TEUK_ERR_INVALID_ARG; the autotuner skips such shapes; variant 10 needs threads_theta
 * <= 128, threads_theta * (rows_per_block + 1) <= 256, the FP64-transform engine and a whole
 * grid, not a slab). Results do not depend on the shape. */
int teuk_set_launch_shape(teuk_t h, int threads_theta, int rows_per_block, int variant);
/* Persistent launches for small problems (FP64, or the FP64 error-free transforms): teuk_step
 * runs steps_per_launch outer steps (k iterations each, Eqs. lw1, lw2) per cooperative launch
 * of ceil((n_r - 1) / rows_per_block) blocks of threads_theta x rows_per_block threads
 * (threads_theta 0: n_theta rounded up to 32, at most 256 / rows_per_block). Block b owns the
 * half rows and nodes [b R, (b + 1) R); neighbouring blocks wait on each other's progress
 * counters (bounded waits: a wait that reaches its limit ends the launch and teuk_sync reports
 * TEUK_ERR_TIMEOUT) instead of the launch boundaries between phases. Results are bit-identical
 * to the other launch shapes. teuk_step returns TEUK_ERR_INVALID_ARG if the blocks cannot all
 * be resident at once; teuk_substep and handles with dissipation use the rows-per-block
 * kernels of the same shape. teuk_launch_shape reports variant 9; teuk_tune tries it (1, 2, 4
 * or 8 rows; 1 or 8 outer steps per launch) against the best other shape run as a CUDA graph,
 * and keeps whichever is faster. 1 <= rows_per_block <= 8, 1 <= steps_per_launch <= 4096. */
int teuk_set_persistent(teuk_t h, int threads_theta, int rows_per_block, int steps_per_launch);

/* Lax-Wendroff iterations that allocate nothing, for callers that cannot let a library
 * allocate device memory while they step (their memory belongs to a pool of their own, or
 * they cannot afford cudaMalloc/cudaFree, which may synchronise the whole device). The paper
 * has no counterpart: this is an interface variant of teuk_substep.
 *  - h: an existing handle; only its constant tables, stream and device are used, its own
 *    state is neither read nor written. An r* slab handle takes one iteration per call.
 *  - u_in / u_out: caller-owned device buffers in the handle's layout
 *    [4][w][n_r][P] doubles, P = n_theta rounded up to a multiple of 16 (128 bytes); they may
 *    be the same buffer. Both must start on a 16-byte boundary (the integer engine copies
 *    their rows into shared memory with bulk copies), else TEUK_ERR_INVALID_ARG; allocators
 *    such as cudaMalloc and torch's return 256-byte aligned blocks. The first iteration reads
 *    u_in, later ones run in place on u_out; rows 0 and n_r-1 of u_out are set to zero.
 *  - The half-step rows live in one fixed device array of 2^21 doubles (16 MiB) that every
 *    GPU loading the library holds until exit; 4 * w * (n_r - 1) * P above 2^21 is rejected
 *    with TEUK_ERR_INVALID_ARG. Every row of it that a call reads is written earlier in the
 *    same call, so nothing needs clearing; calls that overlap on the GPU (other streams,
 *    other handles) share the array and race.
 *  - The first call on a device looks up the array's device address (cudaGetSymbolAddress);
 *    make that first call before any stream capture. The handle's device must be current.
 *  - Calls no cudaMalloc, cudaFree or other allocating routine; work is queued on the
 *    handle's stream and the call returns without waiting for it.
 *  - Errors found by the kernels themselves (a non-finite value, TEUK_ERR_NONFINITE; a bounded
 *    wait that reached its limit, TEUK_ERR_TIMEOUT) are kept in the handle's status word and
 *    reported by the next teuk_sync(h), as for teuk_substep. */
int teuk_substep_noalloc(teuk_t h, const double* u_in, double* u_out, int64_t n_iterations);

/* Per-kernel timing with CUDA events on the handle's stream: enable = 1 starts recording
 * the duration of every half-step and full-step launch; teuk_kernel_times() waits for the
 * stream and returns (and clears) the summed milliseconds and launch counts. Steps replayed
 * as a CUDA graph keep running as a graph and time a sample: the two kernels of the last
 * iteration of the outer step (event nodes of the graph), counted once per drain from the
 * last replay before it (the counts say how many launches were timed). */
int teuk_timing(teuk_t h, int enable);
int teuk_kernel_times(teuk_t h, double* ms_half, double* ms_full, int64_t* n_half, int64_t* n_full);

/* Measured FP64 pipe throughput of the current device (a chain of independent FMAs on every
 * SM): operations per second, counting one per FMA. */
int teuk_fp64_peak(double* ops_per_second);
/* Measured throughput of the integer engine's product window on the current device: 32-bit
 * limb partial products per second (a mad.lo / madc.hi pair with its carry each; a
 * double-double product window has 10, a quad-double one 36), from independent windows on
 * every SM. The roofline unit of the integer engine. */
int teuk_int_peak(double* pairs_per_second);

const char* teuk_strerror(int code);
const char* teuk_last_error(teuk_t h);

/* Multi-word arithmetic self-test: applies op (0 add, 1 sub, 2 mul, 3 div, 4 sqrt, 5 exp,
 * 6 log, 7 dot-accumulate a*b + out, 8 out[t] + sum_{q<11} a[t+q] b[t+q] (indices mod n) through
 * one accumulator, 9 the same sum through the integer engine, 10 / 11 a + b / a - b through
 * the integer engine, 12 a / 2 + b through the engine's products by powers of two (a shift
 * of the other mantissa); 9..12 for double-double and quad-double)
 * elementwise to n values of precision w, on the host (device = 0) or the current CUDA
 * device (device = 1). a, b, out: [w][n] host arrays. */
int teuk_mw_eval(int op, int words, int device, const double* a, const double* b, double* out,
                 int64_t n);

#ifdef __cplusplus
}
#endif
#endif
