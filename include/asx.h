/*
 * asx.h -- C ABI of the GB300 (sm_103a) solver for the porosity-extended
 * Saint-Venant model on a regular hexagonal raster (arxiv 2406.14933, "ASTERIX").
 *
 * The library advances the explicit finite-volume scheme of the paper, Sec. 2.2,
 * Eq. fvm_2D_eq_frac.07, in the fractional form of Appendix A: upwind mass and
 * momentum fluxes on every hexagon edge (Eqs. fvm_2D_eq.04-06, fvm_2D_eq_frac.01),
 * the free-surface pressure term, rain at t^{n+1}, the closed-form implicit
 * soil-friction / plant-drag update (Eq. miu-formula) and the CFL time step
 * (Eqs. fvm_2D_eq_frac.12-13).  Every step runs on the GPU; the host only launches
 * and reads results.
 *
 * Raster: `rows` x `cols` pointy-top hexagons, row-major, every row `cols` cells long,
 * odd rows shifted east by half a centre spacing.  Cell (r, c) is element r*cols + c of
 * every dense field passed in or out.  `edge_m` is the hexagon edge length (the paper's
 * "radius"); cell area sigma = (3 sqrt3 / 2) edge_m^2.
 *
 * State: the prognostic mass m = theta*h lives in float32 as an unevaluated sum
 * hi + lo (a compensated pair), the velocity (v1, v2) in float32.  The global ledger
 * (rain in, outflow, clamped water, storage) is float64.
 *
 * Conventions for every call:
 *   - Inputs are copied in; the caller keeps ownership and may free them on return.
 *   - Output buffers are caller-allocated.  ASX_PTR_DEVICE pointers must be device
 *     memory of `desc.device`, dense (no pitch).
 *   - Work is ordered on `desc.cuda_stream` (NULL = the legacy default stream).  A
 *     call returns once its results are valid for the caller: calls that fill host
 *     memory or return host values synchronise with that stream.
 *   - No exception crosses the ABI: every call returns an asx_status; asx_last_error
 *     gives a one-line description of the last failure on that handle.
 *   - One thread at a time per handle.
 */
#ifndef ASX_H
#define ASX_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    ASX_OK = 0,
    ASX_EINVAL = 1,    /* an argument is out of range (see each call) */
    ASX_ENOMEM = 2,    /* device or host allocation failed */
    ASX_ECUDA = 3,     /* a CUDA runtime call failed (asx_last_error has the text) */
    ASX_ESTATE = 4,    /* the call needs fields / params that were not set */
    ASX_ENUMERIC = 5,  /* the state became non-finite; the clock stops at that step */
    ASX_ETIMEOUT = 6,  /* a bounded wait inside a kernel ran out */
    ASX_EBOUNDS = 7    /* an index outside its buffer (only the bounds-checked debug build
                        * of the library checks; the access was skipped) */
} asx_status;

enum { ASX_BC_WALL = 0, ASX_BC_FREE = 1, ASX_BC_FLUX = 2, ASX_BC_DIRICHLET = 3 };
enum { ASX_SIDE_W = 0, ASX_SIDE_E = 1, ASX_SIDE_S = 2, ASX_SIDE_N = 3 };
enum { ASX_PTR_HOST = 0, ASX_PTR_DEVICE = 1 };
/* Arithmetic of a raster (asx_raster_desc.precision).  The paper states no precision.
 *   ASX_FP32_COMP  float32 state with the mass as a compensated pair and a float64
 *                  ledger: the fast path (the TMA strip kernel).
 *   ASX_FP64       float64 state, bed and porosity, every operation in float64 (one
 *                  thread per cell; float64 runs at 1/64 of the float32 rate on GB300):
 *                  for checks against double-precision references on small rasters. */
enum { ASX_FP32_COMP = 0, ASX_FP64 = 1 };
#define ASX_MAX_CLASSES 16
#define ASX_MAX_RAIN 64

typedef struct asx_raster asx_raster;      /* opaque, owned by the library */

/* Geometry and boundaries of one raster (Sec. 2.2 (a); boundary types of Sec. 3).
 *   bc[side]            ASX_BC_WALL (mirror: the edge carries nothing), ASX_BC_FREE
 *                       (free discharge: a ghost copy of the inner cell, outflow only),
 *                       ASX_BC_FLUX (given mass flux asx_params.bc_q[side] per unit
 *                       length, entering along the side's inward normal; an edge of the
 *                       side admits l q (n_side . n_edge), carrying the velocity q / h of
 *                       the cell's depth h, at least the critical depth (q^2/g)^(1/3);
 *                       no pressure term) or ASX_BC_DIRICHLET (Sec. 4, Eq. numerics-bc: a
 *                       ghost cell on the inner cell's bed and porosity with depth
 *                       asx_params.bc_h[side] and velocity -bc_u[side] n_side, through the
 *                       interior edge formulas).  Mass through FLUX and DIRICHLET edges
 *                       is booked in the ledger's outflow (inflow negative).
 *   free_begin/free_end the side's type applies to the positions [begin, end) along it
 *                       (the column for S/N, the row for W/E) and the rest of the side is
 *                       a wall; begin == end: all of it.
 *   n_classes           0: porosity is a float per cell; 1..ASX_MAX_CLASSES: each cell
 *                       holds a uint8 land-cover class and asx_params gives per-class
 *                       porosity and coefficients.
 *   max_samples         capacity of the outlet hydrograph (0 = no hydrograph).
 *   precision           ASX_FP32_COMP (0, the default of a zeroed struct) or ASX_FP64.
 * A boundary edge belongs to the S or N side when its missing neighbour's row is
 * outside the raster, otherwise to W or E. */
typedef struct {
    int rows, cols;            /* >= 2 each; rows * cols < 2^31 */
    double edge_m;             /* > 0 */
    int bc[4];                 /* indexed by ASX_SIDE_* */
    int free_begin[4], free_end[4];
    int n_classes;
    int max_samples;
    void *cuda_stream;         /* cudaStream_t; NULL = default stream */
    int device;                /* CUDA device ordinal */
    int precision;             /* ASX_FP32_COMP or ASX_FP64 */
} asx_raster_desc;

/* Physical and numerical parameters (Sec. 3 "Parameters"; Eq. eq_K_h_theta).
 *   g                        gravity [m/s^2] (> 0)
 *   cfl                      Courant number in (0, 1] (Eq. fvm_2D_eq_frac.12)
 *   dt_max                   maximum time step [s] (> 0)
 *   alpha_s, alpha_p         soil friction [-] and plant drag [1/m] (>= 0), used when
 *                            n_classes == 0
 *   class_theta/alpha_p/alpha_s  n_classes entries each when n_classes > 0
 *                            (theta in (0, 1], coefficients >= 0); host pointers
 *   n_rain, rain_t, rain_r   piecewise-linear rain rate r(t) [m/s] at increasing times
 *                            [s], zero outside [rain_t[0], rain_t[n-1]]; host
 *                            pointers; n_rain <= ASX_MAX_RAIN (0 = no rain)
 *   sample_dt                hydrograph sample interval [s]; steps are cut at the
 *                            sample times (0 = none)
 *   viscosity                1: add the artificial viscosity l c_(i,j) mu_(i,j) (v_j - v_i)
 *                            to the momentum flux of every interior edge (Appendix A,
 *                            Eqs. eq_artif_visc, eq_visc1: c_(i,j) = max(c_i, c_j) with
 *                            c = |v| + sqrt(g h), mu_(i,j) the harmonic mean of theta h,
 *                            0 when both cells are dry); raster sides add none.  0: off.
 *   tau                      linear soil resistance -tau h v [1/s] (>= 0) of Thacker's
 *                            problem (Sec. 4, Eq. eq_soil_friction_thacker), taken
 *                            implicitly with the other resistances:
 *                            (theta h + dt tau h) v + dt K |v| v = gamma.  0: none.
 *   h_dry                    depth [m] (>= 0) below which a cell's new velocity is set to
 *                            zero (a wet/dry threshold the paper does not print; without
 *                            resistance, films at a moving shoreline otherwise accelerate
 *                            without bound).  0: none (a cell is dry only when empty).
 * ASX_EINVAL on any value out of range. */
typedef struct {
    double g, cfl, dt_max;
    double alpha_s, alpha_p;
    const float *class_theta, *class_alpha_p, *class_alpha_s;
    int n_rain;
    const double *rain_t, *rain_r;
    double sample_dt;
    int viscosity;
    double tau, h_dry;
    double bc_q[4], bc_h[4], bc_u[4];   /* per side, see asx_raster_desc.bc */
} asx_params;

/* Water budget since the last asx_set_fields, all in m^3 (float64):
 *   rain_in   sum over steps of sigma * (applied rain depth) over all cells
 *   outflow   water that left through free-discharge edges
 *   storage   sum over cells of sigma * theta h now (computed on the device)
 *   storage0  the same at asx_set_fields
 *   clamped   water created by setting a negative mass to zero
 *   defect_rel |storage0 + rain_in + clamped - outflow - storage| /
 *              max(rain_in, storage0) (0 when both are 0)
 *   steps     time steps taken */
typedef struct {
    double rain_in, outflow, storage, storage0, clamped, defect_rel;
    long long steps;
} asx_ledger;

/* Create a raster on desc->device.  Allocates all device memory it will use.
 * ASX_EINVAL: rows or cols < 2, rows * cols >= 2^31, edge_m <= 0 or not finite, a bc
 * value outside ASX_BC_WALL .. ASX_BC_DIRICHLET, free_begin < 0 or free_end <
 * free_begin, n_classes outside [0, ASX_MAX_CLASSES], max_samples < 0, a precision
 * other than ASX_FP32_COMP / ASX_FP64.  ASX_ENOMEM when device memory runs out. */
asx_status asx_create_raster(const asx_raster_desc *desc, asx_raster **out);

/* Free the raster and all its device memory (NULL is accepted). */
asx_status asx_destroy_raster(asx_raster *r);

/* Set the parameters; may be called again between steps. */
asx_status asx_set_params(asx_raster *r, const asx_params *p);

/* Set the static fields and the initial state (the paper's "Data In", Sec. 3), reset
 * the clock to t = 0 and the ledger.  z: bed elevation [m] (float64, finite); in
 * ASX_FP32_COMP mode it is rounded to the nearest float32 (round to nearest even: an
 * elevation of 1000 m moves by at most 3.1e-5 m), in ASX_FP64 mode kept as given;
 * theta_or_null: porosity per cell in (0, 1] when n_classes == 0, else NULL;
 * class_or_null: class per cell (< n_classes) when n_classes > 0, else NULL;
 * h0: initial depth [m] (>= 0, finite); v1_0, v2_0: initial velocity [m/s] (finite;
 * NULL = 0).  All dense rows x cols.  ptr_kind: ASX_PTR_HOST or ASX_PTR_DEVICE.
 * Value checks (ASX_EINVAL) are made on host inputs; device inputs are trusted.
 * Needs asx_set_params first (ASX_ESTATE). */
asx_status asx_set_fields(asx_raster *r, const double *z, const float *theta_or_null,
                          const uint8_t *class_or_null, const float *h0, const float *v1_0,
                          const float *v2_0, int ptr_kind);

/* Advance exactly n_steps time steps (n_steps >= 0) of Eq. fvm_2D_eq_frac.07, each
 * with the CFL time step (cut at hydrograph sample times).  *t_out (may be NULL)
 * receives the time reached.  ASX_ENUMERIC if the state became non-finite. */
asx_status asx_step(asx_raster *r, int n_steps, double *t_out);

/* Advance until t == t_end (the last step is cut to land on t_end).  t_end below the
 * current time is a no-op.  *t_out (may be NULL) receives the time reached. */
asx_status asx_run_until(asx_raster *r, double t_end, double *t_out);

/* Water budget (see asx_ledger).  scenario must be 0 for a single raster. */
asx_status asx_mass_ledger(asx_raster *r, int scenario, asx_ledger *out);

/* Depth h = m / theta and velocity of every cell, dense rows x cols float32 (any
 * pointer may be NULL to skip that field). */
asx_status asx_get_fields(asx_raster *r, int scenario, float *h, float *v1, float *v2,
                          int ptr_kind);

/* Depth and velocity of every cell in float64, dense rows x cols: in ASX_FP64 mode the
 * state itself (h = m / theta in float64), in ASX_FP32_COMP mode h = (m_hi + m_lo) /
 * theta in float64 and the float32 velocities widened.  Any pointer may be NULL.  Uses
 * three float64 planes of device scratch for the duration of the call. */
asx_status asx_get_fields64(asx_raster *r, int scenario, double *h, double *v1, double *v2,
                            int ptr_kind);

/* The raw state: compensated mass pair (m_hi, m_lo), v1, v2, dense rows x cols
 * float32 (for checkpoints; any pointer may be NULL).  ASX_EINVAL in ASX_FP64 mode,
 * which has no float32 state. */
asx_status asx_get_state(asx_raster *r, float *m_hi, float *m_lo, float *v1, float *v2,
                         int ptr_kind);

/* Restore a raw state written by asx_get_state together with the clock and ledger of
 * asx_get_clock / asx_mass_ledger at that moment; continuing from it reproduces the
 * uninterrupted run bit for bit.  Needs asx_set_fields first (static fields).
 * samples_cum_outflow: the cumulative outflow [m^3] at each of the n_samples sample times
 * up to t (with sample_dt > 0, n_samples sample_dt <= t < (n_samples + 1) sample_dt is
 * required: ASX_EINVAL otherwise).  ASX_EINVAL in ASX_FP64 mode. */
asx_status asx_set_state(asx_raster *r, const float *m_hi, const float *m_lo,
                         const float *v1, const float *v2, int ptr_kind, double t,
                         long long step, const asx_ledger *ledger, int n_samples,
                         const double *samples_cum_outflow);

/* Outlet hydrograph: q[k] = outflow volume between sample times k and k+1, divided
 * by sample_dt [m^3/s], for the samples recorded so far (at most cap).  *n receives
 * the number of samples recorded. */
asx_status asx_get_hydrograph(asx_raster *r, int scenario, double *q, int cap, int *n);

/* Current time, the time step the next step will take (0 when no step is pending),
 * and the number of steps taken. */
asx_status asx_get_clock(asx_raster *r, int scenario, double *t, double *dt, long long *step);

/* One-line description of the last error on this handle ("" if none; a static string
 * for r == NULL). */
const char *asx_last_error(const asx_raster *r);

/* ---------------------------------------------------------------- ensembles
 * A batch of independent rasters ("scenarios") of uneven sizes advanced together: each
 * with its own CFL time step, clock, ledger and hydrograph, all in one persistent kernel
 * launch (captured in a CUDA graph) in which a thread-block cluster takes a scenario at a
 * time from a queue (longest first).  The per-scenario step is the single-raster step
 * (Eq. fvm_2D_eq_frac.07), so a scenario's state matches a single raster run bit for bit
 * (per-cell porosity; the gather cell code).  Ensembles serve sweeps over coefficients,
 * slopes and storms such as the sensitivity and calibration studies of Secs. 4.3-4.4. */
typedef struct asx_ensemble asx_ensemble;

/* One scenario: geometry, boundaries and parameters as in asx_raster_desc / asx_params
 * (per-cell porosity, scalar alpha_s / alpha_p), a rain table of at most 8 points (host
 * pointers, copied), the end time t_end [s] the scenario runs to, the hydrograph interval
 * sample_dt and capacity max_samples, max_steps (0 = no limit), the per-side values of
 * ASX_BC_FLUX / ASX_BC_DIRICHLET sides (bc_q, bc_h, bc_u as in asx_params), and the
 * optional terms viscosity, tau, h_dry as in asx_params (all 0: the plain scheme). */
typedef struct {
    int rows, cols;
    double edge_m;
    int bc[4], free_begin[4], free_end[4];
    double g, cfl, dt_max, alpha_s, alpha_p;
    int n_rain;
    const double *rain_t, *rain_r;
    double t_end, sample_dt;
    int max_samples;
    long long max_steps;
    double bc_q[4], bc_h[4], bc_u[4];
    int viscosity;
    double tau, h_dry;
} asx_scenario_desc;

/* Launch shape of the ensemble: CTAs per cluster (1, 2, 4, 8) sharing one scenario, and
 * the kernel.  tile_rows = 0: the gather kernel (one thread per cell), threads per CTA
 * (128, 256, 512), cells each thread updates per round (1, 2, 4).  tile_rows = 8, 16 or
 * 32: the strip kernel (each warp a TMA-fed tile worker over tiles of 128 columns x
 * tile_rows rows, the cells along the sides gathered; the same per-cell code, hence the
 * same bits, as a single raster's strip kernel with that tile height), threads per CTA
 * 128, 256 or 512 (4, 8 or 16 tile workers), cells_per_thread 1.  tile_rows = 1: the strip kernel
 * with each scenario's tile height (8, 16 or 32) chosen on the host as the one whose
 * modelled step on this cluster is shortest (few, larger tiles for large rasters; more,
 * smaller ones where large tiles would leave warps idle).  split = 0: every scenario runs
 * on a whole cluster.  split > 0 (strip kernel, cluster >= 2): the `split` scenarios that
 * come first in the queue (the largest) run on whole clusters, and once they are all
 * taken each CTA runs the others alone; the results are the same either way. */
typedef struct {
    int cluster, threads, cells_per_thread;
    int tile_rows;
    int split;
} asx_ensemble_tuning;

/* Create an ensemble of n scenarios on `device`, work ordered on cuda_stream.  Allocates
 * all device memory.  ASX_EINVAL on any description out of range. */
asx_status asx_create_ensemble(int n, const asx_scenario_desc *descs, void *cuda_stream, int device,
                               asx_ensemble **out);
asx_status asx_destroy_ensemble(asx_ensemble *e);

/* Static fields and initial state of scenario s (dense rows x cols; the bed z in
 * float64, rounded to the nearest float32 as in asx_set_fields; theta, h0, v1, v2 in
 * float32, v1, v2 may be NULL = 0); the state is kept so that every run starts from it. */
asx_status asx_ensemble_set_fields(asx_ensemble *e, int s, const double *z, const float *theta,
                                   const float *h0, const float *v1, const float *v2, int ptr_kind);

/* Times every launch shape (the gather kernel's 36, the strip kernel's 24) on the ensemble
 * cut short (after one untimed launch; each shape twice, the faster counts) and keeps the fastest for asx_ensemble_run; *best_out (may be
 * NULL) receives it.  Before the first asx_ensemble_run that takes every scenario to its
 * t_end, each scenario is cut at max_steps steps.  After one, scenario i is cut at its
 * step count in that run times max_steps x (total cells) / (total cells x steps): the same
 * number of cell updates as max_steps per scenario, distributed over the scenarios as in
 * the real run, so that the shape chosen suits the real run's critical path (its longest
 * scenarios) and not only its throughput.  Such a complete run also makes later runs take
 * the scenarios in decreasing order of measured cells x steps (before it: cells x t_end /
 * edge).  The scenarios' states are reset to their initial state afterwards by the next
 * asx_ensemble_run. */
asx_status asx_ensemble_autotune(asx_ensemble *e, int max_steps, asx_ensemble_tuning *best_out);

/* Runs every scenario from its initial state to its t_end in one persistent launch
 * (tuning NULL = the autotuned or default shape).  ASX_ENUMERIC if a scenario's state
 * became non-finite, ASX_ETIMEOUT if a tensor copy of the strip kernel did not arrive
 * within its bounded wait (that scenario stops; the others finish). */
asx_status asx_ensemble_run(asx_ensemble *e, const asx_ensemble_tuning *tuning);

/* Per-scenario results of the last run (see asx_ledger, asx_get_fields, asx_get_state,
 * asx_get_hydrograph). */
asx_status asx_ensemble_ledger(asx_ensemble *e, int s, asx_ledger *out);
asx_status asx_ensemble_get_fields(asx_ensemble *e, int s, float *h, float *v1, float *v2, int ptr_kind);
asx_status asx_ensemble_get_state(asx_ensemble *e, int s, float *m_hi, float *m_lo, float *v1, float *v2,
                                  int ptr_kind);
asx_status asx_ensemble_get_hydrograph(asx_ensemble *e, int s, double *q, int cap, int *n);
asx_status asx_ensemble_get_clock(asx_ensemble *e, int s, double *t, long long *steps);
const char *asx_ensemble_last_error(const asx_ensemble *e);

/* ---------------------------------------------------------------- the surrogate's GEMM
 * D[M x N] = A[M x K] . B[N x K]^T on the tensor cores (tcgen05, BF16 inputs, FP32
 * accumulation in tensor memory): the product the surrogate MLP is made of (not in the
 * paper; the learned hydrograph surrogate is this library's addition).  A(m, k) =
 * A[m*sam + k*sak] and B(n, k) = B[n*sbn + k*sbk] are BF16 device arrays read through
 * these element strides; D is FP32, row stride ldd >= N.  An operand whose base is
 * 16-byte aligned, with one stride 1 and the other a multiple of 8 that is at least the
 * contiguous extent (K, or M / N), is staged by TMA tile copies; any other operand is
 * read element by element (same results either way).  Asynchronous on cuda_stream.
 * ASX_EINVAL on non-positive sizes, null pointers or ldd < N; ASX_ECUDA if the launch
 * fails. */
asx_status asx_gemm_bf16(int M, int N, int K, const void *A, long long sam, long long sak, const void *B,
                         long long sbn, long long sbk, float *D, long long ldd, void *cuda_stream);

/* ---------------------------------------------------------------- the surrogate
 * A learned stand-in for whole hillslope runs (not in the paper): an MLP mapping slope,
 * vegetation cover, porosity, plant drag and a 32-sample hyetograph (ASX_MLP_IN inputs)
 * to a 128-sample outlet hydrograph (ASX_MLP_OUT outputs), three hidden ReLU layers of
 * ASX_MLP_HIDDEN units, trained on hydrographs the solver produces.  BF16 weights and
 * activations, FP32 accumulation on the tensor cores (asx_gemm_bf16), FP32 master weights
 * and Adam moments.  Parameters are packed as W1 (256 x 36, row = output unit), b1 (256),
 * W2 (256 x 256), b2, W3 (256 x 256), b3, W4 (128 x 256), b4 (128): ASX_MLP_PARAMS
 * floats.  x is batch x 36 and y, t are batch x 128, FP32 row-major.  Loss: mean squared
 * error over batch x 128. */
#define ASX_MLP_IN 36
#define ASX_MLP_HIDDEN 256
#define ASX_MLP_OUT 128
#define ASX_MLP_PARAMS 173952
typedef struct asx_mlp asx_mlp;

/* Allocates parameters, Adam state and activations for batches up to max_batch
 * (1 .. 4,194,304); parameters start at zero. */
asx_status asx_mlp_create(int device, void *cuda_stream, int max_batch, asx_mlp **out);
asx_status asx_mlp_destroy(asx_mlp *p);
/* Sets / reads the packed FP32 parameters (setting also resets Adam). */
asx_status asx_mlp_set_params(asx_mlp *p, const float *params, int ptr_kind);
asx_status asx_mlp_get_params(asx_mlp *p, float *params, int ptr_kind);
/* Inference on any batch (processed max_batch rows at a time). */
asx_status asx_mlp_forward(asx_mlp *p, int batch, const float *x, float *y, int ptr_kind);
/* Gradient of the loss with respect to the packed parameters, and the loss (batch <=
 * max_batch); for gradient checks. */
asx_status asx_mlp_gradients(asx_mlp *p, int batch, const float *x, const float *t, float *grad, float *loss,
                             int ptr_kind);
/* One Adam step (beta 0.9 / 0.999, eps 1e-8, decoupled-free L2 weight decay on the weight
 * matrices); *loss (may be NULL) receives the batch loss before the step (and then the
 * call waits for the stream).  From the second step at a batch size the step's kernels
 * replay as a CUDA graph held by the handle (one per batch size; the same results), so
 * x and t are copied into the handle's buffers on the stream before it runs. */
asx_status asx_mlp_train_step(asx_mlp *p, int batch, const float *x, const float *t, float lr,
                              float weight_decay, float *loss, int ptr_kind);
const char *asx_mlp_last_error(const asx_mlp *p);

/* The surrogate's check against the solver, with fallback: for k < n_check, with
 * q = idx[k], computes e_k = ||y_q - ref_k||_2 / ||ref_k||_2 over the ASX_MLP_OUT samples
 * of row q of y (batch x ASX_MLP_OUT, the surrogate's hydrographs) and row k of ref
 * (n_check x ASX_MLP_OUT, the solver's hydrographs of the same queries, same units);
 * where e_k > tol, or e_k is not a number, row q of y is overwritten with ref_k.
 * rel_err[k] receives e_k (0 where both rows are zero, +inf where only ref_k is zero,
 * NaN where idx[k] lies outside [0, batch) -- such a row is skipped), *n_replaced the
 * number of rows replaced.  idx must not repeat.  All pointers are device memory;
 * asynchronous on cuda_stream.  ASX_EINVAL on negative sizes, n_check > batch, tol < 0
 * or null pointers. */
asx_status asx_surrogate_check(int batch, int n_check, const int *idx, float *y, const float *ref, float tol,
                               float *rel_err, int *n_replaced, void *cuda_stream);

/* Allocation-free scan of a state the caller holds (the paper has no counterpart; this
 * serves callers that may not allocate device memory, e.g. a runtime that owns every
 * buffer and forbids allocation once started, or a library that only lends pointers).
 * It writes to *storage_out the water volume sum_i sigma (m_hi + m_lo)_i [m^3] (float64,
 * fixed-order sum) and to *cmax_out the largest wave speed |v| + sqrt(g h), h = m_hi /
 * theta, of the state; both outputs are device pointers and are written asynchronously
 * on cuda_stream.  All arrays are device memory of the current device, rows x cols with
 * a row pitch of `pitch` elements (>= cols); theta in (0, 1].
 * No memory is allocated: the scratch (per-CTA partials and a completion counter) is a
 * fixed 64 KB device array held by the library for as long as it is loaded, one copy
 * per device.  Limit: at most 67,108,864 cells (4096 CTAs of 16,384 cells); larger
 * rasters return ASX_EINVAL.  The first call on a device looks up the array's device
 * address (cudaGetSymbolAddress); make that first call before any stream capture.  All
 * calls on a device share the scratch, so calls that overlap on the GPU (on different
 * streams, or from several threads) race: order them on one stream.
 * Returns ASX_EINVAL on bad sizes, a non-finite or non-positive edge_m or g, or null
 * pointers; ASX_ECUDA when the address lookup, the counter reset or this call's kernel
 * launch fails, or the context was broken by earlier work.  The launch status is the
 * launch's own: a launch error that earlier, unrelated work left for cudaGetLastError is
 * neither reported nor cleared by this call. */
asx_status asx_state_scan_noalloc(int rows, int cols, int pitch, double edge_m, double g,
                                  const float *m_hi, const float *m_lo, const float *v1,
                                  const float *v2, const float *theta, double *storage_out,
                                  float *cmax_out, void *cuda_stream);

/* Failure-detection self-test (no counterpart in the paper): one warp on `device` waits,
 * with the bounded mbarrier wait of the step kernels (which gives up after 2 s), on an
 * mbarrier that nothing arrives at; the wait runs out, the kernel flags it, and the
 * host reads the flag.  Returns ASX_ETIMEOUT when the timeout was detected and reported
 * (the expected outcome; the CUDA context stays usable), ASX_OK if the wait completed,
 * ASX_ECUDA / ASX_ENOMEM on a CUDA error. */
asx_status asx_selftest_wait(int device);

#ifdef __cplusplus
}
#endif
#endif /* ASX_H */
