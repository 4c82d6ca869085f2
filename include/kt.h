/*
 * kt.h -- C ABI of libkt: the Kurganov-Tadmor (KT) semi-discrete step with Heun (RK2) time
 * integration for 3+1d relativistic viscous hydrodynamics in Milne coordinates (tau, x, y, eta_s)
 * with shear stress pi^{mu nu} and bulk pressure Pi, as stated in
 * D. Bazow, U. Heinz, M. Strickland, "Massively parallel simulations of relativistic fluid
 * dynamics on graphics processing units with CUDA", arXiv:1608.06577.
 *
 * Every step of the time integration runs in hand-written CUDA kernels for sm_103a (GB300).
 * There is no CPU fallback: without a CUDA device kt_init fails with KT_ERR_CUDA.
 *
 * Units: hbar = c = 1, lengths in fm.  Energy density, pressures, pi^{mu nu} and Pi in fm^-4,
 * temperature in fm^-1, tau and x, y in fm, eta_s dimensionless.
 *
 * Layouts of the state arguments: physical cells only, x fastest, then y, then eta
 * (index i + nx*(j + ny*k)), component-major (all cells of component 0, then component 1 ...).
 * Internally the state lives in padded structure-of-arrays fields with two ghost layers on
 * each side (Sec. 4.1, Eqs. ghostCells_1/2; Sec. 4.2).
 *
 * Conventions.  Every call returns KT_OK (0) or a negative KT_ERR_* code; on error nothing
 * is written to the caller's outputs and kt_last_error() describes the failure.  No call
 * throws.  A context belongs to one host thread; its work is enqueued on the context's
 * stream.  Pointers passed to a call are only read or written during that call (buffers are
 * copied); the caller keeps ownership of everything it passes.
 */
#ifndef KT_H
#define KT_H
#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ------------------------------------------------------------------ status codes */
enum {
  KT_OK = 0,
  KT_ERR_ARG = -1,        /* invalid argument (null pointer, bad size, bad option) */
  KT_ERR_CUDA = -2,       /* a CUDA runtime call failed (message in kt_last_error) */
  KT_ERR_OOM = -3,        /* device allocation failed or the caller's arena is too small */
  KT_ERR_EOS = -4,        /* EOS table not strictly increasing in e, or too short */
  KT_ERR_STATE = -5,      /* non-finite input state or T^{tau tau} <= |T^{tau i}| after set_state */
  KT_ERR_INVERSION = -6,  /* a cell's root-find (Eq. eInferred) failed during a step */
  KT_ERR_NONFINITE = -7,  /* a non-finite value appeared during a step */
  KT_ERR_TIMEOUT = -8     /* a copy into shared memory did not complete within its bounded wait;
                             the step's results are invalid */
};

enum { KT_MILNE = 0, KT_CARTESIAN = 1 };              /* coordinates (Cartesian: Sec. 5.1) */
enum { KT_BC_COPY = 0, KT_BC_PERIODIC = 1 };          /* ghost cells: Eqs. ghostCells_1/2 or periodic */
enum { KT_FP64 = 0, KT_MIXED = 1 };                   /* precision mode */
enum { KT_STORE_FP64 = 0, KT_STORE_PI_FP32 = 1 };     /* KT_MIXED storage of pi, Pi (kt_options.pi_storage) */
enum { KT_INV_PLAIN = 0, KT_INV_LEARNED = 1, KT_INV_CONFORMAL = 2 };  /* inversion start: previous e, MLP, conformal root */
enum { KT_IFACE_RECON = 0, KT_IFACE_INVERT = 1 };     /* face velocities (see kt_options.iface) */
enum { KT_EOS_CONFORMAL = 0, KT_EOS_TABLE = 1 };
enum { KT_COEF_CONST = 0, KT_COEF_GAUSS = 1, KT_COEF_PAPER_ZETA = 2 };

typedef struct {
  int nx, ny, neta; /* physical cells per axis, each >= 1 */
} kt_grid;

/* Equation of state (Sec. 2.3).
 * KT_EOS_CONFORMAL: e = a T^4, P0 = e/3, c_s^2 = 1/3.
 * KT_EOS_TABLE: n >= 4 nodes, e strictly increasing (fm^-4); P0 (fm^-4), c_s^2 = dP0/de,
 *   T (fm^-1), lndelta = ln(1/3 - c_s^2) per node.  Interpolation: piecewise cubic Hermite in
 *   e with slopes dP0/de = c_s^2 and dT/de = c_s^2 T/(e+P0); c_s^2 between nodes is the
 *   derivative of the P0 interpolant; lndelta is linear in e.  Copied at kt_init. */
typedef struct {
  int kind;
  double a;
  int n;
  const double *e, *p, *cs2, *T, *lndelta;
} kt_eos;

/* Specific viscosity eta/s or zeta/s as a function of T (fm^-1):
 * KT_COEF_CONST: c0;  KT_COEF_GAUSS: c0 exp(-((T - c1)/c2)^2);
 * KT_COEF_PAPER_ZETA: c0 times the zeta/s parametrisation of Sec. 2.2, Eq. (zetas), with
 *   x = T/T_c, T_c = c1 (the paper uses 200 MeV): a quadratic for 0.995 <= x <= 1.05 and
 *   exponential tails above (-> 0.001) and below (-> 0.03).
 * KT_COEF_CONST with c0 = 0 switches the channel off (pi == 0 or Pi == 0). */
typedef struct {
  int kind;
  double c0, c1, c2;
} kt_coef;

typedef struct {
  double theta_limiter;  /* generalised minmod parameter in [1, 2] (Sec. 3.1); default 1 */
  int coords;            /* KT_MILNE (default) or KT_CARTESIAN */
  int bc;                /* KT_BC_COPY (default) or KT_BC_PERIODIC */
  int precision;         /* KT_FP64 (default) or KT_MIXED: FP32 stencil/sources, FP64 Heun + inversion */
  int inversion;         /* KT_INV_PLAIN (default), KT_INV_LEARNED or KT_INV_CONFORMAL (both KT_MIXED
                            only; see the learned root-find start below) */
  int tau_pipi_on;       /* 1 (default): tau_pipi/tau_pi = 10/7; 0: tau_pipi = 0 */
  int regulate;          /* 1 (default): Eq. (regPimunu) after every inversion */
  double rho_max, xi0;   /* regulator parameters of Eq. (rho); defaults 1 and 0.1 */
  double e_min;          /* the inversion clamps e >= e_min (fm^-4); default 0 */
  double tau_relax_min;  /* floor on tau_pi and tau_Pi (fm); default 0 (no floor) */
  void* stream;          /* cudaStream_t for all work; NULL = a stream owned by the context */
  void* arena;           /* optional caller-owned device memory for the state; NULL = cudaMalloc */
  size_t arena_bytes;    /* its size, at least kt_state_bytes() */
  const float* mlp_weights; /* KT_INV_LEARNED: host pointer to KT_MLP_NPARAM floats (see below) */
  int use_graph;         /* 1 (default): kt_step replays a captured CUDA graph of the step loop */
  int autotune;          /* 1 (default): the first kt_step times the candidate tile shapes and grid
                            sizes (side-effect-free first-stage launches) and keeps the fastest;
                            0: 32 x 4 x 2 tiles on a persistent grid */
  int iface;             /* velocities v^+- at the cell faces (Sec. 3.1).  KT_IFACE_RECON (default):
                            u^mu extrapolated to the faces with the same generalised minmod as q.
                            KT_IFACE_INVERT: the extrapolated conserved states q^+- themselves are
                            inverted (Eq. eInferred), 12 root-finds per cell and stage, each started
                            from the e of the cell the state was extrapolated from; a state with no
                            root gets v = 0.  FP64 root-finds in KT_FP64, FP32 in KT_MIXED. */
  int pi_storage;        /* KT_MIXED only.  KT_STORE_FP64 (default): all 15 components of q (Eq.
                            qComponents) are stored and Heun-summed in FP64.  KT_STORE_PI_FP32: only
                            T^{tau mu} is; pi^{mu nu} and Pi -- the dissipative quantities the scheme
                            promotes to conserved variables (Sec. 3.1) -- are stored and summed in FP32
                            (the storage variant of Sec. 4.2's remark on memory).  The inversion and
                            the T^{tau mu} accumulation stay FP64 either way. */
} kt_options;

/* Learned inversion start: an MLP 6 -> 32 -> 32 -> 1 with ReLU; weights row-major
 * W1[32][6], b1[32], W2[32][32], b2[32], W3[32], b3[1]. */
#define KT_MLP_NPARAM (32 * 6 + 32 + 32 * 32 + 32 + 32 + 1)

typedef struct {
  double tau;            /* current proper time */
  long long steps;       /* steps taken since kt_set_state */
  float max_speed;       /* max local propagation speed a (Eq. ax) seen in the last step, times the
                            direction's metric factor (tau for eta): a CFL diagnostic */
  unsigned int status;   /* OR of status bits of the last kt_step: 1 inversion, 2 non-finite, 4 copy timeout */
  long long newton_iters;/* total Newton iterations in the last kt_step (all cells, both stages) */
  long long fallbacks;   /* learned mode: cells that fell back to the plain root-find */
  long long regulated;   /* cells whose pi was scaled by a factor < 0.999 in the last kt_step */
  /* of the current state, over every event's physical cells (reduced on the device when
   * kt_get_stats is called; 0 before any state is set): */
  double e_min, e_max;   /* smallest and largest energy density (fm^-4, in the stored precision) */
  double reg_min;        /* smallest regulation factor tanh(rho)/rho applied to pi in the last step */
} kt_stats;

typedef struct kt_ctx kt_ctx;

/* Fill *opt with the defaults listed above.  Returns KT_OK or KT_ERR_ARG. */
int kt_options_default(kt_options* opt);

/* Device bytes the state of one grid needs with this EOS and these options (the size of a
 * caller-provided kt_options.arena).  eos may be NULL for the conformal EOS; a table of n nodes
 * adds its per-interval coefficients.  Returns KT_ERR_ARG for a bad grid or null bytes,
 * KT_ERR_EOS for a table with fewer than 4 nodes. */
int kt_state_bytes(const kt_grid* grid, const kt_eos* eos, const kt_options* opt, size_t* bytes);

/* Create a context (Sec. 4.3 step 2, memory allocation).  dx is used for x and y.
 * eos, eta_over_s, zeta_over_s: problem definition of Secs. 2.2-2.3 (copied).  opt may be NULL. */
int kt_init(kt_ctx** out, const kt_grid* grid, double dx, double deta, double dtau, const kt_eos* eos,
            const kt_coef* eta_over_s, const kt_coef* zeta_over_s, const kt_options* opt);

/* Set the state at proper time tau from primaries (Sec. 4.3 steps 3-5): the conserved
 * variables are formed with Eqs. (Ttt), (Tti), ghost cells are filled.
 *   e:      [cells] energy density (required)
 *   u:      [3][cells] u^x, u^y, u^eta (NULL = fluid at rest); u^tau from u.u = 1
 *   pi:     [10][cells] pi^{tt,tx,ty,tn,xx,xy,xn,yy,yn,nn} (NULL = 0)
 *   Pi:     [cells] bulk pressure (NULL = 0)
 *   u_prev: [3][cells] u at tau - dtau for the first backward time difference (NULL = u,
 *           i.e. u^{-1} = u^0 as in Sec. 4.3)
 * on_device: 0 = host pointers, 1 = device pointers.  Returns KT_ERR_STATE for non-finite
 * inputs, e < 0, or a cell whose E = T^{tau tau} - pi^{tau tau} and M^i = T^{tau i} - pi^{tau i}
 * admit no inversion (E <= 0 or M^2 >= E^2, Sec. 2.4); the context then has no valid state. */
int kt_set_state(kt_ctx* ctx, double tau, const double* e, const double* u, const double* pi,
                 const double* Pi, const double* u_prev, int on_device);

/* Advance n_steps full Heun steps (Eqs. step1-finalStep; Sec. 4.3 steps 1-9), each two fused
 * stage launches.  Asynchronous on the context's stream; it synchronises once at the end to
 * read the status word.  Returns KT_ERR_INVERSION / KT_ERR_NONFINITE if any cell failed. */
int kt_step(kt_ctx* ctx, int n_steps);

/* Copy the state out (physical cells).  Any output may be NULL.
 *   e [cells], u [4][cells] (u^tau, u^x, u^y, u^eta), pi [10][cells], Pi [cells],
 *   q [15][cells] conserved variables of Eq. (qComponents). */
int kt_get_state(kt_ctx* ctx, double* tau, double* e, double* u, double* pi, double* Pi, double* q,
                 int on_device);

/* Checkpoint and restart (Sec. 4.3: the program writes the state out every m steps; the run can
 * continue from it).  A checkpoint is the complete evolved state of one event, so that
 *   n steps  ==  k steps, kt_get_checkpoint, kt_set_checkpoint (in this or a new context with the
 *                same options), n - k steps
 * bit for bit.  (Primaries alone do not determine q: the regulator of Eq. regPimunu rescales pi
 * after the inversion without re-inverting.)  buf = [KT_CHECKPOINT_ROWS][cells] doubles, layout
 * as kt_get_state, rows:
 *    0-14  q, the conserved variables of Eq. (qComponents) (FP64)
 *   15-29  the copy of q the stencil reads (KT_MIXED: its FP32 values, widened exactly; KT_FP64:
 *          q again, ignored by kt_set_checkpoint)
 *   30     e     31  P0(e)     32-35  u^mu (u^tau, u^x, u^y, u^eta)     36-39  u^mu one step earlier
 *   40     the regulation factor applied in the last step (the diagnostics' last column)
 * kt_get_checkpoint writes buf (host, or device if on_device) and *tau (may be NULL).
 * kt_set_checkpoint reads it (rows stored in FP32 in KT_MIXED are rounded to nearest, which is
 * exact for values that kt_get_checkpoint produced), fills the ghost cells, sets tau for the
 * context and resets the step count and statistics; KT_ERR_ARG for a bad event, a null buffer or
 * tau <= 0 in Milne coordinates.  The caller owns buf. */
#define KT_CHECKPOINT_ROWS 41
int kt_get_checkpoint(kt_ctx* ctx, int event, double* tau, double* buf, int on_device);
int kt_set_checkpoint(kt_ctx* ctx, int event, double tau, const double* buf, int on_device);

/* Validity diagnostics of Sec. 7 (Eqs. inverseReynoldsNumbers, inverseReynoldsNumbers2) at the
 * current state of an event, out = [7][cells] (layout as kt_get_state; host pointer, or device
 * pointer if on_device):
 *   0  Kn_theta_pi = tau_pi theta          1  Kn_theta_Pi = tau_Pi theta
 *   2  R_pi^-1 = sqrt(pi^{mu nu} pi_{mu nu}) / P0      3  R_Pi^-1 = |Pi| / P0
 *   4  (R_pi^(2))^-1 = sqrt(J^{mu nu} J_{mu nu}) / (2 eta sqrt(sigma^{mu nu} sigma_{mu nu}))
 *   5  (R_Pi^(2))^-1 = |J| / (zeta |theta|)
 *   6  the regulation factor tanh(rho)/rho of Eq. (regPimunu) applied to pi in the last step
 *      (1 before the first step or with the regulator off)
 * with J^{mu nu}, J the second-order terms of Eq. (14_moment_terms) (no diffusion), the
 * unfloored relaxation times tau_pi = 5 (eta/s)/T and tau_Pi = (zeta/s)/(15 (1/3 - c_s^2)^2 T),
 * and the time derivative of u taken backward over the last step, as in the first stage.  A
 * quantity whose channel is off, or whose denominator vanishes, is 0.  Computed by one extra
 * kernel over the event (stencil precision of the context). */
int kt_get_diagnostics(kt_ctx* ctx, int event, double* out, int on_device);

/* Self-test of failure detection (the paper has no counterpart): one block waits, with at most
 * `polls` polls, on an mbarrier that nothing arms -- the bounded wait the stage kernels use for
 * their shared-memory copies -- and reports the timeout through the status word instead of
 * hanging.  Returns KT_ERR_TIMEOUT (the expected outcome), KT_ERR_ARG for polls = 0, or a CUDA
 * error.  The context stays usable. */
int kt_selftest_wait(kt_ctx* ctx, unsigned polls);

/* Self-test of the FP64 division the stencil uses for face velocities and coefficients (the paper
 * has no counterpart): q[i] = a[i] / b[i] for n device-resident operands, on `stream`.  For
 * 2^-125 <= b < 2^125 it is a Newton-Raphson reciprocal from a single-precision seed with one
 * quotient correction, accurate to one unit in the last place where the quotient is a normal
 * double; other b take the IEEE division.  KT_ERR_ARG for null pointers or n < 0. */
int kt_selftest_div(const double* a, const double* b, double* q, long long n, void* stream);

/* Self-test of the double -> float conversions the mixed-precision kernels do with integer
 * instructions (the paper has no counterpart): for n device-resident x, rn[i] is x[i] rounded to
 * nearest even (the stored FP32 copies), rz[i] x[i] with its mantissa truncated (values that only
 * steer a computation).  Both flush magnitudes below 2^-126 to zero; rn gives infinity for
 * overflow, infinity and NaN; rz assumes |x| < 2^128.  KT_ERR_ARG for null pointers or n < 0. */
int kt_selftest_cvt(const double* x, float* rn, float* rz, long long n, void* stream);

int kt_get_stats(kt_ctx* ctx, kt_stats* stats);
const char* kt_last_error(const kt_ctx* ctx);
void kt_free(kt_ctx* ctx);

/* ------------------------------------------------------------------ batches of events
 * Many independent events (fluctuating initial conditions, uneven grids) share one context:
 * every field array holds all events, each event's padded lattice at its own offset, and one
 * persistent launch per Runge-Kutta stage walks a table of (event, tile) work items.  All
 * events share the physics parameters, dtau and tau.  kt_init is kt_init_batch with one event;
 * kt_set_state / kt_get_state address event 0.  kt_step advances every event; each event must
 * have been given a state first.  The results of an event do not depend on the batch it is in. */
int kt_state_bytes_batch(int n_events, const kt_grid* grids, const kt_eos* eos, const kt_options* opt,
                         size_t* bytes);
int kt_init_batch(kt_ctx** out, int n_events, const kt_grid* grids, double dx, double deta, double dtau,
                  const kt_eos* eos, const kt_coef* eta_over_s, const kt_coef* zeta_over_s, const kt_options* opt);
int kt_set_state_event(kt_ctx* ctx, int event, double tau, const double* e, const double* u, const double* pi,
                       const double* Pi, const double* u_prev, int on_device);
int kt_get_state_event(kt_ctx* ctx, int event, double* tau, double* e, double* u, double* pi, double* Pi, double* q,
                       int on_device);
/* The tile shape in use (threads per block x, y, z), the grid size in blocks and, after
 * autotuning, the measured first-stage time in ms of each candidate (up to *n_candidates
 * entries; *n_candidates is set to the number of candidates, 36; candidates not timed report 0).
 * Candidate 12 v + 2 s + g is tile shape s of (32,4,2), (32,8,1), (32,2,4), (32,1,8), (32,4,1),
 * (32,2,2) with g = 0 a persistent grid (as many blocks as are resident at once, each walking the
 * tile table) or g = 1 one block per tile, and, for KT_MIXED with FP64 pi storage, the variant v:
 * 0 a right-hand-side and an update launch per stage; 1 the same with the update kernels' inputs
 * staged in shared memory by TMA bulk copies of each tile (double-buffered on a persistent grid);
 * 2 (face velocities by reconstruction) one fused launch per stage, right-hand side and update.
 * The autotuner times the candidates with v = 0 and, where v = 2 applies, v = 2 (v = 1 measured
 * slower over a whole step); kt_set_tuning selects any.  v = 1 applies to KT_MIXED with FP64 pi
 * storage, v = 2 also needs KT_IFACE_RECON; elsewhere (the FP64 mode, FP32 pi storage) the v = 0
 * layout runs whatever v is asked for. */
int kt_get_tuning(kt_ctx* ctx, int* block_xyz, int* grid_blocks, float* candidate_ms, int* n_candidates);
/* Use candidate `candidate` (numbered as above) from now on, without autotuning; KT_ERR_ARG if it
 * is out of range.  The results do not depend on the candidate: every candidate runs the same
 * kernels on the same tiles. */
int kt_set_tuning(kt_ctx* ctx, int candidate);

/* Measurement (the paper has no counterpart): advance n_steps >= 1 steps exactly as kt_step does
 * but launch by launch, without the CUDA graph, with CUDA events on the context's stream between
 * the launches, and return in ms[0..5] the average duration per step of: the learned start's
 * network launch (0 without KT_INV_LEARNED), the stage-1 right-hand-side launch (FP64, fused
 * layout: the fused stage-1 launch), the stage-1 update launch (FP64, fused layout: 0), the
 * stage-2 right-hand-side launch (FP64, fused layout: the fused stage-2 launch), the stage-2
 * update launch (FP64, fused layout: 0) and the tau advance.  *n_kernels must be >= 6 on entry
 * and is set to 6.  The state, tau and statistics advance as with kt_step; errors are those of
 * kt_step.  The per-step event synchronisation makes these steps slower in total than kt_step's. */
int kt_time_kernels(kt_ctx* ctx, int n_steps, float* ms, int* n_kernels);

/* ------------------------------------------------------------------ learned root-find start
 * The paper solves Eq. (eInferred) by Newton-Raphson (Sec. 3.2) and states no starting point.
 * KT_INV_LEARNED starts it from a small network: features (computed by the library from
 * E = T^tt - pi^tt, M^2 = Mx^2 + My^2 + tau^2 Meta^2 and Pi):
 *   x = [(ln E - 1)/6, M^2/E^2, 5 Pi/E, ln(1 - M^2/E^2)/2, e_conf/E, |M|/E],
 * e_conf = sqrt(4E^2 - 3M^2) - E the conformal root; output z, start e = e_conf exp(y/10) with
 * y = (M^2/E^2) z where M^2/E^2 > KT_MLP_GATE_R2, else y = 0 (the correction vanishes at rest,
 * where e_conf = E is the root).  The network runs once per cell and step, in a launch of its
 * own before the first Runge-Kutta stage, on the state at the start of the step (its single-
 * precision copy); both stages apply that z to their own E, M^2 and Pi.
 * At most 2 FP64 Newton steps follow; a cell whose residual |f(e)|/E then exceeds 1e-10 falls
 * back to the plain root-find (the test uses 0.99e-10, formed in single precision, so that every
 * accepted root meets 1e-10 exactly).  Parameters: KT_MLP_NPARAM floats, layout as documented above
 * KT_MLP_NPARAM.  KT_INV_CONFORMAL is the same start without the network (y = 0: e = e_conf,
 * the closed-form root of the conformal EOS, Sec. 2.4) and the same Newton steps and fallback:
 * the ablation that shows what the network adds; it needs no weights.  (It gives the state of
 * KT_INV_LEARNED with all-zero weights bit for bit, without the inference.)
 * All pointers below are device pointers; work goes to `stream`. */
#define KT_MLP_PACKED_BYTES 3396 /* scratch of kt_mlp_predict: packed BF16 weights + FP32 biases */
#define KT_MLP_GATE_R2 1e-3      /* M^2/E^2 above which the network's correction is applied */

/* Training samples from the context's current state: for n physical cells (packed indices
 * i + nx*(j + ny*k), device int64 array `cells`), write the features x [n][6] (float), the
 * target y = 10 ln(e/e_conf) (float) and the exact root e (double, plain FP64 root-find). */
int kt_mlp_features(kt_ctx* ctx, long long n, const long long* cells, float* x, float* y, double* e_exact);

/* Inference on tensor cores (mma.sync BF16, FP32 accumulation) for n feature rows x [n][6]
 * -> y [n].  scratch: caller-owned device memory of at least KT_MLP_PACKED_BYTES that receives
 * the packed weights (overwritten; calls that share it must not overlap). */
int kt_mlp_predict(const float* params, const float* x, long long n, float* y, void* scratch, size_t scratch_bytes,
                   void* stream);

/* Same inference as kt_mlp_predict without a caller-provided scratch buffer and without any
 * device allocation.  (The paper has no counterpart: this serves callers that cannot call
 * cudaMalloc, for example code whose device memory is budgeted up front by a host
 * application or a custom allocator, or latency-critical loops where an allocation and the
 * synchronisation it may imply are not acceptable.)  The packed weights go to a file-scope
 * device array of KT_MLP_PACKED_BYTES bytes that every GPU loading the library holds until
 * the process exits.  The first call on a device looks up that array's device address with
 * cudaGetSymbolAddress (the current device must be the one the pointers live on), and so does
 * the first call after the device's context has been re-created (cudaDeviceReset); make that
 * first call before any stream capture.  All calls on a device share the array and it keeps
 * the last call's contents; each call overwrites all of it before use, so nothing needs
 * clearing, but calls that overlap on the GPU (other streams, other host threads) race on it.
 * n is limited to KT_MLP_STATIC_MAX_ROWS rows; larger n, negative n or null pointers return
 * KT_ERR_ARG with a message on stderr. */
#define KT_MLP_STATIC_MAX_ROWS 2147483647LL
int kt_mlp_predict_static(const float* params, const float* x, long long n, float* y, void* stream);

/* Gradient of the mean squared error over n samples with respect to the KT_MLP_NPARAM
 * parameters: grad [KT_MLP_NPARAM] and loss [1] are overwritten.  bf16_forward = 1 rounds
 * weights and activations to BF16 in the forward pass as the tensor-core inference does;
 * 0 runs it in FP32. */
int kt_mlp_grad(const float* params, const float* x, const float* y_target, long long n, int bf16_forward,
                float* grad, float* loss, void* stream);

/* The network's training set from samples of kt_mlp_features (the paper has no counterpart):
 * of the n rows x [n][6], y [n] (device), keep in their order those the network corrects, feature
 * 1 (M^2/E^2) above KT_MLP_GATE_R2, writing their features to x_out [*n_out][6] and the target
 * z = y / (M^2/E^2) (IEEE division) to z_out; *n_out is a device int64.  x_out and z_out need
 * room for n rows.  workspace: caller-owned device memory of kt_mlp_targets_workspace(n) bytes.
 * Asynchronous on `stream`; KT_ERR_ARG for null pointers, n < 0 or a small workspace. */
int kt_mlp_targets_workspace(long long n, size_t* bytes);
int kt_mlp_targets(const float* x, const float* y, long long n, float* x_out, float* z_out, long long* n_out,
                   void* workspace, size_t workspace_bytes, void* stream);

/* Mini-batch b (>= 0) of epoch `epoch` of a shuffled pass over n training rows (device x [n][6],
 * y [n]): rows p(b batch + i), i < count = min(batch, n - b batch), into xb [count][6], yb [count],
 * where p is a pseudo-random permutation of [0, n) keyed by (seed, epoch) -- a 4-round Feistel
 * network on the smallest 4^h >= n with cycle walking -- so that the batches of an epoch cover
 * every row exactly once.  *flag (device) gets bit 1 if a walk exceeded its bound (not expected;
 * that row is then taken unpermuted).  KT_ERR_ARG for null pointers, n <= 0, batch <= 0 or
 * b batch >= n. */
int kt_mlp_batch(const float* x, const float* y, long long n, unsigned long long seed, int epoch, long long b,
                 long long batch, float* xb, float* yb, unsigned* flag, void* stream);

/* One Adam step (beta1 0.9, beta2 0.999, eps 1e-8) at step number `step` >= 1; m, v are the
 * caller's moment buffers of KT_MLP_NPARAM floats (zero before the first step). */
int kt_mlp_adam(float* params, const float* grad, float* m, float* v, int step, float lr, void* stream);

#ifdef __cplusplus
}
#endif
#endif
