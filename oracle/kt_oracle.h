/*
 * kt_oracle.h -- plain FP64 CPU oracle for the Kurganov-Tadmor (KT) + Heun step of
 * 3+1d relativistic viscous hydrodynamics (Bazow, Heinz, Strickland, arXiv:1608.06577).
 *
 * TEST INFRASTRUCTURE ONLY.  This library checks the CUDA path: only the test suite,
 * the package's smoke check and the benchmark's CPU-baseline leg may load it.  It shares
 * no code, header, table generator or constant with the CUDA path.
 *
 * Units: hbar = c = 1, lengths in fm.  e, P, pi^{mu nu}, Pi in fm^-4; T in fm^-1.
 * Layout: every field is a padded structure-of-arrays, (nx+4)(ny+4)(neta+4) cells,
 * x fastest, eta slowest, 2 ghost layers per side (Sec. 4.1-4.2).
 */
#ifndef KT_ORACLE_H
#define KT_ORACLE_H
#ifdef __cplusplus
extern "C" {
#endif

enum { KO_MILNE = 0, KO_CARTESIAN = 1 };
enum { KO_BC_COPY = 0, KO_BC_PERIODIC = 1 };
enum { KO_EOS_CONFORMAL = 0, KO_EOS_TABLE = 1 };
enum { KO_COEF_CONST = 0, KO_COEF_GAUSS = 1, KO_COEF_PAPER_ZETA = 2 };
enum { KO_IFACE_RECON = 0, KO_IFACE_INVERT = 1 };

/* status bits OR-ed over all cells of a step */
enum { KO_ST_INVERSION = 1, KO_ST_NONFINITE = 2 };

typedef struct {
  int nx, ny, neta;          /* physical cells */
  double dx, dy, deta, dtau; /* fm, fm, 1, fm */
  int coords;                /* KO_MILNE or KO_CARTESIAN */
  int bc;                    /* KO_BC_COPY or KO_BC_PERIODIC */
  double theta;              /* generalised minmod parameter, 1..2 */
  int eos_kind;
  double eos_a;              /* conformal: e = a T^4 */
  int eos_n;                 /* table: nodes uniform in ln e */
  const double *eos_e, *eos_p, *eos_cs2, *eos_T, *eos_lndelta; /* lndelta = ln(1/3 - cs2) */
  int eta_kind;  double eta_c[3];   /* eta/s(T): c0 or c0*exp(-((T-c1)/c2)^2), T in fm^-1 */
  int zeta_kind; double zeta_c[3];  /* zeta/s(T), same forms, or c0 times Eq. (zetas) with T_c = c1 */
  int tau_pipi_on;           /* 1: tau_pipi/tau_pi = 10/7; 0: tau_pipi = 0 */
  int regulate;              /* 1: apply Eq. (regPimunu) after each inversion */
  double rho_max, xi0;
  double e_min;              /* inversion clamps e >= e_min */
  double tau_relax_min;      /* floor on tau_pi and tau_Pi, fm */
  int iface;                 /* KO_IFACE_RECON or KO_IFACE_INVERT */
} ko_params;

typedef struct ko_ctx ko_ctx;

ko_ctx* ko_create(const ko_params* prm);
void ko_free(ko_ctx* c);
/* physical cells, x fastest.  u = [3][cells] (u^x, u^y, u^eta), pi = [10][cells]
 * (tt,tx,ty,tn,xx,xy,xn,yy,yn,nn), Pi = [cells]; any of u, pi, Pi, u_prev may be NULL. */
int ko_set_state(ko_ctx* c, double tau, const double* e, const double* u, const double* pi,
                 const double* Pi, const double* u_prev);
/* The state given directly as the evolved variables (to restart from another program's state):
 * q = [15][cells] conserved variables, e = [cells] and u = [4][cells] (u^tau, u^x, u^y, u^eta) as
 * produced by the last inversion, u_prev = [4][cells] (NULL = u).  P0 is evaluated from e. */
int ko_set_state_q(ko_ctx* c, double tau, const double* q, const double* e, const double* u,
                   const double* u_prev);
int ko_step(ko_ctx* c, int nsteps);
/* e = [cells], u = [4][cells], pi = [10][cells], Pi = [cells], q = [15][cells]; NULL skips */
int ko_get_state(const ko_ctx* c, double* tau, double* e, double* u, double* pi, double* Pi,
                 double* q);
/* C[q] of Eq. (semiDiscreteKT) for the current state at the current tau (no update). */
int ko_rhs(ko_ctx* c, double* out /* [15][cells] */);
int ko_set_threads(int n);
/* The CFL diagnostic of the last ko_step call: the largest local propagation speed a of
 * Eq. (ax) over every face evaluated in its stages, the eta speeds times tau (Milne). */
double ko_max_speed(const ko_ctx* c);
/* Validity diagnostics of Sec. 7 at the current state, out = [7][cells]: tau_pi theta,
 * tau_Pi theta, sqrt(pi.pi)/P0, |Pi|/P0, the second-order inverse Reynolds numbers of shear and
 * bulk (Eq. inverseReynoldsNumbers2), and the regulation factor of the last step. */
int ko_diagnostics(const ko_ctx* c, double* out);
/* eta/s and zeta/s at temperature T (fm^-1): out[0] = eta/s, out[1] = zeta/s */
void ko_coefficients(const ko_ctx* c, double T, double* out);

/* ---- single-formula entry points used by the oracle's own pin tests ---- */
double ko_minmod3(double x, double y, double z);
/* EOS and transport at energy density e: out = {P0, cs2, T} */
void ko_eos(const ko_ctx* c, double e, double* out);
/* inversion of Eq. (eInferred): returns status; out = {e, P0, ut, ux, uy, un} */
int ko_invert(const ko_ctx* c, double tau, const double* q15, double* out);
/* kinematic tensors of App. A at one point from u^mu and d_alpha u^mu:
 * du[alpha*4+mu] = d_alpha u^mu.  pi16 = pi^{mu nu} (row major).
 * out: theta(1) Du_lower(4) sigma(16) omega(16) I1(16) I3(16) I4(16) Gpi(16) = 101 doubles */
void ko_tensor_terms(const ko_ctx* c, double tau, const double* u4, const double* du16,
                     const double* pi16, double* out);
/* regulator factor tanh(rho)/rho of Eq. (rho) for one cell */
double ko_regulator_factor(const ko_ctx* c, double tau, double e, double P0, const double* u4,
                           const double* pi16, double Pi);

#ifdef __cplusplus
}
#endif
#endif
