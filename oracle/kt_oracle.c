/*
 * kt_oracle.c -- plain, slow FP64 CPU oracle of the KT semi-discrete scheme with Heun (RK2)
 * time stepping for 3+1d viscous hydrodynamics in Milne coordinates, following
 * Bazow, Heinz, Strickland, arXiv:1608.06577.
 *
 * TEST INFRASTRUCTURE ONLY: the tests, the smoke check and the benchmark's CPU-baseline leg
 * may load this library; the product path never does.  It shares no code with the CUDA path.
 *
 * Every step is written in the paper's order and notation, with generic 4x4 tensors, an
 * explicit metric and explicit Christoffel symbols.  Nothing is blocked, fused or reordered
 * beyond what the equations state.  Readings of points the paper leaves open are marked
 * "reading:" in the comments.
 *
 * Passages followed:
 *   conservation laws in Milne form ........ Sec. 2.4, Eqs. (dT001)-(dT03)
 *   T^{tau mu}, T^{ij} from primaries ....... Eqs. (Ttt), (Tti), (Tij)
 *   relaxation equations, I_Pi, I_pi ........ Eqs. (relEqs_Pi), (relEqs), (dPi), (I1)-(I4)
 *   transport coefficients .................. Eqs. (betaPi)-(lambdapiPi)
 *   inversion T^{tau mu} -> (e, u) ........... Eqs. (eInferred), (utInferred), (uiInferred)
 *   flux-conservative form, sources ......... Sec. 3.1, Eq. (qComponents); App. B, Eq. (B13)
 *   KT update, flux, speed, extrapolation ... Eqs. (semiDiscreteKT), (Hflux), (ax), minmod
 *   Heun (s = 2, beta_1 = 1/2) .............. Eqs. (step1)-(finalStep), Sec. 4.3 steps 1-9
 *   derivative rules in sources ............. Sec. 3.1 (central in space, backward in time)
 *   regulator ............................... Sec. 3.2, Eqs. (regPimunu), (rho)
 *   ghost cells ............................. Sec. 4.1, Eqs. (ghostCells_1), (ghostCells_2)
 *   kinematic tensors ....................... App. A (covariant definitions)
 */
#include "kt_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define NQ 15

/* q index of pi^{mu nu}, Eq. (qComponents): (Ttt,Ttx,Tty,Ttn, pitt,pitx,pity,pitn,
 * pixx,pixy,pixn, piyy,piyn, pinn, Pi) */
static const int PIX[4][4] = {{4, 5, 6, 7}, {5, 8, 9, 10}, {6, 9, 11, 12}, {7, 10, 12, 13}};

typedef struct {
  double *q[NQ];
  double *u[4];
  double *e, *p;
} fields_t;

struct ko_ctx {
  ko_params P;
  double *te, *tp, *tcs2, *tT, *tlnd;
  int nt;
  int NX, NY, NZ;
  size_t ncell;
  double tau;
  /* q^n, q^*, Q (= q^{n+1} before the swap) */
  double *q[NQ], *qs[NQ], *Q[NQ];
  /* u^n, u^*, u^{n-1}, u^{n+1} */
  double *u[4], *us[4], *up[4], *un[4];
  double *e, *p, *es, *ps;
  double *reg; /* regulation factor applied to pi^{n+1} in the last step (1 before any step) */
  double *spd; /* per cell, the largest local speed of its two faces in each direction (a stage) */
  double max_speed; /* largest local speed over the steps of the last ko_step call */
};

/* ------------------------------------------------------------------ geometry (Sec. 2.4) */
typedef struct {
  double glo[4], gup[4]; /* diagonal metric g_{mu mu}, g^{mu mu} */
  double G[4][4][4];     /* Gamma^mu_{alpha beta} */
  double gnn;            /* |g_{eta eta}| = tau^2 (Milne) or 1 */
} geom_t;

static void geom_at(const ko_ctx* c, double tau, geom_t* g) {
  memset(g, 0, sizeof(*g));
  double t2 = (c->P.coords == KO_MILNE) ? tau * tau : 1.0;
  g->glo[0] = 1.0; g->glo[1] = -1.0; g->glo[2] = -1.0; g->glo[3] = -t2;
  g->gup[0] = 1.0; g->gup[1] = -1.0; g->gup[2] = -1.0; g->gup[3] = -1.0 / t2;
  g->gnn = t2;
  if (c->P.coords == KO_MILNE) {
    /* the only nonvanishing Christoffel symbols in Milne coordinates */
    g->G[3][0][3] = 1.0 / tau;
    g->G[3][3][0] = 1.0 / tau;
    g->G[0][3][3] = tau;
  }
}

/* ------------------------------------------------------------------ EOS (Sec. 2.3) */
/* reading: the table is piecewise cubic Hermite in e on nodes uniform in ln e; its slopes
 * are dP/de = cs2 and dT/de = cs2 T / (e + P) (thermodynamics with mu = 0).  cs2(e) is the
 * derivative of the P interpolant.  ln(1/3 - cs2) is interpolated linearly. */
static void eos_eval(const ko_ctx* c, double e, double* P0, double* cs2, double* T, double* lnd) {
  if (c->P.eos_kind == KO_EOS_CONFORMAL) {
    *P0 = e / 3.0;
    *cs2 = 1.0 / 3.0;
    *T = pow(e / c->P.eos_a, 0.25);
    *lnd = -INFINITY;
    return;
  }
  const double* te = c->te;
  int n = c->nt;
  int lo = 0, hi = n - 1; /* find i with te[i] <= e < te[i+1], clamped to [0, n-2] */
  if (e <= te[0]) {
    lo = 0;
  } else if (e >= te[n - 1]) {
    lo = n - 2;
  } else {
    while (hi - lo > 1) {
      int mid = (lo + hi) / 2;
      if (te[mid] <= e) lo = mid; else hi = mid;
    }
  }
  if (lo > n - 2) lo = n - 2;
  int i = lo;
  double de = te[i + 1] - te[i];
  double t = (e - te[i]) / de;
  double t2 = t * t, t3 = t2 * t;
  double h00 = 2 * t3 - 3 * t2 + 1, h10 = t3 - 2 * t2 + t, h01 = -2 * t3 + 3 * t2, h11 = t3 - t2;
  double m0 = c->tcs2[i] * de, m1 = c->tcs2[i + 1] * de;
  *P0 = h00 * c->tp[i] + h10 * m0 + h01 * c->tp[i + 1] + h11 * m1;
  double d00 = 6 * t2 - 6 * t, d10 = 3 * t2 - 4 * t + 1, d01 = -6 * t2 + 6 * t, d11 = 3 * t2 - 2 * t;
  *cs2 = (d00 * c->tp[i] + d10 * m0 + d01 * c->tp[i + 1] + d11 * m1) / de;
  double s0 = c->tcs2[i] * c->tT[i] / (te[i] + c->tp[i]) * de;
  double s1 = c->tcs2[i + 1] * c->tT[i + 1] / (te[i + 1] + c->tp[i + 1]) * de;
  *T = h00 * c->tT[i] + h10 * s0 + h01 * c->tT[i + 1] + h11 * s1;
  *lnd = (1.0 - t) * c->tlnd[i] + t * c->tlnd[i + 1];
}

/* ------------------------------------------------------ transport coefficients (Sec. 2.2) */
typedef struct {
  int shear_on, bulk_on;
  double eta_over_taupi; /* eta/tau_pi = (e+P0)/5 */
  double rate_pi;        /* 1/tau_pi with tau_pi = 5 (eta/s)/T, floored */
  double zeta_over_tauPi;/* 15 (1/3 - cs2)^2 (e + P0) */
  double rate_Pi;        /* 1/tau_Pi = 15 (1/3-cs2)^2 T / (zeta/s), floored */
  double lam_Pipi;       /* lambda_{Pi pi}/tau_Pi = 8/5 (1/3 - cs2) */
} transport_t;

/* zeta/s of Sec. 2.2, Eq. (zetas), as a function of x = T/T_c: a quadratic around T_c joined to
 * two exponential tails; the printed domain of the quadratic, "0.995 T_c >= T >= 1.05 T_c", is read
 * as 0.995 T_c <= T <= 1.05 T_c (the other two branches cover T > 1.05 T_c and T < 0.995 T_c) */
static double zeta_over_s_paper(double x) {
  if (x > 1.05) return 0.9 * exp(-(x - 1.0) / 0.025) + 0.25 * exp(-(x - 1.0) / 0.13) + 0.001;
  if (x < 0.995) return 0.9 * exp((x - 1.0) / 0.0025) + 0.22 * exp((x - 1.0) / 0.022) + 0.03;
  return -13.45 + 27.55 * x - 13.77 * x * x;
}

static double coef_value(int kind, const double* cc, double T) {
  if (kind == KO_COEF_CONST) return cc[0];
  if (kind == KO_COEF_PAPER_ZETA) return cc[0] * zeta_over_s_paper(T / cc[1]);
  double x = (T - cc[1]) / cc[2];
  return cc[0] * exp(-x * x);
}

static double coef_log(int kind, const double* cc, double T) {
  if (kind == KO_COEF_CONST) return log(cc[0]);
  if (kind == KO_COEF_PAPER_ZETA) return log(coef_value(kind, cc, T));
  double x = (T - cc[1]) / cc[2];
  return log(cc[0]) - x * x;
}

void ko_coefficients(const ko_ctx* c, double T, double* out) {
  out[0] = coef_value(c->P.eta_kind, c->P.eta_c, T);
  out[1] = coef_value(c->P.zeta_kind, c->P.zeta_c, T);
}

static void transport(const ko_ctx* c, double e, double P0, double T, double lnd, transport_t* tr) {
  const ko_params* P = &c->P;
  tr->shear_on = !(P->eta_kind == KO_COEF_CONST && P->eta_c[0] == 0.0);
  tr->bulk_on = !(P->zeta_kind == KO_COEF_CONST && P->zeta_c[0] == 0.0) && P->eos_kind == KO_EOS_TABLE;
  double rmax = (P->tau_relax_min > 0.0) ? 1.0 / P->tau_relax_min : INFINITY;
  tr->eta_over_taupi = (e + P0) / 5.0;
  double es = coef_value(P->eta_kind, P->eta_c, T);
  double rpi = (es > 0.0) ? T / (5.0 * es) : INFINITY;
  tr->rate_pi = (rpi < rmax) ? rpi : rmax;
  /* reading: 1/tau_Pi is formed in logarithms so that a vanishing (1/3 - cs2) and a vanishing
   * zeta/s give a finite, floored rate */
  double lrate = log(15.0) + 2.0 * lnd + log(T) - coef_log(P->zeta_kind, P->zeta_c, T);
  double rPi = exp(lrate);
  tr->rate_Pi = (rPi < rmax) ? rPi : rmax;
  double d = exp(lnd);
  tr->zeta_over_tauPi = 15.0 * d * d * (e + P0);
  tr->lam_Pipi = 1.6 * d;
}

/* ------------------------------------------------------------------ minmod (Sec. 3.1) */
static double sgn(double x) { return (x > 0.0) ? 1.0 : ((x < 0.0) ? -1.0 : 0.0); } /* sgn(0)=0 */
static double minmod2(double x, double y) {
  double ax = fabs(x), ay = fabs(y);
  return (sgn(x) + sgn(y)) * ((ax < ay) ? ax : ay) / 2.0;
}
double ko_minmod3(double x, double y, double z) { return minmod2(x, minmod2(y, z)); }

/* (q_d)_i = minmod(theta (q_i - q_{i-1})/D, (q_{i+1} - q_{i-1})/(2D), theta (q_{i+1} - q_i)/D) */
static double slope(const double* A, size_t i, size_t s, double D, double th) {
  return ko_minmod3(th * (A[i] - A[i - s]) / D, (A[i + s] - A[i - s]) / (2.0 * D),
                    th * (A[i + s] - A[i]) / D);
}

/* ------------------------------------------------------------------ inversion (Sec. 2.4) */
static int invert_core(const ko_ctx* c, double tau, const double* q, double e0, double* out) {
  geom_t g;
  geom_at(c, tau, &g);
  double E = q[0] - q[4];
  double Mx = q[1] - q[5], My = q[2] - q[6], Mn = q[3] - q[7];
  double Pi = q[14];
  double M2 = Mx * Mx + My * My + g.gnn * Mn * Mn;
  double P0, cs2, T, lnd, e;
  int st = 0;
  int bulk = !(c->P.zeta_kind == KO_COEF_CONST && c->P.zeta_c[0] == 0.0) && c->P.eos_kind == KO_EOS_TABLE;
  if (!(E > 0.0) || !isfinite(E) || !isfinite(M2) || !(M2 < E * E)) {
    st = KO_ST_INVERSION;
    e = (c->P.e_min > 0.0) ? c->P.e_min : 1e-30;
  } else if (c->P.eos_kind == KO_EOS_CONFORMAL && (!bulk || Pi == 0.0)) {
    /* conformal closed form e = sqrt(4E^2 - 3M^2) - E, written without cancellation */
    double M = sqrt(M2);
    e = 3.0 * (E - M) * (E + M) / (sqrt(4.0 * E * E - 3.0 * M2) + E);
  } else {
    /* f(e) = e - E + M^2/(E + P0(e) + Pi) = 0, Newton-Raphson (Sec. 3.2) safeguarded by a
     * bisection bracket [lo, hi] with f(lo) <= 0 <= f(hi). */
    double lo = (c->P.e_min > 0.0) ? c->P.e_min : 1e-300, hi = E;
    eos_eval(c, lo, &P0, &cs2, &T, &lnd);
    double flo = lo - E + M2 / (E + P0 + Pi);
    eos_eval(c, hi, &P0, &cs2, &T, &lnd);
    double fhi = hi - E + M2 / (E + P0 + Pi);
    if (!(flo <= 0.0) || !(fhi >= 0.0)) {
      st = KO_ST_INVERSION;
      e = (flo > 0.0) ? lo : hi;
    } else {
      /* start: the cell's previous e if it lies in the bracket, else E */
      e = (e0 >= lo && e0 <= hi) ? e0 : hi;
      int it;
      for (it = 0; it < 200; ++it) {
        eos_eval(c, e, &P0, &cs2, &T, &lnd);
        double A = E + P0 + Pi;
        double f = e - E + M2 / A;
        if (f == 0.0) break;
        if (f < 0.0) lo = e; else hi = e;
        double fp = 1.0 - M2 * cs2 / (A * A);
        double en = e - f / fp;
        if (!(en >= lo && en <= hi)) en = 0.5 * (lo + hi); /* bisect when Newton leaves the bracket */
        double de = fabs(en - e);
        e = en;
        /* f is known to about one ulp of E, so the root is resolved to that level */
        if (de <= ldexp(E, -50)) break;
      }
      if (it >= 200) st = KO_ST_INVERSION;
    }
  }
  if (e < c->P.e_min) e = c->P.e_min;
  eos_eval(c, e, &P0, &cs2, &T, &lnd);
  double Ptot = P0 + Pi;
  double ut, ux, uy, un;
  if (st) {
    ut = 1.0; ux = uy = un = 0.0;
  } else {
    ut = sqrt((E + Ptot) / (e + Ptot));
    double w = (e + Ptot) * ut;
    ux = Mx / w; uy = My / w; un = Mn / w;
  }
  out[0] = e; out[1] = P0; out[2] = ut; out[3] = ux; out[4] = uy; out[5] = un;
  if (!isfinite(e) || !isfinite(ut) || !isfinite(ux) || !isfinite(uy) || !isfinite(un)) st |= KO_ST_NONFINITE;
  return st;
}

int ko_invert(const ko_ctx* c, double tau, const double* q15, double* out) {
  return invert_core(c, tau, q15, -1.0, out);
}

void ko_eos(const ko_ctx* c, double e, double* out) {
  double lnd;
  eos_eval(c, e, &out[0], &out[1], &out[2], &lnd);
}

/* ---------------------------------------------------------- kinematic tensors (App. A) */
typedef struct {
  double theta, Du_lo[4];
  double sigma[4][4], omega[4][4], I1[4][4], I3[4][4], I4[4][4], Gpi[4][4];
  double pisig;
} tens_t;

/* du[alpha][mu] = d_alpha u^mu; pi[mu][nu] = pi^{mu nu} */
static void tensor_terms(const geom_t* g, const double* u, double du[4][4], double pi[4][4], tens_t* t) {
  double cov[4][4]; /* cov[mu][alpha] = u^mu_{;alpha} = d_alpha u^mu + Gamma^mu_{alpha beta} u^beta */
  for (int mu = 0; mu < 4; ++mu)
    for (int al = 0; al < 4; ++al) {
      double s = du[al][mu];
      for (int be = 0; be < 4; ++be) s += g->G[mu][al][be] * u[be];
      cov[mu][al] = s;
    }
  /* theta = u^mu_{;mu} */
  t->theta = cov[0][0] + cov[1][1] + cov[2][2] + cov[3][3];
  /* D u^mu = u^alpha u^mu_{;alpha}; lowered with the metric */
  for (int mu = 0; mu < 4; ++mu) {
    double s = 0.0;
    for (int al = 0; al < 4; ++al) s += u[al] * cov[mu][al];
    t->Du_lo[mu] = g->glo[mu] * s;
  }
  double D[4][4]; /* Delta^{mu nu} = g^{mu nu} - u^mu u^nu */
  for (int mu = 0; mu < 4; ++mu)
    for (int nu = 0; nu < 4; ++nu) D[mu][nu] = ((mu == nu) ? g->gup[mu] : 0.0) - u[mu] * u[nu];
  double nab[4][4]; /* nab[alpha][mu] = nabla^alpha u^mu = Delta^{alpha beta} u^mu_{;beta} */
  for (int al = 0; al < 4; ++al)
    for (int mu = 0; mu < 4; ++mu) {
      double s = 0.0;
      for (int be = 0; be < 4; ++be) s += D[al][be] * cov[mu][be];
      nab[al][mu] = s;
    }
  /* sigma^{mu nu} = (nabla^mu u^nu + nabla^nu u^mu)/2 - theta/3 Delta^{mu nu} */
  for (int mu = 0; mu < 4; ++mu)
    for (int nu = 0; nu < 4; ++nu)
      t->sigma[mu][nu] = 0.5 * (nab[mu][nu] + nab[nu][mu]) - t->theta / 3.0 * D[mu][nu];
  /* reading: omega^{mu nu} = (1/2) Delta^{mu a} Delta^{nu b} (u_{a;b} - u_{b;a}) as in App. A,
   * i.e. (nabla^nu u^mu - nabla^mu u^nu)/2, the convention of the App. A component listing */
  for (int mu = 0; mu < 4; ++mu)
    for (int nu = 0; nu < 4; ++nu) t->omega[mu][nu] = 0.5 * (nab[nu][mu] - nab[mu][nu]);
  double om_mix[4][4]; /* omega^mu_lambda = omega^{mu kappa} g_{kappa lambda} */
  for (int mu = 0; mu < 4; ++mu)
    for (int la = 0; la < 4; ++la) om_mix[mu][la] = t->omega[mu][la] * g->glo[la];
  /* I1^{mu nu} = (pi^{lambda mu} u^nu + pi^{lambda nu} u^mu) D u_lambda, Eq. (I1) */
  for (int mu = 0; mu < 4; ++mu)
    for (int nu = 0; nu < 4; ++nu) {
      double s = 0.0;
      for (int la = 0; la < 4; ++la) s += (pi[la][mu] * u[nu] + pi[la][nu] * u[mu]) * t->Du_lo[la];
      t->I1[mu][nu] = s;
    }
  /* I3^{mu nu} = pi^{mu lambda} omega^nu_lambda + pi^{nu lambda} omega^mu_lambda */
  for (int mu = 0; mu < 4; ++mu)
    for (int nu = 0; nu < 4; ++nu) {
      double s = 0.0;
      for (int la = 0; la < 4; ++la) s += pi[mu][la] * om_mix[nu][la] + pi[nu][la] * om_mix[mu][la];
      t->I3[mu][nu] = s;
    }
  /* pi^alpha_beta sigma^beta_alpha = pi^{mu nu} sigma_{mu nu} */
  double ps = 0.0;
  for (int mu = 0; mu < 4; ++mu)
    for (int nu = 0; nu < 4; ++nu) ps += pi[mu][nu] * t->sigma[mu][nu] * g->glo[mu] * g->glo[nu];
  t->pisig = ps;
  /* I4^{mu nu} = (1/2) g_{lambda kappa}(pi^{mu kappa} sigma^{nu lambda} + pi^{nu kappa} sigma^{mu lambda})
   *             - (1/3) Delta^{mu nu} pi^alpha_beta sigma^beta_alpha, Eq. (I4) */
  for (int mu = 0; mu < 4; ++mu)
    for (int nu = 0; nu < 4; ++nu) {
      double s = 0.0;
      for (int la = 0; la < 4; ++la)
        for (int ka = 0; ka < 4; ++ka) {
          double gl = (la == ka) ? g->glo[la] : 0.0;
          s += gl * (pi[mu][ka] * t->sigma[nu][la] + pi[nu][ka] * t->sigma[mu][la]);
        }
      t->I4[mu][nu] = 0.5 * s - D[mu][nu] * ps / 3.0;
    }
  /* geometric term of the conservative form: with G^{mu nu} = u^a Gamma^mu_{ab} pi^{b nu} +
   * u^a Gamma^nu_{ab} pi^{b mu} (Sec. 2.4), the pi rows of App. B receive -G/u^tau */
  for (int mu = 0; mu < 4; ++mu)
    for (int nu = 0; nu < 4; ++nu) {
      double s = 0.0;
      for (int al = 0; al < 4; ++al)
        for (int be = 0; be < 4; ++be)
          s += u[al] * (g->G[mu][al][be] * pi[be][nu] + g->G[nu][al][be] * pi[be][mu]);
      t->Gpi[mu][nu] = -s / u[0];
    }
}

void ko_tensor_terms(const ko_ctx* c, double tau, const double* u4, const double* du16,
                     const double* pi16, double* out) {
  geom_t g;
  geom_at(c, tau, &g);
  double du[4][4], pi[4][4];
  for (int a = 0; a < 4; ++a)
    for (int b = 0; b < 4; ++b) { du[a][b] = du16[4 * a + b]; pi[a][b] = pi16[4 * a + b]; }
  tens_t t;
  tensor_terms(&g, u4, du, pi, &t);
  int k = 0;
  out[k++] = t.theta;
  for (int a = 0; a < 4; ++a) out[k++] = t.Du_lo[a];
  double(*mats[6])[4] = {t.sigma, t.omega, t.I1, t.I3, t.I4, t.Gpi};
  for (int m = 0; m < 6; ++m)
    for (int a = 0; a < 4; ++a)
      for (int b = 0; b < 4; ++b) out[k++] = mats[m][a][b];
}

/* ------------------------------------------------------------------ regulator (Sec. 3.2) */
static double regulator_factor(const geom_t* g, int milne, double tau, double e, double P0,
                               const double* u, double pi[4][4], double Pi, double rho_max, double xi0) {
  /* Pi^{mu nu} = Pi Delta^{mu nu} + pi^{mu nu} */
  double PP = 0.0;
  for (int mu = 0; mu < 4; ++mu)
    for (int nu = 0; nu < 4; ++nu) {
      double Dmn = ((mu == nu) ? g->gup[mu] : 0.0) - u[mu] * u[nu];
      double X = Pi * Dmn + pi[mu][nu];
      PP += X * X * g->glo[mu] * g->glo[nu];
    }
  /* reading: rho = 0 (factor 1) when Pi^{mu nu} Pi_{mu nu} vanishes; absolute values; P0 in
   * sqrt(e^2 + 3 P0^2); the eta component of pi^{lambda mu} u_mu is scaled by tau */
  if (!(PP > 0.0)) return 1.0;
  double nPP = sqrt(PP);
  double r1 = nPP / (rho_max * sqrt(e * e + 3.0 * P0 * P0));
  double tr = 0.0;
  for (int mu = 0; mu < 4; ++mu) tr += g->glo[mu] * pi[mu][mu];
  double r2 = fabs(tr) / (xi0 * rho_max * nPP);
  double r3 = 0.0;
  for (int la = 0; la < 4; ++la) {
    double s = 0.0;
    for (int mu = 0; mu < 4; ++mu) s += pi[la][mu] * g->glo[mu] * u[mu];
    if (la == 3 && milne) s *= tau;
    double r = fabs(s) / (xi0 * rho_max * nPP);
    if (r > r3) r3 = r;
  }
  double rho = r1;
  if (r2 > rho) rho = r2;
  if (r3 > rho) rho = r3;
  if (rho < 1e-4) return 1.0 - rho * rho / 3.0;
  return tanh(rho) / rho;
}

double ko_regulator_factor(const ko_ctx* c, double tau, double e, double P0, const double* u4,
                           const double* pi16, double Pi) {
  geom_t g;
  geom_at(c, tau, &g);
  double pi[4][4];
  for (int a = 0; a < 4; ++a)
    for (int b = 0; b < 4; ++b) pi[a][b] = pi16[4 * a + b];
  return regulator_factor(&g, c->P.coords == KO_MILNE, tau, e, P0, u4, pi, Pi, c->P.rho_max, c->P.xi0);
}

/* ------------------------------------------------------------------ lattice helpers */
static size_t cidx(const ko_ctx* c, int i, int j, int k) {
  return (size_t)i + (size_t)c->NX * ((size_t)j + (size_t)c->NY * (size_t)k);
}

/* ghost layers (Sec. 4.1, Eqs. ghostCells_1/2): copies of the outermost physical layer, or
 * periodic images; only axis-aligned ghosts are ever read */
static void fill_ghosts(const ko_ctx* c, double* A) {
  int nx = c->P.nx, ny = c->P.ny, nz = c->P.neta;
  int per = (c->P.bc == KO_BC_PERIODIC);
  for (int k = 2; k < nz + 2; ++k)
    for (int j = 2; j < ny + 2; ++j) {
      int gi[4] = {0, 1, nx + 2, nx + 3};
      for (int g = 0; g < 4; ++g) {
        int i = gi[g];
        int src = per ? 2 + (((i - 2) % nx) + nx) % nx : (i < 2 ? 2 : nx + 1);
        A[cidx(c, i, j, k)] = A[cidx(c, src, j, k)];
      }
    }
  for (int k = 2; k < nz + 2; ++k)
    for (int i = 2; i < nx + 2; ++i) {
      int gj[4] = {0, 1, ny + 2, ny + 3};
      for (int g = 0; g < 4; ++g) {
        int j = gj[g];
        int src = per ? 2 + (((j - 2) % ny) + ny) % ny : (j < 2 ? 2 : ny + 1);
        A[cidx(c, i, j, k)] = A[cidx(c, i, src, k)];
      }
    }
  for (int j = 2; j < ny + 2; ++j)
    for (int i = 2; i < nx + 2; ++i) {
      int gk[4] = {0, 1, nz + 2, nz + 3};
      for (int g = 0; g < 4; ++g) {
        int k = gk[g];
        int src = per ? 2 + (((k - 2) % nz) + nz) % nz : (k < 2 ? 2 : nz + 1);
        A[cidx(c, i, j, k)] = A[cidx(c, i, j, src)];
      }
    }
}

/* ------------------------------------------------------------------ KT right-hand side */
/* numerical flux H of Eq. (Hflux) through the face between cells a (left) and b = a + s */
static void face_flux(const ko_ctx* c, const fields_t* F, double tau, size_t a, size_t s, int d,
                      double D, double H[NQ], double* speed) {
  size_t b = a + s;
  double th = c->P.theta;
  double qm[NQ], qp[NQ];
  for (int n = 0; n < NQ; ++n) {
    /* q^-_{i+1/2} = q_i + D/2 (q_d)_i ; q^+_{i+1/2} = q_{i+1} - D/2 (q_d)_{i+1} */
    qm[n] = F->q[n][a] + 0.5 * D * slope(F->q[n], a, s, D, th);
    qp[n] = F->q[n][b] - 0.5 * D * slope(F->q[n], b, s, D, th);
  }
  double vm, vp;
  if (c->P.iface == KO_IFACE_INVERT) {
    /* literal reading of Sec. 3.1: primaries from the extrapolated states q^+- */
    double o[6];
    invert_core(c, tau, qm, F->e[a], o);
    vm = o[3 + d] / o[2];
    invert_core(c, tau, qp, F->e[b], o);
    vp = o[3 + d] / o[2];
  } else {
    /* reading: u^mu at the faces by the same generalised-minmod extrapolation of the
     * cell-centred u^mu */
    double um[4], upp[4];
    for (int m = 0; m < 4; ++m) {
      um[m] = F->u[m][a] + 0.5 * D * slope(F->u[m], a, s, D, th);
      upp[m] = F->u[m][b] - 0.5 * D * slope(F->u[m], b, s, D, th);
    }
    vm = um[d + 1] / um[0];
    vp = upp[d + 1] / upp[0];
  }
  /* local propagation speed, Eq. (ax): a = max(|v^+|, |v^-|) */
  double av = fabs(vp) > fabs(vm) ? fabs(vp) : fabs(vm);
  for (int n = 0; n < NQ; ++n) H[n] = 0.5 * (vp * qp[n] + vm * qm[n]) - 0.5 * av * (qp[n] - qm[n]);
  *speed = av;
}

/* X^{d nu} = P (v^d delta^nu_tau - g^{d nu}) - v^d pi^{tau nu} + pi^{d nu}: the quantity whose
 * d-derivative enters S_c^nu (App. B); P = P0 + Pi */
static double Xterm(const fields_t* F, const geom_t* g, size_t c_, int d, int nu) {
  double P = F->p[c_] + F->q[14][c_];
  double v = F->u[d + 1][c_] / F->u[0][c_];
  double r = -v * F->q[PIX[0][nu]][c_] + F->q[PIX[d + 1][nu]][c_];
  if (nu == 0) r += P * v;
  if (nu == d + 1) r -= P * g->gup[d + 1];
  return r;
}

/* C[q] (Eq. semiDiscreteKT) at one physical cell */
static void cell_rhs(const ko_ctx* c, const fields_t* F, double* const* uprev, double tau, size_t idx,
                     double out[NQ], double* speed) {
  geom_t g;
  geom_at(c, tau, &g);
  size_t str[3] = {1, (size_t)c->NX, (size_t)c->NX * (size_t)c->NY};
  double Dd[3] = {c->P.dx, c->P.dy, c->P.deta};
  for (int n = 0; n < NQ; ++n) out[n] = 0.0;

  /* 1. -(H_{i+1/2} - H_{i-1/2})/D in x, y, eta.  The CFL diagnostic records the largest local
   * speed a of the cell's faces, the eta speeds times sqrt(-g_{eta eta}) = tau (Milne) so that
   * all three are in units of c */
  double amax = 0.0;
  for (int d = 0; d < 3; ++d) {
    double Hp[NQ], Hm[NQ], ap, am;
    face_flux(c, F, tau, idx, str[d], d, Dd[d], Hp, &ap);
    face_flux(c, F, tau, idx - str[d], str[d], d, Dd[d], Hm, &am);
    for (int n = 0; n < NQ; ++n) out[n] -= (Hp[n] - Hm[n]) / Dd[d];
    double a = (ap > am) ? ap : am;
    if (d == 2 && c->P.coords == KO_MILNE) a = a * tau;
    if (a > amax) amax = a;
  }
  *speed = amax;

  /* 2. sources J = S + G (App. B) */
  double u[4];
  for (int m = 0; m < 4; ++m) u[m] = F->u[m][idx];
  double e = F->e[idx], P0 = F->p[idx], Pi = F->q[14][idx];
  double P = P0 + Pi;
  double P0x, cs2, T, lnd;
  eos_eval(c, e, &P0x, &cs2, &T, &lnd);
  transport_t tr;
  transport(c, e, P0, T, lnd, &tr);
  double pi[4][4];
  for (int a = 0; a < 4; ++a)
    for (int b = 0; b < 4; ++b) pi[a][b] = F->q[PIX[a][b]][idx];

  /* derivatives (Sec. 3.1): central in space, backward in time */
  double du[4][4];
  for (int m = 0; m < 4; ++m) du[0][m] = (u[m] - uprev[m][idx]) / c->P.dtau;
  for (int d = 0; d < 3; ++d)
    for (int m = 0; m < 4; ++m) du[d + 1][m] = (F->u[m][idx + str[d]] - F->u[m][idx - str[d]]) / (2.0 * Dd[d]);
  double dv = 0.0; /* d_i v_i */
  for (int d = 0; d < 3; ++d) {
    double vpl = F->u[d + 1][idx + str[d]] / F->u[0][idx + str[d]];
    double vmi = F->u[d + 1][idx - str[d]] / F->u[0][idx - str[d]];
    dv += (vpl - vmi) / (2.0 * Dd[d]);
  }
  tens_t t;
  tensor_terms(&g, u, du, pi, &t);

  /* S_c: -sum_d d_d X^{d nu}, difference of the products at i+-1 */
  for (int nu = 0; nu < 4; ++nu) {
    double s = 0.0;
    for (int d = 0; d < 3; ++d)
      s -= (Xterm(F, &g, idx + str[d], d, nu) - Xterm(F, &g, idx - str[d], d, nu)) / (2.0 * Dd[d]);
    out[nu] += s;
  }
  /* G_c^nu = -Gamma^lambda_{lambda mu} T^{mu nu} - Gamma^nu_{mu lambda} T^{mu lambda}, with
   * T^{tau nu} the evolved q and T^{ij} = (e+P) u^i u^j - P g^{ij} + pi^{ij} (Eq. Tij) */
  double Tf[4][4];
  for (int a = 0; a < 4; ++a)
    for (int b = 0; b < 4; ++b) {
      if (a == 0) Tf[a][b] = F->q[b][idx];
      else if (b == 0) Tf[a][b] = F->q[a][idx];
      else Tf[a][b] = (e + P) * u[a] * u[b] - ((a == b) ? P * g.gup[a] : 0.0) + pi[a][b];
    }
  for (int nu = 0; nu < 4; ++nu) {
    double s = 0.0;
    for (int la = 0; la < 4; ++la)
      for (int mu = 0; mu < 4; ++mu) s += g.G[la][la][mu] * Tf[mu][nu];
    for (int mu = 0; mu < 4; ++mu)
      for (int la = 0; la < 4; ++la) s += g.G[nu][mu][la] * Tf[mu][la];
    out[nu] -= s;
  }

  /* S_pi + G_pi for the 10 pi rows */
  if (tr.shear_on) {
    double tpp = c->P.tau_pipi_on ? 10.0 / 7.0 : 0.0;
    for (int a = 0; a < 4; ++a)
      for (int b = a; b < 4; ++b) {
        double Ipi = t.I1[a][b] + (4.0 / 3.0) * t.theta * pi[a][b] - t.I3[a][b] + tpp * t.I4[a][b] -
                     1.2 * Pi * t.sigma[a][b];
        double S = (2.0 * tr.eta_over_taupi * t.sigma[a][b] - tr.rate_pi * pi[a][b] - Ipi) / u[0] +
                   pi[a][b] * dv;
        out[PIX[a][b]] += S + t.Gpi[a][b];
      }
  }
  /* S_Pi */
  if (tr.bulk_on) {
    double IPi = (2.0 / 3.0) * Pi * t.theta - tr.lam_Pipi * t.pisig;
    out[14] += (-tr.zeta_over_tauPi * t.theta - tr.rate_Pi * Pi - IPi) / u[0] + Pi * dv;
  }
  (void)P;
}

/* ------------------------------------------------------------------ stages (Sec. 4.3) */
static int for_all_cells_stage(ko_ctx* c, const fields_t* F, double* const* uprev, double tau,
                               double** qout, double* const* qbase) {
  int nx = c->P.nx, ny = c->P.ny, nz = c->P.neta;
  /* the threads split the (eta, y) rows of the lattice (timing only; results do not depend on it) */
#pragma omp parallel for collapse(2) schedule(static)
  for (int k = 2; k < nz + 2; ++k)
    for (int j = 2; j < ny + 2; ++j)
      for (int i = 2; i < nx + 2; ++i) {
        size_t idx = cidx(c, i, j, k);
        double C[NQ];
        cell_rhs(c, F, uprev, tau, idx, C, &c->spd[idx]);
        for (int n = 0; n < NQ; ++n) {
          /* forward Euler E[w] = w + dtau C[w] */
          double w = F->q[n][idx] + c->P.dtau * C[n];
          /* convex combination q^{n+1} = (q^n + E[q^*])/2 */
          if (qbase) w = 0.5 * (qbase[n][idx] + w);
          qout[n][idx] = w;
        }
      }
  for (int k = 2; k < nz + 2; ++k)
    for (int j = 2; j < ny + 2; ++j)
      for (int i = 2; i < nx + 2; ++i) {
        double a = c->spd[cidx(c, i, j, k)];
        if (a > c->max_speed) c->max_speed = a;
      }
  return 0;
}

/* set inferred variables, then regulate pi, then ghosts (steps 2-4 and 8 of Sec. 4.3) */
static int infer_regulate_ghost(ko_ctx* c, double** q, double tau, double** u, double* e, double* p, double* reg) {
  int nx = c->P.nx, ny = c->P.ny, nz = c->P.neta;
  int st_all = 0;
  geom_t g;
  geom_at(c, tau, &g);
#pragma omp parallel for collapse(2) schedule(static) reduction(| : st_all)
  for (int k = 2; k < nz + 2; ++k)
    for (int j = 2; j < ny + 2; ++j)
      for (int i = 2; i < nx + 2; ++i) {
        size_t idx = cidx(c, i, j, k);
        double qc[NQ], o[6];
        for (int n = 0; n < NQ; ++n) qc[n] = q[n][idx];
        int st = invert_core(c, tau, qc, e[idx], o);
        st_all |= st;
        e[idx] = o[0];
        p[idx] = o[1];
        for (int m = 0; m < 4; ++m) u[m][idx] = o[2 + m];
        if (c->P.regulate) {
          double pi[4][4];
          for (int a = 0; a < 4; ++a)
            for (int b = 0; b < 4; ++b) pi[a][b] = qc[PIX[a][b]];
          double f = regulator_factor(&g, c->P.coords == KO_MILNE, tau, o[0], o[1], &o[2], pi, qc[14],
                                      c->P.rho_max, c->P.xi0);
          for (int n = 4; n < 14; ++n) q[n][idx] = f * qc[n];
          if (reg) reg[idx] = f;
        }
      }
  for (int n = 0; n < NQ; ++n) fill_ghosts(c, q[n]);
  for (int m = 0; m < 4; ++m) fill_ghosts(c, u[m]);
  fill_ghosts(c, e);
  fill_ghosts(c, p);
  return st_all;
}

int ko_step(ko_ctx* c, int nsteps) {
  int st = 0;
  c->max_speed = 0.0;
  for (int s = 0; s < nsteps; ++s) {
    double tau_n = c->tau, tau_1 = c->tau + c->P.dtau;
    /* 1. q^* = E[q^n; e^n, p^n, u^n, u^{n-1}], sources at tau^n */
    fields_t F = {{0}, {0}, c->e, c->p};
    for (int n = 0; n < NQ; ++n) F.q[n] = c->q[n];
    for (int m = 0; m < 4; ++m) F.u[m] = c->u[m];
    for_all_cells_stage(c, &F, c->up, tau_n, c->qs, NULL);
    /* 2.-4. e^*, p^*, u^* from q^* at tau^{n+1}; regulate; ghosts */
    st |= infer_regulate_ghost(c, c->qs, tau_1, c->us, c->es, c->ps, NULL);
    /* 5.-6. Q = (q^n + E[q^*; e^*, p^*, u^*, u^n])/2, sources at tau^{n+1} */
    fields_t S = {{0}, {0}, c->es, c->ps};
    for (int n = 0; n < NQ; ++n) S.q[n] = c->qs[n];
    for (int m = 0; m < 4; ++m) S.u[m] = c->us[m];
    for_all_cells_stage(c, &S, c->u, tau_1, c->Q, c->q);
    /* 8. e, p, u^{n+1} from Q; regulate; ghosts */
    st |= infer_regulate_ghost(c, c->Q, tau_1, c->un, c->e, c->p, c->reg);
    /* 7. and 9. u^{n-1} <- u^n, u^n <- u^{n+1}, q <-> Q */
    for (int m = 0; m < 4; ++m) {
      double* t = c->up[m];
      c->up[m] = c->u[m];
      c->u[m] = c->un[m];
      c->un[m] = t;
    }
    for (int n = 0; n < NQ; ++n) {
      double* t = c->q[n];
      c->q[n] = c->Q[n];
      c->Q[n] = t;
    }
    c->tau = tau_1;
  }
  return st;
}

int ko_rhs(ko_ctx* c, double* out) {
  fields_t F = {{0}, {0}, c->e, c->p};
  for (int n = 0; n < NQ; ++n) F.q[n] = c->q[n];
  for (int m = 0; m < 4; ++m) F.u[m] = c->u[m];
  int nx = c->P.nx, ny = c->P.ny, nz = c->P.neta;
  size_t ncp = (size_t)nx * ny * nz;
#pragma omp parallel for collapse(2) schedule(static)
  for (int k = 2; k < nz + 2; ++k)
    for (int j = 2; j < ny + 2; ++j)
      for (int i = 2; i < nx + 2; ++i) {
        double C[NQ], a;
        cell_rhs(c, &F, c->up, c->tau, cidx(c, i, j, k), C, &a);
        size_t o = (size_t)(i - 2) + (size_t)nx * ((size_t)(j - 2) + (size_t)ny * (size_t)(k - 2));
        for (int n = 0; n < NQ; ++n) out[(size_t)n * ncp + o] = C[n];
      }
  return 0;
}

/* Validity diagnostics of Sec. 7 at the current state (tau^n, with the backward time derivative
 * u^n - u^{n-1} as in the first stage): Knudsen numbers tau_pi theta and tau_Pi theta (unfloored
 * relaxation times), first-order inverse Reynolds numbers sqrt(pi^{mu nu} pi_{mu nu})/P0 and
 * |Pi|/P0 (Eq. inverseReynoldsNumbers), second-order ones sqrt(J^{mu nu} J_{mu nu}) /
 * (2 eta sqrt(sigma^{mu nu} sigma_{mu nu})) and |J| / (zeta |theta|) (Eq. inverseReynoldsNumbers2)
 * with J^{mu nu}, J of Eq. (14_moment_terms) without diffusion, and the regulation factor of the
 * last step.  A quantity whose channel is off (or whose denominator vanishes) is 0. */
static void cell_diagnostics(const ko_ctx* c, const fields_t* F, double* const* uprev, double tau, size_t idx,
                             double out[6]) {
  geom_t g;
  geom_at(c, tau, &g);
  size_t str[3] = {1, (size_t)c->NX, (size_t)c->NX * (size_t)c->NY};
  double Dd[3] = {c->P.dx, c->P.dy, c->P.deta};
  double u[4];
  for (int m = 0; m < 4; ++m) u[m] = F->u[m][idx];
  double e = F->e[idx], P0 = F->p[idx], Pi = F->q[14][idx];
  double P0x, cs2, T, lnd;
  eos_eval(c, e, &P0x, &cs2, &T, &lnd);
  transport_t tr;
  transport(c, e, P0, T, lnd, &tr);
  double pi[4][4];
  for (int a = 0; a < 4; ++a)
    for (int b = 0; b < 4; ++b) pi[a][b] = F->q[PIX[a][b]][idx];
  double du[4][4];
  for (int m = 0; m < 4; ++m) du[0][m] = (u[m] - uprev[m][idx]) / c->P.dtau;
  for (int d = 0; d < 3; ++d)
    for (int m = 0; m < 4; ++m) du[d + 1][m] = (F->u[m][idx + str[d]] - F->u[m][idx - str[d]]) / (2.0 * Dd[d]);
  tens_t t;
  tensor_terms(&g, u, du, pi, &t);
  double tpp = c->P.tau_pipi_on ? 10.0 / 7.0 : 0.0;
  double pp = 0.0, ss = 0.0, xx = 0.0;
  for (int a = 0; a < 4; ++a)
    for (int b = 0; b < 4; ++b) {
      double w = g.glo[a] * g.glo[b];
      /* J^{ab}/tau_pi = 2 pi_l^<a omega^b>l - (4/3) pi theta - (tau_pipi/tau_pi) pi^l<a sigma_l^b>
       *               + (6/5) Pi sigma, with I3, I4 of App. A */
      double X = t.I3[a][b] - (4.0 / 3.0) * t.theta * pi[a][b] - tpp * t.I4[a][b] + 1.2 * Pi * t.sigma[a][b];
      pp += pi[a][b] * pi[a][b] * w;
      ss += t.sigma[a][b] * t.sigma[a][b] * w;
      xx += X * X * w;
    }
  double es = coef_value(c->P.eta_kind, c->P.eta_c, T);
  double tau_pi = tr.shear_on ? 5.0 * es / T : 0.0;
  double tau_Pi = tr.bulk_on ? exp(-(log(15.0) + 2.0 * lnd + log(T) - coef_log(c->P.zeta_kind, c->P.zeta_c, T)))
                             : 0.0;
  out[0] = tau_pi * t.theta;
  out[1] = tau_Pi * t.theta;
  out[2] = sqrt(pp) / P0;
  out[3] = fabs(Pi) / P0;
  out[4] = (tr.shear_on && ss > 0.0) ? sqrt(xx) / (2.0 * tr.eta_over_taupi * sqrt(ss)) : 0.0;
  double J = (2.0 / 3.0) * Pi * t.theta - tr.lam_Pipi * t.pisig; /* -J / tau_Pi */
  out[5] = (tr.bulk_on && t.theta != 0.0) ? fabs(J) / (tr.zeta_over_tauPi * fabs(t.theta)) : 0.0;
}

int ko_diagnostics(const ko_ctx* c, double* out) {
  fields_t F = {{0}, {0}, c->e, c->p};
  for (int n = 0; n < NQ; ++n) F.q[n] = c->q[n];
  for (int m = 0; m < 4; ++m) F.u[m] = c->u[m];
  int nx = c->P.nx, ny = c->P.ny, nz = c->P.neta;
  size_t ncp = (size_t)nx * ny * nz;
  for (int k = 0; k < nz; ++k)
    for (int j = 0; j < ny; ++j)
      for (int i = 0; i < nx; ++i) {
        size_t o = (size_t)i + (size_t)nx * ((size_t)j + (size_t)ny * (size_t)k);
        size_t idx = cidx(c, i + 2, j + 2, k + 2);
        double d[6];
        cell_diagnostics(c, &F, c->up, c->tau, idx, d);
        for (int m = 0; m < 6; ++m) out[(size_t)m * ncp + o] = d[m];
        out[6 * ncp + o] = c->reg[idx];
      }
  return 0;
}

/* ------------------------------------------------------------------ state in / out */
int ko_set_state(ko_ctx* c, double tau, const double* e, const double* u, const double* pi,
                 const double* Pi, const double* u_prev) {
  int nx = c->P.nx, ny = c->P.ny, nz = c->P.neta;
  size_t ncp = (size_t)nx * ny * nz;
  geom_t g, gp;
  geom_at(c, tau, &g);
  geom_at(c, tau - c->P.dtau, &gp);
  c->tau = tau;
  int st = 0;
  for (int k = 0; k < nz; ++k)
    for (int j = 0; j < ny; ++j)
      for (int i = 0; i < nx; ++i) {
        size_t o = (size_t)i + (size_t)nx * ((size_t)j + (size_t)ny * (size_t)k);
        size_t idx = cidx(c, i + 2, j + 2, k + 2);
        double ec = e[o];
        double ux = u ? u[o] : 0.0, uy = u ? u[ncp + o] : 0.0, un = u ? u[2 * ncp + o] : 0.0;
        double ut = sqrt(1.0 + ux * ux + uy * uy + g.gnn * un * un); /* u.u = 1 */
        double pic[10];
        for (int m = 0; m < 10; ++m) pic[m] = pi ? pi[(size_t)m * ncp + o] : 0.0;
        double Pic = Pi ? Pi[o] : 0.0;
        double P0, cs2, T, lnd;
        eos_eval(c, ec, &P0, &cs2, &T, &lnd);
        double P = P0 + Pic;
        double uu[4] = {ut, ux, uy, un};
        /* Eqs. (Ttt), (Tti) */
        c->q[0][idx] = (ec + P) * ut * ut - P + pic[0];
        for (int m = 1; m < 4; ++m) c->q[m][idx] = (ec + P) * ut * uu[m] + pic[m];
        for (int m = 0; m < 10; ++m) c->q[4 + m][idx] = pic[m];
        c->q[14][idx] = Pic;
        c->e[idx] = ec;
        c->p[idx] = P0;
        c->reg[idx] = 1.0;
        for (int m = 0; m < 4; ++m) c->u[m][idx] = uu[m];
        if (u_prev) {
          double px = u_prev[o], py = u_prev[ncp + o], pn = u_prev[2 * ncp + o];
          c->up[0][idx] = sqrt(1.0 + px * px + py * py + gp.gnn * pn * pn);
          c->up[1][idx] = px; c->up[2][idx] = py; c->up[3][idx] = pn;
        } else {
          for (int m = 0; m < 4; ++m) c->up[m][idx] = uu[m]; /* u^{-1} = u^0 (Sec. 4.3 footnote) */
        }
        if (!isfinite(c->q[0][idx])) st |= KO_ST_NONFINITE;
      }
  for (int n = 0; n < NQ; ++n) fill_ghosts(c, c->q[n]);
  for (int m = 0; m < 4; ++m) { fill_ghosts(c, c->u[m]); fill_ghosts(c, c->up[m]); }
  fill_ghosts(c, c->e);
  fill_ghosts(c, c->p);
  return st;
}

int ko_set_state_q(ko_ctx* c, double tau, const double* q, const double* e, const double* u,
                   const double* u_prev) {
  int nx = c->P.nx, ny = c->P.ny, nz = c->P.neta;
  size_t ncp = (size_t)nx * ny * nz;
  c->tau = tau;
  int st = 0;
  for (int k = 0; k < nz; ++k)
    for (int j = 0; j < ny; ++j)
      for (int i = 0; i < nx; ++i) {
        size_t o = (size_t)i + (size_t)nx * ((size_t)j + (size_t)ny * (size_t)k);
        size_t idx = cidx(c, i + 2, j + 2, k + 2);
        for (int n = 0; n < NQ; ++n) c->q[n][idx] = q[(size_t)n * ncp + o];
        double P0, cs2, T, lnd;
        eos_eval(c, e[o], &P0, &cs2, &T, &lnd);
        c->e[idx] = e[o];
        c->p[idx] = P0;
        c->reg[idx] = 1.0;
        for (int m = 0; m < 4; ++m) {
          c->u[m][idx] = u[(size_t)m * ncp + o];
          c->up[m][idx] = u_prev ? u_prev[(size_t)m * ncp + o] : c->u[m][idx];
        }
        if (!isfinite(c->q[0][idx])) st |= KO_ST_NONFINITE;
      }
  for (int n = 0; n < NQ; ++n) fill_ghosts(c, c->q[n]);
  for (int m = 0; m < 4; ++m) { fill_ghosts(c, c->u[m]); fill_ghosts(c, c->up[m]); }
  fill_ghosts(c, c->e);
  fill_ghosts(c, c->p);
  return st;
}

int ko_get_state(const ko_ctx* c, double* tau, double* e, double* u, double* pi, double* Pi, double* q) {
  int nx = c->P.nx, ny = c->P.ny, nz = c->P.neta;
  size_t ncp = (size_t)nx * ny * nz;
  if (tau) *tau = c->tau;
  for (int k = 0; k < nz; ++k)
    for (int j = 0; j < ny; ++j)
      for (int i = 0; i < nx; ++i) {
        size_t o = (size_t)i + (size_t)nx * ((size_t)j + (size_t)ny * (size_t)k);
        size_t idx = cidx(c, i + 2, j + 2, k + 2);
        if (e) e[o] = c->e[idx];
        if (u) for (int m = 0; m < 4; ++m) u[(size_t)m * ncp + o] = c->u[m][idx];
        if (pi) for (int m = 0; m < 10; ++m) pi[(size_t)m * ncp + o] = c->q[4 + m][idx];
        if (Pi) Pi[o] = c->q[14][idx];
        if (q) for (int n = 0; n < NQ; ++n) q[(size_t)n * ncp + o] = c->q[n][idx];
      }
  return 0;
}

/* ------------------------------------------------------------------ lifetime */
static double* zalloc(size_t n) { return (double*)calloc(n, sizeof(double)); }

ko_ctx* ko_create(const ko_params* prm) {
  if (!prm || prm->nx < 1 || prm->ny < 1 || prm->neta < 1) return NULL;
  ko_ctx* c = (ko_ctx*)calloc(1, sizeof(ko_ctx));
  c->P = *prm;
  c->NX = prm->nx + 4; c->NY = prm->ny + 4; c->NZ = prm->neta + 4;
  c->ncell = (size_t)c->NX * c->NY * c->NZ;
  if (prm->eos_kind == KO_EOS_TABLE) {
    int n = prm->eos_n;
    c->nt = n;
    c->te = zalloc(n); c->tp = zalloc(n); c->tcs2 = zalloc(n); c->tT = zalloc(n); c->tlnd = zalloc(n);
    memcpy(c->te, prm->eos_e, n * sizeof(double));
    memcpy(c->tp, prm->eos_p, n * sizeof(double));
    memcpy(c->tcs2, prm->eos_cs2, n * sizeof(double));
    memcpy(c->tT, prm->eos_T, n * sizeof(double));
    memcpy(c->tlnd, prm->eos_lndelta, n * sizeof(double));
  }
  c->P.eos_e = c->P.eos_p = c->P.eos_cs2 = c->P.eos_T = c->P.eos_lndelta = NULL;
  for (int n = 0; n < NQ; ++n) { c->q[n] = zalloc(c->ncell); c->qs[n] = zalloc(c->ncell); c->Q[n] = zalloc(c->ncell); }
  for (int m = 0; m < 4; ++m) {
    c->u[m] = zalloc(c->ncell); c->us[m] = zalloc(c->ncell); c->up[m] = zalloc(c->ncell); c->un[m] = zalloc(c->ncell);
  }
  c->e = zalloc(c->ncell); c->p = zalloc(c->ncell); c->es = zalloc(c->ncell); c->ps = zalloc(c->ncell);
  c->reg = zalloc(c->ncell);
  c->spd = zalloc(c->ncell);
  /* unused ghost corners keep a harmless rest state */
  for (size_t i = 0; i < c->ncell; ++i) {
    c->u[0][i] = c->us[0][i] = c->up[0][i] = c->un[0][i] = 1.0;
    c->reg[i] = 1.0;
  }
  return c;
}

void ko_free(ko_ctx* c) {
  if (!c) return;
  free(c->te); free(c->tp); free(c->tcs2); free(c->tT); free(c->tlnd);
  for (int n = 0; n < NQ; ++n) { free(c->q[n]); free(c->qs[n]); free(c->Q[n]); }
  for (int m = 0; m < 4; ++m) { free(c->u[m]); free(c->us[m]); free(c->up[m]); free(c->un[m]); }
  free(c->e); free(c->p); free(c->es); free(c->ps);
  free(c->reg);
  free(c->spd);
  free(c);
}

double ko_max_speed(const ko_ctx* c) { return c->max_speed; }

int ko_set_threads(int n) {
#ifdef _OPENMP
  if (n > 0) omp_set_num_threads(n);
  return omp_get_max_threads();
#else
  (void)n;
  return 1;
#endif
}
