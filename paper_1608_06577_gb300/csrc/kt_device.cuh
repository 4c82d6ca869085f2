// kt_device.cuh -- device-side building blocks of libkt (sm_103a).
//
// Lattice: padded structure-of-arrays, two ghost layers per side (Sec. 4.1), x fastest,
// eta slowest (Sec. 4.2).  Each field occupies `fstride` elements; the row pitch is rounded
// up to a multiple of 4 elements and every field starts on a 256-byte boundary.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace kt {

constexpr int NQ = 15;  // T^{tau mu} (4), pi^{mu nu} (10), Pi (1): Eq. (qComponents)

// q index of pi^{mu nu}
__host__ __device__ constexpr int pix(int a, int b) {
  return (a > b) ? pix(b, a)
                 : (a == 0 ? 4 + b : (a == 1 ? 7 + b : (a == 2 ? 9 + b : 13)));
}

enum : unsigned { ST_INVERSION = 1u, ST_NONFINITE = 2u };

struct Lattice {
  int nx, ny, nz;      // physical cells
  int pitch;           // padded row length (>= nx + 4)
  int NY, NZ;          // ny + 4, nz + 4
  long long plane;     // pitch * NY
  long long fstride;   // elements per field (>= plane * NZ, multiple of 32)
  __host__ __device__ long long idx(int i, int j, int k) const {
    return (long long)i + (long long)pitch * ((long long)j + (long long)NY * (long long)k);
  }
};

// Table EOS: one record per interval [e_i, e_{i+1}], cubic polynomials in t = (e - e_i)/(e_{i+1} - e_i)
template <typename R>
struct EosSeg {
  R e0, inv_de;
  R P0, mP, cP2, cP3;   // P(t) = P0 + t (mP + t (cP2 + t cP3)); c_s^2 = P'(t) inv_de
  R T0, mT, cT2, cT3;   // T(t), same form
  R l0, dl;             // ln(1/3 - c_s^2) = l0 + t dl
};

struct Coef {
  int kind;       // 0 const, 1 gauss
  double c0, c1, c2;
  double ln_c0;
};

struct Params {
  Lattice L;
  double dx, dy, deta, dtau;
  double theta;
  int milne;          // 1 Milne, 0 Cartesian
  int periodic;
  int eos_table;      // 0 conformal, 1 table
  double eos_a;       // conformal e = a T^4
  int eos_n;
  float lne0, inv_h;  // index guess: (ln e - ln e_0) * inv_h
  const EosSeg<double>* seg_d;
  const EosSeg<float>* seg_f;
  Coef eta, zeta;
  int shear_on, bulk_on;
  double tpp;         // tau_pipi / tau_pi (10/7 or 0)
  int regulate;
  double rho_max, xi0;
  double e_min;
  double rate_max;    // 1 / tau_relax_min (or +inf)
  double ln_rate_max;
};

template <typename R> __device__ __forceinline__ const EosSeg<R>* eos_table(const Params& P);
template <> __device__ __forceinline__ const EosSeg<double>* eos_table<double>(const Params& P) { return P.seg_d; }
template <> __device__ __forceinline__ const EosSeg<float>* eos_table<float>(const Params& P) { return P.seg_f; }

// Interval search: a single-precision log guess, corrected so that e_i <= e < e_{i+1} exactly
// (clamped to the first / last interval outside the table).
template <typename R>
__device__ __forceinline__ int eos_interval(const Params& P, const EosSeg<R>* seg, R e) {
  int n1 = P.eos_n - 2;
  float g = (__logf((float)e) - P.lne0) * P.inv_h;
  int i = (g > 0.f) ? (int)g : 0;  // NaN compares false -> 0
  i = min(i, n1);
  #pragma unroll 1
  for (int it = 0; it < 64 && i > 0 && e < seg[i].e0; ++it) --i;
  #pragma unroll 1
  for (int it = 0; it < 64 && i < n1 && e >= seg[i + 1].e0; ++it) ++i;
  return i;
}

// P0(e), c_s^2(e) (for the root-find)
template <typename R>
__device__ __forceinline__ void eos_P_cs2(const Params& P, R e, R& P0, R& cs2) {
  if (!P.eos_table) {
    P0 = e * R(1.0 / 3.0);
    cs2 = R(1.0 / 3.0);
    return;
  }
  const EosSeg<R>* seg = eos_table<R>(P);
  const EosSeg<R>& s = seg[eos_interval<R>(P, seg, e)];
  R t = (e - s.e0) * s.inv_de;
  P0 = fma(t, fma(t, fma(t, s.cP3, s.cP2), s.mP), s.P0);
  cs2 = fma(t, fma(t, R(3) * s.cP3, R(2) * s.cP2), s.mP) * s.inv_de;
}

template <typename R>
__device__ __forceinline__ R eos_P(const Params& P, R e) {
  R p, c;
  eos_P_cs2<R>(P, e, p, c);
  return p;
}

// T(e) and ln(1/3 - c_s^2)(e) (for the transport coefficients)
template <typename R>
__device__ __forceinline__ void eos_T_lnd(const Params& P, R e, R& T, R& lnd) {
  if (!P.eos_table) {
    T = sqrt(sqrt(e / R(P.eos_a)));
    lnd = -R(INFINITY);
    return;
  }
  const EosSeg<R>* seg = eos_table<R>(P);
  const EosSeg<R>& s = seg[eos_interval<R>(P, seg, e)];
  R t = (e - s.e0) * s.inv_de;
  T = fma(t, fma(t, fma(t, s.cT3, s.cT2), s.mT), s.T0);
  lnd = fma(t, s.dl, s.l0);
}

// Generalised minmod of (theta dm, (dm + dp)/2, theta dp), Sec. 3.1, with sgn(0) = 0:
// the common-sign smallest magnitude, or 0.  This is the slope times the cell size.
template <typename R>
__device__ __forceinline__ R limited_slope(R qm, R q0, R qp, R theta) {
  R a = theta * (q0 - qm), b = R(0.5) * (qp - qm), c = theta * (qp - q0);
  R mn = fmin(fabs(a), fmin(fabs(b), fabs(c)));
  bool pos = (a > R(0)) & (b > R(0)) & (c > R(0));
  bool neg = (a < R(0)) & (b < R(0)) & (c < R(0));
  return pos ? mn : (neg ? -mn : R(0));
}

template <typename R>
__device__ __forceinline__ R coef_value(const Coef& c, R T) {
  if (c.kind == 0) return R(c.c0);
  R x = (T - R(c.c1)) / R(c.c2);
  return R(c.c0) * exp(-x * x);
}

template <typename R>
__device__ __forceinline__ R coef_log(const Coef& c, R T) {
  if (c.kind == 0) return R(c.ln_c0);
  R x = (T - R(c.c1)) / R(c.c2);
  return R(c.ln_c0) - x * x;
}

// per-cell read of an R-typed field from a buffer that may hold double or float
template <typename R, typename S>
__device__ __forceinline__ R ld(const S* __restrict__ p, long long i) {
  return (R)__ldg(p + i);
}

}  // namespace kt
