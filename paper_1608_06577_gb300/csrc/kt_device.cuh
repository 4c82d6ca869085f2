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

// q index of pi^{mu nu} (not recursive, so that it always inlines)
__host__ __device__ __forceinline__ constexpr int pix(int a, int b) {
  const int lo = (a < b) ? a : b, hi = (a < b) ? b : a;
  return lo == 0 ? 4 + hi : (lo == 1 ? 7 + hi : (lo == 2 ? 9 + hi : 13));
}

enum : unsigned { ST_INVERSION = 1u, ST_NONFINITE = 2u, ST_TIMEOUT = 4u };

__device__ __forceinline__ double f2d_bits(float f);
__device__ __forceinline__ float d2f_bits(double d);
__device__ __forceinline__ float d2f_trunc(double d);

// One event's padded lattice inside the field arrays.  A field array holds every component of
// every event: component n of event e starts at n * fstride + base (fstride is shared by all
// events of a context; a single event has base 0).
struct Lattice {
  int nx, ny, nz;      // physical cells
  int pitch;           // padded row length (>= nx + 4)
  int NY, NZ;          // ny + 4, nz + 4
  long long plane;     // pitch * NY
  long long fstride;   // elements between components (sum of all events' padded sizes)
  long long base;      // first element of this event
  __host__ __device__ long long idx(int i, int j, int k) const {
    return base + (long long)i + (long long)pitch * ((long long)j + (long long)NY * (long long)k);
  }
};

// a block-shaped tile of one event: the persistent stage kernel walks a table of these
struct Tile {
  int event, i0, j0, k0;
};

// Table EOS: one record per interval [e_i, e_{i+1}], cubic polynomials in t = (e - e_i)/(e_{i+1} - e_i)
template <typename R>
struct EosSeg {
  R e0, inv_de;
  R P0, mP, cP2, cP3;   // P(t) = P0 + t (mP + t (cP2 + t cP3)); c_s^2 = P'(t) inv_de
  R T0, mT, cT2, cT3;   // T(t), same form
  R l0, dl;             // ln(1/3 - c_s^2) = l0 + t dl
  R a1, a2, a3;         // the same P in d = e - e0: P = P0 + d (a1 + d (a2 + d a3)), c_s^2 = P'(d)
};

// The root-find's record of interval i of the table EOS, 64 bytes (two 32-byte sectors, fetched
// by four vector loads in one round trip): its ends e0 <= e < e1 (e1 = +inf for the last
// interval), so that the interval guess is checked with the coefficients already loaded; P in
// d = e - e0 as in EosSeg (FP64); and c_s^2 = P'(d) = b1 + d (b2 + d b3) in single precision, with
// b1, b2, b3 the FP32 table's a1, 2 a2, 3 a3 (the products rounded in single precision).
struct alignas(64) RootSeg {
  double e0, e1, P0, a1, a2, a3;
  float b1, b2, b3, unused;
};

// The mixed-precision root-find's record of the same interval: e0, e1, P0 and a1 in FP64, the
// cubic's a2 and a3 rounded to single precision, b1-b3 as in RootSeg.  In d = e - e0 the
// correction d (a2 + d a3) to a1 is below 1e-3 of a1 inside the table (intervals of ~1% in e,
// c_s^2 varying by ~1e-4 across one), so forming it in single precision moves P0(e) by ~1e-12
// of itself -- far inside the root-find's 1e-10 acceptance -- and takes one FP64 instruction
// per residual off the slow FP64 pipe.
struct alignas(64) RootSegM {
  double e0, e1, P0, a1;
  float a2, a3, b1, b2;
  float b3, unused0, unused1, unused2;
};

struct Coef {
  int kind;       // 0 const, 1 gauss
  double c0, c1, c2;
  double ln_c0;
};

// Per-run constants in the stencil precision, computed once on the host so that no thread
// divides or converts them (on GB300 both run on the slow FP64 pipe).
template <typename R>
struct PR {
  R inv_d[3];          // 1/dx, 1/dy, 1/deta
  R half_inv_d[3];     // 1/(2 dx), 1/(2 dy), 1/(2 deta)
  R theta;             // minmod parameter
  R inv_dtau, dtau, half_dtau;
  R rate_max;          // 1/tau_relax_min (or +inf)
  R tpp;               // tau_pipi/tau_pi
  R rho_max, xi0_rho_max;
  R eos_a;
  R eta_c0, eta_c1, eta_inv_c2, eta_ln_c0, eta_inv_c1;
  R zeta_c0, zeta_c1, zeta_inv_c2, zeta_ln_c0, zeta_inv_c1;
};

struct Params {
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
  const RootSeg* seg_r;
  const RootSegM* seg_m;  // the same intervals for the mixed-precision root-find
  Coef eta, zeta;
  int shear_on, bulk_on;
  double tpp;         // tau_pipi / tau_pi (10/7 or 0)
  int regulate;
  int iface_invert;   // face velocities from root-finds of the extrapolated states (KT_IFACE_INVERT)
  int mlp_infer;      // learned start: 1 runs the network (KT_INV_LEARNED), 0 starts from e_conf alone
  double rho_max, xi0;
  double e_min;
  double rate_max;    // 1 / tau_relax_min (or +inf)
  double ln_rate_max;
  PR<double> pd;
  PR<float> pf;
};

template <typename R> __device__ __forceinline__ const PR<R>& pr(const Params& P);
template <> __device__ __forceinline__ const PR<double>& pr<double>(const Params& P) { return P.pd; }
template <> __device__ __forceinline__ const PR<float>& pr<float>(const Params& P) { return P.pf; }

template <typename R> __device__ __forceinline__ const EosSeg<R>* eos_table(const Params& P);
template <> __device__ __forceinline__ const EosSeg<double>* eos_table<double>(const Params& P) { return P.seg_d; }
template <> __device__ __forceinline__ const EosSeg<float>* eos_table<float>(const Params& P) { return P.seg_f; }

// Interval search: a single-precision log guess, corrected so that e_i <= e < e_{i+1} exactly
// (clamped to the first / last interval outside the table).
template <typename R>
__device__ __forceinline__ int eos_interval(const Params& P, const EosSeg<R>* seg, R e) {
  int n1 = P.eos_n - 2;
  float ef;
  if constexpr (sizeof(R) == 8) ef = d2f_trunc(e); else ef = e;
  float g = (__logf(ef) - P.lne0) * P.inv_h;
  int i = (g > 0.f) ? (int)g : 0;  // NaN compares false -> 0
  i = min(i, n1);
  if constexpr (sizeof(R) == 8) {  // nodes are positive: compare bit patterns (e <= 0 orders below all)
    const long long b = __double_as_longlong(e);
#pragma unroll 1
    for (int it = 0; it < 64 && i > 0 && b < __double_as_longlong(seg[i].e0); ++it) --i;
#pragma unroll 1
    for (int it = 0; it < 64 && i < n1 && b >= __double_as_longlong(seg[i + 1].e0); ++it) ++i;
  } else {
#pragma unroll 1
    for (int it = 0; it < 64 && i > 0 && e < seg[i].e0; ++it) --i;
#pragma unroll 1
    for (int it = 0; it < 64 && i < n1 && e >= seg[i + 1].e0; ++it) ++i;
  }
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
    T = sqrt(sqrt(e / pr<R>(P).eos_a));
    lnd = -R(INFINITY);
    return;
  }
  const EosSeg<R>* seg = eos_table<R>(P);
  // FP64: the exact interval.  FP32 (the mixed-precision sources): the interval of the
  // single-precision log guess alone; next to a node that may be the neighbouring interval,
  // whose cubic matches value and slope at the node, so the difference stays far below FP32
  // rounding, and the dependent table loads of the correction are saved.
  int i;
  if constexpr (sizeof(R) == 8) {
    i = eos_interval<R>(P, seg, e);
  } else {
    const float g = (__logf(e) - P.lne0) * P.inv_h;
    i = min((g > 0.f) ? (int)g : 0, P.eos_n - 2);
  }
  const EosSeg<R>& s = seg[i];
  R t = (e - s.e0) * s.inv_de;
  T = fma(t, fma(t, fma(t, s.cT3, s.cT2), s.mT), s.T0);
  lnd = fma(t, s.dl, s.l0);
}

// Generalised minmod of (theta dl, (dl + dr)/2, theta dr), Sec. 3.1, with sgn(0) = 0, from the
// one-sided differences dl = q_i - q_{i-1}, dr = q_{i+1} - q_i: the three arguments share a sign
// exactly when dl and dr do, and then the result is that sign times the smallest magnitude.
// This is the slope times the cell size.
// FP64: the signs and magnitudes are compared as integers (the magnitudes of doubles order like
// their bit patterns), so only the theta branch does FP64 arithmetic.  FP32 with theta = 1: the
// median of (dl, dr, 0) by four min/max instructions.  (FP32 theta != 1 tests the sign by the
// product, which loses slopes whose one-sided differences multiply below ~1e-45.)
// TH1: theta = 1, where (|dl| + |dr|)/2 >= min(|dl|, |dr|) never decides.
template <typename R, bool TH1 = false>
__device__ __forceinline__ R limited_slope_d(R dl, R dr, R theta) {
  if constexpr (sizeof(R) == 8) {
    const long long bl = __double_as_longlong(dl), br = __double_as_longlong(dr);
    const long long ml = bl & 0x7fffffffffffffffLL, mr = br & 0x7fffffffffffffffLL;
    R m = (ml < mr) ? dl : dr;  // the smaller magnitude (0 if either is 0), with the shared sign
    if constexpr (!TH1) {
      const R m1 = theta * m, m2 = R(0.5) * (dl + dr);
      m = ((__double_as_longlong(m1) & 0x7fffffffffffffffLL) < (__double_as_longlong(m2) & 0x7fffffffffffffffLL))
              ? m1 : m2;
    }
    return ((bl ^ br) >= 0) ? m : R(0);
  } else if constexpr (TH1) {
    return fmaxf(fminf(dl, dr), fminf(fmaxf(dl, dr), 0.f));
  } else {
    R mn = fmin(theta * fabs(dl), theta * fabs(dr));
    mn = fmin(mn, R(0.5) * fabs(dl + dr));
    return (dl * dr > R(0)) ? copysign(mn, dl) : R(0);
  }
}

// The three slopes of a five-point stencil, s_{i-1}, s_i, s_{i+1}, from its one-sided differences
// d0..d3.  FP32 with theta = 1: minmod(a, b) = clamp(a, min(0, b), max(0, b)) (zero when the signs
// differ or either is zero, else the smaller magnitude), so s_i and s_{i+1} share the bounds from
// d2: ten min/max instructions for the three.  Otherwise limited_slope_d for each.
template <typename R, bool TH1>
__device__ __forceinline__ void three_slopes(R d0, R d1, R d2, R d3, R th, R& sm, R& s0, R& sp) {
  if constexpr (sizeof(R) == 4 && TH1) {
    const R lo1 = fminf(d1, 0.f), hi1 = fmaxf(d1, 0.f), lo2 = fminf(d2, 0.f), hi2 = fmaxf(d2, 0.f);
    sm = fminf(fmaxf(d0, lo1), hi1);
    s0 = fminf(fmaxf(d1, lo2), hi2);
    sp = fminf(fmaxf(d3, lo2), hi2);
  } else {
    sm = limited_slope_d<R, TH1>(d0, d1, th);
    s0 = limited_slope_d<R, TH1>(d1, d2, th);
    sp = limited_slope_d<R, TH1>(d2, d3, th);
  }
}

// max(a, b) of non-negative a, b (FP64: compared as integers, off the FP64 pipe)
__device__ __forceinline__ float nmax(float a, float b) { return fmaxf(a, b); }
__device__ __forceinline__ double nmax(double a, double b) {
  return (__double_as_longlong(a) < __double_as_longlong(b)) ? b : a;
}

// a / b for b > 0 (face velocities: b is an extrapolated u^tau >= 1).  FP32: the fast hardware
// division.  FP64, for b within [2^-125, 2^125): Newton-Raphson for 1/b from a single-precision
// seed (b's leading 20 mantissa bits, approximate reciprocal: relative error ~2^-20), one step
// r <- r + r (1 - b r) (~2^-40), then the quotient corrected once, q <- q + r (a - b q), which
// leaves about one ulp; five FP64 instructions.  Other b take the IEEE division.
__device__ __forceinline__ float vdiv(float a, float b) { return __fdividef(a, b); }
__device__ __forceinline__ double vdiv(double a, double b) {
  const unsigned hi = (unsigned)__double2hiint(b);
  if ((hi >> 20) - 898u > 249u) return a / b;  // also b <= 0, NaN, infinity
  const float bf = __uint_as_float((hi - 0x38000000u) << 3);
  float rf;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(rf) : "f"(bf));
  const unsigned rb = __float_as_uint(rf);
  const double r0 = __hiloint2double((int)((rb >> 3) + 0x38000000u), (int)(rb << 29));
  const double r1 = fma(r0, fma(-b, r0, 1.0), r0);
  const double q0 = a * r1;
  return fma(r1, fma(-b, q0, a), q0);
}

// a / b, exp, ln in the stencil precision.  FP64: the division of vdiv (about one ulp; the IEEE
// division for denominators outside its range), the library exp and log.  FP32: the fast
// hardware forms (a few ulp; division operands are velocities, u^tau >= 1 and transport scales,
// far from the range where the fast division degrades).
__device__ __forceinline__ double sdiv(double a, double b) { return vdiv(a, b); }
__device__ __forceinline__ float sdiv(float a, float b) { return __fdividef(a, b); }
__device__ __forceinline__ double sexp(double x) { return exp(x); }
__device__ __forceinline__ float sexp(float x) { return __expf(x); }
__device__ __forceinline__ double slog(double x) { return log(x); }
__device__ __forceinline__ float slog(float x) { return __logf(x); }

// zeta/s of Sec. 2.2, Eq. (zetas), at x = T/T_c (the quadratic on 0.995 <= x <= 1.05)
template <typename R>
__device__ __forceinline__ R zeta_over_s_paper(R x) {
  const R y = x - R(1);
  if (x > R(1.05)) return R(0.9) * sexp(-y * R(1.0 / 0.025)) + R(0.25) * sexp(-y * R(1.0 / 0.13)) + R(0.001);
  if (x < R(0.995)) return R(0.9) * sexp(y * R(1.0 / 0.0025)) + R(0.22) * sexp(y * R(1.0 / 0.022)) + R(0.03);
  return R(-13.45) + R(27.55) * x - R(13.77) * x * x;
}

// eta/s(T) and ln(zeta/s)(T): const c0, c0 exp(-((T - c1)/c2)^2), or c0 times Eq. (zetas)
template <typename R>
__device__ __forceinline__ R eta_over_s(const Params& P, R T) {
  const PR<R>& p = pr<R>(P);
  if (P.eta.kind == 0) return p.eta_c0;
  if (P.eta.kind == 2) return p.eta_c0 * zeta_over_s_paper<R>(T * p.eta_inv_c1);
  R x = (T - p.eta_c1) * p.eta_inv_c2;
  return p.eta_c0 * sexp(-x * x);
}

template <typename R>
__device__ __forceinline__ R ln_zeta_over_s(const Params& P, R T) {
  const PR<R>& p = pr<R>(P);
  if (P.zeta.kind == 0) return p.zeta_ln_c0;
  if (P.zeta.kind == 2) return slog(p.zeta_c0 * zeta_over_s_paper<R>(T * p.zeta_inv_c1));
  R x = (T - p.zeta_c1) * p.zeta_inv_c2;
  return p.zeta_ln_c0 - x * x;
}

// Conversions between float and double on the integer pipe.  On GB300 the F2F conversion
// instructions issue on the FP64 pipe, which has 1/64 of the FP32 rate; these bit-level
// versions leave it free.  float -> double is exact (subnormal floats flush to zero);
// double -> float rounds to nearest even (results below the smallest normal float flush to
// zero; overflow, infinity and NaN give infinity, so a non-finite input stays non-finite).
__device__ __forceinline__ double f2d_bits(float f) {
  const unsigned b = __float_as_uint(f);
  const unsigned ex = (b >> 23) & 0xffu;
  const unsigned s = b & 0x80000000u;
  const unsigned m = b & 0x7fffffu;
  const unsigned ed = (ex == 0xffu) ? 0x7ffu : ex + 896u;
  const unsigned hi = (ex == 0u) ? s : (s | (ed << 20) | (m >> 3));
  const unsigned lo = (ex == 0u) ? 0u : (m << 29);
  return __hiloint2double((int)hi, (int)lo);
}

__device__ __forceinline__ float d2f_bits(double d) {
  // round to nearest even at bit 29 of the magnitude: adding 0x0fffffff plus the lowest kept bit
  // carries into the kept bits exactly when the dropped ones exceed half an ulp, or equal it with
  // an odd kept part; the exponent is rebiased by 896 in the same 64-bit addition
  const unsigned hi = (unsigned)__double2hiint(d), lo = (unsigned)__double2loint(d);
  const unsigned ah = hi & 0x7fffffffu;
  const unsigned long long r =
      ((((unsigned long long)ah << 32) | lo) + (0x0fffffffull + ((lo >> 29) & 1u))) - (896ull << 52);
  unsigned bits = (unsigned)(r >> 29);
  bits = (ah < (897u << 20)) ? 0u : bits;              // below the smallest normal float
  bits = (ah >= (1151u << 20)) ? 0x7f800000u : bits;   // overflow, infinity or NaN
  return __uint_as_float((hi & 0x80000000u) | bits);
}

// double -> float by truncating the mantissa (rounding toward zero), for values that only steer a
// computation -- the network's features, the Newton step length, the table-interval guess -- and
// never reach a stored result: magnitudes below the smallest normal float flush to zero; finite
// |x| < 2^128 is assumed.  Six integer instructions against about twenty for d2f_bits.
__device__ __forceinline__ float d2f_trunc(double d) {
  const unsigned hi = (unsigned)__double2hiint(d), lo = (unsigned)__double2loint(d);
  const int hm = (int)(hi & 0x7fffffffu) - (896 << 20);  // exponent rebiased to the float's
  const unsigned mag = __funnelshift_l(lo, (unsigned)hm, 3);
  return __uint_as_float((hi & 0x80000000u) | ((hm >= (1 << 20)) ? mag : 0u));
}

template <typename R> __device__ __forceinline__ double to_f64(R x);
template <> __device__ __forceinline__ double to_f64<double>(double x) { return x; }
template <> __device__ __forceinline__ double to_f64<float>(float x) { return f2d_bits(x); }
__device__ __forceinline__ float to_f32(float x) { return x; }
__device__ __forceinline__ float to_f32(double x) { return d2f_bits(x); }
template <typename R> __device__ __forceinline__ R from_f64(double x);
template <> __device__ __forceinline__ double from_f64<double>(double x) { return x; }
template <> __device__ __forceinline__ float from_f64<float>(double x) { return d2f_bits(x); }

// per-cell read of an R-typed field from a buffer that may hold double or float
template <typename R, typename S>
__device__ __forceinline__ R ld(const S* __restrict__ p, long long i) {
  return (R)__ldg(p + i);
}

}  // namespace kt
