// flops.hpp -- an operation-counting stand-in for double, for the algorithmic flop count of the
// oracle (kt_oracle_flops.cpp compiles kt_oracle.c with it in place of double).
//
// TEST AND MEASUREMENT INFRASTRUCTURE ONLY, like the oracle itself.  Every arithmetic operation on
// a counted value increments one counter per kind; the values themselves are computed exactly as
// with double (the same operations in the same order, no contraction), so the counting build
// reproduces the plain oracle bit for bit.  Single-threaded: the counters are plain globals.
#pragma once
#include <cmath>

enum FlopKind { FK_ADD, FK_MUL, FK_DIV, FK_SQRT, FK_TRANSC, FK_CMP, FK_N };
extern unsigned long long ko_flop_count[FK_N];

struct fdouble {
  double v;
  fdouble() = default;  // trivial, so calloc'd arrays of fdouble are valid
  constexpr fdouble(double x) : v(x) {}
  explicit operator double() const { return v; }
  explicit operator int() const { return (int)v; }
  explicit operator long long() const { return (long long)v; }
  explicit operator unsigned long() const { return (unsigned long)v; }
  explicit operator float() const { return (float)v; }
};
static_assert(sizeof(fdouble) == sizeof(double), "fdouble must have the layout of double");

inline fdouble fc_op(FlopKind k, double r) {
  ++ko_flop_count[k];
  return fdouble(r);
}
inline fdouble operator+(fdouble a, fdouble b) { return fc_op(FK_ADD, a.v + b.v); }
inline fdouble operator-(fdouble a, fdouble b) { return fc_op(FK_ADD, a.v - b.v); }
inline fdouble operator*(fdouble a, fdouble b) { return fc_op(FK_MUL, a.v * b.v); }
inline fdouble operator/(fdouble a, fdouble b) { return fc_op(FK_DIV, a.v / b.v); }
inline fdouble operator-(fdouble a) { return fdouble(-a.v); }  // a sign flip, not counted
inline fdouble operator+(fdouble a) { return a; }
inline fdouble& operator+=(fdouble& a, fdouble b) { return a = a + b; }
inline fdouble& operator-=(fdouble& a, fdouble b) { return a = a - b; }
inline fdouble& operator*=(fdouble& a, fdouble b) { return a = a * b; }
inline fdouble& operator/=(fdouble& a, fdouble b) { return a = a / b; }
inline bool fc_cmp(bool r) {
  ++ko_flop_count[FK_CMP];
  return r;
}
inline bool operator<(fdouble a, fdouble b) { return fc_cmp(a.v < b.v); }
inline bool operator>(fdouble a, fdouble b) { return fc_cmp(a.v > b.v); }
inline bool operator<=(fdouble a, fdouble b) { return fc_cmp(a.v <= b.v); }
inline bool operator>=(fdouble a, fdouble b) { return fc_cmp(a.v >= b.v); }
inline bool operator==(fdouble a, fdouble b) { return fc_cmp(a.v == b.v); }
inline bool operator!=(fdouble a, fdouble b) { return fc_cmp(a.v != b.v); }

// library functions: sqrt counts as one square root, exp/log/pow/tanh as one transcendental
// each; |x|, scaling by a power of two and finiteness tests are free
inline fdouble sqrt(fdouble a) { return fc_op(FK_SQRT, std::sqrt(a.v)); }
inline fdouble exp(fdouble a) { return fc_op(FK_TRANSC, std::exp(a.v)); }
inline fdouble log(fdouble a) { return fc_op(FK_TRANSC, std::log(a.v)); }
inline fdouble tanh(fdouble a) { return fc_op(FK_TRANSC, std::tanh(a.v)); }
inline fdouble pow(fdouble a, fdouble b) { return fc_op(FK_TRANSC, std::pow(a.v, b.v)); }
inline fdouble fabs(fdouble a) { return fdouble(std::fabs(a.v)); }
inline fdouble ldexp(fdouble a, int e) { return fdouble(std::ldexp(a.v, e)); }
inline bool isfinite(fdouble a) { return std::isfinite(a.v); }
